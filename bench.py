"""Benchmark: angular-spectrum propagation of 2048 x 2048 complex64 fields on GB300.

One step = one batched call of the whole hot path (row forward FFT with fused zero padding,
column FFT + transfer function + inverse column FFT, row inverse FFT with fused crop) over a
batch of B synthetic 2048^2 fields resident in HBM (B * 32 MiB of input > L2, so no L2 flush is
needed between steps).  Metric: propagations/s (whole job), plus HBM GB/s against the roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]

Under torchrun each rank runs its own batch (independent items, no collective on the data
path: weak scaling); the time is the max over ranks.  ``--impl reference`` times the FP64 CPU
oracle on this host's cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 2048
PITCH = 10e-6
LAM = 633e-9
Z = 0.05
METRIC = "propagations/s (2048^2 angular spectrum, padded to 4096^2)"
UNIT = "propagations/s"
BYTES_PER_PROP = 80 * N * N          # 3 passes: 8N^2 + 16N^2 | 16N^2 + 16N^2 | 16N^2 + 8N^2
COL_BYTES_PER_PROP = 32 * N * N      # column pass: read + write the Ny x Px intermediate


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel at
# batch 16, from one ncu capture of the current column kernel (profiles/asm_2048_batch16_launches.md);
# scaled by the batch (traffic grows in proportion to the fields processed).  The column pass reads
# the 67 MB transfer-function table of the plan once per launch besides its 16 fields.
NCU_TRAFFIC_B16 = {"col_fwd_h_inv": 2154.40e6}


def traffic_bytes(kernel, batch):
    t = NCU_TRAFFIC_B16.get(kernel)
    return None if t is None else round(t * batch / 16)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # wait (at most 3 s) for the first sample; only samples taken after it are summarised
        self.skip = 0
        t0 = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t0 < 3.0:
            with open(self.path) as f:
                self.skip = sum(1 for _ in f)
            if self.skip:
                break
            time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if len(rows) > self.skip:
            rows = rows[self.skip:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- FP32 arithmetic of the passes, counted from the kernels' own butterflies (P = 4096: three
# radix-16 DIF stages).  FP32 instructions per 16 points: a radix-16 butterfly done as 4 x 4
# (eight radix-4 DFTs of 16 additions, eight non-trivial inner twiddles of 4 instructions) = 160;
# the first forward stage, whose upper 8 inputs are the zero padding, 128; the last inverse stage,
# of which only the lower 8 outputs are kept, 144; the 15 inter-stage twiddle multiplications
# (complex multiply = 2 FMUL + 2 FFMA) 60.  ncu counts of the same kernels (fadd + fmul + ffma
# thread instructions) agree within 4% (profiles/asm_2048_kernels_full.md).
FP32_R16, FP32_R16_ZERO_HALF_IN, FP32_R16_HALF_OUT, FP32_TWIDDLES = 160, 128, 144, 60
FP32_FWD = (FP32_R16_ZERO_HALF_IN + FP32_TWIDDLES + FP32_R16 + FP32_TWIDDLES + FP32_R16) / 16.0   # per point
FP32_INV = (FP32_R16 + FP32_TWIDDLES + FP32_R16 + FP32_TWIDDLES + FP32_R16_HALF_OUT) / 16.0       # per point
FP32_PER_PASS = {   # FP32 instructions per propagation of an N x N field (P = 2N)
    "row_fwd": FP32_FWD * N * 2 * N,                      # N rows of P points
    "col_fwd_h_inv": (FP32_FWD + 4.0 + FP32_INV) * (2 * N) ** 2,   # P columns: FFT, x H (loaded), IFFT
    "row_inv": (FP32_INV + 1.0) * N * 2 * N,              # N rows: IFFT, 1/(Px Py) on the kept half
}


def fp32_peak(dev):
    """FP32 instruction rate of this GPU (instructions/s): sixteen independent FFMA chains per
    thread, 32 warps per SM, timed with CUDA events, best of 5 (cwo_debug_ffma_rate)."""
    import torch
    from paper_1107_5578_gb300 import cwo
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = sms * 8, 2048
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    L = cwo.lib()
    stream = torch.cuda.current_stream()
    best = float("inf")
    for k in range(6):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cwo.check(L.cwo_debug_ffma_rate(blocks, iters, out.data_ptr(), stream.cuda_stream), "cwo_debug_ffma_rate")
        b.record(stream)
        torch.cuda.synchronize()
        if k:
            best = min(best, a.elapsed_time(b) / 1e3)
    return blocks * 256 * iters * 16 / best


class NvmlClockSampler:
    """SM clock and throttle reasons sampled every 2 ms by NVML queries (read only) during the
    timed region; falls back to the nvidia-smi sampler where NVML cannot be loaded."""
    BITS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, torch_index: int):
        self.index = torch_index
        self.fallback = None
        self.samples = []

    def _handle(self):
        import ctypes
        import torch
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(self.index)
        uuid = getattr(props, "uuid", None)
        ok = False
        if uuid is not None:
            u = str(uuid)
            u = u if u.startswith("GPU-") else "GPU-" + u
            ok = nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
        if not ok:
            bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
            ok = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        if not ok:
            raise OSError("no NVML handle for the device")
        return nv, h

    def __enter__(self):
        import ctypes
        import threading
        try:
            nv, h = self._handle()
        except Exception:
            self.fallback = ClockSampler(self.index).__enter__()
            return self
        reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or nv.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
        self.max_mhz = float(mx.value)
        self.stop = threading.Event()

        def run():
            clk, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
            while not self.stop.is_set():
                if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and reasons_fn(h, ctypes.byref(rs)) == 0:
                    self.samples.append((float(clk.value), int(rs.value)))
                time.sleep(0.002)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 1.0:
            time.sleep(0.001)
        self.skip = len(self.samples)
        return self

    def __exit__(self, *a):
        if self.fallback is not None:
            return self.fallback.__exit__(*a)
        self.stop.set()
        self.thread.join(timeout=2)

    def summary(self):
        if self.fallback is not None:
            return self.fallback.summary()
        rows = self.samples[self.skip:] or self.samples[-1:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = sorted({name for _, r in rows for bit, name in self.BITS.items() if r & bit})
        return {"sm_mhz": float(np.median([c for c, _ in rows])), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(rows), "sampler": "nvml, 2 ms"}


def oracle_times(fn, reps=2):
    """Seconds per call of fn() with the oracle on one thread and on all of them."""
    import oracle
    cores = oracle.max_threads()
    out = {}
    for label, th in (("1_thread", 1), (f"{cores}_threads", cores)):
        oracle.set_threads(th)
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        out[label] = round((time.perf_counter() - t0) / reps, 4)
    oracle.set_threads(cores)
    return out, cores


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def config_asm_512(dev, steps=200):
    """512^2 ASM (633 nm, 10 um, z = 0.05 m, padded to 1024^2) from a complex128 field: relative
    L2 against the FP64 oracle, device throughput as a batch of 64 and one propagation at a time,
    and the oracle's time on 1 and all host threads."""
    import torch
    import oracle
    from paper_1107_5578_gb300 import cwo, synth
    n, z = 512, 0.05
    u = synth.random_field(n, seed=1)
    plan = cwo.Plan(n, n, PITCH, PITCH, LAM, z, cwo.ANGULAR)
    plan.reserve(64)
    x1 = torch.from_numpy(u.astype(np.complex64)).to(dev)
    got = plan.propagate(x1).cpu().numpy().astype(np.complex128)
    want = oracle.propagate(u, PITCH, PITCH, LAM, z, oracle.ANGULAR)
    xb = torch.from_numpy(np.stack([synth.random_field(n, seed=10 + k) for k in range(64)]).astype(np.complex64)).to(dev)
    yb = torch.empty_like(xb)
    y1 = torch.empty_like(x1)

    def timed(f, reps):
        for _ in range(5):
            f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            f()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_b = timed(lambda: plan.propagate_batch(xb, out=yb), steps)
    ms_1 = timed(lambda: plan.propagate(x1, out=y1), steps)
    plan.close()
    ot, cores = oracle_times(lambda: oracle.propagate(u, PITCH, PITCH, LAM, z, oracle.ANGULAR), reps=3)
    return {"workload": "asm_512_pad1024", "rel_l2_vs_oracle": rel_l2(got, want),
            "batch64_propagations_per_s": round(64 / (ms_b / 1e3), 1), "single_us": round(1e3 * ms_1, 2),
            "single_propagations_per_s": round(1 / (ms_1 / 1e3), 1),
            "oracle_s_per_propagation": ot, "oracle_cores": cores}


def config_fresnel_stack_errors(dev):
    """The 16-plane Fresnel stack of 2048^2 (one call): planes 0, 7 and 15 against the FP64 oracle
    propagating the same source to the same distance, and the oracle's time per plane."""
    import torch
    import oracle
    from paper_1107_5578_gb300 import cwo, synth
    n, planes = 2048, 16
    zs = [float(v) for v in np.linspace(0.1, 0.4, planes)]
    u = synth.masked_gaussian(n, seed=2)
    plan = cwo.Plan(n, n, 8e-6, 8e-6, 532e-9, zs[0], cwo.FRESNEL_CONV)
    y = plan.propagate_stack(torch.from_numpy(u.astype(np.complex64)).to(dev), zs)
    torch.cuda.synchronize()
    errs = {}
    for j in (0, 7, 15):
        want = oracle.propagate(u.astype(np.complex64), 8e-6, 8e-6, 532e-9, zs[j], oracle.FRESNEL_CONV)
        errs[f"plane_{j}_z_{zs[j]:.3f}"] = rel_l2(y[j].cpu().numpy().astype(np.complex128), want)
    plan.close()
    ot, cores = oracle_times(lambda: oracle.propagate(u, 8e-6, 8e-6, 532e-9, zs[7], oracle.FRESNEL_CONV), reps=1)
    return {"rel_l2_vs_oracle": errs, "oracle_s_per_plane": ot, "oracle_cores": cores}


def config_precision_4096(dev):
    """Precision study at 4096^2 (padded to 8192^2; unit amplitude, random phase; 532 nm, 3.74 um):
    relative L2 and the largest wrapped phase error (|U| > 1e-3 max |U|) of the three
    transfer-function phase arms against the FP64 oracle, for z = 0.05, 0.2 and 1.0 m."""
    import oracle
    from paper_1107_5578_gb300 import precision, synth
    n, lam, pitch = 4096, 532e-9, 3.74e-6
    u = synth.random_phase_field(n, seed=3).astype(np.complex64)
    out = {}
    for z in (0.05, 0.2, 1.0):
        ref = oracle.propagate(u, pitch, pitch, lam, z, oracle.ANGULAR)
        out[f"z_{z}"] = {arm: {k: float(f"{v:.3e}") for k, v in precision.errors(precision.run_arm(u, pitch, lam, z, arm), ref).items()}
                         for arm in precision.ARMS}
    return {"workload": "asm_4096_pad8192", "arms": out}


def config_hologram(dev, steps=200):
    """Phase-only hologram (1920 x 1080 phase in a 2048^2 canvas, padded to 4096^2, 520 nm,
    6.4 um, z = 0.15 m): 200 Adam steps through the hand-written adjoint; seconds per step and the
    first and last loss."""
    from paper_1107_5578_gb300 import hologram
    prob = hologram.HologramProblem(device=dev)
    # untimed warm-up from the same start: first-use costs (kernel attributes, autograd, Adam state)
    # stay out of the timed run, which starts again from the initial phase
    hologram.optimise(prob, steps=3, lr=0.05)
    _, losses, dt = hologram.optimise(prob, steps=steps, lr=0.05)
    prob.plan.close()
    return {"workload": "hologram_1920x1080_canvas2048_pad4096", "steps": steps, "ms_per_step": round(1e3 * dt / steps, 3),
            "loss_first": float(f"{losses[0]:.5e}"), "loss_last": float(f"{losses[-1]:.5e}")}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle
    from paper_1107_5578_gb300 import synth
    oracle.build()
    u = synth.random_field(N, seed=1)
    oracle.propagate(u, PITCH, PITCH, LAM, Z, oracle.ANGULAR)   # warm page cache / threads
    times = []
    for _ in range(max(1, args.warmup)):
        oracle.propagate(u, PITCH, PITCH, LAM, Z, oracle.ANGULAR)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.propagate(u, PITCH, PITCH, LAM, Z, oracle.ANGULAR)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = 1e3 / ms
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "asm_2048_pad4096", "n": N, "batch_per_step": 1,
                                            "pitch_m": PITCH, "wavelength_m": LAM, "z_m": Z},
            "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"1 propagation of one 2048^2 field per step, {args.steps} steps"},
            "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    """Oracle throughput on this host (bounded: a few 2048^2 propagations, ~seconds), on all
    threads, with one single-threaded propagation beside it."""
    import oracle
    from paper_1107_5578_gb300 import synth
    oracle.build()
    u = synth.random_field(N, seed=1)
    oracle.propagate(u, PITCH, PITCH, LAM, Z, oracle.ANGULAR)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.propagate(u, PITCH, PITCH, LAM, Z, oracle.ANGULAR)
        reps += 1
        if time.perf_counter() - t0 > 8.0 or reps >= 5:
            break
    dt = (time.perf_counter() - t0) / reps
    cores = oracle.max_threads()
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.propagate(u, PITCH, PITCH, LAM, Z, oracle.ANGULAR)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": round(1.0 / dt, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} propagation(s) of one 2048^2 ASM field (FP64, OpenMP over rows/columns)",
            "single_thread": {"value": round(1.0 / dt1, 4), "unit": UNIT, "cores": 1,
                              "sample": "1 propagation of one 2048^2 ASM field on one thread"}}


def stack_measurement(dev, hbm_peak):
    """The 2048^2 Fresnel z-stack: a seeded Bernoulli(0.5) mask times a Gaussian envelope
    (sigma = 400 px), 532 nm, 8 um, 16 planes z = linspace(0.1, 0.4, 16), all planes in one
    batched call, which runs as two separable line passes: every source row is transformed once
    and convolved per plane into that plane's N x N intermediate, then every plane's columns.
    Algorithmic bytes 8 N^2 (1 + 3 J): source read once; per plane the intermediate written and
    read once and the plane written (392 N^2 at J = 16, against 680 N^2 for the three-pass stack
    with its N x 2N spectra)."""
    import torch
    from paper_1107_5578_gb300 import cwo, synth
    n, planes = 2048, 16
    zs = [float(v) for v in np.linspace(0.1, 0.4, planes)]
    x = torch.from_numpy(synth.masked_gaussian(n, seed=2).astype(np.complex64)).to(dev)
    plan = cwo.Plan(n, n, 8e-6, 8e-6, 532e-9, zs[0], cwo.FRESNEL_CONV)
    plan.reserve(planes)
    y = torch.empty((planes, n, n), dtype=torch.complex64, device=dev)
    for _ in range(3):
        plan.propagate_stack(x, zs, out=y)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    a.record()
    for _ in range(reps):
        plan.propagate_stack(x, zs, out=y)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    nbytes = 8 * (1 + 3 * planes) * n * n
    gbs = nbytes / (ms / 1e3) / 1e9
    launches = plan.launches_per_call
    plan.close()
    return {"workload": "fresnel_2048_pad4096_stack16", "ms_per_stack": round(ms, 4),
            "planes_per_s": round(planes / (ms / 1e3), 1), "hbm_gbs_algorithmic": round(gbs, 1),
            "frac_of_measured_hbm": round(gbs / hbm_peak, 4), "bytes_per_stack": nbytes,
            "launches_per_stack": launches}


def serving_measurement(dev, n_req, rate_hz):
    """Mixed-size serving on an open-loop Poisson stream (seeded): N in {256..4096} weighted
    .3/.3/.2/.15/.05, 70 % ASM / 30 % Fresnel, z ~ U[0.01, 0.5] m, lambda in {450, 532, 633} nm,
    pitch ~ U[4, 10] um, fields from a device-resident pool.  Continuous batching (per-size slots,
    mixed per-item batches, memory admission, concurrent streams) against the serial baseline
    (one request at a time) on the same stream; latency = arrival -> observed completion."""
    import torch
    from paper_1107_5578_gb300 import serving, synth
    sizes = synth.SERVING_SIZES
    pools = serving.make_pools(sizes, per_size=4, device=dev)
    server = serving.Server(sizes=sizes, pools=pools, device=dev)
    server.warm_up()
    server.run(serving.make_requests(2000, seed=77, rate_hz=4 * rate_hz))       # warm-up
    reqs = serving.make_requests(n_req, seed=78, rate_hz=rate_hz)
    b0 = server.batches
    server.run(reqs)
    cont = serving.latency_stats(reqs)
    cont["batches"] = server.batches - b0
    cont["mem_peak_bytes"] = server.mem_peak
    plans = {}
    serving.serve_serial(serving.make_requests(400, seed=77, rate_hz=rate_hz), pools, device=dev, plans=plans)
    sreqs = serving.make_requests(n_req, seed=78, rate_hz=rate_hz)
    serving.serve_serial(sreqs, pools, device=dev, plans=plans)
    ser = serving.latency_stats(sreqs)
    server.close()
    for v in plans.values():
        v.close()
    del server, plans, pools
    torch.cuda.empty_cache()
    return {"workload": "mixed_256_to_4096_poisson", "requests": n_req, "rate_hz": rate_hz,
            "continuous": cont, "serial": ser}


def timed_steps(plan, x, y, steps, stream, before=None):
    """Run `steps` propagations of the batch x back to back on `stream`; return the event time of
    the whole run (ms) and the summed per-pass times (ms), read after the run from one set of
    pass events per step (recorded by the library on the launching stream)."""
    import torch
    step_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for evs in step_ev:
        for e_ in evs:
            e_.record(stream)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if before is not None:
        before()
    t0.record(stream)
    for i in range(steps):
        plan.set_timing_events(step_ev[i])
        plan.propagate_batch(x, out=y)
    t1.record(stream)
    return t0, t1, step_ev


def pass_sums(plan, step_ev):
    plan.set_timing_events(None)
    pp = np.zeros(3)
    for evs in step_ev:
        pp += [evs[0].elapsed_time(evs[1]), evs[1].elapsed_time(evs[2]), evs[2].elapsed_time(evs[3])]
    return pp


def recalc_h_measurement(x, y, steps):
    """The same 2048^2 ASM batch with the transfer function evaluated per element in the column
    pass (the paper's "re-calculation"; no per-plan table): propagations/s and per-pass times."""
    import torch
    from paper_1107_5578_gb300 import cwo
    B = x.shape[0]
    plan = cwo.Plan(N, N, PITCH, PITCH, LAM, Z, cwo.ANGULAR)
    plan.reserve(B)
    for _ in range(3):
        plan.propagate_batch(x, out=y)
    a, b, step_ev = timed_steps(plan, x, y, steps, torch.cuda.current_stream())
    torch.cuda.synchronize()
    pp = pass_sums(plan, step_ev)
    ms = a.elapsed_time(b) / steps
    plan.close()
    return {"workload": "asm_2048_pad4096, transfer function evaluated per element", "value": round(B / (ms / 1e3), 2),
            "unit": UNIT, "passes_ms": {k: round(v / steps, 4) for k, v in zip(("row_fwd", "col_fwd_h_inv", "row_inv"), pp)}}


def asm_4096_measurement(dev, steps, hbm_peak, batch=2):
    """The 4096^2 angular spectrum method (padded to 8192^2; the precision study's size), batch 2,
    transfer function materialised per plan: propagations/s, per-pass times and algorithmic
    TB/s (80 N^2 bytes per propagation)."""
    import torch
    from paper_1107_5578_gb300 import cwo
    n = 4096
    x = torch.randn(batch, n, n, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    plan = cwo.Plan(n, n, 3.74e-6, 3.74e-6, 532e-9, 0.2, cwo.ANGULAR, cwo.FLAG_CACHE_H)
    plan.reserve(batch)
    for _ in range(3):
        plan.propagate_batch(x, out=y)
    a, b, step_ev = timed_steps(plan, x, y, steps, torch.cuda.current_stream())
    torch.cuda.synchronize()
    pp = pass_sums(plan, step_ev) / steps
    ms = a.elapsed_time(b) / steps
    plan.close()
    del x, y
    torch.cuda.empty_cache()
    gbs = 80 * n * n * batch / (ms / 1e3) / 1e9
    return {"workload": f"asm_4096_pad8192_batch{batch}", "value": round(batch / (ms / 1e3), 2), "unit": UNIT,
            "passes_ms": {k: round(v, 4) for k, v in zip(("row_fwd", "col_fwd_h_inv", "row_inv"), pp)},
            "hbm_gbs_algorithmic": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm_peak, 4)}


def fresnel_batch_measurement(x, y, steps, hbm_peak):
    """Fresnel diffraction (convolution form) of the same 16 fields of 2048^2 (532 nm, 8 um,
    z = 0.2 m): two separable line passes, 32 N^2 algorithmic bytes per propagation."""
    import torch
    from paper_1107_5578_gb300 import cwo
    B = x.shape[0]
    plan = cwo.Plan(N, N, 8e-6, 8e-6, 532e-9, 0.2, cwo.FRESNEL_CONV)
    plan.reserve(B)
    for _ in range(3):
        plan.propagate_batch(x, out=y)
    a, b, step_ev = timed_steps(plan, x, y, steps, torch.cuda.current_stream())
    torch.cuda.synchronize()
    pp = pass_sums(plan, step_ev) / steps
    ms = a.elapsed_time(b) / steps
    launches = plan.launches_per_call
    plan.close()
    gbs = 32 * N * N * B / (ms / 1e3) / 1e9
    return {"workload": f"fresnel_conv_2048_pad4096_batch{B}", "value": round(B / (ms / 1e3), 2), "unit": UNIT,
            "passes_ms": {"line_x": round(pp[0], 4), "line_y": round(pp[1], 4)},
            "hbm_gbs_algorithmic": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm_peak, 4),
            "bytes_per_prop": 32 * N * N, "launches_per_call": launches}


# Table "Calculation times of the GS algorithm on the CPU and GPUs", 40 iterations, GeForce GTX580
GS_PAPER_MS_40 = {512: 338.0, 1024: 1.19e3, 2048: 4.65e3}


def gs_measurement(dev, iterations=40):
    """GS kinoform loop (Section "GS algorithm"): object = sqrt of a synthetic test image with a
    random phase, ASM at +-0.1 m, 633 nm, 10 um, the plan's transfer function materialised once
    (gs.GSProblem); the timed region covers the first propagation,
    `iterations` iterations and the final reconstruction (2 * iterations + 2 propagations), as
    the paper times its loop, with everything resident on the device."""
    import torch
    from paper_1107_5578_gb300 import gs
    out = []
    for n in (512, 1024, 2048):
        prob = gs.GSProblem(n, seed=1, device=dev)
        prob.run(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, inten = prob.run(iterations)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out.append({"n": n, "iterations": iterations, "ms": round(ms, 3),
                    "propagations_per_s": round((2 * iterations + 2) / (ms / 1e3), 1),
                    "amplitude_error": round(gs.amplitude_error(inten, prob.amplitude), 5),
                    "paper_gtx580_ms": GS_PAPER_MS_40[n]})
        prob.plan.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 500 for this implementation, 20 for the reference arm)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="the headline workload only (no e2e, secondary workloads, serving or CPU baseline): "
                         "for profiler launch lists")
    ap.add_argument("--serving-requests", type=int, default=100000,
                    help="requests of the mixed-size serving stream (0 skips the serving measurements)")
    ap.add_argument("--serving-rate", type=float, default=2000.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.headline_only:
        args.serving_requests, args.no_cpu_baseline = 0, True
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 500
    world, rank, local = dist_setup()

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist
    from paper_1107_5578_gb300 import cwo, replicas, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    B = args.batch
    # the paper's "once-calculation": the transfer function is materialised when the plan is made
    # (outside the timed region, like the twiddles and axis tables) and loaded by the column pass
    plan = cwo.Plan(N, N, PITCH, PITCH, LAM, Z, cwo.ANGULAR, cwo.FLAG_CACHE_H)
    plan.reserve(B)
    # synthetic inputs: B random fields per rank (amplitude U[0,1), phase U[0, 2 pi))
    base = torch.from_numpy(synth.random_field(N, seed=replicas.rank_seed(1000, rank)).astype(np.complex64))
    g = torch.Generator(device="cpu").manual_seed(rank)
    host_in = torch.empty((B, N, N), dtype=torch.complex64).pin_memory()
    for i in range(B):
        host_in[i].copy_(base * torch.exp(1j * 2 * np.pi * torch.rand((), generator=g)).to(torch.complex64))
    x = host_in.to(dev)
    y = torch.empty_like(x)
    host_out = torch.empty((B, N, N), dtype=torch.complex64).pin_memory()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing
    for _ in range(args.warmup):
        plan.propagate_batch(x, out=y)
    barrier()
    wall = {}

    def start():
        barrier()
        wall["t0"] = time.perf_counter()

    with NvmlClockSampler(torch.cuda.current_device()) as clk:
        t_start, t_end, step_ev = timed_steps(plan, x, y, args.steps, stream, before=start)
        barrier()
        wall1 = time.perf_counter()
    wall0 = wall["t0"]
    per_pass = pass_sums(plan, step_ev)
    clocks = clk.summary()
    ms_total = replicas.max_over_ranks(t_start.elapsed_time(t_end), dev)
    ms_step = ms_total / args.steps
    value = replicas.job_rate(B * args.steps, world, ms_total / 1e3)

    # per-pass averages (ms per launch); each pass against the HBM roofline (algorithmic bytes)
    # and the FP32 arithmetic roofline (counted FP32 instructions against the measured rate)
    pp = per_pass / args.steps
    hbm_peak, sm_max, peak_kind = peaks()
    fp32_rate = fp32_peak(dev)
    names = ["row_fwd", "col_fwd_h_inv", "row_inv"]
    dom = int(np.argmax(pp))
    pass_bytes = [24 * N * N * B, 32 * N * N * B, 24 * N * N * B]
    passes = {}
    for k, nm in enumerate(names):
        gbs = pass_bytes[k] / (pp[k] / 1e3) / 1e9
        tis = FP32_PER_PASS[nm] * B / (pp[k] / 1e3) / 1e12
        passes[nm] = {"ms": round(pp[k], 4), "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
                      "fp32_tinst_s": round(tis, 2), "alu_frac": round(tis / (fp32_rate / 1e12), 4)}
    achieved = pass_bytes[dom] / (pp[dom] / 1e3) / 1e9
    path_gbs = BYTES_PER_PROP * B / (sum(pp) / 1e3) / 1e9
    hbm_roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": traffic_bytes(names[dom], B),
                "kernel": names[dom], "peak_kind": peak_kind}
    alu_roof = {"bound": "alu", "achieved": passes[names[dom]]["fp32_tinst_s"], "peak": round(fp32_rate / 1e12, 2),
                "unit": "FP32 Tinst/s", "frac": passes[names[dom]]["alu_frac"], "traffic": traffic_bytes(names[dom], B),
                "kernel": names[dom], "peak_kind": "measured (cwo_debug_ffma_rate: 16 FFMA chains per thread, best of 5)",
                "fp32_inst_per_launch": int(FP32_PER_PASS[names[dom]] * B)}
    roofline, roofline_other = (alu_roof, hbm_roof) if alu_roof["frac"] > hbm_roof["frac"] else (hbm_roof, alu_roof)

    # ---- end to end through the public API with host buffers: every step uploads its inputs
    # from pinned host memory and downloads its results; uploads, propagations and downloads of
    # neighbouring steps overlap on three streams (pipeline.HostPipeline)
    from paper_1107_5578_gb300 import pipeline
    pipe = pipeline.HostPipeline(plan, B, dev)
    host_outs = [host_out, torch.empty_like(host_out).pin_memory()]
    e_steps = max(3, args.steps // 2)
    pipe.run([host_in] * 2, host_outs)                   # warm-up
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in pipe.up:
        st.wait_stream(stream)                           # the timed region starts at e0
    for i in range(e_steps):
        pipe.enqueue(host_in, host_outs[i % 2], i)
    for st in pipe.down:
        stream.wait_stream(st)
    e1.record(stream)
    barrier()
    e_ms = replicas.max_over_ranks(e0.elapsed_time(e1), dev)
    e_value = replicas.job_rate(B * e_steps, world, e_ms / 1e3)
    # the copy engines alone (context for e2e): one upload and one download of a step's bytes
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    x.copy_(host_in, non_blocking=True)
    c1.record(stream)
    host_out.copy_(y, non_blocking=True)
    c2.record(stream)
    torch.cuda.synchronize()
    copy_gbs = {"h2d": round(host_in.numel() * 8 / (c0.elapsed_time(c1) / 1e3) / 1e9, 1),
                "d2h": round(host_out.numel() * 8 / (c1.elapsed_time(c2) / 1e3) / 1e9, 1)}

    extra = rank == 0 and not args.headline_only        # the secondary workloads and configs
    stack = stack_measurement(dev, peaks()[0]) if extra else None
    recalc_h = recalc_h_measurement(x, y, args.steps) if extra else None
    fresnel_b = fresnel_batch_measurement(x, y, args.steps, peaks()[0]) if extra else None
    asm_4096 = asm_4096_measurement(dev, min(args.steps, 20), peaks()[0]) if extra else None
    gs_res = gs_measurement(dev) if extra else None
    cfg_512 = config_asm_512(dev) if extra else None
    cfg_stack = config_fresnel_stack_errors(dev) if extra else None
    if cfg_stack is not None:
        stack.update(cfg_stack)
    cfg_prec = config_precision_4096(dev) if extra else None
    cfg_holo = config_hologram(dev) if extra else None
    serve = serving_measurement(dev, args.serving_requests, args.serving_rate) \
        if args.serving_requests > 0 and rank == 0 else None
    serve_high = serving_measurement(dev, min(args.serving_requests, 20000), 4 * args.serving_rate) \
        if args.serving_requests > 0 and rank == 0 else None
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline_sample()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "asm_2048_pad4096", "n": N, "padded": 2 * N, "batch_per_step": B,
                   "transfer_function": "materialised per plan (once-calculation), cache_bytes "
                                        f"{(N + 1) * 2 * N * 8}",
                   "pitch_m": PITCH, "wavelength_m": LAM, "z_m": Z,
                   "l2": "inputs larger than L2 (B x 32 MiB per step), no flush",
                   "parallelism": f"independent items per rank x{world}"},
        "hbm_gbs_path": round(path_gbs, 1),
        "roofline": roofline,
        "roofline_other": roofline_other,
        "passes": passes,
        "fp32_peak_tinst_s": round(fp32_rate / 1e12, 2),
        "roofline_path": {"achieved": round(path_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                          "frac": round(path_gbs / hbm_peak, 4), "bytes_per_prop": BYTES_PER_PROP},
        "passes_ms": {n: round(v, 4) for n, v in zip(names, pp)},
        "clocks": clocks,
        "e2e": {"value": round(e_value, 2), "unit": UNIT,
                "h2d_bytes_per_step": B * N * N * 8, "d2h_bytes_per_step": B * N * N * 8,
                "overlap": f"uploads, propagations and downloads of neighbouring steps overlapped; "
                           f"{len(pipe.chunks)} copy streams per direction",
                "copy_gbs": copy_gbs},
        "gpu_launches": plan.launches_per_call * args.steps,
        "fresnel_stack": stack,
        "asm_512": cfg_512,
        "precision_4096": cfg_prec,
        "hologram": cfg_holo,
        "asm_recalc_h": recalc_h,
        "fresnel_batch": fresnel_b,
        "asm_4096": asm_4096,
        "gs_kinoform": gs_res,
        "serving": serve,
        "serving_4x_rate": serve_high,
        "wall_s": round(wall1 - wall0, 3),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
