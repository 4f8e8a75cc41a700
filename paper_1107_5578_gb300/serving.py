"""Serving: continuous batching of mixed-size diffraction requests on one GPU.

Requests carry their own field size N, type (ASM / Fresnel), distance, wavelength and pitch.
The server keeps, per size, a few slots -- a plan (tables and scratch resident), a CUDA stream and
input/output buffers -- and a queue.  Whenever a slot of a size is free and the device-memory
budget admits the batch, the pending requests of that size (up to the slot's capacity) are
gathered into the slot's input buffer and propagated in one mixed batch (cwo_propagate_items:
one set of three launches for the whole batch, each item with its own parameters).  Requests that
arrive while others are on the GPU are admitted as soon as a slot and memory free up, and batches
of different sizes run concurrently on different streams (small sizes on higher-priority
streams), so short requests do not queue behind large ones.  Completion is observed by polling
the slot's event; latency is arrival -> observed completion on the host clock.

The baseline (``serve_serial``) propagates the same requests one at a time in arrival order.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import cwo, synth

DEFAULT_MAX_BATCH = {256: 64, 512: 32, 1024: 16, 2048: 8, 4096: 2}


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    kind: int
    z: float
    wavelength: float
    pitch: float
    t_arrival: float = 0.0            # seconds from the start of the run
    pool_index: int = 0               # which resident field of the pool to propagate
    field: torch.Tensor | None = None  # or an explicit [n, n] complex64 CUDA field
    t_done: float | None = None
    result: torch.Tensor | None = None

    def done(self) -> bool:
        return self.t_done is not None

    def item(self) -> dict:
        return {"type": self.kind, "z": self.z, "wavelength": self.wavelength, "dx": self.pitch, "dy": self.pitch}


def validate(req: Request) -> None:
    """Host-side admission check; raises ValueError without touching the device."""
    if req.n not in DEFAULT_MAX_BATCH and not (16 <= req.n <= 4096 and (req.n & (req.n - 1)) == 0):
        raise ValueError(f"request {req.rid}: unsupported size {req.n}")
    if req.kind not in (cwo.ANGULAR, cwo.FRESNEL_CONV):
        raise ValueError(f"request {req.rid}: unsupported type {req.kind}")
    if not (req.wavelength > 0 and req.pitch > 0 and np.isfinite(req.z)):
        raise ValueError(f"request {req.rid}: wavelength and pitch must be > 0, z finite")
    if req.kind == cwo.FRESNEL_CONV and req.z == 0.0:
        raise ValueError(f"request {req.rid}: Fresnel needs z != 0")


def batch_bytes(n: int, b: int) -> int:
    """Device bytes a batch of b fields of n x n occupies while in flight (scratch + in + out)."""
    return cwo.device_bytes(n, n, b) + 2 * b * n * n * 8


def admit(queued: int, capacity: int, in_use: int, budget: int, bytes_of) -> int:
    """How many of `queued` requests one free slot takes now: up to its capacity, halved until
    the batch fits the memory budget next to what is in flight (0: wait for completions)."""
    b = min(queued, capacity)
    while b > 0 and in_use + bytes_of(b) > budget:
        b //= 2
    return b


class _Slot:
    def __init__(self, n, capacity, device, priority):
        self.n, self.capacity = n, capacity
        self.plan = cwo.Plan(n, n, cwo.DEFAULT_PITCH, None, cwo.DEFAULT_WAVELENGTH, 0.1, cwo.ANGULAR)
        self.plan.reserve(capacity)
        self.stream = torch.cuda.Stream(device=device, priority=priority)
        self.inbuf = torch.empty((capacity, n, n), dtype=torch.complex64, device=device)
        self.outbuf = torch.empty_like(self.inbuf)
        self.event = torch.cuda.Event()
        self.idx_host = torch.empty(capacity, dtype=torch.int64).pin_memory()
        self.idx_dev = torch.empty(capacity, dtype=torch.int64, device=device)
        self.reqs: list[Request] = []
        self.bytes = 0

    @property
    def busy(self):
        return bool(self.reqs)


class Server:
    def __init__(self, sizes=(256, 512, 1024, 2048, 4096), max_batch=None, slots_per_size=2,
                 mem_budget: int | None = None, device="cuda", pools=None, keep_results=False):
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.max_batch = dict(DEFAULT_MAX_BATCH if max_batch is None else max_batch)
        self.sizes = sorted(sizes)
        self.slots = {}
        for n in self.sizes:
            prio = -1 if n <= 512 else 0            # short requests on high-priority streams
            self.slots[n] = [_Slot(n, self.max_batch[n], self.device, prio) for _ in range(slots_per_size)]
        self.queues = {n: collections.deque() for n in self.sizes}
        self.mem_budget = mem_budget if mem_budget is not None else sum(
            batch_bytes(n, self.max_batch[n]) * slots_per_size for n in self.sizes)
        self.mem_in_use = 0
        self.mem_peak = 0
        self.pools = pools or {}
        self.keep_results = keep_results
        self.batches = 0
        self._next_rid = 1 << 40

    def submit(self, req: Request) -> Request:
        """Queue a request; the returned object is its future (done(), result after completion)."""
        validate(req)
        if req.n not in self.queues:
            raise ValueError(f"request {req.rid}: size {req.n} is not served")
        if batch_bytes(req.n, 1) > self.mem_budget:
            raise ValueError(f"request {req.rid}: one {req.n}^2 field needs more than the memory budget")
        self.queues[req.n].append(req)
        return req

    def submit_field(self, field: torch.Tensor, z: float, wavelength: float = cwo.DEFAULT_WAVELENGTH,
                     pitch: float = cwo.DEFAULT_PITCH, kind: int = cwo.ANGULAR) -> Request:
        """Queue one explicit [n, n] complex64 CUDA field; returns its future."""
        if field.dim() != 2 or field.shape[0] != field.shape[1] or field.dtype != torch.complex64 \
                or field.device != self.device:
            raise ValueError("field must be a square complex64 tensor on the server's device")
        self._next_rid += 1
        req = Request(self._next_rid, int(field.shape[0]), kind, z, wavelength, pitch, field=field)
        return self.submit(req)

    def step(self, now: float | None = None) -> int:
        """Admit what fits and collect what finished; returns the number of completions."""
        self.dispatch()
        return self.poll(time.perf_counter() if now is None else now)

    def wait(self, req: Request) -> torch.Tensor | None:
        """Drive the server until `req` completes; returns its result when results are kept."""
        while not req.done():
            self.step()
        return req.result

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values()) + sum(len(s.reqs) for v in self.slots.values() for s in v)

    def poll(self, now: float) -> int:
        done = 0
        for n in self.sizes:
            for s in self.slots[n]:
                if s.reqs and s.event.query():
                    for i, r in enumerate(s.reqs):
                        r.t_done = now
                        if self.keep_results:
                            r.result = s.outbuf[i].clone()
                    done += len(s.reqs)
                    s.reqs = []
                    self.mem_in_use -= s.bytes
                    s.bytes = 0
        return done

    def dispatch(self) -> None:
        for n in self.sizes:                        # smallest first
            q = self.queues[n]
            for s in self.slots[n]:
                if not q:
                    break
                if s.busy:
                    continue
                b = admit(len(q), s.capacity, self.mem_in_use, self.mem_budget, lambda k: batch_bytes(n, k))
                if b == 0:
                    break                           # retried after completions free memory
                need = batch_bytes(n, b)
                reqs = [q.popleft() for _ in range(b)]
                self._launch(s, reqs)
                self.mem_in_use += need
                self.mem_peak = max(self.mem_peak, self.mem_in_use)
                s.bytes = need

    def _launch(self, s: _Slot, reqs: list[Request]) -> None:
        b = len(reqs)
        if any(r.field is not None for r in reqs):  # caller-made fields: order after their producer
            s.stream.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s.stream):
            if b == 1:                              # no gather: propagate straight from the source
                r = reqs[0]
                if r.field is not None:
                    x = r.field.unsqueeze(0)
                else:
                    pool = self.pools[s.n]
                    k = r.pool_index % pool.shape[0]
                    x = pool[k:k + 1]
            elif all(r.field is None for r in reqs):
                pool = self.pools[s.n]
                s.idx_host[:b].copy_(torch.tensor([r.pool_index % pool.shape[0] for r in reqs]))
                s.idx_dev[:b].copy_(s.idx_host[:b], non_blocking=True)
                torch.index_select(pool, 0, s.idx_dev[:b], out=s.inbuf[:b])
                x = s.inbuf[:b]
            else:
                for i, r in enumerate(reqs):
                    s.inbuf[i].copy_(r.field if r.field is not None else self.pools[s.n][r.pool_index])
                x = s.inbuf[:b]
            s.plan.propagate_items(x, [r.item() for r in reqs], out=s.outbuf[:b], stream=s.stream)
            s.event.record(s.stream)
        s.reqs = reqs
        self.batches += 1

    def warm_up(self) -> None:
        """Touch every code path a run takes (single and gathered batches of every size) so that
        no first-use cost (module loading, allocator growth) lands inside a measured run."""
        for n in self.sizes:
            pool = self.pools.get(n)
            if pool is None:
                continue
            for s in self.slots[n]:
                for b in (1, min(2, s.capacity)):
                    for kind in (cwo.ANGULAR, cwo.FRESNEL_CONV):
                        reqs = [Request(-1, n, kind, 0.1, 532e-9, 8e-6, pool_index=k) for k in range(b)]
                        self._launch(s, reqs)
                        s.event.synchronize()
                        s.reqs = []
        self.batches = 0

    def run(self, requests: list[Request]) -> float:
        """Open-loop run: requests are released at their arrival times (seconds from start).
        Python's cyclic garbage collector is paused for the run (a collection over a large heap
        would stall the loop for its duration)."""
        import gc
        requests = sorted(requests, key=lambda r: r.t_arrival)
        gc.collect()
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            i, total, done = 0, len(requests), 0
            while done < total:
                now = time.perf_counter() - t0
                while i < total and requests[i].t_arrival <= now:
                    self.submit(requests[i])
                    i += 1
                self.dispatch()
                done += self.poll(time.perf_counter() - t0)
            return time.perf_counter() - t0
        finally:
            if was_enabled:
                gc.enable()


def serve_serial(requests: list[Request], pools, device="cuda", keep_results=False, plans=None) -> float:
    """Baseline: one request at a time in arrival order, each propagated alone and waited for
    (garbage collector paused as in Server.run)."""
    import gc
    gc.collect()
    was_enabled = gc.isenabled()
    gc.disable()
    try:
        return _serve_serial(requests, pools, device, keep_results, plans)
    finally:
        if was_enabled:
            gc.enable()


def _serve_serial(requests, pools, device, keep_results, plans) -> float:
    requests = sorted(requests, key=lambda r: r.t_arrival)
    dev = torch.device(device)
    plans = {} if plans is None else plans
    outs = {}
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in requests:
        if r.n not in plans:
            plans[r.n] = cwo.Plan(r.n, r.n, cwo.DEFAULT_PITCH, None, cwo.DEFAULT_WAVELENGTH, 0.1, cwo.ANGULAR)
            outs[r.n] = torch.empty((1, r.n, r.n), dtype=torch.complex64, device=dev)
        if r.n not in outs:
            outs[r.n] = torch.empty((1, r.n, r.n), dtype=torch.complex64, device=dev)
        while time.perf_counter() - t0 < r.t_arrival:
            pass
        x = (r.field if r.field is not None else pools[r.n][r.pool_index % pools[r.n].shape[0]]).unsqueeze(0)
        plans[r.n].propagate_items(x, [r.item()], out=outs[r.n], stream=stream)
        stream.synchronize()
        r.t_done = time.perf_counter() - t0
        if keep_results:
            r.result = outs[r.n][0].clone()
    return time.perf_counter() - t0


def make_pools(sizes, per_size=4, device="cuda", seed=100):
    return {n: torch.from_numpy(np.stack([synth.random_field(n, seed=seed + 7 * n + k).astype(np.complex64)
                                          for k in range(per_size)])).to(device)
            for n in sizes}


def make_requests(n_req, seed, rate_hz=2000.0, sizes=synth.SERVING_SIZES, weights=synth.SERVING_WEIGHTS):
    d = synth.serving_requests(n_req, seed, rate_hz, sizes, weights)
    return [Request(rid=k, n=int(d["n"][k]), kind=int(d["kind"][k]), z=float(d["z"][k]),
                    wavelength=float(d["lam"][k]), pitch=float(d["pitch"][k]), t_arrival=float(d["t"][k]),
                    pool_index=int(d["pool"][k])) for k in range(n_req)]


def latency_stats(requests) -> dict:
    lat = np.array([r.t_done - r.t_arrival for r in requests]) * 1e3
    span = max(r.t_done for r in requests) - min(r.t_arrival for r in requests)
    sizes = np.array([r.n for r in requests])
    by_size = {int(n): {"p50_ms": round(float(np.percentile(lat[sizes == n], 50)), 4),
                        "p99_ms": round(float(np.percentile(lat[sizes == n], 99)), 4)}
               for n in sorted(set(sizes.tolist()))}
    arr = np.array([r.t_arrival for r in requests])
    slow = np.where(lat > 10.0)[0]
    return {"requests": len(requests), "p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4), "mean_ms": round(float(lat.mean()), 4),
            "max_ms": round(float(lat.max()), 4), "throughput_rps": round(len(requests) / span, 1),
            "over_10ms": int(len(slow)),
            "over_10ms_arrivals_s": [round(float(arr[slow[0]]), 3), round(float(arr[slow[-1]]), 3)] if len(slow) else None,
            "by_size": by_size}
