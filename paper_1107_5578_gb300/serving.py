"""Serving: continuous batching of mixed-size diffraction requests on one GPU.

Requests carry their own field size N, type (ASM / Fresnel), distance, wavelength and pitch.  The
scheduling runtime is native (include/cwo_serve.h): per size it keeps a few slots -- a plan
(tables and scratch resident), a CUDA stream (higher priority for small sizes), an event and
input/output buffers -- and a queue.  Whenever a slot of a size is free and the device-memory
budget admits the batch, the pending requests of that size (up to the slot's capacity) are
gathered into the slot's input buffer and propagated in one mixed batch (cwo_propagate_items: one
set of launches for the whole batch, each item with its own parameters).  Requests that arrive
while others are on the GPU are admitted as soon as a slot and memory free up, and batches of
different sizes run concurrently on different streams, so short requests do not queue behind
large ones.  Completion is observed by polling the slots' events; latency is arrival -> observed
completion on the host clock.  This module marshals requests and results; every scheduling
decision is taken by the runtime.

The baseline (``serve_serial``) propagates the same requests one at a time in arrival order,
also natively (cwo_server_run_serial).
"""
from __future__ import annotations

import ctypes
import dataclasses

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
    ticket: int = -1

    def done(self) -> bool:
        return self.t_done is not None

    def item(self) -> dict:
        return {"type": self.kind, "z": self.z, "wavelength": self.wavelength, "dx": self.pitch, "dy": self.pitch}


# cwo_request of include/cwo_serve.h
REQUEST_DTYPE = np.dtype([("n", "<i4"), ("type", "<i4"), ("z", "<f8"), ("wavelength", "<f8"), ("pitch", "<f8"),
                          ("field", "<u8"), ("out", "<u8"), ("t_arrival", "<f8")], align=True)
assert REQUEST_DTYPE.itemsize == 56


class _Stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("mem_in_use", ctypes.c_size_t),
                ("mem_peak", ctypes.c_size_t), ("mem_budget", ctypes.c_size_t)]


_SIGS = {
    "cwo_server_create": ([ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "cwo_server_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "cwo_server_batch_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "cwo_server_admit": ([ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int,
                          ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cwo_server_submit": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "cwo_server_after": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "cwo_server_step": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cwo_server_done": ([ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cwo_server_run": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "cwo_server_run_serial": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "cwo_server_warm_up": ([ctypes.c_void_p], ctypes.c_int),
    "cwo_server_get_stats": ([ctypes.c_void_p, ctypes.POINTER(_Stats)], ctypes.c_int),
}


def _lib():
    L = cwo.lib()
    if not getattr(L, "_cwo_serve_bound", False):
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        L._cwo_serve_bound = True
    return L


def validate(req: Request) -> None:
    """Host-side argument check of one request (the runtime checks again, with the device
    pointers); raises ValueError without touching the device."""
    if not (16 <= req.n <= 4096 and (req.n & (req.n - 1)) == 0):
        raise ValueError(f"request {req.rid}: unsupported size {req.n}")
    if req.kind not in (cwo.ANGULAR, cwo.FRESNEL_CONV):
        raise ValueError(f"request {req.rid}: unsupported type {req.kind}")
    if not (req.wavelength > 0 and req.pitch > 0 and np.isfinite(req.z)):
        raise ValueError(f"request {req.rid}: wavelength and pitch must be > 0, z finite")
    if req.kind == cwo.FRESNEL_CONV and req.z == 0.0:
        raise ValueError(f"request {req.rid}: Fresnel needs z != 0")


def batch_bytes(n: int, b: int) -> int:
    """Device bytes a batch of b fields of n x n occupies while in flight (scratch + in + out)."""
    out = ctypes.c_size_t(0)
    cwo.check(_lib().cwo_server_batch_bytes(int(n), int(b), ctypes.byref(out)), "cwo_server_batch_bytes")
    return int(out.value)


def admit(queued: int, capacity: int, in_use: int, budget: int, n: int) -> int:
    """How many of `queued` requests of size n one free slot takes now (the runtime's rule: up to
    its capacity, halved until the batch fits the memory budget next to what is in flight)."""
    out = ctypes.c_int(0)
    cwo.check(_lib().cwo_server_admit(int(queued), int(capacity), int(in_use), int(budget), int(n), ctypes.byref(out)),
              "cwo_server_admit")
    return int(out.value)


class Server:
    def __init__(self, sizes=(256, 512, 1024, 2048, 4096), max_batch=None, slots_per_size=2,
                 mem_budget: int | None = None, device="cuda", pools=None, keep_results=False):
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.max_batch = dict(DEFAULT_MAX_BATCH if max_batch is None else max_batch)
        self.sizes = sorted(sizes)
        self.pools = pools or {}
        self.keep_results = keep_results
        self._handle = ctypes.c_void_p()
        sz = (ctypes.c_int * len(self.sizes))(*self.sizes)
        mb = (ctypes.c_int * len(self.sizes))(*[self.max_batch[n] for n in self.sizes])
        with torch.cuda.device(self.device):
            cwo.check(_lib().cwo_server_create(len(self.sizes), sz, mb, int(slots_per_size), int(mem_budget or 0),
                                               ctypes.byref(self._handle)), "cwo_server_create")
        self._pending: dict[int, Request] = {}
        self._next_rid = 1 << 40

    def close(self) -> None:
        if self._handle:
            _lib().cwo_server_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stats(self) -> _Stats:
        st = _Stats()
        cwo.check(_lib().cwo_server_get_stats(self._handle, ctypes.byref(st)), "cwo_server_get_stats")
        return st

    @property
    def batches(self) -> int:
        return int(self._stats().batches)

    @property
    def mem_peak(self) -> int:
        return int(self._stats().mem_peak)

    @property
    def mem_budget(self) -> int:
        return int(self._stats().mem_budget)

    @property
    def mem_in_use(self) -> int:
        return int(self._stats().mem_in_use)

    def _fill(self, rec, r: Request) -> None:
        validate(r)
        if r.field is not None:
            src = r.field
        else:
            pool = self.pools[r.n]
            src = pool[r.pool_index % pool.shape[0]]
        if self.keep_results:
            r.result = torch.empty((r.n, r.n), dtype=torch.complex64, device=self.device)
        rec["n"], rec["type"], rec["z"] = r.n, r.kind, r.z
        rec["wavelength"], rec["pitch"] = r.wavelength, r.pitch
        rec["field"] = src.data_ptr()
        rec["out"] = r.result.data_ptr() if r.result is not None else 0
        rec["t_arrival"] = r.t_arrival

    def submit(self, req: Request) -> Request:
        """Queue a request; the returned object is its future (done(), result after completion)."""
        if req.n not in self.sizes:
            raise ValueError(f"request {req.rid}: size {req.n} is not served")
        rec = np.zeros(1, dtype=REQUEST_DTYPE)
        self._fill(rec[0], req)
        if req.field is not None:                   # caller-made field: order after its producer
            cwo.check(_lib().cwo_server_after(self._handle, torch.cuda.current_stream(self.device).cuda_stream),
                      "cwo_server_after")
        t = ctypes.c_longlong(-1)
        st = _lib().cwo_server_submit(self._handle, rec.ctypes.data, ctypes.byref(t))
        if st == cwo.ERR_INVALID_ARG:
            raise ValueError(f"request {req.rid}: {cwo.last_error()}")
        cwo.check(st, "cwo_server_submit")
        req.ticket = int(t.value)
        self._pending[req.ticket] = req
        return req

    def submit_field(self, field: torch.Tensor, z: float, wavelength: float = cwo.DEFAULT_WAVELENGTH,
                     pitch: float = cwo.DEFAULT_PITCH, kind: int = cwo.ANGULAR) -> Request:
        """Queue one explicit [n, n] complex64 CUDA field; returns its future."""
        if field.dim() != 2 or field.shape[0] != field.shape[1] or field.dtype != torch.complex64 \
                or field.device != self.device:
            raise ValueError("field must be a square complex64 tensor on the server's device")
        self._next_rid += 1
        req = Request(self._next_rid, int(field.shape[0]), kind, z, wavelength, pitch, field=field.contiguous())
        return self.submit(req)

    def step(self) -> int:
        """Admit what fits and collect what finished; returns the number of completions."""
        c = ctypes.c_int(0)
        cwo.check(_lib().cwo_server_step(self._handle, ctypes.byref(c)), "cwo_server_step")
        if c.value:
            t = ctypes.c_double(0.0)
            for k in [k for k in self._pending if _lib().cwo_server_done(self._handle, k, ctypes.byref(t)) == 1]:
                self._pending.pop(k).t_done = t.value
        return int(c.value)

    def wait(self, req: Request) -> torch.Tensor | None:
        """Drive the server until `req` completes; returns its result when results are kept."""
        while not req.done():
            self.step()
        return req.result

    def pending(self) -> int:
        return len(self._pending)

    def warm_up(self) -> None:
        """Touch every path a run takes (single and gathered batches of every size and type) so
        that no first-use cost lands inside a measured run."""
        cwo.check(_lib().cwo_server_warm_up(self._handle), "cwo_server_warm_up")

    def run(self, requests: list[Request]) -> float:
        """Open-loop run: requests are released at their arrival times (seconds from start) and
        scheduled by the runtime; sets each request's t_done; returns the makespan."""
        recs = np.zeros(len(requests), dtype=REQUEST_DTYPE)
        for rec, r in zip(recs, requests):
            self._fill(rec, r)
        t_done = np.zeros(len(requests), dtype=np.float64)
        st = _lib().cwo_server_run(self._handle, recs.ctypes.data, len(requests), t_done.ctypes.data)
        if st == cwo.ERR_INVALID_ARG:
            raise ValueError(cwo.last_error())
        cwo.check(st, "cwo_server_run")
        for r, t in zip(requests, t_done):
            r.t_done = float(t)
        return float(t_done.max()) if len(requests) else 0.0


def serve_serial(requests: list[Request], pools, device="cuda", keep_results=False, plans=None) -> float:
    """Baseline: one request at a time in arrival order, each propagated alone and waited for
    (native, cwo_server_run_serial).  ``plans``: a dict in which the baseline keeps its server
    between calls (so that a warm-up call leaves it ready)."""
    sizes = sorted({r.n for r in requests} | set(pools.keys()))
    cache = {} if plans is None else plans
    key = ("serial", tuple(sizes), bool(keep_results))
    srv = cache.get(key)
    if srv is None:
        srv = Server(sizes=sizes, max_batch={n: 1 for n in sizes}, slots_per_size=1, device=device, pools=pools,
                     keep_results=keep_results)
        srv.warm_up()
        cache[key] = srv
    srv.pools = pools
    recs = np.zeros(len(requests), dtype=REQUEST_DTYPE)
    for rec, r in zip(recs, requests):
        srv._fill(rec, r)
    t_done = np.zeros(len(requests), dtype=np.float64)
    cwo.check(_lib().cwo_server_run_serial(srv._handle, recs.ctypes.data, len(requests), t_done.ctypes.data),
              "cwo_server_run_serial")
    for r, t in zip(requests, t_done):
        r.t_done = float(t)
    return float(t_done.max()) if len(requests) else 0.0


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
