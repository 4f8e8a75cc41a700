"""Thin Python binding of libcwo_gb300.so (the C ABI of include/cwo.h).

Argument marshalling only: every step of a propagation runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  If the shared library has not been built the
import of this module's functions fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcwo_gb300.so")

# cwo_type
ANGULAR = 0
FRESNEL_CONV = 1
FRESNEL_FOURIER = 2
SHIFTED_FRESNEL = 3
SHIFTED_ANGULAR = 4
# flags
FLAG_PHASE_FP32 = 0x1
FLAG_PHASE_FP64 = 0x2
EPI_NONE, EPI_PHASE, EPI_AMPLITUDE, EPI_INTENSITY = 0, 1, 2, 3
FLAG_CACHE_H = 0x8
FLAG_LITERAL_SCALE = 0x4
# status
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = range(6)
STATUS_NAMES = {0: "CWO_OK", 1: "CWO_ERR_INVALID_ARG", 2: "CWO_ERR_UNSUPPORTED", 3: "CWO_ERR_OOM",
                4: "CWO_ERR_CUDA", 5: "CWO_ERR_TIMEOUT"}
DEFAULT_WAVELENGTH = 633e-9
DEFAULT_PITCH = 10e-6

_lock = threading.Lock()
_lib = None


class Shift(ctypes.Structure):
    """cwo_shift: shift (m) and Rect band-limit windows (centre, full width in 1/m; width <= 0:
    none) of the shifted angular spectrum method."""
    _fields_ = [("ox", ctypes.c_double), ("oy", ctypes.c_double), ("cx", ctypes.c_double),
                ("wx", ctypes.c_double), ("cy", ctypes.c_double), ("wy", ctypes.c_double)]


class ShiftedFresnel(ctypes.Structure):
    """cwo_shifted_fresnel: destination pitches and the centres of both grids (metres)."""
    _fields_ = [("dx1", ctypes.c_double), ("dy1", ctypes.c_double), ("ox0", ctypes.c_double),
                ("oy0", ctypes.c_double), ("ox1", ctypes.c_double), ("oy1", ctypes.c_double)]


def band_limit(nx: int, ny: int, dx: float, dy: float, wavelength: float, z: float) -> Shift:
    """The on-axis band-limited ASM windows (no shift) for this geometry."""
    out = Shift()
    check(lib().cwo_band_limit(int(nx), int(ny), float(dx), float(dy), float(wavelength), float(z), ctypes.byref(out)),
          "cwo_band_limit")
    return out


class Item(ctypes.Structure):
    """cwo_item: one entry of a mixed batch (cwo_propagate_items)."""
    _fields_ = [("z", ctypes.c_double), ("wavelength", ctypes.c_double), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("type", ctypes.c_int), ("flags", ctypes.c_uint)]


class CwoError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def lib() -> ctypes.CDLL:
    """Load the shared library (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it first "
                                  "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            vp, i, u, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_longlong
            pp = ctypes.POINTER(ctypes.c_void_p)
            sz = ctypes.POINTER(ctypes.c_size_t)
            dpp = ctypes.POINTER(ctypes.c_double)
            sig = {
                "cwo_plan_create": ([i, i, d, d, d, d, i, u, pp], i),
                "cwo_plan_destroy": ([vp], i),
                "cwo_plan_create_shifted": ([i, i, d, d, d, d, ctypes.POINTER(Shift), u, pp], i),
                "cwo_band_limit": ([i, i, d, d, d, d, ctypes.POINTER(Shift)], i),
                "cwo_plan_create_shifted_fresnel": ([i, i, d, d, d, d, ctypes.POINTER(ShiftedFresnel), u, pp], i),
                "cwo_plan_device_bytes": ([i, i, i, sz], i),
                "cwo_plan_reserve": ([vp, i], i),
                "cwo_propagate": ([vp, vp, vp, vp], i),
                "cwo_propagate_batch": ([vp, vp, ll, vp, i, dpp, vp], i),
                "cwo_propagate_adjoint": ([vp, vp, vp, vp], i),
                "cwo_propagate_adjoint_batch": ([vp, vp, ll, vp, i, dpp, vp], i),
                "cwo_propagate_items": ([vp, vp, ll, vp, i, ctypes.POINTER(Item), vp], i),
                "cwo_launches_per_call": ([vp], i),
                "cwo_propagate_epilogue": ([vp, vp, vp, i, i, i, vp, vp, vp], i),
                "cwo_gs_run": ([vp, vp, vp, vp, i, i, vp], i),
                "cwo_plan_check": ([vp], i),
                "cwo_plan_set_timing_events": ([vp, ctypes.POINTER(ctypes.c_void_p)], i),
                "cwo_last_error": ([], ctypes.c_char_p),
                "cwo_version": ([], i),
                "cwo_debug_axis_bins": ([i, vp], i),
                "cwo_debug_split_axis": ([i, vp, vp], i),
                "cwo_debug_fresnel_axis": ([i, d, d, d, vp], i),
                "cwo_debug_twiddles": ([i, vp], i),
                "cwo_debug_asm_axis": ([i, d, d, d, i, vp], i),
                "cwo_debug_emulate": ([i, i, d, d, d, d, i, u, i, vp, vp], i),
                "cwo_debug_line_fft": ([i, i, vp, vp], i),
                "cwo_debug_asm_h": ([i, i, d, d, d, d, ctypes.POINTER(ctypes.c_int), vp], i),
                "cwo_debug_emulate_shifted_fresnel": ([i, i, d, d, d, d, ctypes.POINTER(ShiftedFresnel), i, vp, vp], i),
                "cwo_debug_emulate_shifted": ([i, i, d, d, d, d, ctypes.POINTER(Shift), i, vp, vp], i),
                "cwo_debug_bounded_wait": ([u, i, ctypes.POINTER(ctypes.c_int)], i),
                "cwo_debug_ffma_rate": ([i, i, vp, vp], i),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def last_error() -> str:
    return lib().cwo_last_error().decode("utf-8", "replace")


def check(status: int, where: str) -> None:
    if status != OK:
        raise CwoError(status, where, last_error())


def device_bytes(nx: int, ny: int, batch: int = 1) -> int:
    out = ctypes.c_size_t(0)
    check(lib().cwo_plan_device_bytes(nx, ny, batch, ctypes.byref(out)), "cwo_plan_device_bytes")
    return int(out.value)


def _stream_handle(stream) -> ctypes.c_void_p:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(int(s.cuda_stream))


def _check_field(t, nx: int, ny: int, name: str, batch: int | None = None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.complex64:
        raise TypeError(f"{name} must be complex64 (got {t.dtype})")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape[-2:]) != (ny, nx):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected [..., {ny}, {nx}]")
    if batch is not None and t.numel() != batch * nx * ny:
        raise ValueError(f"{name} holds {t.numel() // (nx * ny)} fields, expected {batch}")


def _check_real(t, nx: int, ny: int, name: str, batch: int):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32 (got {t.dtype})")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if tuple(t.shape[-2:]) != (ny, nx) or t.numel() != batch * nx * ny:
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {batch} x [{ny}, {nx}]")


class Plan:
    """A propagation plan (tables resident on the device, scratch owned by the plan)."""

    def __init__(self, nx: int, ny: int | None = None, dx: float = DEFAULT_PITCH,
                 dy: float | None = None, wavelength: float = DEFAULT_WAVELENGTH, z: float = 0.1,
                 kind: int = ANGULAR, flags: int = 0, shift: "Shift | None" = None,
                 shifted_fresnel: "ShiftedFresnel | None" = None):
        """``shift`` (a Shift) makes a shifted angular-spectrum plan (kind SHIFTED_ANGULAR);
        ``shifted_fresnel`` (a ShiftedFresnel) a shifted Fresnel plan (kind SHIFTED_FRESNEL)."""
        self.nx, self.ny = int(nx), int(nx if ny is None else ny)
        self.dx, self.dy = float(dx), float(dx if dy is None else dy)
        self.wavelength, self.z, self.kind, self.flags = float(wavelength), float(z), int(kind), int(flags)
        h = ctypes.c_void_p(0)
        self._sfr = shifted_fresnel
        if shifted_fresnel is not None:
            self.kind = SHIFTED_FRESNEL
            check(lib().cwo_plan_create_shifted_fresnel(self.nx, self.ny, self.dx, self.dy, self.wavelength, self.z,
                                                        ctypes.byref(shifted_fresnel), self.flags, ctypes.byref(h)),
                  "cwo_plan_create_shifted_fresnel")
        elif shift is not None:
            self.kind = SHIFTED_ANGULAR
            check(lib().cwo_plan_create_shifted(self.nx, self.ny, self.dx, self.dy, self.wavelength, self.z,
                                                ctypes.byref(shift), self.flags, ctypes.byref(h)),
                  "cwo_plan_create_shifted")
        else:
            check(lib().cwo_plan_create(self.nx, self.ny, self.dx, self.dy, self.wavelength, self.z,
                                        self.kind, self.flags, ctypes.byref(h)), "cwo_plan_create")
        self._h = h

    @property
    def output_pitch(self) -> tuple:
        """(dx2, dy2) of the destination plane: the source pitches, except for the Fourier form
        (lambda z / (Nx dx), lambda z / (Ny dy))."""
        if self.kind == FRESNEL_FOURIER:
            return (self.wavelength * self.z / (self.nx * self.dx), self.wavelength * self.z / (self.ny * self.dy))
        if self.kind == SHIFTED_FRESNEL:
            return (self._sfr.dx1, self._sfr.dy1)
        return (self.dx, self.dy)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None or not self._h.value:
            raise RuntimeError("plan has been destroyed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().cwo_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self) -> None:
        """Synchronise and raise CwoError(CWO_ERR_TIMEOUT) if a bounded wait of an earlier call
        on this plan expired."""
        check(lib().cwo_plan_check(self.handle), "cwo_plan_check")

    def reserve(self, batch: int) -> None:
        check(lib().cwo_plan_reserve(self.handle, int(batch)), "cwo_plan_reserve")

    def set_timing_events(self, events) -> None:
        """Record 4 torch.cuda.Event (enable_timing=True) around the passes of every later call
        (None switches it off): events[0] before the row forward pass, [1] after it, [2] after
        the column pass, [3] after the row inverse pass."""
        if events is None:
            check(lib().cwo_plan_set_timing_events(self.handle, None), "cwo_plan_set_timing_events")
            self._events = None
            return
        if len(events) != 4:
            raise ValueError("need 4 events")
        import torch
        for ev in events:
            if not ev.cuda_event:   # torch creates the cudaEvent_t on first record
                ev.record(torch.cuda.current_stream())
        arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(ev.cuda_event) for ev in events])
        check(lib().cwo_plan_set_timing_events(self.handle, arr), "cwo_plan_set_timing_events")
        self._events = list(events)

    @property
    def launches_per_call(self) -> int:
        return int(lib().cwo_launches_per_call(self.handle))

    def _out(self, x, batch_shape):
        import torch
        return torch.empty((*batch_shape, self.ny, self.nx), dtype=torch.complex64, device=x.device)

    def propagate(self, x, out=None, stream=None):
        """One field [Ny][Nx] (complex64, CUDA) -> propagated field."""
        _check_field(x, self.nx, self.ny, "input", 1)
        out = self._out(x, x.shape[:-2]) if out is None else out
        _check_field(out, self.nx, self.ny, "output", 1)
        check(lib().cwo_propagate(self.handle, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "cwo_propagate")
        return out

    def adjoint(self, x, out=None, stream=None):
        _check_field(x, self.nx, self.ny, "input", 1)
        out = self._out(x, x.shape[:-2]) if out is None else out
        _check_field(out, self.nx, self.ny, "output", 1)
        check(lib().cwo_propagate_adjoint(self.handle, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "cwo_propagate_adjoint")
        return out

    def propagate_batch(self, x, z=None, out=None, stream=None, adjoint=False):
        """Batch [B][Ny][Nx] -> [B][Ny][Nx].  ``z``: None (plan z) or B distances (host floats)."""
        b = x.shape[0] if x.dim() == 3 else 1
        _check_field(x, self.nx, self.ny, "input", b)
        return self._batch(x, self.nx * self.ny, b, z, out, stream, adjoint)

    def propagate_items(self, x, items, out=None, stream=None):
        """Mixed batch [B][Ny][Nx]: item i propagated with items[i] = (type, z, wavelength, dx, dy)
        given as dicts or Item structures; the plan supplies only the shape and resources."""
        b = x.shape[0] if x.dim() == 3 else 1
        _check_field(x, self.nx, self.ny, "input", b)
        if len(items) != b:
            raise ValueError(f"{len(items)} items for {b} fields")
        arr = (Item * b)()
        for k, it in enumerate(items):
            if isinstance(it, Item):
                arr[k] = it
            else:
                arr[k] = Item(float(it["z"]), float(it["wavelength"]), float(it["dx"]),
                              float(it.get("dy", it["dx"])), int(it["type"]), int(it.get("flags", 0)))
        out = self._out(x, (b,)) if out is None else out
        _check_field(out, self.nx, self.ny, "output", b)
        check(lib().cwo_propagate_items(self.handle, ctypes.c_void_p(x.data_ptr()), self.nx * self.ny,
                                        ctypes.c_void_p(out.data_ptr()), b, arr, _stream_handle(stream)),
              "cwo_propagate_items")
        return out

    def propagate_epilogue(self, x, epilogue, amplitude=None, out=None, adjoint=False, stream=None):
        """Batch [B][Ny][Nx] (or one field) propagated (adjoint: by conj(H)) with an output
        epilogue: EPI_PHASE (unit amplitude), EPI_AMPLITUDE (amplitude * phase; ``amplitude`` a
        float32 tensor shaped like x) or EPI_INTENSITY (returns |u|^2 as float32)."""
        import torch
        b = x.shape[0] if x.dim() == 3 else 1
        _check_field(x, self.nx, self.ny, "input", b)
        inten = None
        if epilogue == EPI_INTENSITY:
            inten = torch.empty(x.shape, dtype=torch.float32, device=x.device) if out is None else out
            _check_real(inten, self.nx, self.ny, "intensity", b)
            optr = None
        else:
            out = self._out(x, x.shape[:-2]) if out is None else out
            _check_field(out, self.nx, self.ny, "output", b)
            optr = out.data_ptr()
        aptr = None
        if epilogue == EPI_AMPLITUDE:
            _check_real(amplitude, self.nx, self.ny, "amplitude", b)
            aptr = amplitude.data_ptr()
        check(lib().cwo_propagate_epilogue(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(optr), b,
                                           int(bool(adjoint)), int(epilogue), ctypes.c_void_p(aptr),
                                           ctypes.c_void_p(inten.data_ptr() if inten is not None else None),
                                           _stream_handle(stream)), "cwo_propagate_epilogue")
        return inten if epilogue == EPI_INTENSITY else out

    def gs_run(self, amplitude, field, iterations, intensity=True, stream=None):
        """Gerchberg-Saxton kinoform iteration in place on ``field`` ([B][Ny][Nx] or one field;
        in: amplitude * initial phase, out: the kinoform).  Returns the reconstructed intensity
        (float32, like ``amplitude``) or None."""
        import torch
        b = field.shape[0] if field.dim() == 3 else 1
        _check_field(field, self.nx, self.ny, "field", b)
        _check_real(amplitude, self.nx, self.ny, "amplitude", b)
        inten = torch.empty(amplitude.shape, dtype=torch.float32, device=field.device) if intensity else None
        check(lib().cwo_gs_run(self.handle, ctypes.c_void_p(amplitude.data_ptr()), ctypes.c_void_p(field.data_ptr()),
                               ctypes.c_void_p(inten.data_ptr() if inten is not None else None), b, int(iterations),
                               _stream_handle(stream)), "cwo_gs_run")
        return inten

    def propagate_stack(self, x, zs, out=None, stream=None):
        """One source [Ny][Nx] propagated to len(zs) planes in one batched call (shared spectrum)."""
        _check_field(x, self.nx, self.ny, "input", 1)
        return self._batch(x, 0, len(zs), zs, out, stream, False)

    def _batch(self, x, stride, b, z, out, stream, adjoint):
        out = self._out(x, (b,)) if out is None else out
        _check_field(out, self.nx, self.ny, "output", b)
        zp = None
        if z is not None:
            if len(z) != b:
                raise ValueError(f"{len(z)} distances for {b} items")
            zarr = (ctypes.c_double * b)(*[float(v) for v in z])
            zp = ctypes.cast(zarr, ctypes.POINTER(ctypes.c_double))
        fn = lib().cwo_propagate_adjoint_batch if adjoint else lib().cwo_propagate_batch
        check(fn(self.handle, ctypes.c_void_p(x.data_ptr()), int(stride), ctypes.c_void_p(out.data_ptr()),
                 int(b), zp, _stream_handle(stream)), fn.__name__)
        return out


def emulate(u, dx, dy, wavelength, z, kind=ANGULAR, flags=0, adjoint=False):
    """Host emulation of the kernels (test support): numpy complex64 [ny][nx] -> same."""
    import numpy as np
    a = np.ascontiguousarray(u, dtype=np.complex64)
    ny, nx = a.shape
    out = np.empty_like(a)
    check(lib().cwo_debug_emulate(nx, ny, dx, dy, wavelength, z, kind, flags, int(adjoint),
                                  a.ctypes.data, out.ctypes.data), "cwo_debug_emulate")
    return out


def asm_h(px, py, dx, dy, wavelength, z):
    """Host evaluation of the ASM transfer function in the column pass's own mode (test
    support): (mode, complex64 [py][px] in axis index order)."""
    import numpy as np
    out = np.empty((py, px), dtype=np.complex64)
    mode = ctypes.c_int(99)
    check(lib().cwo_debug_asm_h(px, py, dx, dy, wavelength, z, ctypes.byref(mode), out.ctypes.data),
          "cwo_debug_asm_h")
    return mode.value, out


def emulate_shifted(u, dx, dy, wavelength, z, shift, adjoint=False):
    """Host emulation of a shifted angular-spectrum plan's kernels (test support): numpy
    complex64 [ny][nx] -> same."""
    import numpy as np
    a = np.ascontiguousarray(u, dtype=np.complex64)
    ny, nx = a.shape
    out = np.empty_like(a)
    check(lib().cwo_debug_emulate_shifted(nx, ny, dx, dy, wavelength, z, ctypes.byref(shift), int(adjoint),
                                          a.ctypes.data, out.ctypes.data), "cwo_debug_emulate_shifted")
    return out


def emulate_shifted_fresnel(u, dx0, dy0, wavelength, z, params, adjoint=False):
    """Host emulation of a shifted Fresnel plan's kernels (test support): numpy complex64
    [ny][nx] -> same."""
    import numpy as np
    a = np.ascontiguousarray(u, dtype=np.complex64)
    ny, nx = a.shape
    out = np.empty_like(a)
    check(lib().cwo_debug_emulate_shifted_fresnel(nx, ny, dx0, dy0, wavelength, z, ctypes.byref(params),
                                                  int(adjoint), a.ctypes.data, out.ctypes.data),
          "cwo_debug_emulate_shifted_fresnel")
    return out


def line_fft(x, inverse=False):
    """Host emulation of one padded line transform (test support)."""
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.complex64)
    p = a.size if inverse else 2 * a.size
    out = np.empty(p // 2 if inverse else p, dtype=np.complex64)
    check(lib().cwo_debug_line_fft(p, int(inverse), a.ctypes.data, out.ctypes.data), "cwo_debug_line_fft")
    return out


def axis_bins(p: int):
    import numpy as np
    out = np.empty(p, dtype=np.int32)
    check(lib().cwo_debug_axis_bins(p, out.ctypes.data), "cwo_debug_axis_bins")
    return out


def split_axis(p: int):
    import numpy as np
    index = np.empty(p, dtype=np.int32)
    phase = np.empty(p // 2, dtype=np.complex64)
    check(lib().cwo_debug_split_axis(p, index.ctypes.data, phase.ctypes.data), "cwo_debug_split_axis")
    return index, phase


def fresnel_axis(p: int, pitch: float, wavelength: float, z: float):
    import numpy as np
    out = np.empty(p, dtype=np.complex128)
    check(lib().cwo_debug_fresnel_axis(p, pitch, wavelength, z, out.ctypes.data), "cwo_debug_fresnel_axis")
    return out


def twiddles(p: int):
    """Inter-stage twiddle table of an axis of length p as complex64: per stage s the block
    [kp][j] of (W^{j(2kp+1)}, W^{j(2kp+2)}) pairs, j < S_s = (p >> 4s) / 16."""
    import numpy as np
    nst = (int(p).bit_length() - 1 + 3) // 4
    words = sum(8 * ((p >> (4 * s)) // 16) for s in range(max(nst - 1, 0)))
    out = np.empty(2 * words, dtype=np.complex64)
    check(lib().cwo_debug_twiddles(p, out.ctypes.data), "cwo_debug_twiddles")
    return out


def debug_bounded_wait(spin_limit: int, complete: bool) -> int:
    """Run the bounded mbarrier wait on the current device against a barrier that completes
    (complete=True) or that nothing completes, and return the status word it left (bit 0 =
    the wait gave up)."""
    st = ctypes.c_int(-1)
    check(lib().cwo_debug_bounded_wait(int(spin_limit), int(bool(complete)), ctypes.byref(st)), "cwo_debug_bounded_wait")
    return st.value


def asm_axis(p: int, pitch: float, wavelength: float, z: float, is_x: bool):
    import numpy as np
    out = np.empty((p, 4), dtype=np.float32)
    check(lib().cwo_debug_asm_axis(p, pitch, wavelength, z, int(is_x), out.ctypes.data), "cwo_debug_asm_axis")
    return out
