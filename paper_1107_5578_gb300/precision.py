"""Precision study of the angular-spectrum transfer-function phase.

At z / lambda ~ 1e5 .. 2e6 cycles the phase 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2) of Eq. ang2 is
far beyond what FP32 can hold to a fraction of a cycle.  Three arms of the same propagation:
  reduced  default: per-axis parts reduced modulo one cycle in FP64 on the host, O(1) remainder
           per element in float-float / FP32
  fp32     the phase of Eq. ang2 evaluated literally in FP32 per element (CWO_FLAG_PHASE_FP32)
  fp64     the phase evaluated literally in FP64 per element (CWO_FLAG_PHASE_FP64)
Each is compared with a reference field computed in FP64 (the caller supplies it; the tests use
the FP64 oracle): relative L2 error over all pixels and the largest wrapped phase error over the
pixels with |U| > 1e-3 max |U|.
"""
from __future__ import annotations

import numpy as np

from . import cwo

ARMS = {"reduced": 0, "fp32": cwo.FLAG_PHASE_FP32, "fp64": cwo.FLAG_PHASE_FP64}


def errors(got: np.ndarray, ref: np.ndarray) -> dict:
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    mag = np.abs(ref)
    mask = mag > 1e-3 * mag.max()
    dph = np.angle(got[mask] * np.conj(ref[mask]))
    return {"rel_l2": rel, "max_phase_err_rad": float(np.max(np.abs(dph)))}


def run_arm(u: np.ndarray, pitch: float, wavelength: float, z: float, arm: str) -> np.ndarray:
    import torch
    ny, nx = u.shape
    plan = cwo.Plan(nx, ny, pitch, pitch, wavelength, z, cwo.ANGULAR, ARMS[arm])
    x = torch.from_numpy(np.ascontiguousarray(u, dtype=np.complex64)).cuda()
    y = plan.propagate(x)
    torch.cuda.synchronize()
    out = y.cpu().numpy().astype(np.complex128)
    plan.close()
    return out
