"""Gerchberg-Saxton kinoform generation with the angular spectrum method (Section "GS
algorithm", Table "Calculation times of the GS algorithm on the CPU and GPUs").

The object is the amplitude sqrt(I) of a test image with a random initial phase; the kinoform
(a phase-only field) sits at distance z.  The whole loop runs on the device through
``cwo_gs_run``: each half-iteration is one three-pass propagation whose last pass applies the
constraint (phase only, or object amplitude with the propagated phase).  Every propagation of
the loop has the same distance (the backward ones use conj(H)), so the plan materialises its
transfer function once (the paper's once-calculation), about 3% faster per loop than evaluating
it per element.

    python -m paper_1107_5578_gb300.gs --n 2048 --iterations 40
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import cwo, synth

PITCH = 10e-6          # the paper's default pitch and wavelength (Section "CWO class")
WAVELENGTH = 633e-9
DISTANCE = 0.1         # Section "GS algorithm": +-0.1 m


class GSProblem:
    def __init__(self, n=2048, seed=1, batch=1, pitch=PITCH, wavelength=WAVELENGTH, z=DISTANCE, device="cuda"):
        self.n, self.batch, self.z = n, batch, z
        amps, fields = [], []
        for k in range(batch):
            a, f = synth.gs_problem(n, seed=seed + k)
            amps.append(a)
            fields.append(f)
        self.amplitude_np = np.stack(amps)
        self.field0_np = np.stack(fields)
        self.amplitude = torch.from_numpy(self.amplitude_np.astype(np.float32)).to(device)
        self.field0 = torch.from_numpy(self.field0_np.astype(np.complex64)).to(device)
        self.plan = cwo.Plan(n, n, pitch, pitch, wavelength, z, cwo.ANGULAR, cwo.FLAG_CACHE_H)
        self.plan.reserve(batch)

    def run(self, iterations: int):
        """(kinoform [B][n][n] complex64, reconstructed intensity [B][n][n] float32)."""
        field = self.field0.clone()
        inten = self.plan.gs_run(self.amplitude, field, iterations)
        return field, inten


def amplitude_error(inten: torch.Tensor, amplitude: torch.Tensor) -> float:
    """Relative error of the reconstructed amplitude against the object amplitude, after the
    best scalar gain (the kinoform carries no information about the absolute energy)."""
    rec = inten.double().clamp_min(0).sqrt()
    a = amplitude.double()
    g = (rec * a).sum() / (rec * rec).sum()
    return float((g * rec - a).norm() / a.norm())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--iterations", type=int, default=40)
    args = ap.parse_args()
    prob = GSProblem(args.n)
    prob.run(2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    _, inten = prob.run(args.iterations)
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"workload": f"gs_{args.n}", "iterations": args.iterations, "ms": a.elapsed_time(b),
                      "amplitude_error": amplitude_error(inten, prob.amplitude)}))


if __name__ == "__main__":
    main()
