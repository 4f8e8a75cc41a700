"""Phase-only hologram optimisation through the differentiable propagation.

A phase phi [h][w] (1080 x 1920 by default) drives a unit-amplitude field exp(i phi), placed at
the centre of a square canvas of zeros (2048^2); the angular spectrum method (padded by the
library to 4096^2) propagates it by z, and the loss is the mean squared difference between the
intensity |U|^2 on the phi-sized window and a smooth target.  Adam updates phi; gradients come
from the hand-written adjoint kernel (autograd.propagate).

Usable as a module (HologramProblem, optimise) or as a script:
    python -m paper_1107_5578_gb300.hologram --steps 200
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import autograd, cwo, synth


class HologramProblem:
    def __init__(self, h=1080, w=1920, canvas=2048, pitch=6.4e-6, wavelength=520e-9, z=0.15,
                 seed=1, device="cuda"):
        self.h, self.w, self.canvas = h, w, canvas
        self.oy, self.ox = (canvas - h) // 2, (canvas - w) // 2
        self.pitch, self.wavelength, self.z = pitch, wavelength, z
        self.device = torch.device(device)
        self.plan = cwo.Plan(canvas, canvas, pitch, pitch, wavelength, z, cwo.ANGULAR)
        phi0, tgt = synth.hologram_problem(seed, h, w)
        self.phi0 = phi0
        # scale the target so that its energy matches the initial field's intensity on the window
        with torch.no_grad():
            i0 = self.intensity(torch.from_numpy(phi0).float().to(self.device))
        e0 = float(i0.sum())
        self.target_np = tgt * (e0 / float(tgt.sum()))
        self.target = torch.from_numpy(self.target_np).float().to(self.device)

    def field(self, phi: torch.Tensor) -> torch.Tensor:
        x = torch.zeros(self.canvas, self.canvas, dtype=torch.complex64, device=phi.device)
        x[self.oy:self.oy + self.h, self.ox:self.ox + self.w] = torch.polar(torch.ones_like(phi), phi)
        return x

    def intensity(self, phi: torch.Tensor) -> torch.Tensor:
        u = autograd.propagate(self.field(phi), self.plan)
        uw = u[self.oy:self.oy + self.h, self.ox:self.ox + self.w]
        return uw.real ** 2 + uw.imag ** 2

    def loss(self, phi: torch.Tensor) -> torch.Tensor:
        d = self.intensity(phi) - self.target
        return (d * d).mean()


def optimise(problem: HologramProblem, steps=200, lr=0.05, log_every=0):
    phi = torch.from_numpy(problem.phi0).float().to(problem.device).requires_grad_(True)
    opt = torch.optim.Adam([phi], lr=lr)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        opt.zero_grad(set_to_none=True)
        L = problem.loss(phi)
        L.backward()
        opt.step()
        losses.append(L.detach())
        if log_every and (s % log_every == 0 or s == steps - 1):
            print(f"step {s:4d} loss {float(L.detach()):.6e}", flush=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return phi.detach(), [float(v) for v in losses], dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=0.05)
    args = ap.parse_args()
    prob = HologramProblem()
    _, losses, dt = optimise(prob, args.steps, args.lr, log_every=20)
    print(json.dumps({"workload": "hologram_1920x1080_canvas2048_pad4096", "steps": args.steps,
                      "s_per_step": dt / args.steps, "loss_first": losses[0], "loss_last": losses[-1]}))


if __name__ == "__main__":
    main()
