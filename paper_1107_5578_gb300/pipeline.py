"""Propagation of batches held in host memory with the transfers overlapped.

Each batch is copied host -> device, propagated and copied back; with three CUDA streams (upload,
compute, download) and two device buffer sets, the upload of batch i + 1 and the download of
batch i - 1 run while batch i is propagated, so a stream of batches costs about
max(upload, propagate, download) per batch instead of their sum.  Every batch still moves its own
inputs and results; nothing is cached between batches.  Host buffers should be pinned.
"""
from __future__ import annotations

import torch

from . import cwo


class HostPipeline:
    def __init__(self, plan: cwo.Plan, batch: int, device=None):
        self.plan = plan
        self.batch = int(batch)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        shape = (self.batch, plan.ny, plan.nx)
        self.x = [torch.empty(shape, dtype=torch.complex64, device=self.device) for _ in range(2)]
        self.y = [torch.empty(shape, dtype=torch.complex64, device=self.device) for _ in range(2)]
        self.up = torch.cuda.Stream(device=self.device)
        self.comp = torch.cuda.Stream(device=self.device)
        self.down = torch.cuda.Stream(device=self.device)
        self.uploaded = [torch.cuda.Event() for _ in range(2)]
        self.computed = [torch.cuda.Event() for _ in range(2)]
        self.downloaded = [torch.cuda.Event() for _ in range(2)]
        plan.reserve(self.batch)
        for s in range(2):                      # every event starts in the completed state
            self.computed[s].record(self.comp)
            self.downloaded[s].record(self.down)

    def enqueue(self, host_in: torch.Tensor, host_out: torch.Tensor, i: int) -> None:
        """Batch i: host_in [B][ny][nx] -> propagate -> host_out, on buffer set i % 2."""
        s = i % 2
        self.up.wait_event(self.computed[s])             # x[s] consumed by batch i - 2
        with torch.cuda.stream(self.up):
            self.x[s].copy_(host_in, non_blocking=True)
            self.uploaded[s].record(self.up)
        self.comp.wait_event(self.uploaded[s])
        self.comp.wait_event(self.downloaded[s])         # y[s] read out by batch i - 2
        self.plan.propagate_batch(self.x[s], out=self.y[s], stream=self.comp)
        self.computed[s].record(self.comp)
        self.down.wait_event(self.computed[s])
        with torch.cuda.stream(self.down):
            host_out.copy_(self.y[s], non_blocking=True)
            self.downloaded[s].record(self.down)

    def run(self, host_inputs, host_outputs) -> None:
        """Propagate every batch of host_inputs into host_outputs (same lengths) and wait."""
        for i, (hi, ho) in enumerate(zip(host_inputs, host_outputs)):
            self.enqueue(hi, ho, i)
        self.down.synchronize()
