"""Propagation of batches held in host memory with the transfers overlapped.

Each batch is copied host -> device, propagated and copied back; with upload streams, a compute
stream, download streams and two device buffer sets, the upload of batch i + 1 and the download
of batch i - 1 run while batch i is propagated, so a stream of batches costs about
max(upload, propagate, download) per batch instead of their sum.  A transfer may be split into
`copy_streams` contiguous chunks on as many streams (measured on GB300: no gain; the host link
carries ~210 GB/s up, ~193 GB/s down and ~270 GB/s with both directions busy, whether copy
engines or SMs move the data).  Every batch still moves its own inputs and results; nothing is
cached between batches.  Host buffers should be pinned.
"""
from __future__ import annotations

import torch

from . import cwo


class HostPipeline:
    def __init__(self, plan: cwo.Plan, batch: int, device=None, copy_streams: int = 1):
        self.plan = plan
        self.batch = int(batch)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        shape = (self.batch, plan.ny, plan.nx)
        self.x = [torch.empty(shape, dtype=torch.complex64, device=self.device) for _ in range(2)]
        self.y = [torch.empty(shape, dtype=torch.complex64, device=self.device) for _ in range(2)]
        k = max(1, min(int(copy_streams), self.batch))
        bounds = [self.batch * j // k for j in range(k + 1)]
        self.chunks = [(bounds[j], bounds[j + 1]) for j in range(k)]
        self.up = [torch.cuda.Stream(device=self.device) for _ in range(k)]
        self.down = [torch.cuda.Stream(device=self.device) for _ in range(k)]
        self.comp = torch.cuda.Stream(device=self.device)
        self.uploaded = [[torch.cuda.Event() for _ in range(k)] for _ in range(2)]
        self.downloaded = [[torch.cuda.Event() for _ in range(k)] for _ in range(2)]
        self.computed = [torch.cuda.Event() for _ in range(2)]
        plan.reserve(self.batch)
        for s in range(2):                      # every event starts in the completed state
            self.computed[s].record(self.comp)
            for j in range(k):
                self.downloaded[s][j].record(self.down[j])

    def enqueue(self, host_in: torch.Tensor, host_out: torch.Tensor, i: int) -> None:
        """Batch i: host_in [B][ny][nx] -> propagate -> host_out, on buffer set i % 2."""
        s = i % 2
        for j, (a, b) in enumerate(self.chunks):
            self.up[j].wait_event(self.computed[s])     # x[s] consumed by batch i - 2
            with torch.cuda.stream(self.up[j]):
                self.x[s][a:b].copy_(host_in[a:b], non_blocking=True)
                self.uploaded[s][j].record(self.up[j])
        for j in range(len(self.chunks)):
            self.comp.wait_event(self.uploaded[s][j])
            self.comp.wait_event(self.downloaded[s][j])  # y[s] read out by batch i - 2
        self.plan.propagate_batch(self.x[s], out=self.y[s], stream=self.comp)
        self.computed[s].record(self.comp)
        for j, (a, b) in enumerate(self.chunks):
            self.down[j].wait_event(self.computed[s])
            with torch.cuda.stream(self.down[j]):
                host_out[a:b].copy_(self.y[s][a:b], non_blocking=True)
                self.downloaded[s][j].record(self.down[j])

    def synchronize(self) -> None:
        for st in self.down:
            st.synchronize()

    def run(self, host_inputs, host_outputs) -> None:
        """Propagate every batch of host_inputs into host_outputs (same lengths) and wait."""
        for i, (hi, ho) in enumerate(zip(host_inputs, host_outputs)):
            self.enqueue(hi, ho, i)
        self.synchronize()
