"""The host pipeline (overlapped upload / propagate / download on three streams) returns, for
every batch, exactly what a plain synchronous propagation of that batch returns."""
import numpy as np
import pytest

from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu


def test_pipeline_matches_serial(gpu):
    import torch
    from paper_1107_5578_gb300 import cwo, pipeline
    plan = cwo.Plan(256, 128, 8e-6, 8e-6, 532e-9, 0.03, cwo.ANGULAR)
    batches = [torch.from_numpy(np.stack([synth.random_field(256, seed=90 + 4 * i + k, ny=128) for k in range(3)])
                                .astype(np.complex64)).pin_memory() for i in range(5)]
    outs = [torch.empty_like(b).pin_memory() for b in batches]
    pipe = pipeline.HostPipeline(plan, 3)
    pipe.run(batches, outs)
    ref = cwo.Plan(256, 128, 8e-6, 8e-6, 532e-9, 0.03, cwo.ANGULAR)
    for b, o in zip(batches, outs):
        want = ref.propagate_batch(b.cuda()).cpu()
        assert torch.equal(o, want)
