"""Serving on the GPU: every result is the same alone and in the mixed, continuously batched
stream (bit for bit: no arithmetic depends on the batch), results match the oracle, and the
memory budget bounds what is in flight."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv(gpu):
    import torch
    from paper_1107_5578_gb300 import cwo, serving
    cwo.lib()
    return torch, serving


def _requests(serving, n_req, sizes, seed=11, rate=4000.0):
    from paper_1107_5578_gb300 import synth
    w = [1.0 / len(sizes)] * len(sizes)
    return serving.make_requests(n_req, seed, rate_hz=rate, sizes=sizes, weights=w)


def test_results_are_the_same_alone_and_in_the_mix(srv):
    torch, serving = srv
    sizes = (256, 512, 1024)
    pools = serving.make_pools(sizes, per_size=3)
    # a dense stream (5 us between arrivals): requests arrive while others are on the GPU, so
    # they travel in mixed batches
    mix = _requests(serving, 60, sizes, rate=2e5)
    server = serving.Server(sizes=sizes, max_batch={256: 16, 512: 8, 1024: 4}, pools=pools, keep_results=True)
    server.run(mix)
    assert server.batches < len(mix)                 # batching happened
    alone = _requests(serving, 60, sizes, rate=2e5)
    serving.serve_serial(alone, pools, keep_results=True)
    for a, b in zip(sorted(mix, key=lambda r: r.rid), sorted(alone, key=lambda r: r.rid)):
        assert torch.equal(a.result, b.result), a.rid
    # and against the FP64 oracle for a few of them
    for r in sorted(mix, key=lambda r: r.rid)[:6]:
        u = pools[r.n][r.pool_index % 3].cpu().numpy().astype(np.complex128)
        want = oracle.propagate(u, r.pitch, r.pitch, r.wavelength, r.z, r.kind)
        got = r.result.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 2e-5


def test_memory_budget_bounds_what_is_in_flight(srv):
    torch, serving = srv
    sizes = (256, 512)
    pools = serving.make_pools(sizes, per_size=2)
    budget = serving.batch_bytes(512, 2)
    server = serving.Server(sizes=sizes, max_batch={256: 16, 512: 8}, pools=pools, mem_budget=budget)
    reqs = _requests(serving, 80, sizes, rate=20000.0)
    server.run(reqs)
    assert all(r.t_done is not None for r in reqs)
    assert 0 < server.mem_peak <= budget


def test_submit_field_returns_a_future(srv):
    torch, serving = srv
    from paper_1107_5578_gb300 import synth
    server = serving.Server(sizes=(128,), max_batch={128: 4}, keep_results=True)
    u = [synth.random_field(128, seed=200 + k) for k in range(3)]
    futs = [server.submit_field(torch.from_numpy(v.astype(np.complex64)).cuda(), z=0.03 * (k + 1),
                                wavelength=532e-9, pitch=8e-6, kind=k % 2) for k, v in enumerate(u)]
    for k, f in enumerate(futs):
        got = server.wait(f).cpu().numpy().astype(np.complex128)
        want = oracle.propagate(u[k], 8e-6, 8e-6, 532e-9, 0.03 * (k + 1), k % 2)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 2e-5
    with pytest.raises(ValueError):
        server.submit_field(torch.zeros(64, 64, dtype=torch.complex64, device="cuda"), z=0.1)   # size not served
    small = serving.Server(sizes=(128,), max_batch={128: 4}, mem_budget=1000)
    with pytest.raises(ValueError):                                # one field exceeds the budget
        small.submit_field(torch.zeros(128, 128, dtype=torch.complex64, device="cuda"), z=0.1)


def test_server_refuses_a_host_field_before_queueing_it(srv):
    torch, serving = srv
    server = serving.Server(sizes=(128,), max_batch={128: 4}, keep_results=True)
    host = torch.zeros(128, 128, dtype=torch.complex64)             # host memory
    req = serving.Request(1, 128, 0, 0.05, 532e-9, 8e-6, field=host)
    with pytest.raises(ValueError):
        server.submit(req)
    assert server.pending() == 0
    ok = server.submit_field(torch.ones(128, 128, dtype=torch.complex64, device="cuda"), z=0.05,
                             wavelength=532e-9, pitch=8e-6)
    assert server.wait(ok) is not None                               # the server still serves
    server.close()
