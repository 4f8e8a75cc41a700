"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bar: relative L2 error <= 2e-5 (FP32 field/FFT arithmetic against FP64)."""
import numpy as np
import pytest

import oracle
from paper_1107_5578_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def cwo(gpu):
    import paper_1107_5578_gb300.cwo as m
    m.lib()
    return m


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(u):
    import torch
    return torch.from_numpy(np.ascontiguousarray(u, dtype=np.complex64)).cuda()


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def gpu_prop(cwo, u, dx, dy, lam, z, kind, flags=0, adjoint=False):
    ny, nx = u.shape
    plan = cwo.Plan(nx, ny, dx, dy, lam, z, kind, flags)
    x = to_dev(u)
    y = plan.adjoint(x) if adjoint else plan.propagate(x)
    out = to_host(y)
    plan.close()
    return out


ORC_KIND = {0: oracle.ANGULAR, 1: oracle.FRESNEL_CONV}


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512, 1024])
@pytest.mark.parametrize("kind", [0, 1])
def test_square_sizes(cwo, n, kind):
    u = synth.random_field(n, seed=100 + n)
    z = 0.05 if kind == 0 else 0.08
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, z, kind)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, z, ORC_KIND[kind])
    assert rel(got, want) <= TOL


@pytest.mark.parametrize("nx,ny", [(64, 16), (16, 128), (256, 32), (32, 512), (2048, 16)])
@pytest.mark.parametrize("kind", [0, 1])
def test_rectangular(cwo, nx, ny, kind):
    u = synth.random_field(nx, seed=7, ny=ny)
    got = gpu_prop(cwo, u, 8e-6, 6e-6, 532e-9, 0.03, kind)
    want = oracle.propagate(u, 8e-6, 6e-6, 532e-9, 0.03, ORC_KIND[kind])
    assert rel(got, want) <= TOL


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("n", [32, 256])
def test_adjoint(cwo, kind, n):
    u = synth.random_field(n, seed=5)
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, 0.07, kind, adjoint=True)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.07, ORC_KIND[kind], oracle.ADJOINT)
    assert rel(got, want) <= TOL


def test_asm_512_config(cwo):
    # 512 x 512 field, amplitude U[0,1), phase U[0, 2 pi), padded to 1024^2, 633 nm, 10 um, 5 cm
    u = synth.random_field(512, seed=1)
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, 0.05, 0)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
    assert rel(got, want) <= TOL


def test_asm_zero_distance_identity(cwo):
    u = synth.random_field(128, seed=3)
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, 0.0, 0)
    assert rel(got, u) <= 2e-6


def test_asm_negative_distance(cwo):
    u = synth.random_field(128, seed=4)
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, -0.12, 0)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, -0.12, oracle.ANGULAR)
    assert rel(got, want) <= TOL


def test_asm_evanescent(cwo):
    # pitch below lambda / sqrt(2): the corners of the band are evanescent and cut
    u = synth.random_field(64, seed=6)
    got = gpu_prop(cwo, u, 0.4e-6, 0.4e-6, 633e-9, 20e-6, 0)
    want = oracle.propagate(u, 0.4e-6, 0.4e-6, 633e-9, 20e-6, oracle.ANGULAR)
    assert rel(got, want) <= TOL


def test_fresnel_literal_scale(cwo):
    u = synth.random_field(64, seed=8)
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, 0.05, 1, flags=cwo.FLAG_LITERAL_SCALE)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.05, oracle.FRESNEL_CONV, oracle.LITERAL_SCALE)
    assert rel(got, want) <= TOL


@pytest.mark.parametrize("kind", [0, 1])
def test_batch_per_item_z(cwo, kind):
    import torch
    n, b = 128, 5
    zs = [0.01, 0.05, 0.1, 0.2, 0.35]
    us = np.stack([synth.random_field(n, seed=20 + i) for i in range(b)])
    plan = cwo.Plan(n, None, 8e-6, None, 532e-9, 0.1, kind)
    y = to_host(plan.propagate_batch(to_dev(us), z=zs))
    for i in range(b):
        want = oracle.propagate(us[i], 8e-6, 8e-6, 532e-9, zs[i], ORC_KIND[kind])
        assert rel(y[i], want) <= TOL
    # the same batch again with the plan's z equals independent single calls bit for bit
    yb = plan.propagate_batch(to_dev(us))
    for i in range(b):
        single = plan.propagate(to_dev(us[i]))
        assert torch.equal(yb[i], single)
    plan.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_stack_shared_source(cwo, kind):
    n = 128
    zs = list(np.linspace(0.1, 0.4, 6))
    u = synth.masked_gaussian(n, seed=2, sigma_px=25.0)
    plan = cwo.Plan(n, None, 8e-6, None, 532e-9, 0.1, kind)
    y = to_host(plan.propagate_stack(to_dev(u), zs))
    for i, z in enumerate(zs):
        want = oracle.propagate(u, 8e-6, 8e-6, 532e-9, float(z), ORC_KIND[kind])
        assert rel(y[i], want) <= TOL
    plan.close()


def test_in_place(cwo):
    u = synth.random_field(64, seed=9)
    plan = cwo.Plan(64, None, 10e-6, None, 633e-9, 0.05, 0)
    x = to_dev(u)
    plan.propagate(x, out=x)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
    assert rel(to_host(x), want) <= TOL
    plan.close()


def test_rejects_host_and_short_buffers(cwo):
    import torch
    plan = cwo.Plan(64, None, 10e-6, None, 633e-9, 0.05, 0)
    x = torch.zeros(64, 64, dtype=torch.complex64)
    host = x.numpy()
    out = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
    st = cwo.lib().cwo_propagate(plan.handle, host.ctypes.data, out.data_ptr(), None)
    assert st == cwo.ERR_INVALID_ARG
    short = torch.zeros(100, dtype=torch.complex64, device="cuda")
    # a buffer whose allocation is too small for a field is refused before any launch
    big = torch.zeros(1 << 20, dtype=torch.complex64, device="cuda")
    end = big.data_ptr() + big.numel() * 8 - 100 * 8
    st = cwo.lib().cwo_propagate(plan.handle, end, out.data_ptr(), None)
    del short
    if st != cwo.OK:       # the caching allocator may hand out a larger segment
        assert st == cwo.ERR_INVALID_ARG
    torch.cuda.synchronize()
    plan.close()


# ---------------------------------------------------------------------- full-size workloads

@pytest.mark.slow
def test_asm_2048_full(cwo):
    u = synth.random_field(2048, seed=11)
    got = gpu_prop(cwo, u, 10e-6, 10e-6, 633e-9, 0.05, 0)
    want = oracle.propagate(u, 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
    assert rel(got, want) <= TOL


@pytest.mark.slow
@pytest.mark.parametrize("cached", [True, False], ids=["once_h", "recalc_h"])
def test_asm_2048_batch16_as_benchmarked(cwo, cached):
    # the benchmark's launch configuration: one batched call of 16 fields of 2048^2 (each field a
    # random phase rotation of one random field), persistent row passes over 16 x 512 row groups,
    # the column pass's item-fastest grid, with the transfer function materialised per plan (the
    # headline) or evaluated per element; two sampled items against the oracle, every item
    # against the first up to its rotation
    import torch
    n, b = 2048, 16
    base = synth.random_field(n, seed=1000)
    rot = np.exp(2j * np.pi * synth.rng(5).random(b))
    x = torch.from_numpy((base[None] * rot[:, None, None]).astype(np.complex64)).cuda()
    plan = cwo.Plan(n, n, 10e-6, 10e-6, 633e-9, 0.05, cwo.ANGULAR, cwo.FLAG_CACHE_H if cached else 0)
    plan.reserve(b)
    y = plan.propagate_batch(x)
    plan.check()
    got = y.cpu().numpy().astype(np.complex128)
    for k in (0, 11):
        want = oracle.propagate(x[k].cpu().numpy(), 10e-6, 10e-6, 633e-9, 0.05, oracle.ANGULAR)
        assert rel(got[k], want) <= TOL
    # linearity: item k = rot_k / rot_0 * item 0 up to the FP32 rounding of the input rotation
    for k in range(1, b):
        assert rel(got[k], got[0] * (rot[k] / rot[0])) <= 2 * TOL


@pytest.mark.slow
def test_fresnel_stack_2048_sampled_planes(cwo):
    # 2048^2 binary mask (p = 0.5) x Gaussian (sigma 400 px), 532 nm, 8 um, 16 planes z in [0.1, 0.4]
    n = 2048
    zs = np.linspace(0.1, 0.4, 16)
    u = synth.masked_gaussian(n, seed=2)
    plan = cwo.Plan(n, None, 8e-6, None, 532e-9, 0.1, 1)
    y = plan.propagate_stack(to_dev(u), list(zs))
    for j in (0, 7, 15):
        want = oracle.propagate(u, 8e-6, 8e-6, 532e-9, float(zs[j]), oracle.FRESNEL_CONV)
        assert rel(to_host(y[j]), want) <= TOL
    plan.close()


def test_status_word_stays_clean(cwo):
    # the bounded waits of the row passes never expire in normal operation
    u = synth.random_field(256, seed=12)
    plan = cwo.Plan(256, None, 10e-6, None, 633e-9, 0.05, 0)
    for _ in range(3):
        plan.propagate(to_dev(u))
    plan.check()
    plan.close()


@pytest.mark.slow
def test_4096_rows_cluster_path_aligned_and_not(cwo):
    # 4096-wide rows (padded to 8192) take the two-CTA cluster row pass; an input that does not
    # start on a 16-byte boundary takes its per-thread-load variant: same arithmetic, same bits
    import torch
    n = 4096
    u = synth.random_field(n, seed=12)
    plan = cwo.Plan(n, n, 3.74e-6, 3.74e-6, 532e-9, 0.2, cwo.ANGULAR)
    x = to_dev(u)
    a = plan.propagate(x)
    buf = torch.empty(n * n + 1, dtype=torch.complex64, device="cuda")
    xm = buf[1:].view(n, n)
    xm.copy_(x)
    assert xm.data_ptr() % 16 == 8
    b = plan.propagate(xm)
    plan.check()
    assert torch.equal(a, b)
    want = oracle.propagate(u.astype(np.complex64), 3.74e-6, 3.74e-6, 532e-9, 0.2, oracle.ANGULAR)
    assert rel(to_host(a), want) <= TOL


@pytest.mark.parametrize("n,z,lam,pitch", [(256, 0.05, 633e-9, 10e-6), (512, -0.2, 532e-9, 4e-6), (128, 2e-4, 633e-9, 0.9e-6)])
def test_cached_transfer_function(cwo, n, z, lam, pitch):
    # CWO_FLAG_CACHE_H: the transfer function materialised at plan creation by the same device
    # functions; forward, adjoint and batches equal the on-the-fly plan, and per-item distances
    # (which cannot use the cache) still propagate correctly
    import torch
    u = synth.random_field(n, seed=400 + n)
    x = to_dev(u)
    fly = cwo.Plan(n, n, pitch, pitch, lam, z, cwo.ANGULAR)
    cache = cwo.Plan(n, n, pitch, pitch, lam, z, cwo.ANGULAR, cwo.FLAG_CACHE_H)
    a, b = fly.propagate(x), cache.propagate(x)
    assert rel(to_host(b), to_host(a)) <= 1e-6
    want = oracle.propagate(u, pitch, pitch, lam, z, oracle.ANGULAR)
    assert rel(to_host(b), want) <= TOL
    assert rel(to_host(cache.adjoint(x)), to_host(fly.adjoint(x))) <= 1e-6
    xb = torch.stack([x, x * 0.5j])
    assert rel(to_host(cache.propagate_batch(xb)), to_host(fly.propagate_batch(xb))) <= 1e-6
    y = to_host(cache.propagate_batch(xb, z=[z / 2, 2 * z]))
    for k, zz in enumerate((z / 2, 2 * z)):
        w = oracle.propagate(to_host(xb[k]), pitch, pitch, lam, zz, oracle.ANGULAR)
        assert rel(y[k], w) <= TOL
    cache.check()
    with pytest.raises(cwo.CwoError):
        cwo.Plan(n, n, pitch, pitch, lam, z, cwo.FRESNEL_CONV, cwo.FLAG_CACHE_H)


@pytest.mark.slow
@pytest.mark.parametrize("nx,ny", [(4096, 4096), (1024, 4096), (64, 4096)])
def test_cached_transfer_function_split_columns(cwo, nx, ny):
    # at Py = 8192 a cached transfer function runs the split column pass (each zero-padded column
    # as the 4096-point DFTs of x_n and x_n W_8192^n, the cache in that order): forward, adjoint
    # and a batch equal the per-element plan, which runs the radix-16,16,16,2 column transform,
    # and the forward result matches the oracle
    import torch
    pitch, lam, z = 3.74e-6, 532e-9, 0.2
    u = synth.random_field(nx, seed=77, ny=ny)
    x = to_dev(u)
    fly = cwo.Plan(nx, ny, pitch, pitch, lam, z, cwo.ANGULAR)
    cache = cwo.Plan(nx, ny, pitch, pitch, lam, z, cwo.ANGULAR, cwo.FLAG_CACHE_H)
    a, b = fly.propagate(x), cache.propagate(x)
    assert rel(to_host(b), to_host(a)) <= 1e-6
    assert rel(to_host(cache.adjoint(x)), to_host(fly.adjoint(x))) <= 1e-6
    xb = torch.stack([x, x * 0.5j])
    assert rel(to_host(cache.propagate_batch(xb)), to_host(fly.propagate_batch(xb))) <= 1e-6
    cache.check()
    if nx != ny:
        want = oracle.propagate(u, pitch, pitch, lam, z, oracle.ANGULAR)
        assert rel(to_host(b), want) <= TOL
        want = oracle.propagate(u, pitch, pitch, lam, z, oracle.ANGULAR, oracle.ADJOINT)
        assert rel(to_host(cache.adjoint(x)), want) <= TOL


# ------------------------------------------------- properties at full size (no oracle output)

@pytest.mark.slow
@pytest.mark.parametrize("kind,z", [(0, 0.05), (1, 0.2)])
def test_adjoint_dot_product_2048(cwo, kind, z):
    # <A x, y> = <x, A^H y> for the cropped linear operator A of one plan (its adjoint conjugates
    # H and C); bounded by 1e-6 of ||A x|| ||y||, the Cauchy-Schwarz scale of either side
    n = 2048
    x = synth.random_field(n, seed=61)
    y = synth.random_field(n, seed=62)
    plan = cwo.Plan(n, n, 10e-6, 10e-6, 633e-9, z, kind)
    ax = to_host(plan.propagate(to_dev(x)))
    ahy = to_host(plan.adjoint(to_dev(y)))
    plan.check()
    plan.close()
    lhs = np.vdot(y, ax)
    rhs = np.vdot(ahy, x)
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(ax) * np.linalg.norm(y)


@pytest.mark.slow
def test_asm_zero_distance_identity_4096(cwo):
    # H = 1 at z = 0: the largest field comes back through both padded transforms unchanged
    n = 4096
    u = synth.random_field(n, seed=63)
    got = gpu_prop(cwo, u, 3.74e-6, 3.74e-6, 532e-9, 0.0, 0)
    assert rel(got, u) <= 2e-6


@pytest.mark.parametrize("nx,ny,adjoint", [(256, 256, False), (512, 64, True), (32, 1024, False), (1024, 32, True)])
def test_fresnel_separable_equals_three_pass(cwo, nx, ny, adjoint):
    # the convolution-form Fresnel plan runs two separable line passes; an output that does not
    # start on a 16-byte boundary takes the three-pass method: both agree with each other and the
    # oracle
    import torch
    u = synth.random_field(nx, seed=70 + nx, ny=ny)
    plan = cwo.Plan(nx, ny, 8e-6, 6e-6, 532e-9, 0.04, cwo.FRESNEL_CONV)
    assert plan.launches_per_call == 2
    x = to_dev(u)
    run = plan.adjoint if adjoint else plan.propagate
    a = to_host(run(x))
    buf = torch.empty(nx * ny + 1, dtype=torch.complex64, device="cuda")
    out = buf[1:].view(ny, nx)
    assert out.data_ptr() % 16 == 8
    run(x, out=out)
    b = to_host(out)
    # an input off a 16-byte boundary: the first line pass loads per thread (no bulk copies)
    ibuf = torch.empty(nx * ny + 1, dtype=torch.complex64, device="cuda")
    xm = ibuf[1:].view(ny, nx)
    xm.copy_(x)
    c = to_host(run(xm))
    plan.check()
    plan.close()
    want = oracle.propagate(u, 8e-6, 6e-6, 532e-9, 0.04, oracle.FRESNEL_CONV, oracle.ADJOINT if adjoint else 0)
    assert rel(a, want) <= TOL and rel(b, want) <= TOL
    assert rel(a, b) <= 1e-5
    assert np.array_equal(a, c)


@pytest.mark.slow
def test_fresnel_4096_and_batch16_2048(cwo):
    # the largest field (lines padded to 8192: two lines per CTA) and a 16-field batch as the
    # serving and stack workloads size it; sampled items against the oracle
    import torch
    u = synth.random_field(4096, seed=71)
    plan = cwo.Plan(4096, 4096, 3.74e-6, 3.74e-6, 532e-9, 0.3, cwo.FRESNEL_CONV)
    got = to_host(plan.propagate(to_dev(u)))
    plan.close()
    assert rel(got, oracle.propagate(u, 3.74e-6, 3.74e-6, 532e-9, 0.3, oracle.FRESNEL_CONV)) <= TOL
    n, b = 2048, 16
    base = synth.random_field(n, seed=72)
    zs = list(np.linspace(0.1, 0.4, b))
    x = to_dev(np.broadcast_to(base, (b, n, n)))
    plan = cwo.Plan(n, n, 8e-6, 8e-6, 532e-9, 0.2, cwo.FRESNEL_CONV)
    y = to_host(plan.propagate_batch(x, z=zs))
    plan.check()
    plan.close()
    for k in (0, 9):
        assert rel(y[k], oracle.propagate(base, 8e-6, 8e-6, 532e-9, zs[k], oracle.FRESNEL_CONV)) <= TOL


@pytest.mark.parametrize("nx,ny", [(512, 256), (256, 1024)])
def test_fresnel_stack_separable_equals_three_pass(cwo, nx, ny):
    # a Fresnel z-stack runs as two separable passes (each source row transformed once for all
    # planes); an output off a 16-byte boundary takes the three-pass stack: both agree with each
    # other and the oracle
    import torch
    zs = [0.05, 0.11, -0.2, 0.3, 0.07]
    u = synth.random_field(nx, seed=80 + nx, ny=ny)
    plan = cwo.Plan(nx, ny, 8e-6, 6e-6, 532e-9, 0.1, cwo.FRESNEL_CONV)
    x = to_dev(u)
    a = to_host(plan.propagate_stack(x, zs))
    buf = torch.empty(len(zs) * nx * ny + 1, dtype=torch.complex64, device="cuda")
    out = buf[1:].view(len(zs), ny, nx)
    plan.propagate_stack(x, zs, out=out)
    b = to_host(out)
    plan.check()
    plan.close()
    for i, z in enumerate(zs):
        assert rel(a[i], oracle.propagate(u, 8e-6, 6e-6, 532e-9, z, oracle.FRESNEL_CONV)) <= TOL
    assert rel(a, b) <= 1e-5
