"""Host-side serving logic: request validation and the request stream recipe (no GPU)."""
import numpy as np
import pytest

from paper_1107_5578_gb300 import synth


def test_request_stream_recipe():
    d = synth.serving_requests(20000, seed=5)
    n = d["n"]
    frac = {s: float(np.mean(n == s)) for s in synth.SERVING_SIZES}
    for s, w in zip(synth.SERVING_SIZES, synth.SERVING_WEIGHTS):
        assert abs(frac[s] - w) < 0.02
    assert abs(float(np.mean(d["kind"] == 1)) - 0.3) < 0.02
    gaps = np.diff(d["t"])
    assert abs(gaps.mean() - 1 / 2000.0) < 0.05 / 2000.0          # Poisson, mean 2000 req/s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05             # exponential gaps
    assert d["z"].min() >= 0.01 and d["z"].max() <= 0.5
    assert set(np.unique(d["lam"])) == set(synth.SERVING_WAVELENGTHS)
    assert d["pitch"].min() >= 4e-6 and d["pitch"].max() <= 10e-6
    # same seed, same stream
    d2 = synth.serving_requests(20000, seed=5)
    assert np.array_equal(d["t"], d2["t"]) and np.array_equal(d["n"], d2["n"])


def test_validation_rejects_bad_requests_without_a_device():
    pytest.importorskip("torch")
    from paper_1107_5578_gb300 import serving
    ok = serving.Request(0, 256, 0, 0.1, 532e-9, 8e-6)
    serving.validate(ok)
    for bad in [serving.Request(1, 300, 0, 0.1, 532e-9, 8e-6), serving.Request(2, 256, 5, 0.1, 532e-9, 8e-6),
                serving.Request(3, 256, 0, 0.1, 0.0, 8e-6), serving.Request(4, 256, 1, 0.0, 532e-9, 8e-6),
                serving.Request(5, 256, 0, float("inf"), 532e-9, 8e-6)]:
        with pytest.raises(ValueError):
            serving.validate(bad)


def test_admission_by_memory_budget():
    """The runtime's admission rule (cwo_server_admit, host only): up to the slot's capacity and
    the queue, halved until the batch fits the budget next to the bytes in flight."""
    pytest.importorskip("torch")
    from paper_1107_5578_gb300 import build, serving
    build.build()
    n = 256
    per = {k: serving.batch_bytes(n, k) for k in range(1, 9)}
    assert all(per[k + 1] > per[k] for k in range(1, 8))          # bytes grow with the batch
    assert per[1] > 2 * n * n * 8                                 # plan scratch + input + output
    big = 10 * per[8]
    assert serving.admit(10, 8, 0, big, n) == 8                   # capacity bound
    assert serving.admit(3, 8, 0, big, n) == 3                    # queue bound
    assert serving.admit(8, 8, big - per[4], big, n) == 4         # halved to fit
    assert serving.admit(8, 8, big - per[1] + 1, big, n) == 0     # nothing fits: wait for completions
    assert serving.admit(0, 8, 0, big, n) == 0
    for q in range(0, 12):
        for used in range(0, big + 1, big // 17):
            b = serving.admit(q, 8, used, big, n)
            assert 0 <= b <= min(q, 8) and (b == 0 or used + per[b] <= big)
            c = min(q, 8)                                         # the first fit of c, c // 2, ...
            while c > 0 and used + per[c] > big:
                c //= 2
            assert b == c


def test_native_server_refuses_bad_arguments_before_touching_a_device():
    """The runtime's argument checks run on the host first (no GPU is needed to see them)."""
    pytest.importorskip("torch")
    import ctypes
    from paper_1107_5578_gb300 import build, cwo, serving
    build.build()
    L = serving._lib()
    out = ctypes.c_void_p()

    def create(sizes, caps, slots=2, budget=0):
        s = (ctypes.c_int * len(sizes))(*sizes)
        c = (ctypes.c_int * len(caps))(*caps)
        return L.cwo_server_create(len(sizes), s, c, slots, budget, ctypes.byref(out))

    assert create([], []) == cwo.ERR_INVALID_ARG                         # no size
    assert create([300], [4]) == cwo.ERR_INVALID_ARG                     # not a power of two
    assert create([8192], [1]) == cwo.ERR_INVALID_ARG                    # above 4096
    assert create([256], [65]) == cwo.ERR_INVALID_ARG                    # batch capacity above 64
    assert create([256], [0]) == cwo.ERR_INVALID_ARG
    assert create([256, 256], [4, 4]) == cwo.ERR_INVALID_ARG             # size given twice
    assert create([256], [4], slots=0) == cwo.ERR_INVALID_ARG
    assert create([256], [4], slots=9) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_create(1, None, None, 2, 0, ctypes.byref(out)) == cwo.ERR_INVALID_ARG
    b = ctypes.c_size_t(0)
    assert L.cwo_server_batch_bytes(100, 1, ctypes.byref(b)) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_batch_bytes(256, 0, ctypes.byref(b)) == cwo.ERR_INVALID_ARG
    take = ctypes.c_int(0)
    assert L.cwo_server_admit(-1, 4, 0, 1 << 30, 256, ctypes.byref(take)) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_admit(4, 0, 0, 1 << 30, 256, ctypes.byref(take)) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_admit(4, 4, 0, 1 << 30, 256, None) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_submit(None, None, None) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_step(None, None) == cwo.ERR_INVALID_ARG
    assert L.cwo_server_done(None, 0, None) == -1
    assert L.cwo_server_destroy(None) == cwo.OK
