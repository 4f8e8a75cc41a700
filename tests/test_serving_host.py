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
    pytest.importorskip("torch")
    from paper_1107_5578_gb300 import serving
    per = lambda k: 100 * k                                   # bytes of a batch of k
    assert serving.admit(10, 8, 0, 10_000, per) == 8            # capacity bound
    assert serving.admit(3, 8, 0, 10_000, per) == 3             # queue bound
    assert serving.admit(8, 8, 9_500, 10_000, per) == 4         # halved to fit: 9500 + 400 <= 10000
    assert serving.admit(8, 8, 9_950, 10_000, per) == 0         # nothing fits: wait for completions
    assert serving.admit(0, 8, 0, 10_000, per) == 0
    for q in range(0, 20):
        for used in range(0, 10_001, 250):
            b = serving.admit(q, 8, used, 10_000, per)
            assert 0 <= b <= min(q, 8) and (b == 0 or used + per(b) <= 10_000)
