"""The request loop (serving): NNFFT and sinc requests of mixed sizes and tolerances,
each result identical alone and in a mix, within its tolerance of the oracle, under a
device-memory budget that forces plan eviction."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2107_02671_gb300 import nnfft as B  # noqa: E402
from paper_2107_02671_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


# (kind, N, M1, M2, tol, rule, complex)
MIX = [("nnfft", 64, 128, 128, 1e-12, None, True), ("nnfft", 100, 3000, 2000, 1e-5, None, True),
       ("sinc", 128, 700, 500, 1e-12, "gl", False), ("nnfft", 1000, 5000, 4000, 1e-9, None, True),
       ("sinc", 300, 2000, 1500, 1e-5, "cc", False), ("nnfft", 3000, 800, 6000, 1e-12, None, True),
       ("sinc", 90, 400, 300, 1e-9, "cc", True), ("nnfft", 50, 0, 10, 1e-12, None, True),
       ("nnfft", 4096, 6000, 100, 1e-5, None, True), ("sinc", 1000, 3000, 3000, 1e-12, "gl", False),
       ("nnfft", 777, 1, 1, 1e-9, None, True), ("sinc", 64, 10, 2000, 1e-5, "gl", True)]


def make_inputs(i, spec):
    kind, N, M1, M2, tol, rule, cplx = spec
    dt, _ = B.tolerance_params(tol)
    c = np.complex128 if dt == B.NNFFT_C128 else np.complex64
    r = np.float64 if dt == B.NNFFT_C128 else np.float32
    rng = np.random.default_rng(100 + i)
    v = rng.uniform(-0.5, 0.5, M1)
    x = rng.uniform(-0.5, 0.5, M2)
    if cplx:
        f = W.draw_complex(rng, M1, c)
    else:
        f = rng.standard_normal(M1).astype(r)
    return v, x, f, np.zeros(M2, dtype=f.dtype)


def submit(S, spec, v, x, f, y):
    kind, N, M1, M2, tol, rule, cplx = spec
    if kind == "nnfft":
        return S.submit_nnfft(N, v, x, f, y, tol)
    return S.submit_sinc(N, v, f, x, y, tol, rule)


def exact(spec, v, x, f):
    kind, N = spec[0], spec[1]
    f64 = f.astype(np.complex128)
    if kind == "nnfft":
        return oracle.nnfft_direct(N, v, f64, x)
    return oracle.sinc_direct(N, v, f64, x)


def test_results_alone_equal_results_in_the_mix_and_meet_tolerance():
    S = B.Server(mem_budget_bytes=8 << 30, slots=4, max_points=1 << 14)
    inputs = [make_inputs(i, s) for i, s in enumerate(MIX)]
    alone = []
    for spec, (v, x, f, y) in zip(MIX, inputs):
        out = np.zeros_like(y)
        S.wait(submit(S, spec, v, x, f, out))
        alone.append(out)
    mixed = [np.zeros_like(y) for (_, _, _, y) in inputs]
    ids = [submit(S, spec, v, x, f, out) for spec, (v, x, f, _), out in zip(MIX, inputs, mixed)]
    lat = [S.wait(i) for i in ids]
    st = S.stats()
    S.close()
    assert all(t > 0 for t in lat)
    assert st["completed"] == 2 * len(MIX) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for spec, (v, x, f, _), a, m in zip(MIX, inputs, alone, mixed):
        assert np.array_equal(a, m), spec
        if spec[3] == 0 or spec[2] == 0:
            assert not np.any(a), spec
            continue
        err = np.max(np.abs(a.astype(np.complex128) - exact(spec, v, x, f))) / np.sum(np.abs(f))
        assert err <= spec[4], (spec, err)


def test_budget_forces_eviction_and_results_stay_correct():
    """Plans for 600k-point requests hold about 70 MB each; the budget (300 MB with about
    50 MB of slot buffers) admits one such plan next to its admission estimate, so each new
    bandwidth bucket evicts the previous plan.  Sampled rows against the oracle."""
    budget = 300 << 20
    S = B.Server(mem_budget_bytes=budget, slots=1, max_points=1 << 20)
    M = 600_000
    for i, N in enumerate([64, 200, 700, 64]):
        rng = np.random.default_rng(50 + i)
        v, x = rng.uniform(-0.5, 0.5, M), rng.uniform(-0.5, 0.5, M)
        f, y = W.draw_complex(rng, M), np.zeros(M, np.complex128)
        S.wait(S.submit_nnfft(N, v, x, f, y, 1e-12))
        rows = W.sample_rows(M, 64, i)
        want = oracle.nnfft_direct(N, v, f, x, rows=rows)
        assert np.max(np.abs(y[rows] - want)) / np.sum(np.abs(f)) <= 1e-12
    st = S.stats()
    S.close()
    assert st["plans_evicted"] >= 2 and st["device_bytes"] <= budget


def test_request_larger_than_the_budget_fails():
    S = B.Server(mem_budget_bytes=40 << 20, slots=1, max_points=4096)
    spec = ("nnfft", 64, 100, 100, 1e-12, None, True)
    v, x, f, y = make_inputs(8, spec)
    with pytest.raises(B.NNFFTError) as e:
        S.wait(S.submit_nnfft(64, v, x, f, y, 1e-12))
    S.close()
    assert e.value.code == 3                                 # NNFFT_ENOMEM


def test_request_errors_do_not_stop_the_loop():
    S = B.Server(mem_budget_bytes=4 << 30, slots=2, max_points=4096)
    spec = ("nnfft", 64, 100, 100, 1e-12, None, True)
    v, x, f, y = make_inputs(7, spec)
    with pytest.raises(B.NNFFTError):                        # above max_points
        S.submit_nnfft(64, np.zeros(5000), x, np.zeros(5000, np.complex128), y, 1e-12)
    vbad = v.copy()
    vbad[3] = 0.75                                           # outside [-1/2, 1/2]
    with pytest.raises(B.NNFFTError):
        S.wait(S.submit_nnfft(64, vbad, x, f, np.zeros_like(y), 1e-12))
    S.wait(S.submit_nnfft(64, v, x, f, y, 1e-12))          # the next request is served
    S.close()
    assert np.max(np.abs(y - exact(spec, v, x, f))) / np.sum(np.abs(f)) <= 1e-12
