"""The request loop (serving): NNFFT and sinc requests of mixed sizes and tolerances,
each result identical alone and in a mix, within its tolerance of the oracle, under a
device-memory budget that forces plan eviction."""
import time

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


@pytest.mark.parametrize("tol", [1e-5, 1e-9, 1e-12])
@pytest.mark.parametrize("kind", ["nnfft", "sinc"])
def test_tolerance_classes_at_the_largest_bandwidth_with_clustered_nodes(kind, tol):
    """The stream's upper end: N = 16384 with Chebyshev-distributed nodes (cos(pi u)/2,
    dense at +-1/2, where 1/phihat1(N x) and hence the second term of Theorem 4.1 is
    largest).  Each tolerance class must hold on sampled and extreme rows."""
    N, M1, M2 = 16384, 60000, 50000
    S = B.Server(mem_budget_bytes=8 << 30, slots=2, max_points=1 << 17)
    rng = np.random.default_rng(77)
    v = np.cos(np.pi * rng.uniform(0, 1, M1)) / 2
    x = np.cos(np.pi * rng.uniform(0, 1, M2)) / 2
    dt, _ = B.tolerance_params(tol)
    if kind == "nnfft":
        f = W.draw_complex(rng, M1, np.complex128 if dt == B.NNFFT_C128 else np.complex64)
        y = np.zeros(M2, f.dtype)
        S.wait(S.submit_nnfft(N, v, x, f, y, tol))
    else:
        f = rng.standard_normal(M1).astype(np.float64 if dt == B.NNFFT_C128 else np.float32)
        y = np.zeros(M2, f.dtype)
        S.wait(S.submit_sinc(N, v, f, x, y, tol, "gl"))
    S.close()
    rows = W.sample_rows(M2, 200, 9, extremes=[int(np.argmin(x)), int(np.argmax(x))])
    f64 = f.astype(np.complex128)
    want = (oracle.nnfft_direct(N, v, f64, x, rows=rows) if kind == "nnfft"
            else oracle.sinc_direct(N, v, f64, x, rows=rows))
    err = np.max(np.abs(y[rows].astype(np.complex128) - want)) / np.sum(np.abs(f))
    assert err <= tol, (kind, tol, err)


def test_work_of_two_slots_overlaps_on_the_device():
    """Continuous batching: two large requests submitted together run on two slots, and
    their device intervals (CUDA events on the slot streams, from before the uploads to
    after the download) intersect: the second request's work starts on the device before
    the first one's has ended.  Pinned host buffers, so that every copy is asynchronous."""
    M, N = 1 << 22, 4096
    S = B.Server(mem_budget_bytes=16 << 30, slots=2, max_points=M)
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()      # noqa: E731
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(2):
        v = pin(rng.uniform(-0.5, 0.5, M))
        x = pin(rng.uniform(-0.5, 0.5, M))
        f = pin(W.draw_complex(rng, M))
        y = pin(np.zeros(M, np.complex128))
        reqs.append((v, x, f, y))
    # warm-up: two requests at once, so that the cache ends up with two plans of this
    # bucket (a plan serves one slot at a time; the second is made on the builder thread
    # while the first request runs); then the two requests back to back
    for i in [S.submit_nnfft(N, v, x, f, y, 1e-12) for v, x, f, y in reqs]:
        S.wait(i)
    t_end = time.time() + 60
    while S.stats()["plans_cached"] < 2 and time.time() < t_end:
        time.sleep(0.01)
    assert S.stats()["plans_cached"] >= 2
    ids = [S.submit_nnfft(N, v, x, f, y, 1e-12) for v, x, f, y in reqs]
    t = [S.wait_device(i)[1] for i in ids]
    S.close()
    for a in t:
        assert 0 <= a[0] <= a[1] < a[2] <= a[3], t
    (a0, _, _, a1), (b0, _, _, b1) = t
    assert a0 < b1 and b0 < a1, t              # the two device intervals intersect
    rows = W.sample_rows(M, 16, 1)
    v, x, f, y = reqs[1]
    want = oracle.nnfft_direct(N, v, f, x, rows=rows)
    assert np.max(np.abs(y[rows] - want)) / np.sum(np.abs(f)) <= 1e-12
