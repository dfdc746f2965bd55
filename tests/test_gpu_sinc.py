"""GPU parity of the fast sinc transform (Algorithm 6.1 with a 2N-node
Gauss-Legendre rule on [-1/2, 1/2]) against the oracle: the direct sum of
eq. (6.2) and the Gauss-Legendre definition of eq. (6.3)
evaluated by direct sums (which isolates the NNFFT error from the quadrature error)."""
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
    yield
    B.sinc_release()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,L1,L2", [(64, 500, 300), (256, 3000, 2000), (1024, 4097, 999)])
def test_sinc_fp64_m8(N, L1, L2):
    a, c, b = W.sinc_inputs(L1, L2, 0)
    h = B.sinc(N, dev(a), dev(c), dev(b), m=8).cpu().numpy()
    B.sinc_sync()
    gl = oracle.sinc_gl(N, a, c, b).real
    assert np.max(np.abs(h - gl)) / np.sum(np.abs(c)) <= 1e-12
    direct = oracle.sinc_direct(N, a, c, b).real
    assert np.max(np.abs(h - direct)) / np.sum(np.abs(c)) <= 1e-12


@pytest.mark.parametrize("N,L1,L2", [(256, 3000, 2000), (1024, 4097, 999)])
def test_sinc_fp32_m4(N, L1, L2):
    a, c, b = W.sinc_inputs(L1, L2, 1)
    c32 = c.astype(np.float32)
    h = B.sinc(N, dev(a), dev(c32), dev(b), m=4).cpu().numpy().astype(np.float64)
    B.sinc_sync()
    direct = oracle.sinc_direct(N, a, c32.astype(np.float64), b).real
    assert np.max(np.abs(h - direct)) / np.sum(np.abs(c)) <= 2e-5


def test_sinc_complex_coefficients():
    N, L1, L2 = 128, 700, 500
    a, c, b = W.sinc_inputs(L1, L2, 2, complex_coeffs=True)
    h = B.sinc(N, dev(a), dev(c), dev(b), m=8).cpu().numpy()
    B.sinc_sync()
    direct = oracle.sinc_direct(N, a, c, b)
    assert np.max(np.abs(h - direct)) / np.sum(np.abs(c)) <= 1e-12


def test_sinc_shannon_identity():
    """a_k = b_k = k/N (Section 6): sinc(pi (l - k)) = delta_lk, so h = c."""
    N = 512
    k = np.arange(-(N // 2), N - N // 2) / N
    rng = np.random.default_rng(3)
    c = rng.standard_normal(N)
    h = B.sinc(N, dev(k), dev(c), dev(k), m=8).cpu().numpy()
    B.sinc_sync()
    assert np.max(np.abs(h - c)) / np.sum(np.abs(c)) <= 1e-12


def test_sinc_repeated_calls_reuse_cache():
    N = 256
    for seed in range(3):
        a, c, b = W.sinc_inputs(1000 + 0, 800, seed)
        h = B.sinc(N, dev(a), dev(c), dev(b), m=8).cpu().numpy()
        B.sinc_sync()
        direct = oracle.sinc_direct(N, a, c, b).real
        assert np.max(np.abs(h - direct)) / np.sum(np.abs(c)) <= 1e-12


def test_sinc_full_size_sampled_rows():
    """N = 1024, L1 = L2 = 2^18, c real N(0,1), m = 8 (fp64) and m = 4 (fp32)."""
    N, L = 1024, 1 << 18
    a, c, b = W.sinc_inputs(L, L, 0)
    rows = W.sample_rows(L, 64, 5, extremes=[int(np.argmin(b)), int(np.argmax(b))])
    h = B.sinc(N, dev(a), dev(c), dev(b), m=8).cpu().numpy()
    B.sinc_sync()
    direct = oracle.sinc_direct(N, a, c, b, rows=rows).real
    assert np.max(np.abs(h[rows] - direct)) / np.sum(np.abs(c)) <= 1e-12
    c32 = c.astype(np.float32)
    h32 = B.sinc(N, dev(a), dev(c32), dev(b), m=4).cpu().numpy().astype(np.float64)
    B.sinc_sync()
    direct = oracle.sinc_direct(N, a, c32.astype(np.float64), b, rows=rows).real
    assert np.max(np.abs(h32[rows] - direct)) / np.sum(np.abs(c)) <= 2e-5


# --------------------------------------------------------------------------------------
# Clenshaw-Curtis rule (Algorithm 6.1 as printed; weights by Algorithm 5.4 on the GPU)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("N,n", [(16, 0), (64, 0), (1024, 0), (100, 0), (97, 0), (64, 384)])
def test_cc_weights_from_gpu(N, n):
    """Device DCT-I weights against the explicit sum of eq. (5.4); n = 4N by default,
    rounded up to 5-smooth (N = 97: 388 -> 400)."""
    t, w = B.sinc_quadrature("cc", N, n)
    nn = len(t) - 1
    want = n if n else 4 * N
    r = nn
    for p in (2, 3, 5):
        while r % p == 0:
            r //= p
    assert nn >= want and r == 1 and (nn == want or N == 97)
    z, wo = oracle.cc_weights(nn)
    assert np.max(np.abs(w - wo)) * nn <= 1e-13
    assert np.max(np.abs(2 * t - z)) <= 1e-15
    assert abs(w.sum() - 1.0) <= 1e-14


@pytest.mark.parametrize("N,L1,L2", [(64, 500, 300), (256, 3000, 2000), (1024, 4097, 999)])
def test_sinc_cc_fp64_m8(N, L1, L2):
    a, c, b = W.sinc_inputs(L1, L2, 7)
    h = B.sinc(N, dev(a), dev(c), dev(b), m=8, rule="cc").cpu().numpy()
    B.sinc_sync()
    cc = oracle.sinc_cc(N, a, c, b).real
    assert np.max(np.abs(h - cc)) / np.sum(np.abs(c)) <= 1e-12
    direct = oracle.sinc_direct(N, a, c, b).real
    assert np.max(np.abs(h - direct)) / np.sum(np.abs(c)) <= 1e-12


@pytest.mark.parametrize("N,L1,L2", [(256, 3000, 2000), (1024, 4097, 999)])
def test_sinc_cc_fp32_m4(N, L1, L2):
    a, c, b = W.sinc_inputs(L1, L2, 8)
    c32 = c.astype(np.float32)
    h = B.sinc(N, dev(a), dev(c32), dev(b), m=4, rule="cc").cpu().numpy().astype(np.float64)
    B.sinc_sync()
    direct = oracle.sinc_direct(N, a, c32.astype(np.float64), b).real
    assert np.max(np.abs(h - direct)) / np.sum(np.abs(c)) <= 2e-5


@pytest.mark.parametrize("k", [5, 7, 9])
@pytest.mark.parametrize("nu", [4, 6, 8])
def test_sinc_cc_figure_6_1_protocol(k, nu):
    """The Fig. 6.1 experiment: N = 2^k, L1 = N/2 random a_k, b_l = l/N (L2 = N), complex
    c, n = nu N; maximum error over repetitions (3 here) against the direct sum."""
    N = 1 << k
    worst = 0.0
    for rep in range(3):
        rng = np.random.default_rng(1000 * k + 10 * nu + rep)
        a = rng.uniform(-0.5, 0.5, N // 2)
        b = np.arange(-(N // 2), N - N // 2) / N
        c = rng.standard_normal(N // 2) + 1j * rng.standard_normal(N // 2)
        h = B.sinc(N, dev(a), dev(c), dev(b), m=8, rule="cc", n=nu * N).cpu().numpy()
        B.sinc_sync()
        d = oracle.sinc_direct(N, a, c, b)
        worst = max(worst, float(np.max(np.abs(h - d)) / np.sum(np.abs(c))))
    assert worst <= 1e-12


def test_sinc_cc_full_size_sampled_rows():
    """N = 1024, L1 = L2 = 2^18 with the Clenshaw-Curtis rule, m = 8 (fp64)."""
    N, L = 1024, 1 << 18
    a, c, b = W.sinc_inputs(L, L, 0)
    rows = W.sample_rows(L, 64, 6, extremes=[int(np.argmin(b)), int(np.argmax(b))])
    h = B.sinc(N, dev(a), dev(c), dev(b), m=8, rule="cc").cpu().numpy()
    B.sinc_sync()
    direct = oracle.sinc_direct(N, a, c, b, rows=rows).real
    assert np.max(np.abs(h[rows] - direct)) / np.sum(np.abs(c)) <= 1e-12


def test_sinc_rule_errors():
    a, c, b = W.sinc_inputs(10, 10, 0)
    with pytest.raises(ValueError):
        B.sinc(64, dev(a), dev(c), dev(b), rule="simpson")
    with pytest.raises(B.NNFFTError):
        B.sinc(64, dev(a), dev(c), dev(b), rule="cc", n=600000)   # 2n > 2^20
