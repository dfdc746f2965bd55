"""GPU parity of the NNFFT (forward and adjoint) against the CPU oracle.

Every case calls the CUDA library through the C ABI (Python binding) and compares
element by element with the oracle on the same seeded inputs:
  * the direct sum of eq. (1.2) (and its adjoint) with the tolerances
    ||err||_inf / ||f||_1 <= 1e-12 (fp64, m = 8, sigma = 2) and <= 2e-5 (fp32, m = 4);
  * Algorithm 2.2 step by step (oracle.nnfft_alg22), which isolates implementation
    error from the window error at small m;
  * at the full 2^20-point size, a seeded sample of output rows plus the extreme rows.
"""
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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run_forward(N, v, x, f, m, dtype, sigma=2.0):
    plan = B.Plan(N, len(v), len(x), sigma, sigma, m, m, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    y = plan.exec(dev(f, dtype))
    plan.sync()
    return y.cpu().numpy().astype(np.complex128), plan


def run_adjoint(N, v, x, g, m, dtype, sigma=2.0):
    plan = B.Plan(N, len(v), len(x), sigma, sigma, m, m, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    z = plan.adjoint(dev(g, dtype))
    plan.sync()
    return z.cpu().numpy().astype(np.complex128), plan


# ------------------------------------------------------------------------------------------
# small configurations, full comparison
# ------------------------------------------------------------------------------------------
def test_config1_plain_fp64():
    """N = 64, M1 = M2 = 128, m = 4, sigma = 2, seed 0 (complex128)."""
    v, x, f = W.nnfft_inputs(128, 128, 0)
    y, plan = run_forward(64, v, x, f, 4, torch.complex128)
    exact = oracle.nnfft_direct(64, v, f, x)
    P = oracle.make_params(64, 2, 2, 4, 4)
    alg = oracle.nnfft_alg22(P, v, f, x)
    E, _, _ = oracle.bound_sinh(P.N1, 4, 4, P.sigma1, P.sigma2)
    assert oracle.relative_error(y, exact, f) <= E
    # same algorithm as Algorithm 2.2 up to the window fit (5e-9 at m = 4) and rounding
    assert oracle.relative_error(y, alg, f) < 2e-7
    assert oracle.relative_error(y, exact, f) < 2 * oracle.relative_error(alg, exact, f) + 1e-7


@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
@pytest.mark.parametrize("N,M1,M2", [(256, 3000, 2500), (64, 1000, 333), (1000, 4097, 129)])
def test_fp64_m8_within_1e12(N, M1, M2, nodes):
    v, x, f = W.nnfft_inputs(M1, M2, 1, nodes=nodes)
    y, _ = run_forward(N, v, x, f, 8, torch.complex128)
    exact = oracle.nnfft_direct(N, v, f, x)
    assert oracle.relative_error(y, exact, f) <= 1e-12


@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_fp64_m8_matches_algorithm_2_2(nodes):
    N, M1, M2 = 200, 700, 600
    v, x, f = W.nnfft_inputs(M1, M2, 2, nodes=nodes)
    y, _ = run_forward(N, v, x, f, 8, torch.complex128)
    P = oracle.make_params(N, 2, 2, 8, 8)
    alg = oracle.nnfft_alg22(P, v, f, x)
    assert oracle.relative_error(y, alg, f) < 1e-13


@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
@pytest.mark.parametrize("N,M1,M2", [(256, 3000, 2500), (64, 128, 128), (1024, 5000, 4000)])
def test_fp32_m4_within_2e5(N, M1, M2, nodes):
    v, x, f = W.nnfft_inputs(M1, M2, 3, nodes=nodes)
    y, _ = run_forward(N, v, x, f.astype(np.complex64), 4, torch.complex64)
    exact = oracle.nnfft_direct(N, v, f.astype(np.complex64).astype(np.complex128), x)
    assert oracle.relative_error(y, exact, f) <= 2e-5


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5),
                                         (torch.complex128, 4, 1e-5)])
@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_adjoint_against_direct(dtype, m, tol, nodes):
    N, M1, M2 = 300, 2000, 1700
    v, x, _ = W.nnfft_inputs(M1, M2, 4, nodes=nodes)
    g = W.adjoint_inputs(M2, 4)
    if dtype == torch.complex64:
        g = g.astype(np.complex64).astype(np.complex128)
    z, _ = run_adjoint(N, v, x, g, m, dtype)
    exact = oracle.nnfft_adjoint_direct(N, v, x, g)
    assert oracle.relative_error(z, exact, g) <= tol


def test_adjoint_matches_transpose_of_algorithm_2_2():
    N, M1, M2 = 64, 300, 250
    v, x, _ = W.nnfft_inputs(M1, M2, 5)
    g = W.adjoint_inputs(M2, 5)
    z, _ = run_adjoint(N, v, x, g, 4, torch.complex128)
    P = oracle.make_params(N, 2, 2, 4, 4)
    za = oracle.nnfft_alg22_adjoint(P, v, x, g)
    assert oracle.relative_error(z, za, g) < 2e-7


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-13), (torch.complex64, 1e-5)])
def test_adjoint_identity_on_gpu(dtype, tol):
    """<A f, g> = <f, A^H g> for the fast maps themselves (exact transpose construction)."""
    N, M1, M2 = 512, 5000, 3000
    v, x, f = W.nnfft_inputs(M1, M2, 6, nodes="chebyshev")
    g = W.adjoint_inputs(M2, 6)
    plan = B.Plan(N, M1, M2, 2, 2, 8 if dtype == torch.complex128 else 4, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    Af = plan.exec(dev(f, dtype)).cpu().numpy().astype(np.complex128)
    Ag = plan.adjoint(dev(g, dtype)).cpu().numpy().astype(np.complex128)
    plan.sync()
    lhs = np.vdot(g, Af)
    rhs = np.vdot(Ag, f)
    assert abs(lhs - rhs) <= tol * np.sum(np.abs(f)) * np.sum(np.abs(g)) / np.sqrt(M1 * M2)


def test_linearity_and_single_coefficient():
    """One nonzero f_k gives exp(-2 pi i N v_k x_j) (a pure exponential)."""
    N, M1, M2 = 777, 50, 4000
    v, x, _ = W.nnfft_inputs(M1, M2, 7)
    f = np.zeros(M1, complex)
    f[17] = 1.0
    y, _ = run_forward(N, v, x, f, 8, torch.complex128)
    exact = oracle.nnfft_direct(N, v, f, x)
    assert np.max(np.abs(y - exact)) < 1e-12
    assert np.max(np.abs(np.abs(y) - 1)) < 1e-12


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("M1,M2", [(1, 1), (1, 37), (33, 1), (255, 257), (0, 10), (10, 0), (0, 0)])
def test_ragged_and_empty_sizes(M1, M2):
    N = 48
    v, x, f = W.nnfft_inputs(M1, M2, 8)
    g = W.adjoint_inputs(M2, 8)
    plan = B.Plan(N, M1, M2, 2, 2, 8, dtype=torch.complex128)
    plan.set_nodes(dev(v) if M1 else torch.empty(0, dtype=torch.float64, device="cuda"),
                   dev(x) if M2 else torch.empty(0, dtype=torch.float64, device="cuda"))
    y = plan.exec(dev(f, torch.complex128) if M1 else torch.empty(0, dtype=torch.complex128, device="cuda"))
    z = plan.adjoint(dev(g, torch.complex128) if M2 else torch.empty(0, dtype=torch.complex128, device="cuda"))
    plan.sync()
    if M2:
        exact = oracle.nnfft_direct(N, v, f, x) if M1 else np.zeros(M2)
        assert np.max(np.abs(y.cpu().numpy() - exact)) <= 1e-12 * max(1.0, np.sum(np.abs(f)))
    if M1:
        exact = oracle.nnfft_adjoint_direct(N, v, x, g) if M2 else np.zeros(M1)
        assert np.max(np.abs(z.cpu().numpy() - exact)) <= 1e-12 * max(1.0, np.sum(np.abs(g)))


def test_boundary_nodes_and_one_cell():
    """Nodes at exactly -1/2 and +1/2, and every node of one side in a single cell."""
    N = 100
    rng = np.random.default_rng(9)
    v = np.concatenate([[-0.5, 0.5, 0.0], 0.123 + 1e-5 * rng.random(600)])
    x = np.concatenate([[-0.5, 0.5, 0.0, 0.25], rng.uniform(-0.5, 0.5, 300)])
    f = W.draw_complex(rng, len(v))
    y, _ = run_forward(N, v, x, f, 8, torch.complex128)
    exact = oracle.nnfft_direct(N, v, f, x)
    assert oracle.relative_error(y, exact, f) <= 1e-12


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_node_edge_values(dtype, m, tol):
    """Nodes on cell boundaries (k / scale and their neighbours one ulp away), +-0,
    subnormal and tiny nodes, +-1/2: the fixed-point binning puts each in a valid cell
    with its local coordinate, so the sums match the direct sum."""
    N = 96
    info = B.params(N, 10, 10, 2.0, 2.0, m, m, "complex128")
    us1 = info["N1"] * N / info["Nstar"]
    us2 = info["N2"] * info["Nstar"] / info["N1"]
    edges1 = np.arange(-40, 41) / us1
    edges2 = np.arange(-40, 41) / us2
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-300, -1e-300, 1e-17, -1e-17, 0.5, -0.5,
                        np.nextafter(0.5, 0), np.nextafter(-0.5, 0)])
    v = np.concatenate([edges1, np.nextafter(edges1, 1), np.nextafter(edges1, -1), special])
    x = np.concatenate([edges2, np.nextafter(edges2, 1), np.nextafter(edges2, -1), special])
    v, x = np.clip(v, -0.5, 0.5), np.clip(x, -0.5, 0.5)
    rng = np.random.default_rng(12)
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    f = W.draw_complex(rng, len(v), npd)
    y, _ = run_forward(N, v, x, f, m, dtype)
    exact = oracle.nnfft_direct(N, v, f.astype(np.complex128), x)
    assert oracle.relative_error(y.astype(np.complex128), exact, f.astype(np.complex128)) <= tol
    g = W.draw_complex(rng, len(x), npd)
    z, _ = run_adjoint(N, v, x, g, m, dtype)
    exact = oracle.nnfft_adjoint_direct(N, v, x, g.astype(np.complex128))
    assert oracle.relative_error(z.astype(np.complex128), exact, g.astype(np.complex128)) <= tol


def test_heavy_cells_split_into_items():
    """Chebyshev nodes at small N put thousands of points in the edge cells (> ITEM_CAP)."""
    N, M1, M2 = 32, 60000, 50000
    v, x, f = W.nnfft_inputs(M1, M2, 10, nodes="chebyshev")
    y, _ = run_forward(N, v, x, f, 8, torch.complex128)
    rows = W.sample_rows(M2, 400, 10, extremes=[int(np.argmin(x)), int(np.argmax(x))])
    exact = oracle.nnfft_direct(N, v, f, x, rows=rows)
    assert np.max(np.abs(y[rows] - exact)) / np.sum(np.abs(f)) <= 1e-12
    g = W.adjoint_inputs(M2, 10)
    z, _ = run_adjoint(N, v, x, g, 8, torch.complex128)
    rows = W.sample_rows(M1, 400, 11, extremes=[int(np.argmin(v)), int(np.argmax(v))])
    exact = oracle.nnfft_adjoint_direct(N, v, x, g, rows=rows)
    assert np.max(np.abs(z[rows] - exact)) / np.sum(np.abs(g)) <= 1e-12


def test_unequal_parameters():
    """m1 != m2 and sigma1 != sigma2 (Section 4 recommends m2 > m1, sigma2 >= sigma1)."""
    N, M1, M2 = 300, 2000, 1500
    v, x, f = W.nnfft_inputs(M1, M2, 12)
    plan = B.Plan(N, M1, M2, 1.5, 2.5, 6, 9, dtype=torch.complex128)
    plan.set_nodes(dev(v), dev(x))
    y = plan.exec(dev(f)).cpu().numpy()
    plan.sync()
    exact = oracle.nnfft_direct(N, v, f, x)
    P = oracle.make_params(N, 1.5, 2.5, 6, 9)
    alg = oracle.nnfft_alg22(P, v, f, x)
    # Fixed tolerance against the exact-window algorithm: the plan fits each side's taps to
    # within eps_j = 1e-3 x (24 m_j^{3/2} + 10) e^{-2 pi m_j sqrt(1 - 1/sigma_j)} (the first term
    # of Theorem 4.1 for that side), and a tap error eps moves a result by at most
    # 2 eps / omegahat1(m1/(2 sigma1)) relative to ||f||_1 (2m taps of weight error eps per node,
    # divided by N1 phihat1(N/2) = m1 omegahat1(m1/(2 sigma1))).  Nothing here comes from the plan.
    eps = max(1e-3 * (24 * m ** 1.5 + 10) * np.exp(-2 * np.pi * m * np.sqrt(1 - 1 / s))
              for m, s in ((6, P.sigma1), (9, P.sigma2)))
    tol = 2 * max(eps, 1e-14) / oracle.omega_sinh_hat(6 / (2 * P.sigma1), P.beta1)
    assert tol < 2e-8
    assert oracle.relative_error(y, alg, f) <= tol
    E, _, _ = oracle.bound_sinh(P.N1, 6, 9, P.sigma1, P.sigma2)
    assert oracle.relative_error(y, exact, f) <= E


def test_deterministic_repeat():
    N, M1, M2 = 512, 20000, 20000
    v, x, f = W.nnfft_inputs(M1, M2, 13, nodes="chebyshev")
    plan = B.Plan(N, M1, M2, 2, 2, 8, dtype=torch.complex128)
    plan.set_nodes(dev(v), dev(x))
    ft = dev(f)
    y1 = plan.exec(ft).clone()
    plan.set_nodes(dev(v), dev(x))
    y2 = plan.exec(ft).clone()
    plan.sync()
    assert torch.equal(y1, y2)


def test_host_buffer_api_matches_device_api():
    N, M1, M2 = 256, 3000, 2000
    v, x, f = W.nnfft_inputs(M1, M2, 14)
    g = W.adjoint_inputs(M2, 14)
    plan = B.Plan(N, M1, M2, 2, 2, 8, dtype=torch.complex128)
    plan.set_nodes_host(v, x)
    yh = plan.exec_host(f)
    zh = plan.adjoint_host(g)
    plan.set_nodes(dev(v), dev(x))
    yd = plan.exec(dev(f)).cpu().numpy()
    zd = plan.adjoint(dev(g)).cpu().numpy()
    plan.sync()
    assert np.array_equal(yh, yd) and np.array_equal(zh, zd)


# ------------------------------------------------------------------------------------------
# error reporting
# ------------------------------------------------------------------------------------------
def test_out_of_range_and_nan_nodes_report_erange():
    for bad in (0.5000001, -0.75, np.nan):
        v = np.array([0.1, bad, -0.2])
        x = np.array([0.0, 0.3])
        plan = B.Plan(32, 3, 2, 2, 2, 4, dtype=torch.complex128)
        plan.set_nodes(dev(v), dev(x))
        plan.exec(dev(np.ones(3, complex)))
        with pytest.raises(B.NNFFTError) as ei:
            plan.sync()
        assert ei.value.code == 2
        plan.sync()   # status is cleared after being reported


def test_exec_before_set_nodes_is_a_state_error():
    plan = B.Plan(32, 3, 2, 2, 2, 4, dtype=torch.complex128)
    with pytest.raises(B.NNFFTError) as ei:
        plan.exec(dev(np.ones(3, complex)))
    assert ei.value.code == 6


def test_wrong_tensor_types_rejected():
    plan = B.Plan(32, 3, 2, 2, 2, 4, dtype=torch.complex128)
    with pytest.raises(TypeError):
        plan.set_nodes(torch.zeros(3, dtype=torch.float32, device="cuda"), None)
    with pytest.raises(ValueError):
        plan.set_nodes(torch.zeros(4, dtype=torch.float64, device="cuda"), None)


# ------------------------------------------------------------------------------------------
# the full-size workload: N = 4096, M1 = M2 = 2^20, sigma = 2, m = 8 (fp64) and m = 4 (fp32)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_full_size_fp64_sampled_rows(nodes):
    N, M = 4096, 1 << 20
    v, x, f = W.nnfft_inputs(M, M, 0, nodes=nodes)
    g = W.adjoint_inputs(M, 0)
    plan = B.Plan(N, M, M, 2, 2, 8, dtype=torch.complex128)
    plan.set_nodes(dev(v), dev(x))
    y = plan.exec(dev(f)).cpu().numpy()
    z = plan.adjoint(dev(g)).cpu().numpy()
    plan.sync()
    rows = W.sample_rows(M, 96, 1, extremes=[int(np.argmin(x)), int(np.argmax(x))])
    exact = oracle.nnfft_direct(N, v, f, x, rows=rows)
    assert np.max(np.abs(y[rows] - exact)) / np.sum(np.abs(f)) <= 1e-12
    rows = W.sample_rows(M, 96, 2, extremes=[int(np.argmin(v)), int(np.argmax(v))])
    exact = oracle.nnfft_adjoint_direct(N, v, x, g, rows=rows)
    assert np.max(np.abs(z[rows] - exact)) / np.sum(np.abs(g)) <= 1e-12


def test_full_size_fp32_sampled_rows():
    N, M = 4096, 1 << 20
    v, x, f = W.nnfft_inputs(M, M, 0, dtype=np.complex64)
    plan = B.Plan(N, M, M, 2, 2, 4, dtype=torch.complex64)
    plan.set_nodes(dev(v), dev(x))
    y = plan.exec(dev(f)).cpu().numpy().astype(np.complex128)
    plan.sync()
    rows = W.sample_rows(M, 96, 3)
    exact = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows)
    assert np.max(np.abs(y[rows] - exact)) / np.sum(np.abs(f)) <= 2e-5


# ------------------------------------------------------------------------------------------
# fp64 arithmetic modes: native FP64 and split precision (double-float + FP32 by degree)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_fp64_native_and_split_modes(nodes):
    N, M1, M2 = 1024, 20000, 15000
    v, x, f = W.nnfft_inputs(M1, M2, 30, nodes=nodes)
    g = W.adjoint_inputs(M2, 30)
    rows_y = W.sample_rows(M2, 300, 30)
    rows_z = W.sample_rows(M1, 300, 31)
    ey = oracle.nnfft_direct(N, v, f, x, rows=rows_y)
    ez = oracle.nnfft_adjoint_direct(N, v, x, g, rows=rows_z)
    out = {}
    for arith in (B.ARITH_FP64, B.ARITH_FP64_SPLIT):
        plan = B.Plan(N, M1, M2, 2, 2, 8, dtype=torch.complex128)
        assert plan.info["arith"] == B.ARITH_FP64_SPLIT      # the default when available
        plan.set_arith(arith)
        assert plan.info["arith"] == arith
        plan.set_nodes(dev(v), dev(x))
        y = plan.exec(dev(f)).cpu().numpy()
        z = plan.adjoint(dev(g)).cpu().numpy()
        plan.sync()
        assert np.max(np.abs(y[rows_y] - ey)) / np.sum(np.abs(f)) <= 1e-12
        assert np.max(np.abs(z[rows_z] - ez)) / np.sum(np.abs(g)) <= 1e-12
        out[arith] = (y, z)
    (y1, z1), (y2, z2) = out[B.ARITH_FP64], out[B.ARITH_FP64_SPLIT]
    assert np.max(np.abs(y1 - y2)) / np.sum(np.abs(f)) <= 1e-13
    assert np.max(np.abs(z1 - z2)) / np.sum(np.abs(g)) <= 1e-13


def test_set_arith_requires_new_nodes_and_rejects_fp32():
    plan = B.Plan(64, 10, 10, 2, 2, 8, dtype=torch.complex128)
    v, x, f = W.nnfft_inputs(10, 10, 31)
    plan.set_nodes(dev(v), dev(x))
    plan.set_arith(B.ARITH_FP64)
    with pytest.raises(B.NNFFTError) as ei:
        plan.exec(dev(f))
    assert ei.value.code == 6
    p32 = B.Plan(64, 10, 10, 2, 2, 4, dtype=torch.complex64)
    assert p32.info["arith"] == B.ARITH_FP32
    with pytest.raises(B.NNFFTError):
        p32.set_arith(B.ARITH_FP64_SPLIT)


@pytest.mark.parametrize("dtype,m", [(torch.complex128, 8), (torch.complex64, 4)])
def test_exec_adjoint_concurrent_equals_separate(dtype, m):
    """nnfft_exec_adjoint (both directions on two streams) gives bit for bit the results of
    nnfft_exec and nnfft_adjoint, for a single plan and a batch."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M1, M2 = 300, 20000, 15000
    v, x, f = W.nnfft_inputs(M1, M2, 31, dtype=npd)
    g = W.adjoint_inputs(M2, 31, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    y1 = plan.exec(dev(f, dtype)).cpu().numpy()
    z1 = plan.adjoint(dev(g, dtype)).cpu().numpy()
    y2, z2 = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
    plan.sync()
    assert np.array_equal(y1, y2.cpu().numpy()) and np.array_equal(z1, z2.cpu().numpy())
    Nb, M1b, M2b = np.array([64, 500, 33]), np.array([1000, 3000, 10]), np.array([2000, 5, 700])
    vb, xb, fb = W.batch_inputs(M1b, M2b, 32, dtype=npd)
    gb = W.draw_complex(np.random.default_rng(3), int(M2b.sum()), npd)
    P = B.BatchPlan(Nb, M1b, M2b, 2.0, 2.0, m, dtype=dtype)
    P.set_nodes(dev(vb), dev(xb))
    y1, z1 = P.exec(dev(fb, dtype)).cpu().numpy(), P.adjoint(dev(gb, dtype)).cpu().numpy()
    y2, z2 = P.exec_adjoint(dev(fb, dtype), dev(gb, dtype))
    P.sync()
    assert np.array_equal(y1, y2.cpu().numpy()) and np.array_equal(z1, z2.cpu().numpy())


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_autotune_keeps_results_within_tolerance(dtype, m, tol):
    """nnfft_autotune picks among the kernel variants; every variant is a correct transform
    (within tolerance of the direct sum, deterministic), and the choice is reported."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M1, M2 = 500, 30000, 20000
    v, x, f = W.nnfft_inputs(M1, M2, 41, dtype=npd)
    g = W.adjoint_inputs(M2, 41, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    t = plan.autotune(dev(f, dtype), dev(g, dtype), reps=2)
    assert t["tuned"] == 1 and t["moments_lanes_v"] in (4, 8, 16, 32) and t["moments_lanes_x"] in (4, 8, 16, 32)
    assert t["eval_lanes_v"] in (1, 2, 3, 8, 32) and t["eval_lanes_x"] in (1, 2, 3, 8, 32)
    assert t["fft_variant"] in (0, 1, 2, 3) and 0 < t["best_ms"] <= 1.1 * t["default_ms"]
    assert t["timed_transform"] == 0
    t = plan.autotune(dev(f, dtype), dev(g, dtype), reps=1, v=dev(v), x=dev(x), flush_l2=True)
    assert t["timed_transform"] == 1 and t["item_split"] in (0, 1)
    assert t["item_cap"] in (32, 64, 128, 256) and 0 < t["best_ms"] <= 1.1 * t["default_ms"]
    y1, z1 = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
    y2, z2 = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
    plan.sync()
    y1, z1 = y1.cpu().numpy(), z1.cpu().numpy()
    assert np.array_equal(y1, y2.cpu().numpy()) and np.array_equal(z1, z2.cpu().numpy())
    rows = W.sample_rows(M2, 64, 3)
    want = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows)
    assert np.max(np.abs(y1[rows] - want)) / np.sum(np.abs(f)) <= tol
    rows = W.sample_rows(M1, 64, 4)
    want = oracle.nnfft_adjoint_direct(N, v, x, g.astype(np.complex128), rows=rows)
    assert np.max(np.abs(z1[rows] - want)) / np.sum(np.abs(g)) <= tol


def test_every_moments_and_fft_variant_is_correct():
    """Both split-precision moments kernels (16 and 32 lanes per item) and both FFT
    packings give the transform within 1e-12, forward and adjoint."""
    N, M1, M2 = 700, 40000, 30000
    v, x, f = W.nnfft_inputs(M1, M2, 43)
    g = W.adjoint_inputs(M2, 43)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, 8, 8)
    plan.set_nodes(dev(v), dev(x))
    rows2, rows1 = W.sample_rows(M2, 48, 5), W.sample_rows(M1, 48, 6)
    want_y = oracle.nnfft_direct(N, v, f, x, rows=rows2)
    want_z = oracle.nnfft_adjoint_direct(N, v, x, g, rows=rows1)
    for lanes, fv, split, el in ((16, 0, 1, 32), (16, 1, 0, 8), (32, 0, 0, 32), (32, 1, 1, 8),
                                 (8, 0, 0, 8), (8, 1, 1, 32), (4, 0, 0, 1), (4, 2, 1, 2),
                                 (8, 2, 0, 32)):
        plan.set_tuning(lanes, lanes, fv, split, el, el)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f), dev(g))
        plan.sync()
        y, z = y.cpu().numpy(), z.cpu().numpy()
        assert np.max(np.abs(y[rows2] - want_y)) / np.sum(np.abs(f)) <= 1e-12, (lanes, fv)
        assert np.max(np.abs(z[rows1] - want_z)) / np.sum(np.abs(g)) <= 1e-12, (lanes, fv)


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_small_item_split_on_and_off(dtype, m, tol):
    """Sparse nodes (few points per cell) take the one-thread-per-item kernels when
    item_split is on; both settings give the transform within tolerance."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M1, M2 = 4000, 3000, 5000                 # about 0.4-0.6 points per cell
    v, x, f = W.nnfft_inputs(M1, M2, 71, dtype=npd)
    g = W.adjoint_inputs(M2, 71, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    want_y = oracle.nnfft_direct(N, v, f.astype(np.complex128), x)
    want_z = oracle.nnfft_adjoint_direct(N, v, x, g.astype(np.complex128))
    for split in (1, 0):
        plan.set_tuning(32, 32, 0, split)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
        plan.sync()
        assert oracle.relative_error(y.cpu().numpy().astype(np.complex128), want_y, f) <= tol
        assert oracle.relative_error(z.cpu().numpy().astype(np.complex128), want_z, g) <= tol


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_transform_host_equals_separate_host_calls(dtype):
    """nnfft_transform_host (overlapped uploads, both directions concurrently) returns
    bit for bit what set_nodes_host + exec_host + adjoint_host return; either direction
    can be skipped; a node out of range reports ERANGE."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    m = 8 if dtype == torch.complex128 else 4
    N, M1, M2 = 800, 50000, 40000
    v, x, f = W.nnfft_inputs(M1, M2, 51, dtype=npd)
    g = W.adjoint_inputs(M2, 51, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    plan.set_nodes_host(v, x)
    y1, z1 = plan.exec_host(f), plan.adjoint_host(g)
    y2, z2 = plan.transform_host(v, x, f, g)
    assert np.array_equal(y1, y2) and np.array_equal(z1, z2)
    y3, z3 = plan.transform_host(v, x, f=f)
    assert np.array_equal(y1, y3) and z3 is None
    y4, z4 = plan.transform_host(v, x, g=g)
    assert y4 is None and np.array_equal(z1, z4)
    vb = v.copy()
    vb[7] = 0.6
    with pytest.raises(B.NNFFTError) as e:
        plan.transform_host(vb, x, f, g)
    assert e.value.code == 2


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_transform_host_graph_replays_the_host_transform(dtype):
    """nnfft_transform_host_graph over page-locked host arrays: each launch uploads the
    arrays' current contents and returns bit for bit what nnfft_transform_host returns on
    them (new nodes and values written in place between launches); one direction alone; a
    pageable array is rejected with EINVAL; a node out of range reports ERANGE at sync."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    m = 8 if dtype == torch.complex128 else 4
    N, M1, M2 = 700, 30000, 20000
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    v, x, f = (pin(a) for a in W.nnfft_inputs(M1, M2, 61, dtype=npd))
    g = pin(W.adjoint_inputs(M2, 61, dtype=npd))
    y, z = pin(np.zeros(M2, npd)), pin(np.zeros(M1, npd))
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    graph = plan.transform_host_graph(v, x, f, g, y, z)
    assert graph.kernels > 0
    for seed in (61, 62):
        v2, x2, f2 = W.nnfft_inputs(M1, M2, seed, dtype=npd)
        v[:], x[:], f[:], g[:] = v2, x2, f2, W.adjoint_inputs(M2, seed, dtype=npd)
        graph.launch()
        plan.sync()
        want_y, want_z = plan.transform_host(v.copy(), x.copy(), f.copy(), g.copy())
        assert np.array_equal(y, want_y) and np.array_equal(z, want_z)
    one = plan.transform_host_graph(v, x, f=f)
    y1 = one.launch()[0]
    plan.sync()
    assert np.array_equal(y1, plan.transform_host(v.copy(), x.copy(), f=f.copy())[0])
    with pytest.raises(B.NNFFTError) as e:
        plan.transform_host_graph(v.copy(), x, f, g, y, z)       # pageable v
    assert e.value.code == 1
    v[5] = 0.75
    graph.launch()
    with pytest.raises(B.NNFFTError) as e:
        plan.sync()
    assert e.value.code == 2
    one.close()
    graph.close()
    plan.close()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_transform_device_equals_separate_calls(dtype):
    """nnfft_transform (sorts and both directions overlapped, device buffers) returns bit
    for bit set_nodes + exec + adjoint, for a single plan and a batch; directions can be
    skipped."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    m = 8 if dtype == torch.complex128 else 4
    N, M1, M2 = 900, 60000, 30000
    v, x, f = W.nnfft_inputs(M1, M2, 61, dtype=npd)
    g = W.adjoint_inputs(M2, 61, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    y1 = plan.exec(dev(f, dtype)).cpu().numpy()
    z1 = plan.adjoint(dev(g, dtype)).cpu().numpy()
    y2, z2 = plan.transform(dev(v), dev(x), dev(f, dtype), dev(g, dtype))
    y3, _ = plan.transform(dev(v), dev(x), f=dev(f, dtype))
    _, z4 = plan.transform(dev(v), dev(x), g=dev(g, dtype))
    plan.sync()
    assert np.array_equal(y1, y2.cpu().numpy()) and np.array_equal(z1, z2.cpu().numpy())
    assert np.array_equal(y1, y3.cpu().numpy()) and np.array_equal(z1, z4.cpu().numpy())
    Nb, M1b, M2b = np.array([100, 2000, 50]), np.array([4000, 100, 900]), np.array([300, 5000, 1])
    vb, xb, fb = W.batch_inputs(M1b, M2b, 62, dtype=npd)
    gb = W.draw_complex(np.random.default_rng(9), int(M2b.sum()), npd)
    P = B.BatchPlan(Nb, M1b, M2b, 2.0, 2.0, m, dtype=dtype)
    P.set_nodes(dev(vb), dev(xb))
    y1, z1 = P.exec(dev(fb, dtype)).cpu().numpy(), P.adjoint(dev(gb, dtype)).cpu().numpy()
    y2, z2 = P.transform(dev(vb), dev(xb), dev(fb, dtype), dev(gb, dtype))
    P.sync()
    assert np.array_equal(y1, y2.cpu().numpy()) and np.array_equal(z1, z2.cpu().numpy())


@pytest.mark.parametrize("sigma", [1.25, 1.5, 2.0])
def test_figure_4_1b_protocol(sigma):
    """The Fig. 4.1(b) experiment with the sinh window itself: N = 1200, m1 = m2 = m in
    2..8, sigma1 = sigma2, M1 = 2400, M2 = 1600, x uniform in [-1/2, 1/2], v uniform in
    [-1/(2a), 1/(2a)] with a = 1 + 2m/N1, complex N(0,1) coefficients, 100 repetitions as in
    the paper; the maximum over the repetitions of the error eq. (4.5) lies below the
    bound E(phi_sinh) of Theorem 4.1 and falls with m."""
    N, M1, M2, reps = 1200, 2400, 1600, 100
    worst = {}
    for m in range(2, 9):
        P = oracle.make_params(N, sigma, sigma, m, m)
        a = 1.0 + 2.0 * m / P.N1
        E, _, _ = oracle.bound_sinh(P.N1, m, m, P.sigma1, P.sigma2)
        plan = B.Plan(N, M1, M2, sigma, sigma, m, m, dtype=torch.complex128)
        err = 0.0
        for rep in range(reps):
            rng = np.random.default_rng(1000 * m + rep)
            x = rng.uniform(-0.5, 0.5, M2)
            v = rng.uniform(-0.5 / a, 0.5 / a, M1)
            f = rng.standard_normal(M1) + 1j * rng.standard_normal(M1)
            plan.set_nodes(dev(v), dev(x))
            y = plan.exec(dev(f)).cpu().numpy()
            err = max(err, oracle.relative_error(y, oracle.nnfft_direct(N, v, f, x), f))
        plan.sync()
        worst[m] = err
        assert err <= E, (sigma, m, err, E)
    assert worst[8] < 1e-3 * worst[2]


@pytest.mark.parametrize("dtype,arith,m,tol", [(torch.complex64, None, 4, 2e-5),
                                               (torch.complex128, "fp64", 8, 1e-12)])
@pytest.mark.parametrize("N,M1,M2", [(300, 40000, 30000), (3000, 2500, 3500)])
def test_team_kernels_eight_lanes_per_item(dtype, arith, m, tol, N, M1, M2):
    """The all-real moments and evaluation kernels with 8 lanes per work item (four items
    per warp) against the direct sums, dense (~60 points per cell) and sparse (< 1)."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.nnfft_inputs(M1, M2, 81, dtype=npd)
    g = W.adjoint_inputs(M2, 81, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    if arith == "fp64":
        plan.set_arith(B.ARITH_FP64)
    rows2, rows1 = W.sample_rows(M2, 64, 7), W.sample_rows(M1, 64, 8)
    want_y = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows2)
    want_z = oracle.nnfft_adjoint_direct(N, v, x, g.astype(np.complex128), rows=rows1)
    for ml, el in ((8, 8), (8, 32), (32, 8)):
        plan.set_tuning(ml, ml, 0, 0, el, el)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
        plan.sync()
        y, z = y.cpu().numpy().astype(np.complex128), z.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(y[rows2] - want_y)) / np.sum(np.abs(f)) <= tol, (ml, el)
        assert np.max(np.abs(z[rows1] - want_z)) / np.sum(np.abs(g)) <= tol, (ml, el)


@pytest.mark.parametrize("dtype,arith,m,tol", [(torch.complex64, None, 4, 2e-5),
                                               (torch.complex128, "fp64", 8, 1e-12),
                                               (torch.complex128, None, 8, 1e-12)])
@pytest.mark.parametrize("N,M1,M2", [(300, 40000, 30000), (3000, 2500, 3500)])
def test_flat_evaluation_equals_item_evaluation(dtype, arith, m, tol, N, M1, M2):
    """The flat evaluation kernels (one thread per sorted point, cell from the sorted keys)
    compute each point exactly as the per-item kernels do: bitwise equal outputs for every
    arithmetic path, dense and sparse cells, and within tolerance of the direct sums; with
    a reduced active size (set_sizes) only the active points are written."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.nnfft_inputs(M1, M2, 91, dtype=npd)
    g = W.adjoint_inputs(M2, 91, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    if arith == "fp64":
        plan.set_arith(B.ARITH_FP64)
    outs = {}
    for el in (32, 8, 1, 2):                   # 2: flat with TMA-staged cell tiles
        plan.set_tuning(32, 32, 0, 0, el, el)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
        plan.sync()
        outs[el] = (y.cpu().numpy(), z.cpu().numpy())
    for el in (8, 1, 2):
        assert np.array_equal(outs[el][0], outs[32][0]) and np.array_equal(outs[el][1], outs[32][1]), el
    rows2, rows1 = W.sample_rows(M2, 64, 9), W.sample_rows(M1, 64, 10)
    y, z = (a.astype(np.complex128) for a in outs[1])
    want_y = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows2)
    want_z = oracle.nnfft_adjoint_direct(N, v, x, g.astype(np.complex128), rows=rows1)
    assert np.max(np.abs(y[rows2] - want_y)) / np.sum(np.abs(f)) <= tol
    assert np.max(np.abs(z[rows1] - want_z)) / np.sum(np.abs(g)) <= tol
    # reduced active sizes: the flat kernels cover exactly the active points
    m1, m2 = M1 // 3, M2 // 2
    plan.set_sizes(m1, m2)
    for el in (1, 2):
        plan.set_tuning(32, 32, 0, 0, el, el)
        plan.set_nodes(dev(v[:m1]), dev(x[:m2]))
        sentinel = torch.full((M2,), 7.0 + 7.0j, dtype=dtype, device="cuda")
        plan.exec(dev(f[:m1], dtype), out=sentinel[:m2])
        plan.sync()
        ys = sentinel.cpu().numpy()
        assert np.all(ys[m2:] == 7.0 + 7.0j)
        rows = W.sample_rows(m2, 32, 11)
        want = oracle.nnfft_direct(N, v[:m1], f[:m1].astype(np.complex128), x[:m2], rows=rows)
        assert np.max(np.abs(ys[:m2][rows].astype(np.complex128) - want)) / np.sum(np.abs(f[:m1])) <= tol


def test_bulk_copy_waits_are_bounded():
    """The bulk (TMA) copy helpers: a staged copy arrives intact; a barrier armed for bytes
    that never come gives up after its cycle limit, sets the timeout bit (4) and leaves the
    context usable (the next copy works)."""
    src = torch.arange(4096, dtype=torch.float32, device="cuda")
    dst, st = B.selftest_bulk_copy(src)
    assert st == 0 and torch.equal(dst, src)
    dst, st = B.selftest_bulk_copy(src, arm_only=True, limit_cycles=2_000_000)
    assert st == 4 and not torch.any(dst)
    dst, st = B.selftest_bulk_copy(src[:1000])
    assert st == 0 and torch.equal(dst, src[:1000])


@pytest.mark.parametrize("dtype,m", [(torch.complex128, 8), (torch.complex64, 4)])
def test_transform_graph_replays_the_transform(dtype, m):
    """A captured transform (CUDA graph) replays set_nodes + forward + adjoint: bitwise the
    result of nnfft_transform on the same buffers; new contents written into the buffers
    are used by the next replay; every replay counts its kernels."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M1, M2 = 600, 30000, 20000
    v, x, f = W.nnfft_inputs(M1, M2, 95, dtype=npd)
    g = W.adjoint_inputs(M2, 95, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    vd, xd, fd, gd = dev(v), dev(x), dev(f, dtype), dev(g, dtype)
    y0, z0 = plan.transform(vd, xd, fd, gd)
    plan.sync()
    y0, z0 = y0.cpu().numpy(), z0.cpu().numpy()
    gr = plan.transform_graph(vd, xd, fd, gd)
    assert gr.kernels > 10
    l0 = B.launch_count()
    y, z = gr.launch()
    plan.sync()
    assert B.launch_count() - l0 == gr.kernels
    assert np.array_equal(y.cpu().numpy(), y0) and np.array_equal(z.cpu().numpy(), z0)
    # new nodes and values in the same buffers
    v2, x2, f2 = W.nnfft_inputs(M1, M2, 96, dtype=npd)
    g2 = W.adjoint_inputs(M2, 96, dtype=npd)
    vd.copy_(dev(v2)); xd.copy_(dev(x2)); fd.copy_(dev(f2, dtype)); gd.copy_(dev(g2, dtype))
    gr.launch()
    plan.sync()
    y2, z2 = y.cpu().numpy().astype(np.complex128), z.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if dtype == torch.complex128 else 2e-5
    rows2, rows1 = W.sample_rows(M2, 32, 12), W.sample_rows(M1, 32, 13)
    want_y = oracle.nnfft_direct(N, v2, f2.astype(np.complex128), x2, rows=rows2)
    want_z = oracle.nnfft_adjoint_direct(N, v2, x2, g2.astype(np.complex128), rows=rows1)
    assert np.max(np.abs(y2[rows2] - want_y)) / np.sum(np.abs(f2)) <= tol
    assert np.max(np.abs(z2[rows1] - want_z)) / np.sum(np.abs(g2)) <= tol
    gr.close()
    with pytest.raises(B.NNFFTError):
        gr.launch()
    plan.close()


def test_transform_graph_batch_plan():
    N, M1, M2 = np.array([64, 300, 7]), np.array([500, 2000, 1]), np.array([400, 0, 90])
    v, x, f = W.batch_inputs(M1, M2, 97)
    g = W.draw_complex(np.random.default_rng(98), int(M2.sum()), np.complex128)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, 8)
    vd, xd, fd, gd = dev(v), dev(x), dev(f), dev(g)
    y0, z0 = P.transform(vd, xd, fd, gd)
    P.sync()
    y0, z0 = y0.cpu().numpy(), z0.cpu().numpy()
    gr = P.transform_graph(vd, xd, fd, gd)
    y, z = gr.launch()
    gr.launch()
    P.sync()
    assert np.array_equal(y.cpu().numpy(), y0) and np.array_equal(z.cpu().numpy(), z0)
    P.close()


def test_fixed_point_coordinate_conversion_error_bounds():
    """The node kernel builds the fp32 coordinate and the split plans' float pair from the
    fixed-point value Y (y = Y 2^-63) with 32-bit conversions: the float is within
    2^-31 + half an ulp of y, the pair within 2^-49 + 2^-56 and normalised (|l| <= ulp(h)/2),
    for edge values (0, +-1, -2^63, powers of two +- 1, rounding ties at 24 and 32 bits) and
    random values of every magnitude, checked in exact rational arithmetic."""
    from fractions import Fraction
    rng = np.random.default_rng(123)
    edge = [0, 1, -1, 2**63 - 1, -2**63, -2**63 + 1, 2**62, -2**62]
    for k in range(0, 63):
        for d in (-1, 0, 1):
            edge += [2**k + d, -(2**k + d)]
    for k in range(25, 63):                      # ties and neighbours at 24 bits
        base = (2**23 + 1) << (k - 23)
        half = 1 << (k - 24)
        edge += [base + half, base + half - 1, base + half + 1, -(base + half), base - half]
    for t in (2**31 - 1, 2**31 - 64, 2**31 - 65, -2**31, -2**31 + 64, 2**24 + 1, -(2**24 + 1)):
        for low in (0, 1, 2**31, 2**32 - 1):     # top words that round up to 2^31 and others
            edge.append(t * 2**32 + low)
    edge = [e for e in edge if -2**63 <= e < 2**63]
    mags = rng.integers(0, 63, 20000)
    rand = (rng.integers(0, 2**62, 20000, dtype=np.int64) >> (62 - mags).astype(np.int64))
    rand *= np.where(rng.random(20000) < 0.5, -1, 1)
    y = np.concatenate([np.array(edge, dtype=np.int64), rand.astype(np.int64)])
    out = B.selftest_fixed63(torch.from_numpy(y).cuda()).cpu().numpy()
    b_single = Fraction(1, 2**31)
    b_pair = Fraction(1, 2**49) + Fraction(1, 2**56)
    for v, (f, h, lo, ref) in zip(y.tolist(), out.tolist()):
        exact = Fraction(int(v), 2**63)
        assert abs(Fraction(f) - exact) < b_single + Fraction(float(np.spacing(np.float32(abs(f))))) / 2
        assert abs(Fraction(h) + Fraction(lo) - exact) <= b_pair
        assert h == 0 or abs(lo) <= float(np.spacing(np.float32(abs(h)))) / 2
        assert abs(Fraction(ref) - exact) <= Fraction(float(np.spacing(np.float32(abs(ref))))) / 2


@pytest.mark.parametrize("dtype,arith,m,tol", [(torch.complex64, None, 4, 2e-5),
                                               (torch.complex128, "fp64", 8, 1e-12),
                                               (torch.complex128, None, 8, 1e-12)])
def test_item_caps(dtype, arith, m, tol):
    """Work items of at most 256, 128, 64 or 32 points: the transform within tolerance of the
    direct sums for each cap and moments width, on dense cells (~60 points per cell) and
    on nodes crowded into a few cells (thousands of points: one cell becomes many items);
    repeated runs bitwise equal; an invalid cap is rejected."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M1, M2 = 300, 40000, 30000
    v, x, f = W.nnfft_inputs(M1, M2, 101, dtype=npd)
    g = W.adjoint_inputs(M2, 101, dtype=npd)
    rng = np.random.default_rng(102)
    vc = (rng.random(M1) * 2e-3 - 1e-3) + 0.25          # a few cells hold all v nodes
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    if arith == "fp64":
        plan.set_arith(B.ARITH_FP64)
    rows2, rows1 = W.sample_rows(M2, 48, 14), W.sample_rows(M1, 48, 15)
    for nodes_v in (v, vc):
        want_y = oracle.nnfft_direct(N, nodes_v, f.astype(np.complex128), x, rows=rows2)
        want_z = oracle.nnfft_adjoint_direct(N, nodes_v, x, g.astype(np.complex128), rows=rows1)
        for cap in (256, 128, 64, 32):
            for ml in (32, 8):
                plan.set_tuning(ml, ml, 0, 0, 1, 1, item_cap=cap)
                plan.set_nodes(dev(nodes_v), dev(x))
                y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
                y2, z2 = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
                plan.sync()
                assert plan.tuning()["item_cap"] == cap
                y, z = y.cpu().numpy(), z.cpu().numpy()
                assert np.array_equal(y, y2.cpu().numpy()) and np.array_equal(z, z2.cpu().numpy())
                y, z = y.astype(np.complex128), z.astype(np.complex128)
                assert np.max(np.abs(y[rows2] - want_y)) / np.sum(np.abs(f)) <= tol, (cap, ml)
                assert np.max(np.abs(z[rows1] - want_z)) / np.sum(np.abs(g)) <= tol, (cap, ml)
    with pytest.raises(B.NNFFTError):
        plan.set_tuning(32, 32, 0, 0, 32, 32, item_cap=48)


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_equispaced_special_cases(dtype, m, tol):
    """The NNFFT's equispaced special cases, checked with numpy alone: v_k = k/N gives the
    NFFT y_j = sum_k f_k e^{-2 pi i k x_j}; x_j = j/N gives its transpose
    y_j = sum_k f_k e^{-2 pi i j v_k}; both equispaced give a length-N DFT (numpy FFT)."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N = 256
    k = np.arange(-N // 2, N // 2)
    grid = k / N
    rng = np.random.default_rng(103)
    xr = rng.uniform(-0.5, 0.5, 3000)
    vr = rng.uniform(-0.5, 0.5, 3000)
    fN = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(npd)
    fM = (rng.standard_normal(3000) + 1j * rng.standard_normal(3000)).astype(npd)

    def run(v, x, f):
        plan = B.Plan(N, len(v), len(x), 2.0, 2.0, m, m, dtype=dtype)
        plan.set_nodes(dev(v), dev(x))
        y = plan.exec(dev(f, dtype))
        plan.sync()
        return y.cpu().numpy().astype(np.complex128)

    f = fN.astype(np.complex128)
    want = np.exp(-2j * np.pi * np.outer(xr, k)) @ f                  # NFFT
    assert np.max(np.abs(run(grid, xr, fN) - want)) / np.sum(np.abs(f)) <= tol
    f = fM.astype(np.complex128)
    want = np.exp(-2j * np.pi * np.outer(k, vr)) @ f                  # transposed NFFT
    assert np.max(np.abs(run(vr, grid, fM) - want)) / np.sum(np.abs(f)) <= tol
    f = fN.astype(np.complex128)
    # y_j = sum_k f_k e^{-2 pi i k j / N}, k, j in I_N: a DFT of the coefficients reordered
    # to k mod N, read back at j mod N
    want = np.fft.fft(np.fft.ifftshift(f))[np.arange(-N // 2, N // 2) % N]
    assert np.max(np.abs(run(grid, grid, fN) - want)) / np.sum(np.abs(f)) <= tol


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_large_sort_sampled_rows(dtype, m, tol):
    """More than 2^23 points per side (the size from which the radix scatter ranks digits
    with match instructions): sampled rows of the forward and adjoint against the direct
    sums."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M = 1024, (1 << 23) + 12345
    v, x, f = W.nnfft_inputs(M, M, 105, dtype=npd)
    g = W.adjoint_inputs(M, 105, dtype=npd)
    plan = B.Plan(N, M, M, 2.0, 2.0, m, m, dtype=dtype)
    plan.set_nodes(dev(v), dev(x))
    y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
    plan.sync()
    y, z = y.cpu().numpy().astype(np.complex128), z.cpu().numpy().astype(np.complex128)
    rows = W.sample_rows(M, 16, 16)
    want = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows)
    assert np.max(np.abs(y[rows] - want)) / np.sum(np.abs(f)) <= tol
    want = oracle.nnfft_adjoint_direct(N, v, x, g.astype(np.complex128), rows=rows)
    assert np.max(np.abs(z[rows] - want)) / np.sum(np.abs(g)) <= tol
    plan.close()


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_three_pass_sort(dtype, m, tol, nodes):
    """A bandwidth whose cells need 17-bit keys (N = 40000: ~80K cells on the v side,
    three radix passes: 8 + 8 + 1 bits where the last pass gathers 8-byte coordinates,
    5 + 6 + 6 where 4-byte ones travel with the keys), forward and adjoint in full against
    the direct sums."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    N, M1, M2 = 40000, 6000, 5000
    v, x, f = W.nnfft_inputs(M1, M2, 106, nodes=nodes, dtype=npd)
    g = W.adjoint_inputs(M2, 106, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    assert plan.info["K1"] > 1 << 16
    plan.set_nodes(dev(v), dev(x))
    y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
    plan.sync()
    y, z = y.cpu().numpy().astype(np.complex128), z.cpu().numpy().astype(np.complex128)
    f64, g64 = f.astype(np.complex128), g.astype(np.complex128)
    assert oracle.relative_error(y, oracle.nnfft_direct(N, v, f64, x), f64) <= tol
    assert oracle.relative_error(z, oracle.nnfft_adjoint_direct(N, v, x, g64), g64) <= tol
    plan.close()


@pytest.mark.parametrize("dtype,arith,m", [(torch.complex128, None, 8), (torch.complex128, "fp64", 8),
                                           (torch.complex64, None, 4)])
@pytest.mark.parametrize("N,M1,M2,nodes", [(4096, 300000, 200001, "chebyshev"),
                                            (700, 80000, 50000, "uniform"),
                                            (3000, 5000, 4000, "uniform"),
                                            (300, 60000, 3, "chebyshev")])
def test_two_stage_sort_equals_lsd_sort(dtype, arith, m, N, M1, M2, nodes):
    """The two-stage node sort (high-digit scatter, then a shared-memory sort per bucket that
    also writes the cell offsets and work items) orders the nodes exactly as the LSD radix
    passes: the transforms are bitwise equal.  Cases: clustered nodes whose edge buckets
    span several shared-memory chunks and hold cells above the item cap, dense uniform
    nodes (one item per cell), sparse nodes (scan-built items), a side of three points."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.nnfft_inputs(M1, M2, 95, nodes=nodes, dtype=npd)
    g = W.adjoint_inputs(M2, 95, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    if arith == "fp64":
        plan.set_arith(B.ARITH_FP64)
    outs = []
    for lsd in (1, 0):
        plan.set_tuning(32, 32, 0, 0, 32, 32, sort_lsd=lsd)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f, dtype), dev(g, dtype))
        plan.sync()
        outs.append((y.cpu().numpy(), z.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    tol = 1e-12 if dtype == torch.complex128 else 2e-5
    rows2 = W.sample_rows(M2, 48, 12, extremes=[int(np.argmin(x)), int(np.argmax(x))])
    want = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows2)
    assert np.max(np.abs(outs[1][0][rows2].astype(np.complex128) - want)) / np.sum(np.abs(f)) <= tol


@pytest.mark.parametrize("dtype,m", [(torch.complex128, 8), (torch.complex64, 4)])
@pytest.mark.parametrize("N,M1,M2,nodes", [(4096, 300000, 200001, "chebyshev"),
                                            (700, 80000, 50000, "uniform"),
                                            (300, 60000, 3, "chebyshev")])
def test_node_order_is_the_stable_sort_by_cell(dtype, m, N, M1, M2, nodes):
    """Step 0 read back through nnfft_node_order, for both node sorts: the order is a
    permutation, the cell offsets run from 0 to M without decreasing, within every cell the
    caller indices increase (the sort is stable), and the cells are consecutive intervals of
    the node axis (the largest node of a non-empty cell is at most the smallest of the next).
    The two sorts give the same order.  Cases: clustered nodes whose edge buckets span several
    shared-memory chunks, dense uniform nodes, a side of three points; complex128 plans sort
    without carrying coordinates, complex64 plans carry 4-byte ones."""
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, _ = W.nnfft_inputs(M1, M2, 96, nodes=nodes, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    orders = []
    for lsd in (1, 0):
        plan.set_tuning(32, 32, 0, 0, 32, 32, sort_lsd=lsd)
        plan.set_nodes(dev(v), dev(x))
        plan.sync()
        sides = []
        for side, t in ((0, v), (1, x)):
            perm, off = plan.node_order(side)
            M = len(t)
            assert np.array_equal(np.sort(perm), np.arange(M))
            assert off[0] == 0 and off[-1] == M and np.all(np.diff(off) >= 0)
            cell = np.repeat(np.arange(len(off) - 1), np.diff(off))
            same = cell[1:] == cell[:-1]
            assert np.all(np.diff(perm)[same] > 0)
            s = t[perm]
            starts = off[:-1][np.diff(off) > 0]
            assert np.all(np.maximum.reduceat(s, starts)[:-1] <= np.minimum.reduceat(s, starts)[1:])
            sides.append((perm, off))
        orders.append(sides)
    for a, b in zip(orders[0], orders[1]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    plan.close()


@pytest.mark.parametrize("N", [4096, 1000, 64])
@pytest.mark.parametrize("dtype,m,arith", [(torch.complex128, 8, None), (torch.complex128, 8, "fp64"),
                                           (torch.complex64, 4, None)])
def test_cluster_fft_equals_two_pass_fft(N, dtype, m, arith):
    """The FFT of step 3 as one launch of a thread-block cluster (the grid in distributed
    shared memory) runs the same butterflies and twiddles as the two-pass kernels: the
    transforms are bitwise equal, forward and adjoint, and the graph of a transform with it
    replays it."""
    M1, M2 = 50000, 40000
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.nnfft_inputs(M1, M2, 97, dtype=npd)
    g = W.adjoint_inputs(M2, 97, dtype=npd)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    if arith == "fp64":
        plan.set_arith(B.ARITH_FP64)
    outs = []
    for fv in (0, 2):
        plan.set_tuning(8, 8, fv, 0, 32, 32)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f), dev(g))
        plan.sync()
        outs.append((y.cpu().numpy(), z.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    vd, xd, fd, gd = dev(v), dev(x), dev(f), dev(g)
    graph = plan.transform_graph(vd, xd, fd, gd)
    yg, zg = graph.launch()
    plan.sync()
    assert np.array_equal(yg.cpu().numpy(), outs[1][0]) and np.array_equal(zg.cpu().numpy(), outs[1][1])
    graph.close()
    rows = W.sample_rows(M2, 32, 13)
    want = oracle.nnfft_direct(N, v, f.astype(np.complex128), x, rows=rows)
    tol = 1e-12 if dtype == torch.complex128 else 2e-5
    assert np.max(np.abs(outs[1][0][rows].astype(np.complex128) - want)) / np.sum(np.abs(f)) <= tol


def test_grid_barrier_waits_are_bounded():
    """The fused grid stage's barrier: blocks that all arrive pass both barriers (the arrival
    counter grows by 2 x blocks and stays a multiple of the block count); a barrier expecting
    one block more than were launched is never completed, so every wait gives up after its
    cycle limit, sets the timeout bit (4) and the abort word, and the context stays usable
    (the next launch over fresh words passes)."""
    import torch as T
    words, st = B.selftest_grid_barrier(blocks=8, extra=0)
    assert st == 0 and words.tolist() == [16, 0]
    words, st = B.selftest_grid_barrier(blocks=8, extra=0, words=words)
    assert st == 0 and words.tolist() == [32, 0]
    words, st = B.selftest_grid_barrier(blocks=4, extra=1, limit_cycles=2_000_000)
    assert st == 4 and int(words[1].item()) == 1 and int(words[0].item()) == 4
    words, st = B.selftest_grid_barrier(blocks=4, extra=0, words=T.zeros(2, dtype=T.int64, device="cuda"))
    assert st == 0 and words.tolist() == [8, 0]


@pytest.mark.parametrize("N,M1,M2,nodes", [(4096, 50000, 40000, "uniform"), (1000, 30000, 70000, "chebyshev"),
                                           (64, 3000, 2000, "uniform")])
def test_fused_grid_stage_equals_stage_launches(N, M1, M2, nodes):
    """fft_variant 3 runs the cell fold, spread convolution, both FFT passes and the gather
    convolution of each direction in one cooperative launch with grid barriers: the same
    block bodies and arithmetic as the stage-wide launches, so exec, adjoint, the concurrent
    pair and the transform graph are bitwise equal to them, and the result is within the
    fp64 tolerance of the direct sum."""
    v, x, f = W.nnfft_inputs(M1, M2, 61, nodes=nodes)
    g = W.adjoint_inputs(M2, 61)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, 8, 8, dtype=torch.complex128)
    outs = []
    for fv in (0, 3):
        plan.set_tuning(8, 8, fv, 0, 32, 32)
        plan.set_nodes(dev(v), dev(x))
        y = plan.exec(dev(f))
        z = plan.adjoint(dev(g))
        y2, z2 = plan.exec_adjoint(dev(f), dev(g))
        plan.sync()
        outs.append([a.cpu().numpy() for a in (y, z, y2, z2)])
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    vd, xd, fd, gd = dev(v), dev(x), dev(f), dev(g)
    graph = plan.transform_graph(vd, xd, fd, gd)
    for _ in range(3):
        yg, zg = graph.launch()
    plan.sync()
    assert np.array_equal(yg.cpu().numpy(), outs[0][0]) and np.array_equal(zg.cpu().numpy(), outs[0][1])
    graph.close()
    rows = W.sample_rows(M2, 32, 17)
    want = oracle.nnfft_direct(N, v, f, x, rows=rows)
    assert np.max(np.abs(outs[1][0][rows] - want)) / np.sum(np.abs(f)) <= 1e-12


def test_fused_grid_stage_needs_equal_degrees():
    """The fused kernel is instantiated for one Chebyshev degree D on both sides: a plan with
    m1 != m2 (D1 != D2) rejects fft_variant 3 with EINVAL and keeps working."""
    plan = B.Plan(256, 2000, 2000, 2.0, 2.0, 8, 5, dtype=torch.complex128)
    if plan.info["D1"] == plan.info["D2"]:
        pytest.skip("equal degrees for these window sizes")
    with pytest.raises(B.NNFFTError):
        plan.set_tuning(8, 8, 3, 0, 32, 32)
    plan.set_tuning(8, 8, 0, 0, 32, 32)


@pytest.mark.parametrize("N,M1,M2,nodes,split", [(4096, 50000, 40000, "uniform", 0),
                                                 (1000, 300000, 200000, "chebyshev", 0),
                                                 (700, 3000, 2000, "uniform", 1)])
def test_gather_inside_evaluation_equals_gather_kernel(N, M1, M2, nodes, split):
    """Evaluation lanes value 3: each work item's warp forms its cell's window sums from the
    FFT output itself (scaled grid values, tap sums, the 1/phihat1 fold on the x side) in the
    gather kernel's order, then evaluates its points: bitwise the gather kernel followed by
    the 32-lane evaluation, forward and adjoint, with cells split into several items
    (clustered nodes), with small-item splitting (where the gather kernel runs instead), and
    replayed from the transform graph; within the fp64 tolerance of the direct sum."""
    v, x, f = W.nnfft_inputs(M1, M2, 83, nodes=nodes)
    g = W.adjoint_inputs(M2, 83)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, 8, 8, dtype=torch.complex128)
    outs = []
    for el in (32, 3):
        plan.set_tuning(8, 8, 0, split, el, el)
        plan.set_nodes(dev(v), dev(x))
        y, z = plan.exec_adjoint(dev(f), dev(g))
        plan.sync()
        outs.append((y.cpu().numpy(), z.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    vd, xd, fd, gd = dev(v), dev(x), dev(f), dev(g)
    graph = plan.transform_graph(vd, xd, fd, gd)
    yg, zg = graph.launch()
    plan.sync()
    assert np.array_equal(yg.cpu().numpy(), outs[0][0]) and np.array_equal(zg.cpu().numpy(), outs[0][1])
    graph.close()
    rows = W.sample_rows(M2, 32, 19)
    want = oracle.nnfft_direct(N, v, f, x, rows=rows)
    assert np.max(np.abs(outs[1][0][rows] - want)) / np.sum(np.abs(f)) <= 1e-12
    rows = W.sample_rows(M1, 32, 20)
    want = oracle.nnfft_adjoint_direct(N, v, x, g, rows=rows)
    assert np.max(np.abs(outs[1][1][rows] - want)) / np.sum(np.abs(g)) <= 1e-12
