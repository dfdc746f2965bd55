"""GPU parity of the sharded transform (Algorithm 2.2 split at its grid): the node sets
are divided among several plans, as among processes with one GPU each, and the grids are
summed in between (here one process runs every share and adds the grids on the device;
across processes the sum is an all-reduce).  The concatenated shares must equal one plan
over all nodes up to the rounding of the grid sum, and the oracle's direct sums within the
usual tolerances (fp64 m = 8: 1e-12, fp32 m = 4: 2e-5, relative to the 1-norm of the
coefficients)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2107_02671_gb300 import nnfft as B  # noqa: E402
from paper_2107_02671_gb300 import sharded as S  # noqa: E402
from paper_2107_02671_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def run_sharded(N, v, x, f, g, m, dtype, cuts_v, cuts_x, arith=None):
    """Shares [cuts[r], cuts[r+1]) of the v and x nodes, one plan each; returns the
    concatenated forward and adjoint results and the summed forward grid."""
    plans = []
    for r in range(len(cuts_v) - 1):
        a, b = cuts_v[r], cuts_v[r + 1]
        c, d = cuts_x[r], cuts_x[r + 1]
        p = B.Plan(N, b - a, d - c, 2.0, 2.0, m, m, dtype=dtype)
        if arith is not None:
            p.set_arith(arith)
        p.set_nodes(dev(v[a:b]), dev(x[c:d]))
        plans.append((p, a, b, c, d))
    sum_f = sum(p.spread_grid(dev(f[a:b], dtype)) for p, a, b, c, d in plans)
    sum_a = sum(p.adjoint_spread_grid(dev(g[c:d], dtype)) for p, a, b, c, d in plans)
    y = torch.cat([p.exec_grid(sum_f) for p, a, b, c, d in plans])
    z = torch.cat([p.adjoint_grid(sum_a) for p, a, b, c, d in plans])
    for p, *_ in plans:
        p.sync()
    return (y.cpu().numpy().astype(np.complex128), z.cpu().numpy().astype(np.complex128),
            sum_f, sum_a)


CASES = [(torch.complex128, 8, None, 1e-12, 1e-14),
         (torch.complex128, 8, B.ARITH_FP64, 1e-12, 1e-14),
         (torch.complex64, 4, None, 2e-5, 2e-6)]


@pytest.mark.parametrize("dtype,m,arith,tol,tol_full", CASES)
@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_sharded_equals_one_plan(dtype, m, arith, tol, tol_full, nodes):
    N, M1, M2, world = 1000, 50001, 40003, 3
    v, x, f = W.nnfft_inputs(M1, M2, 31, nodes=nodes)
    g = W.adjoint_inputs(M2, 31)
    cuts_v = [0] + [S.shard_bounds(M1, world, r)[1] for r in range(world)]
    cuts_x = [0] + [S.shard_bounds(M2, world, r)[1] for r in range(world)]
    y, z, grid_f, grid_a = run_sharded(N, v, x, f, g, m, dtype, cuts_v, cuts_x, arith)
    full = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    if arith is not None:
        full.set_arith(arith)
    full.set_nodes(dev(v), dev(x))
    yf = full.exec(dev(f, dtype)).cpu().numpy().astype(np.complex128)
    zf = full.adjoint(dev(g, dtype)).cpu().numpy().astype(np.complex128)
    gf = full.spread_grid(dev(f, dtype))
    ga = full.adjoint_spread_grid(dev(g, dtype))
    full.sync()
    nf, ng = np.sum(np.abs(f)), np.sum(np.abs(g))
    # the summed grids are the one plan's grids (eq. (2.12) is a sum over k)
    tol_grid = 1e-13 if dtype == torch.complex128 else 1e-5
    assert torch.max(torch.abs(grid_f - gf)).item() <= tol_grid * torch.max(torch.abs(gf)).item()
    assert torch.max(torch.abs(grid_a - ga)).item() <= tol_grid * torch.max(torch.abs(ga)).item()
    assert np.max(np.abs(y - yf)) <= tol_full * nf
    assert np.max(np.abs(z - zf)) <= tol_full * ng
    rows_x = W.sample_rows(M2, 64, 3, extremes=[int(np.argmin(x)), int(np.argmax(x))])
    rows_v = W.sample_rows(M1, 64, 4, extremes=[int(np.argmin(v)), int(np.argmax(v))])
    fy = f.astype(np.complex128)
    assert np.max(np.abs(y[rows_x] - oracle.nnfft_direct(N, v, fy, x, rows=rows_x))) <= tol * nf
    assert np.max(np.abs(z[rows_v] - oracle.nnfft_adjoint_direct(N, v, x, g, rows=rows_v))) <= tol * ng


def test_sharded_with_empty_and_ragged_shares():
    """One share has no frequency nodes, another no spatial nodes: an empty share adds a
    zero grid and evaluates nothing."""
    N, M1, M2 = 300, 2001, 1777
    v, x, f = W.nnfft_inputs(M1, M2, 32)
    g = W.adjoint_inputs(M2, 32)
    cuts_v = [0, 0, 1000, M1]          # share 0: no v nodes
    cuts_x = [0, 900, 900, M2]         # share 1: no x nodes
    y, z, _, _ = run_sharded(N, v, x, f, g, 8, torch.complex128, cuts_v, cuts_x)
    assert np.max(np.abs(y - oracle.nnfft_direct(N, v, f, x))) <= 1e-12 * np.sum(np.abs(f))
    assert np.max(np.abs(z - oracle.nnfft_adjoint_direct(N, v, x, g))) <= 1e-12 * np.sum(np.abs(g))


def test_grid_layout_is_the_deconvolved_step_2_grid():
    """The forward grid of one plan holds ghat_l / N2 = g_l / (N2 phihat2(l)), l in I_K1
    (centered, index l + K1/2): checked against the oracle's Algorithm 2.2 step-1 grid
    g_l divided by N2 phihat2(l)."""
    N, M1, M2, m = 64, 300, 200, 8
    v, x, f = W.nnfft_inputs(M1, M2, 33)
    p = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=torch.complex128)
    p.set_nodes(dev(v), dev(x))
    grid = p.spread_grid(dev(f)).cpu().numpy()
    info = p.info
    P = oracle.make_params(N, 2.0, 2.0, m, m)
    assert (P.K1, P.N2) == (info["K1"], info["N2"])
    _, g, _ = oracle.nnfft_alg22(P, v, f, x, return_stages=True)
    ell = np.arange(-P.K1 // 2, P.K1 // 2).astype(float)
    want = g / (P.N2 * oracle.phi_hat(ell, P.N2, m, P.beta2))
    assert np.max(np.abs(grid - want)) <= 1e-13 * np.max(np.abs(want))


def test_sharded_calls_reject_batches_and_unset_nodes():
    p = B.Plan(64, 10, 10, 2.0, 2.0, 4, 4, dtype=torch.complex128)
    with pytest.raises(B.NNFFTError) as ei:
        p.spread_grid(torch.zeros(10, dtype=torch.complex128, device="cuda"))
    assert ei.value.code == 6                       # NNFFT_ESTATE: set_nodes first
    bp = B.BatchPlan([64, 64], [10, 12], [9, 8], 2.0, 2.0, 4, dtype=torch.complex128)
    bp.set_nodes(dev(np.zeros(22)), dev(np.zeros(17)))
    lib = B.load_library()
    grid = torch.zeros(1 << 14, dtype=torch.complex128, device="cuda")
    f = torch.zeros(22, dtype=torch.complex128, device="cuda")
    rc = lib.nnfft_spread_grid(bp._h, f.data_ptr(), grid.data_ptr())
    assert rc == 1                                  # NNFFT_EINVAL: single-instance plans only
