"""GPU parity of batched plans (many independent Algorithm 2.2 instances in one plan,
one launch per stage) against the oracle's direct sums, instance by instance, and
against single-instance plans."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def err(got, want, f):
    s = np.sum(np.abs(f))
    return float(np.max(np.abs(got - want)) / s) if got.size and s > 0 else 0.0


SMALL = dict(N=[64, 100, 512, 7, 256, 33], M1=[500, 1, 0, 300, 2000, 77], M2=[400, 300, 50, 0, 1500, 1])


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_batch_forward_adjoint_vs_direct(dtype, m, tol):
    N, M1, M2 = (np.array(SMALL[k]) for k in ("N", "M1", "M2"))
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.batch_inputs(M1, M2, 11, dtype=npd)
    g = W.draw_complex(np.random.default_rng(5), int(M2.sum()), npd)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, m, dtype=dtype)
    P.set_nodes(dev(v), dev(x))
    y = P.exec(dev(f)).cpu().numpy()
    z = P.adjoint(dev(g)).cpu().numpy()
    P.sync()
    for i in range(len(N)):
        a1, b1 = P.off1[i], P.off1[i + 1]
        a2, b2 = P.off2[i], P.off2[i + 1]
        fi, gi = f[a1:b1].astype(np.complex128), g[a2:b2].astype(np.complex128)
        if b2 > a2:
            assert err(y[a2:b2], oracle.nnfft_direct(int(N[i]), v[a1:b1], fi, x[a2:b2]), fi) <= tol, i
        if b1 > a1:
            assert err(z[a1:b1], oracle.nnfft_adjoint_direct(int(N[i]), v[a1:b1], x[a2:b2], gi), gi) <= tol, i


def test_batch_matches_single_plans():
    N, M1, M2 = (np.array(SMALL[k]) for k in ("N", "M1", "M2"))
    v, x, f = W.batch_inputs(M1, M2, 21)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, 8)
    P.set_nodes(dev(v), dev(x))
    y = P.exec(dev(f)).cpu().numpy()
    P.sync()
    for i in range(len(N)):
        a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
        S = B.Plan(int(N[i]), int(M1[i]), int(M2[i]), 2.0, 2.0, 8)
        S.set_nodes(dev(v[a1:b1]), dev(x[a2:b2]))
        ys = S.exec(dev(f[a1:b1])).cpu().numpy()
        S.sync()
        if b2 > a2 and b1 > a1:
            assert err(y[a2:b2], ys, f[a1:b1]) <= 1e-14, i
        info, single = P.instance_info(i), S.info
        for k in ("N", "Nstar", "N1", "K1", "N2", "M1", "M2", "ncell1", "ncell2", "fft_n1", "fft_n2"):
            assert info[k] == single[k], (i, k)


@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_batch_64_instances_sampled_rows(nodes):
    """64 instances with N log-uniform in [64, 8192] and M1, M2 log-uniform in
    [1e3, 1e5] (the batched workload's shape, smaller); sampled rows of every instance."""
    N, M1, M2 = W.batch_sizes(64, 3, M_range=(1e3, 1e5))
    v, x, f = W.batch_inputs(M1, M2, 300, nodes)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, 8)
    P.set_nodes(dev(v), dev(x))
    y = P.exec(dev(f)).cpu().numpy()
    P.sync()
    worst = 0.0
    for i in range(64):
        a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
        rows = W.sample_rows(int(M2[i]), 8, i)
        want = oracle.nnfft_direct(int(N[i]), v[a1:b1], f[a1:b1], x[a2:b2], rows=rows)
        worst = max(worst, err(y[a2:b2][rows], want, f[a1:b1]))
    assert worst <= 1e-12


def test_batch_fp32_64_instances_sampled_rows():
    N, M1, M2 = W.batch_sizes(64, 4, M_range=(1e3, 1e5))
    v, x, f = W.batch_inputs(M1, M2, 400, dtype=np.complex64)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, 4, dtype=torch.complex64)
    P.set_nodes(dev(v), dev(x))
    y = P.exec(dev(f)).cpu().numpy()
    P.sync()
    for i in range(64):
        a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
        rows = W.sample_rows(int(M2[i]), 8, i)
        fi = f[a1:b1].astype(np.complex128)
        want = oracle.nnfft_direct(int(N[i]), v[a1:b1], fi, x[a2:b2], rows=rows)
        assert err(y[a2:b2][rows], want, fi) <= 2e-5, i


def test_batch_all_fp64_mode_and_determinism():
    N, M1, M2 = (np.array(SMALL[k]) for k in ("N", "M1", "M2"))
    v, x, f = W.batch_inputs(M1, M2, 31)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, 8)
    P.set_nodes(dev(v), dev(x))
    y1 = P.exec(dev(f)).cpu().numpy()
    y2 = P.exec(dev(f)).cpu().numpy()
    assert np.array_equal(y1, y2)
    P.set_arith(B.ARITH_FP64)
    P.set_nodes(dev(v), dev(x))
    y3 = P.exec(dev(f)).cpu().numpy()
    P.sync()
    for i in range(len(N)):
        a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
        if b2 > a2:
            want = oracle.nnfft_direct(int(N[i]), v[a1:b1], f[a1:b1], x[a2:b2])
            assert err(y3[a2:b2], want, f[a1:b1]) <= 1e-12


def test_batch_errors():
    with pytest.raises(B.NNFFTError) as e:
        B.BatchPlan([64, 0, 32], [10, 10, 10], [10, 10, 10])
    assert "instance 1" in str(e.value)
    N, M1, M2 = np.array([64, 64]), np.array([10, 10]), np.array([10, 10])
    P = B.BatchPlan(N, M1, M2)
    v = np.zeros(20); v[13] = 0.75                      # out of range in instance 1
    P.set_nodes(dev(v), dev(np.zeros(20)))
    with pytest.raises(B.NNFFTError) as e:
        P.sync()
    assert e.value.code == 2                            # NNFFT_ERANGE


@pytest.mark.parametrize("dtype,m", [(torch.complex128, 8), (torch.complex64, 4)])
def test_batch_flat_evaluation_bitwise(dtype, m):
    """Flat evaluation over a batch (cell keys carry each instance's cell base): bitwise
    the per-item evaluation's result, both directions, empty instances included."""
    N, M1, M2 = (np.array(SMALL[k]) for k in ("N", "M1", "M2"))
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.batch_inputs(M1, M2, 51, dtype=npd)
    g = W.draw_complex(np.random.default_rng(6), int(M2.sum()), npd)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, m, dtype=dtype)
    res = []
    for el in (32, 1, 2):                      # 2: flat with TMA-staged cell tiles
        P.set_tuning(32, 32, 0, 0, el, el)
        P.set_nodes(dev(v), dev(x))
        y, z = P.exec_adjoint(dev(f), dev(g))
        P.sync()
        res.append((y.cpu().numpy(), z.cpu().numpy()))
    for r in res[1:]:
        assert np.array_equal(res[0][0], r[0]) and np.array_equal(res[0][1], r[1])


@pytest.mark.parametrize("dtype,m,arith", [(torch.complex128, 8, None), (torch.complex128, 8, "fp64"),
                                           (torch.complex64, 4, None)])
@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_batch_two_stage_sort_equals_lsd_sort(dtype, m, arith, nodes):
    """The two-stage node sort of a batch (per-instance high-digit scatter, then one block
    per instance and bucket of cells) orders every instance's nodes exactly as the LSD
    passes: bitwise equal transforms.  Instances without points, with one point, small and
    large (clustered nodes: buckets over several shared-memory chunks)."""
    N = np.array([2048, 64, 512, 7, 4096, 33, 300])
    M1 = np.array([60000, 1, 0, 300, 90000, 77, 5000])
    M2 = np.array([50000, 300, 50, 0, 70001, 1, 9000])
    npd = np.complex128 if dtype == torch.complex128 else np.complex64
    v, x, f = W.batch_inputs(M1, M2, 61, nodes=nodes, dtype=npd)
    g = W.draw_complex(np.random.default_rng(8), int(M2.sum()), npd)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, m, dtype=dtype)
    if arith == "fp64":
        P.set_arith(B.ARITH_FP64)
    res = []
    for lsd in (1, 0):
        P.set_tuning(32, 32, 0, 0, 32, 32, sort_lsd=lsd)
        P.set_nodes(dev(v), dev(x))
        y, z = P.exec_adjoint(dev(f), dev(g))
        P.sync()
        res.append((y.cpu().numpy(), z.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    tol = 1e-12 if dtype == torch.complex128 else 2e-5
    i = 4                                      # the largest instance against the oracle
    a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
    rows = W.sample_rows(int(M2[i]), 32, 3)
    fi = f[a1:b1].astype(np.complex128)
    want = oracle.nnfft_direct(int(N[i]), v[a1:b1], fi, x[a2:b2], rows=rows)
    assert err(res[1][0][a2:b2][rows].astype(np.complex128), want, fi) <= tol


@pytest.mark.parametrize("nodes", ["uniform", "chebyshev"])
def test_batch_fused_grid_stage_equals_stage_launches(nodes):
    """fft_variant 3 on a batch: the persistent blocks of the cooperative grid-stage launch
    take every instance's fold, spread, FFT and gather blocks in turn (instances without
    points, with one point, small and large); bitwise the stage-wide launches, forward and
    adjoint, also replayed from the transform graph."""
    N = np.array([2048, 64, 512, 7, 4096, 33, 300])
    M1 = np.array([60000, 1, 0, 300, 90000, 77, 5000])
    M2 = np.array([50000, 300, 50, 0, 70001, 1, 9000])
    v, x, f = W.batch_inputs(M1, M2, 67, nodes=nodes)
    g = W.draw_complex(np.random.default_rng(9), int(M2.sum()), np.complex128)
    P = B.BatchPlan(N, M1, M2, 2.0, 2.0, 8, dtype=torch.complex128)
    res = []
    for fv in (0, 3):
        P.set_tuning(8, 8, fv, 0, 32, 32)
        P.set_nodes(dev(v), dev(x))
        y, z = P.exec_adjoint(dev(f), dev(g))
        P.sync()
        res.append((y.cpu().numpy(), z.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    vd, xd, fd, gd = dev(v), dev(x), dev(f), dev(g)
    graph = P.transform_graph(vd, xd, fd, gd)
    yg, zg = graph.launch()
    P.sync()
    assert np.array_equal(yg.cpu().numpy(), res[0][0]) and np.array_equal(zg.cpu().numpy(), res[0][1])
    graph.close()
    i = 4
    a1, b1, a2, b2 = P.off1[i], P.off1[i + 1], P.off2[i], P.off2[i + 1]
    rows = W.sample_rows(int(M2[i]), 32, 5)
    want = oracle.nnfft_direct(int(N[i]), v[a1:b1], f[a1:b1], x[a2:b2], rows=rows)
    assert err(res[1][0][a2:b2][rows], want, f[a1:b1]) <= 1e-12
