"""The multi-process path of the sharded transform on CPU: two gloo ranks run the
orchestration of paper_2107_02671_gb300.sharded (shard bounds, the library calls around
one in-place all-reduce of the grid) and their assembled shares are checked against the
oracle.  Without a GPU the library calls are stood in for by a test plan whose "grid" is
the rank's partial direct sums at every spatial node (the same all-reduce and share
bookkeeping, a different grid); a second check all-reduces the oracle's own Algorithm 2.2
step-1 grids of each rank's frequency share, which must sum to the step-1 grid of all
nodes (eq. (2.12) is a sum over k), the property the sharded design rests on."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, M1, M2, SEED = 200, 301, 257, 41


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class DirectSumShare:
    """Test stand-in for a library plan holding one rank's shares (CPU, oracle sums)."""

    def __init__(self, v_r, x_all, x_range, v_all, v_range):
        self.v_r, self.x_all, self.x_range = v_r, x_all, x_range
        self.v_all, self.v_range = v_all, v_range

    def spread_grid(self, f_r):
        import oracle
        return torch.from_numpy(oracle.nnfft_direct(N, self.v_r, f_r.numpy(), self.x_all))

    def exec_grid(self, grid, out=None):
        a, b = self.x_range
        return grid[a:b].clone()

    def adjoint_spread_grid(self, g_r):
        import oracle
        a, b = self.x_range
        return torch.from_numpy(oracle.nnfft_adjoint_direct(N, self.v_all, self.x_all[a:b],
                                                            g_r.numpy()))

    def adjoint_grid(self, grid, out=None):
        a, b = self.v_range
        return grid[a:b].clone()


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2107_02671_gb300 import sharded as S
        from paper_2107_02671_gb300 import workloads as W
        v, x, f = W.nnfft_inputs(M1, M2, SEED)
        g = W.adjoint_inputs(M2, SEED)
        vr, xr = S.shard_bounds(M1, world, rank), S.shard_bounds(M2, world, rank)
        share = DirectSumShare(v[vr[0]:vr[1]], x, xr, v, vr)
        y_r = S.sharded_exec(share, torch.from_numpy(f[vr[0]:vr[1]].copy()), dist.all_reduce)
        z_r = S.sharded_adjoint(share, torch.from_numpy(g[xr[0]:xr[1]].copy()), dist.all_reduce)
        # eq. (2.12) is linear in the nodes: the ranks' step-1 grids add up to the full one
        P = oracle.make_params(N, 2.0, 2.0, 6, 6)
        _, g_r, _ = oracle.nnfft_alg22(P, v[vr[0]:vr[1]], f[vr[0]:vr[1]], x[:1],
                                       return_stages=True)
        g_sum = torch.from_numpy(g_r.copy())
        dist.all_reduce(g_sum)
        q.put((rank, vr, xr, y_r.numpy(), z_r.numpy(), g_sum.numpy()))
    finally:
        dist.destroy_process_group()


def test_sharded_orchestration_two_gloo_ranks():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2107_02671_gb300 import workloads as W
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    v, x, f = W.nnfft_inputs(M1, M2, SEED)
    g = W.adjoint_inputs(M2, SEED)
    # the shares tile the index ranges in rank order
    assert [r[1] for r in res] == [(0, 151), (151, 301)]
    assert [r[2] for r in res] == [(0, 129), (129, 257)]
    y = np.concatenate([r[3] for r in res])
    z = np.concatenate([r[4] for r in res])
    assert np.max(np.abs(y - oracle.nnfft_direct(N, v, f, x))) < 1e-12 * np.sum(np.abs(f))
    assert np.max(np.abs(z - oracle.nnfft_adjoint_direct(N, v, x, g))) < 1e-12 * np.sum(np.abs(g))
    P = oracle.make_params(N, 2.0, 2.0, 6, 6)
    _, g_full, _ = oracle.nnfft_alg22(P, v, f, x[:1], return_stages=True)
    for r in res:
        assert np.max(np.abs(r[5] - g_full)) < 1e-13 * np.max(np.abs(g_full))


def test_shard_bounds():
    sys.path.insert(0, ROOT)
    from paper_2107_02671_gb300 import sharded as S
    for M in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            b = [S.shard_bounds(M, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == M
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        S.shard_bounds(10, 2, 2)
