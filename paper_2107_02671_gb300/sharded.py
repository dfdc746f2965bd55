"""Sharded NNFFT: Algorithm 2.2 split at its grid for node sets divided among processes.

Step 1 of Algorithm 2.2 (eq. (2.12)) sums over the frequency nodes v_k and step 4
evaluates each spatial node x_j on its own, so P processes (one GPU each) that hold
disjoint shares of the v nodes and of the x nodes compute one transform together:

    forward  y = A f:   grid_r = spread_grid(f_r)        steps 1-2, own v share
                        grid   = sum_r grid_r            one all-reduce (K1 values)
                        y_r    = exec_grid(grid)         steps 3-4, own x share
    adjoint  z = A^H g: grid_r = adjoint_spread_grid(g_r)   own x share
                        grid   = sum_r grid_r               one all-reduce (N2 values)
                        z_r    = adjoint_grid(grid)         own v share

The exchanged grid has K1 = N1 + 2 m1 (forward) or N2 (adjoint) complex values, about
0.1-0.5 MB at the bandwidths of the paper's experiments, whatever M1 and M2 are.  The
FFT of step 3 runs on every process (it is N2 log N2 work, small against M1 + M2).

This module holds only the orchestration: shard bounds and the order of the library
calls around a caller-supplied all-reduce (in place, sum), e.g.
``torch.distributed.all_reduce`` on a NCCL process group.  Every arithmetic step runs in
the library's kernels (Plan.spread_grid & co.)."""
from __future__ import annotations


def shard_bounds(M: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of M items, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or M < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, M >= 0")
    q, r = divmod(M, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def sharded_exec(plan, f_r, all_reduce, y_r=None):
    """y_r = (A f)[own x share] from this process's share f_r of the coefficients.
    ``plan`` holds this process's v and x shares (set_nodes done); ``all_reduce(t)``
    sums t over the processes in place."""
    grid = plan.spread_grid(f_r)
    all_reduce(grid)
    return plan.exec_grid(grid, y_r)


def sharded_adjoint(plan, g_r, all_reduce, z_r=None):
    """z_r = (A^H g)[own v share] from this process's share g_r of the values."""
    grid = plan.adjoint_spread_grid(g_r)
    all_reduce(grid)
    return plan.adjoint_grid(grid, z_r)


class ShardedPlan:
    """This process's part of a sharded NNFFT over M1 frequency and M2 spatial nodes.

    Makes a library plan for the rank's shares (shard_bounds) with the common N, sigma,
    m and dtype; ``set_nodes`` takes the rank's shares of the nodes, ``exec`` and
    ``adjoint`` its shares of the values and return its shares of the results."""

    def __init__(self, N, M1, M2, rank, world, sigma1=2.0, sigma2=2.0, m1=8, m2=None,
                 dtype=None, all_reduce=None):
        from . import nnfft
        self.v_range = shard_bounds(M1, world, rank)
        self.x_range = shard_bounds(M2, world, rank)
        self.plan = nnfft.Plan(N, self.v_range[1] - self.v_range[0],
                               self.x_range[1] - self.x_range[0], sigma1, sigma2, m1, m2,
                               dtype=dtype)
        if all_reduce is None:
            import torch.distributed as dist
            all_reduce = dist.all_reduce
        self.all_reduce = all_reduce

    def set_nodes(self, v_r, x_r):
        self.plan.set_nodes(v_r, x_r)
        return self

    def exec(self, f_r, y_r=None):
        return sharded_exec(self.plan, f_r, self.all_reduce, y_r)

    def adjoint(self, g_r, z_r=None):
        return sharded_adjoint(self.plan, g_r, self.all_reduce, z_r)

    def sync(self):
        self.plan.sync()
