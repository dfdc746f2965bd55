"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws random nodes and
coefficients with numpy's ``default_rng(seed)``.  Draw order is fixed: nodes v,
nodes x, then Re f, Im f (or the real sinc coefficients c).

Node distributions follow the workloads of the paper's experiments (random nodes
in [-1/2, 1/2], Sections 4 and 6) plus a clustered Chebyshev set:
  * ``"uniform"``:   i.i.d. U[-1/2, 1/2)
  * ``"chebyshev"``: cos(pi u) / 2 with u ~ U[0, 1)  (density peaks at +-1/2)
Coefficients are i.i.d. standard normal (real and imaginary parts).
"""
from __future__ import annotations

import numpy as np

NODE_SETS = ("uniform", "chebyshev")


def draw_nodes(rng, M, kind="uniform"):
    """M float64 nodes in [-1/2, 1/2] of the given distribution."""
    if kind == "uniform":
        return rng.uniform(-0.5, 0.5, size=M)
    if kind == "chebyshev":
        return 0.5 * np.cos(np.pi * rng.uniform(0.0, 1.0, size=M))
    raise ValueError(f"unknown node set {kind!r}")


def draw_complex(rng, M, dtype=np.complex128):
    """M complex values with i.i.d. N(0,1) real and imaginary parts."""
    re = rng.standard_normal(M)
    im = rng.standard_normal(M)
    return (re + 1j * im).astype(dtype)


def nnfft_inputs(M1, M2, seed=0, nodes="uniform", dtype=np.complex128):
    """(v, x, f): M1 frequency nodes, M2 spatial nodes, M1 coefficients."""
    rng = np.random.default_rng(seed)
    v = draw_nodes(rng, M1, nodes)
    x = draw_nodes(rng, M2, nodes)
    f = draw_complex(rng, M1, dtype)
    return v, x, f


def adjoint_inputs(M2, seed=0, dtype=np.complex128):
    """g: M2 coefficients for the adjoint transform (independent stream seed+10**6)."""
    rng = np.random.default_rng(seed + 1_000_000)
    return draw_complex(rng, M2, dtype)


def sinc_inputs(L1, L2, seed=0, nodes="uniform", complex_coeffs=False):
    """(a, c, b): L1 sample nodes, L1 coefficients (real N(0,1) unless complex), L2 targets."""
    rng = np.random.default_rng(seed)
    a = draw_nodes(rng, L1, nodes)
    b = draw_nodes(rng, L2, nodes)
    c = draw_complex(rng, L1) if complex_coeffs else rng.standard_normal(L1)
    return a, c, b


def sample_rows(M, count, seed=0, extremes=None):
    """Sorted unique row indices: ``count`` random rows plus the optional ``extremes``."""
    rng = np.random.default_rng(seed + 2_000_000)
    rows = rng.choice(M, size=min(count, M), replace=False) if M > 0 else np.zeros(0, np.int64)
    if extremes is not None:
        rows = np.concatenate([rows, np.asarray(extremes, dtype=np.int64)])
    return np.unique(rows.astype(np.int64))


def batch_sizes(count, seed=0, M_range=(1e3, 1e6), N_range=(64, 8192)):
    """Instance sizes of a batch: M1, M2 drawn separately and N, each log-uniform in its
    range (rounded to integers), from stream seed + 3*10**6."""
    rng = np.random.default_rng(seed + 3_000_000)
    lm = np.log(np.asarray(M_range, dtype=np.float64))
    ln = np.log(np.asarray(N_range, dtype=np.float64))
    M1 = np.rint(np.exp(rng.uniform(lm[0], lm[1], size=count))).astype(np.int64)
    M2 = np.rint(np.exp(rng.uniform(lm[0], lm[1], size=count))).astype(np.int64)
    N = np.rint(np.exp(rng.uniform(ln[0], ln[1], size=count))).astype(np.int64)
    return N, M1, M2


def batch_inputs(M1, M2, seed=0, nodes="uniform", dtype=np.complex128):
    """(v, x, f) of a batch: the instances' nnfft_inputs concatenated; instance i uses
    seed + i."""
    vs, xs, fs = [], [], []
    for i, (m1, m2) in enumerate(zip(M1, M2)):
        v, x, f = nnfft_inputs(int(m1), int(m2), seed + i, nodes, dtype)
        vs.append(v)
        xs.append(x)
        fs.append(f)
    return np.concatenate(vs), np.concatenate(xs), np.concatenate(fs)
