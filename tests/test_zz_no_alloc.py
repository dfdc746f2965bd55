"""nnfft_exec_host_noalloc: the host-buffer forward transform for callers that
cannot allocate device memory at call time (their GPU memory belongs to another
allocator, or an allocation stall is not acceptable).  It stages f and y in the
library's static 4 MiB device array instead of buffers allocated on first use.

Checked through the C ABI against the existing nnfft_exec_host on two calls in a
row (the array keeps the previous call's contents, so the second call must not
see stale data), plus the size limit.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_02671_gb300 import nnfft as B  # noqa: E402
from paper_2107_02671_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load_library()
    lib.nnfft_exec_host_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return lib


def noalloc(lib, plan, f):
    y = np.empty(plan.M2, dtype=plan.np_cdtype)
    rc = lib.nnfft_exec_host_noalloc(plan._h, ctypes.c_void_p(f.ctypes.data),
                                     ctypes.c_void_p(y.ctypes.data))
    B._check(rc)
    return y


@pytest.mark.parametrize("dtype,m,tol", [(torch.complex128, 8, 1e-12), (torch.complex64, 4, 2e-5)])
def test_noalloc_matches_exec_host_twice(lib, dtype, m, tol):
    N, M1, M2 = 512, 30000, 20000
    v, x, _ = W.nnfft_inputs(M1, M2, 21)
    plan = B.Plan(N, M1, M2, 2.0, 2.0, m, m, dtype=dtype)
    plan.set_nodes_host(v, x)
    for call in range(2):                      # two calls in a row, different inputs
        f = W.draw_complex(np.random.default_rng(100 + call), M1, plan.np_cdtype)
        ref = plan.exec_host(f)
        out = noalloc(lib, plan, f)
        err = np.max(np.abs(out.astype(np.complex128) - ref)) / np.sum(np.abs(f))
        assert err <= tol


def test_noalloc_rejects_sizes_beyond_the_static_array(lib):
    M = 200000                                  # 2 * 200000 * 16 bytes > 4 MiB
    plan = B.Plan(64, M, M, 2.0, 2.0, 4, 4, dtype=torch.complex128)
    v, x, f = W.nnfft_inputs(M, M, 22)
    plan.set_nodes_host(v, x)
    with pytest.raises(B.NNFFTError) as ei:
        noalloc(lib, plan, f)
    assert ei.value.code == 1
