"""Thin Python binding of the C ABI in include/nnfft.h.

Argument marshalling only: every step of the transforms runs in the CUDA
library ``_build/libnnfft_gb300.so``.  PyTorch supplies device memory and the
stream; tensors are passed by pointer.  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import weakref
import os
import threading

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

NNFFT_C64, NNFFT_C128 = 0, 1
ARITH_FP32, ARITH_FP64, ARITH_FP64_SPLIT = 0, 1, 2
_CODES = {0: "OK", 1: "EINVAL", 2: "ERANGE", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT", 6: "ESTATE"}


STAGES = ("nodes_v", "nodes_x", "fwd_moments", "fwd_spread_conv", "fwd_fft", "fwd_gather_conv",
          "fwd_eval", "adj_moments", "adj_spread_conv", "adj_fft", "adj_gather_conv", "adj_eval",
          "fwd_cell_fold", "adj_cell_fold")


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rule", ctypes.c_int), ("is_complex", ctypes.c_int),
                ("reserved", ctypes.c_int), ("N", ctypes.c_int64), ("M1", ctypes.c_int64),
                ("M2", ctypes.c_int64), ("tol", ctypes.c_double), ("v", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("f", ctypes.c_void_p), ("y", ctypes.c_void_p)]


class ServerReport(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("points", ctypes.c_double), ("seconds", ctypes.c_double),
                ("plans_cached", ctypes.c_int64), ("plans_made", ctypes.c_int64),
                ("plans_evicted", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("moments_lanes_v", ctypes.c_int), ("moments_lanes_x", ctypes.c_int),
                ("fft_variant", ctypes.c_int), ("tuned", ctypes.c_int),
                ("default_ms", ctypes.c_double), ("best_ms", ctypes.c_double),
                ("item_split", ctypes.c_int), ("timed_transform", ctypes.c_int),
                ("eval_lanes_v", ctypes.c_int), ("eval_lanes_x", ctypes.c_int),
                ("item_cap", ctypes.c_int), ("sort_lsd", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 16), ("count", ctypes.c_int64 * 16)]


class NNFFTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64), ("Nstar", ctypes.c_int64), ("N1", ctypes.c_int64),
        ("K1", ctypes.c_int64), ("N2", ctypes.c_int64),
        ("M1", ctypes.c_int64), ("M2", ctypes.c_int64),
        ("m1", ctypes.c_int), ("m2", ctypes.c_int),
        ("sigma1", ctypes.c_double), ("sigma2", ctypes.c_double),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("dtype", ctypes.c_int), ("D1", ctypes.c_int), ("D2", ctypes.c_int),
        ("fit_err1", ctypes.c_double), ("fit_err2", ctypes.c_double),
        ("ncell1", ctypes.c_int64), ("ncell2", ctypes.c_int64),
        ("fft_n1", ctypes.c_int64), ("fft_n2", ctypes.c_int64),
        ("arith", ctypes.c_int), ("window", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"NNFFT CUDA library not built: {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, i64, cint, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER
        lib.nnfft_params.argtypes = [i64, i64, i64, dbl, dbl, cint, cint, cint, P(Info)]
        lib.nnfft_params_window.argtypes = [i64, i64, i64, dbl, dbl, cint, cint, cint, cint, P(Info)]
        lib.nnfft_plan_window.argtypes = [P(vp), i64, i64, i64, dbl, dbl, cint, cint, cint, cint, vp]
        lib.nnfft_batch_plan_window.argtypes = [P(vp), i64, P(i64), P(i64), P(i64), dbl, dbl, cint,
                                                cint, cint, cint, vp]
        lib.nnfft_window.argtypes = [cint, cint, dbl, dbl, dbl, P(dbl), P(dbl)]
        lib.nnfft_plan.argtypes = [P(vp), i64, i64, i64, dbl, dbl, cint, cint, cint, vp]
        lib.nnfft_plan_info.argtypes = [vp, P(Info)]
        lib.nnfft_batch_plan.argtypes = [P(vp), i64, P(i64), P(i64), P(i64), dbl, dbl, cint, cint,
                                         cint, vp]
        lib.nnfft_batch_count.argtypes = [vp, P(i64)]
        lib.nnfft_set_sizes.argtypes = [vp, i64, i64]
        lib.nnfft_set_bandwidth.argtypes = [vp, i64]
        lib.nnfft_tolerance_params.argtypes = [dbl, P(cint), P(cint)]
        lib.nnfft_server_create.argtypes = [P(vp), i64, cint, i64]
        lib.nnfft_server_submit.argtypes = [vp, P(Request), P(i64)]
        lib.nnfft_server_wait.argtypes = [vp, i64, P(dbl)]
        lib.nnfft_server_wait_device.argtypes = [vp, i64, P(dbl), P(dbl)]
        lib.nnfft_server_stats.argtypes = [vp, P(ServerReport), cint]
        lib.nnfft_server_destroy.argtypes = [vp]
        lib.nnfft_set_stream.argtypes = [vp, vp]
        lib.nnfft_batch_info.argtypes = [vp, i64, P(Info)]
        lib.nnfft_set_nodes.argtypes = [vp, vp, vp]
        lib.nnfft_exec.argtypes = [vp, vp, vp]
        lib.nnfft_adjoint.argtypes = [vp, vp, vp]
        lib.nnfft_exec_adjoint.argtypes = [vp, vp, vp, vp, vp]
        lib.nnfft_transform_host.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.nnfft_transform.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.nnfft_transform_graph.argtypes = [vp, vp, vp, vp, vp, vp, vp, P(vp)]
        lib.nnfft_transform_host_graph.argtypes = [vp, vp, vp, vp, vp, vp, vp, P(vp)]
        lib.nnfft_graph_launch.argtypes = [vp]
        lib.nnfft_graph_kernels.argtypes = [vp]
        lib.nnfft_graph_kernels.restype = i64
        lib.nnfft_graph_destroy.argtypes = [vp]
        lib.nnfft_autotune.argtypes = [vp, vp, vp, vp, vp, vp, vp, cint, cint]
        lib.nnfft_get_tuning.argtypes = [vp, P(Tuning)]
        lib.nnfft_set_tuning.argtypes = [vp, P(Tuning)]
        lib.nnfft_set_nodes_host.argtypes = [vp, vp, vp]
        lib.nnfft_exec_host.argtypes = [vp, vp, vp]
        lib.nnfft_adjoint_host.argtypes = [vp, vp, vp]
        lib.nnfft_sync.argtypes = [vp]
        lib.nnfft_node_order.argtypes = [vp, cint, vp, vp, P(i64)]
        lib.nnfft_destroy.argtypes = [vp]
        lib.sinc_exec.argtypes = [i64, i64, i64, cint, cint, vp, vp, vp, vp, cint, vp]
        lib.sinc_exec_rule.argtypes = [i64, i64, i64, cint, cint, cint, i64, vp, vp, vp, vp, cint,
                                       vp]
        lib.sinc_quadrature.argtypes = [cint, i64, i64, vp, vp, P(i64)]
        lib.sinc_sync.argtypes = [vp]
        lib.sinc_release.argtypes = []
        lib.nnfft_gauss_legendre.argtypes = [i64, vp, vp]
        lib.nnfft_set_arith.argtypes = [vp, cint]
        lib.nnfft_spread_grid.argtypes = [vp, vp, vp]
        lib.nnfft_exec_grid.argtypes = [vp, vp, vp]
        lib.nnfft_adjoint_spread_grid.argtypes = [vp, vp, vp]
        lib.nnfft_adjoint_grid.argtypes = [vp, vp, vp]
        lib.nnfft_timing_enable.argtypes = [vp, cint]
        lib.nnfft_timing_read.argtypes = [vp, P(Timing), cint]
        lib.nnfft_selftest_fixed63.argtypes = [vp, vp, i64]
        lib.nnfft_selftest_bulk_copy.argtypes = [vp, vp, cint, cint, i64, vp]
        lib.nnfft_selftest_grid_barrier.argtypes = [cint, cint, i64, vp, vp]
        lib.nnfft_launch_count.argtypes = []
        lib.nnfft_launch_count.restype = i64
        lib.nnfft_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc):
    if rc != 0:
        msg = _lib.nnfft_last_error().decode(errors="replace")
        raise NNFFTError(rc, msg)


def _dtype_code(dtype):
    import torch
    if dtype in (torch.complex128, np.complex128, "complex128", "c128", NNFFT_C128):
        return NNFFT_C128
    if dtype in (torch.complex64, np.complex64, "complex64", "c64", NNFFT_C64):
        return NNFFT_C64
    raise ValueError(f"unsupported dtype {dtype!r}")


WINDOWS = {"sinh": 0, "kaiser_bessel": 1, "bspline": 2, "algebraic": 3}


def _window_code(window):
    try:
        return WINDOWS[window]
    except KeyError:
        raise ValueError(f"unknown window {window!r} (use one of {sorted(WINDOWS)})") from None


def params(N, M1, M2, sigma1=2.0, sigma2=2.0, m1=8, m2=None, dtype="complex128",
           window="sinh") -> dict:
    """Derived plan parameters (no GPU needed)."""
    lib = load_library()
    info = Info()
    m2 = m1 if m2 is None else m2
    _check(lib.nnfft_params_window(int(N), int(M1), int(M2), float(sigma1), float(sigma2),
                                   int(m1), int(m2), _dtype_code(dtype), _window_code(window),
                                   ctypes.byref(info)))
    return info.as_dict()


def window(name, m, sigma, x, v):
    """The library's window omega(x) and its Fourier transform omegahat(v) (host only)."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib.nnfft_window(_window_code(name), int(m), float(sigma), float(x), float(v),
                            ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def gauss_legendre(n):
    """The library's n-point Gauss-Legendre rule on [-1/2, 1/2] (host arrays)."""
    lib = load_library()
    tau = np.zeros(int(n)); w = np.zeros(int(n))
    _check(lib.nnfft_gauss_legendre(int(n), tau.ctypes.data, w.ctypes.data))
    return tau, w


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_tensor(t, dtype, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr() if n > 0 else 0)


class Plan:
    """NNFFT plan (Algorithm 2.2): y = A f with A_jk = exp(-2 pi i N v_k x_j), and A^H.

    dtype torch.complex128 runs the fp64 path, torch.complex64 the fp32 path.
    Nodes are float64 CUDA tensors in [-1/2, 1/2].
    """

    def __init__(self, N, M1, M2, sigma1=2.0, sigma2=2.0, m1=8, m2=None, dtype=None,
                 stream=None, window="sinh"):
        import torch
        lib = load_library()
        dtype = torch.complex128 if dtype is None else dtype
        self.dtype = dtype
        self.cdtype = torch.complex128 if _dtype_code(dtype) == NNFFT_C128 else torch.complex64
        self.np_cdtype = np.complex128 if self.cdtype == torch.complex128 else np.complex64
        self.M1, self.M2, self.N = int(M1), int(M2), int(N)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._h = ctypes.c_void_p()
        m2 = m1 if m2 is None else m2
        _check(lib.nnfft_plan_window(ctypes.byref(self._h), int(N), int(M1), int(M2),
                                     float(sigma1), float(sigma2), int(m1), int(m2),
                                     _dtype_code(dtype), _window_code(window),
                                     _stream_ptr(self.stream)))
        self._lib = lib

    @property
    def info(self) -> dict:
        info = Info()
        _check(self._lib.nnfft_plan_info(self._h, ctypes.byref(info)))
        return info.as_dict()

    def set_sizes(self, M1, M2):
        """Serve M1 <= capacity frequency and M2 <= capacity spatial nodes (set_nodes next)."""
        _check(self._lib.nnfft_set_sizes(self._h, int(M1), int(M2)))
        self.M1, self.M2 = int(M1), int(M2)
        return self

    def set_bandwidth(self, N):
        """Use the plan (made for bandwidth N') for bandwidth N <= N' (set_nodes next)."""
        _check(self._lib.nnfft_set_bandwidth(self._h, int(N)))
        self.N = int(N)
        return self

    def set_arith(self, arith):
        """ARITH_FP64 or ARITH_FP64_SPLIT for complex128 plans; call set_nodes afterwards."""
        _check(self._lib.nnfft_set_arith(self._h, int(arith)))
        return self

    def set_nodes(self, v=None, x=None):
        import torch
        pv = _dev_tensor(v, torch.float64, self.M1, "v") if v is not None else None
        px = _dev_tensor(x, torch.float64, self.M2, "x") if x is not None else None
        _check(self._lib.nnfft_set_nodes(self._h, pv, px))
        return self

    def exec(self, f, out=None):
        import torch
        pf = _dev_tensor(f, self.cdtype, self.M1, "f")
        if out is None:
            out = torch.empty(self.M2, dtype=self.cdtype, device=f.device)
        po = _dev_tensor(out, self.cdtype, self.M2, "out")
        _check(self._lib.nnfft_exec(self._h, pf, po))
        return out

    def adjoint(self, g, out=None):
        import torch
        pg = _dev_tensor(g, self.cdtype, self.M2, "g")
        if out is None:
            out = torch.empty(self.M1, dtype=self.cdtype, device=g.device)
        po = _dev_tensor(out, self.cdtype, self.M1, "out")
        _check(self._lib.nnfft_adjoint(self._h, pg, po))
        return out

    # sharded transform: Algorithm 2.2 split at its grid (nnfft_spread_grid & co.)
    def spread_grid(self, f, grid=None):
        """Steps 1-2 for this plan's v nodes: the K1 grid values ghat_l / N2 (plan dtype)."""
        import torch
        pf = _dev_tensor(f, self.cdtype, self.M1, "f")
        K1 = self.info["K1"]
        if grid is None:
            grid = torch.empty(K1, dtype=self.cdtype, device=f.device)
        pgr = _dev_tensor(grid, self.cdtype, K1, "grid")
        _check(self._lib.nnfft_spread_grid(self._h, pf, pgr))
        return grid

    def exec_grid(self, grid, out=None):
        """Steps 3-4 and the output division for this plan's x nodes from a K1 grid."""
        import torch
        pgr = _dev_tensor(grid, self.cdtype, self.info["K1"], "grid")
        if out is None:
            out = torch.empty(self.M2, dtype=self.cdtype, device=grid.device)
        po = _dev_tensor(out, self.cdtype, self.M2, "out")
        _check(self._lib.nnfft_exec_grid(self._h, pgr, po))
        return out

    def adjoint_spread_grid(self, g, grid=None):
        """The adjoint's first half for this plan's x nodes: the N2 grid values u_s."""
        import torch
        pg = _dev_tensor(g, self.cdtype, self.M2, "g")
        N2 = self.info["N2"]
        if grid is None:
            grid = torch.empty(N2, dtype=self.cdtype, device=g.device)
        pgr = _dev_tensor(grid, self.cdtype, N2, "grid")
        _check(self._lib.nnfft_adjoint_spread_grid(self._h, pg, pgr))
        return grid

    def adjoint_grid(self, grid, out=None):
        """The adjoint's second half for this plan's v nodes from an N2 grid."""
        import torch
        pgr = _dev_tensor(grid, self.cdtype, self.info["N2"], "grid")
        if out is None:
            out = torch.empty(self.M1, dtype=self.cdtype, device=grid.device)
        po = _dev_tensor(out, self.cdtype, self.M1, "out")
        _check(self._lib.nnfft_adjoint_grid(self._h, pgr, po))
        return out

    def exec_adjoint(self, f, g, y=None, z=None):
        """(A f, A^H g) for the same nodes, both directions running concurrently."""
        import torch
        pf = _dev_tensor(f, self.cdtype, self.M1, "f")
        pg = _dev_tensor(g, self.cdtype, self.M2, "g")
        if y is None:
            y = torch.empty(self.M2, dtype=self.cdtype, device=f.device)
        if z is None:
            z = torch.empty(self.M1, dtype=self.cdtype, device=f.device)
        py = _dev_tensor(y, self.cdtype, self.M2, "y")
        pz = _dev_tensor(z, self.cdtype, self.M1, "z")
        _check(self._lib.nnfft_exec_adjoint(self._h, pf, py, pg, pz))
        return y, z

    def autotune(self, f, g, y=None, z=None, reps=3, v=None, x=None, flush_l2=False) -> dict:
        """Time the kernel variants and keep the fastest: full transforms when the nodes
        v, x are given (else exec + adjoint on the current nodes); flush_l2 writes a buffer
        larger than L2 before every timed run."""
        import torch
        if y is None:
            y = torch.empty(self.M2, dtype=self.cdtype, device=f.device)
        if z is None:
            z = torch.empty(self.M1, dtype=self.cdtype, device=f.device)
        pv = _dev_tensor(v, torch.float64, self.M1, "v") if v is not None else None
        px = _dev_tensor(x, torch.float64, self.M2, "x") if x is not None else None
        _check(self._lib.nnfft_autotune(self._h, pv, px, _dev_tensor(f, self.cdtype, self.M1, "f"),
                                        _dev_tensor(y, self.cdtype, self.M2, "y"),
                                        _dev_tensor(g, self.cdtype, self.M2, "g"),
                                        _dev_tensor(z, self.cdtype, self.M1, "z"), int(reps),
                                        1 if flush_l2 else 0))
        return self.tuning()

    def set_tuning(self, moments_lanes_v=32, moments_lanes_x=32, fft_variant=0, item_split=0,
                   eval_lanes_v=32, eval_lanes_x=32, item_cap=256, sort_lsd=None):
        """Apply a kernel-variant configuration (see autotune); a changed item_split,
        item_cap or sort_lsd needs set_nodes again (sort_lsd None: keep the plan's)."""
        if sort_lsd is None:
            sort_lsd = self.tuning()["sort_lsd"]
        t = Tuning(int(moments_lanes_v), int(moments_lanes_x), int(fft_variant), 0, 0.0, 0.0,
                   int(item_split), 0, int(eval_lanes_v), int(eval_lanes_x), int(item_cap),
                   int(sort_lsd))
        _check(self._lib.nnfft_set_tuning(self._h, ctypes.byref(t)))
        return self

    def tuning(self) -> dict:
        t = Tuning()
        _check(self._lib.nnfft_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    # host-buffer variants (numpy in, numpy out; copies inside the call)
    def set_nodes_host(self, v=None, x=None):
        args = []
        for arr, n in ((v, self.M1), (x, self.M2)):
            if arr is None:
                args.append(None)
                continue
            if not (isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.size == n
                    and arr.flags.c_contiguous):
                raise TypeError("host nodes must be contiguous float64 numpy arrays of the plan size")
            args.append(ctypes.c_void_p(arr.ctypes.data))
        _check(self._lib.nnfft_set_nodes_host(self._h, *args))
        return self

    def _host_arr(self, arr, n, name):
        if not (isinstance(arr, np.ndarray) and arr.dtype == self.np_cdtype and arr.size == n
                and arr.flags.c_contiguous):
            raise TypeError(f"{name} must be a contiguous {np.dtype(self.np_cdtype)} numpy array of {n}")
        return ctypes.c_void_p(arr.ctypes.data)

    def transform(self, v, x, f=None, g=None, y=None, z=None):
        """New nodes and both directions in one call (device tensors): returns (A f, A^H g);
        a direction is skipped when its input is None."""
        import torch
        pv = _dev_tensor(v, torch.float64, self.M1, "v")
        px = _dev_tensor(x, torch.float64, self.M2, "x")
        pf = py = pg = pz = None
        if f is not None:
            pf = _dev_tensor(f, self.cdtype, self.M1, "f")
            y = torch.empty(self.M2, dtype=self.cdtype, device=f.device) if y is None else y
            py = _dev_tensor(y, self.cdtype, self.M2, "y")
        if g is not None:
            pg = _dev_tensor(g, self.cdtype, self.M2, "g")
            z = torch.empty(self.M1, dtype=self.cdtype, device=g.device) if z is None else z
            pz = _dev_tensor(z, self.cdtype, self.M1, "z")
        _check(self._lib.nnfft_transform(self._h, pv, px, pf, py, pg, pz))
        return (y if f is not None else None), (z if g is not None else None)

    def transform_graph(self, v, x, f=None, g=None, y=None, z=None):
        """Capture one transform over these device buffers as a CUDA graph (nothing runs
        yet): returns a TransformGraph whose launch() replays set_nodes + forward + adjoint
        on the buffers' current contents; y and z receive the results."""
        import torch
        pv = _dev_tensor(v, torch.float64, self.M1, "v")
        px = _dev_tensor(x, torch.float64, self.M2, "x")
        pf = py = pg = pz = None
        if f is not None:
            pf = _dev_tensor(f, self.cdtype, self.M1, "f")
            y = torch.empty(self.M2, dtype=self.cdtype, device=f.device) if y is None else y
            py = _dev_tensor(y, self.cdtype, self.M2, "y")
        if g is not None:
            pg = _dev_tensor(g, self.cdtype, self.M2, "g")
            z = torch.empty(self.M1, dtype=self.cdtype, device=g.device) if z is None else z
            pz = _dev_tensor(z, self.cdtype, self.M1, "z")
        h = ctypes.c_void_p()
        _check(self._lib.nnfft_transform_graph(self._h, pv, px, pf, py, pg, pz, ctypes.byref(h)))
        return TransformGraph(self, h, (v, x, f, g, y, z))

    def transform_host_graph(self, v, x, f=None, g=None, y=None, z=None):
        """Capture one transform_host over these page-locked host arrays as a CUDA graph
        (nothing runs yet): launch() uploads their current contents, transforms and writes
        y and z back; sync() waits for it."""
        for arr, n, name in ((v, self.M1, "v"), (x, self.M2, "x")):
            if not (isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.size == n
                    and arr.flags.c_contiguous):
                raise TypeError(f"{name} must be a contiguous float64 numpy array of {n}")
        import torch
        if f is not None and y is None:       # page-locked result arrays
            y = torch.empty(self.M2, dtype=self.cdtype).pin_memory().numpy()
        if g is not None and z is None:
            z = torch.empty(self.M1, dtype=self.cdtype).pin_memory().numpy()
        pf = self._host_arr(f, self.M1, "f") if f is not None else None
        py = self._host_arr(y, self.M2, "y") if f is not None else None
        pg = self._host_arr(g, self.M2, "g") if g is not None else None
        pz = self._host_arr(z, self.M1, "z") if g is not None else None
        h = ctypes.c_void_p()
        _check(self._lib.nnfft_transform_host_graph(
            self._h, ctypes.c_void_p(v.ctypes.data), ctypes.c_void_p(x.ctypes.data), pf, py, pg,
            pz, ctypes.byref(h)))
        return TransformGraph(self, h, (v, x, f, g, y if f is not None else None,
                                        z if g is not None else None))

    def transform_host(self, v, x, f=None, g=None, y=None, z=None):
        """New nodes and both directions from host arrays in one call (overlapped copies):
        returns (A f, A^H g); a direction is skipped when its input is None."""
        for arr, n, name in ((v, self.M1, "v"), (x, self.M2, "x")):
            if not (isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.size == n
                    and arr.flags.c_contiguous):
                raise TypeError(f"{name} must be a contiguous float64 numpy array of {n}")
        if f is not None and y is None:
            y = np.empty(self.M2, dtype=self.np_cdtype)
        if g is not None and z is None:
            z = np.empty(self.M1, dtype=self.np_cdtype)
        pf = self._host_arr(f, self.M1, "f") if f is not None else None
        py = self._host_arr(y, self.M2, "y") if f is not None else None
        pg = self._host_arr(g, self.M2, "g") if g is not None else None
        pz = self._host_arr(z, self.M1, "z") if g is not None else None
        _check(self._lib.nnfft_transform_host(self._h, ctypes.c_void_p(v.ctypes.data),
                                              ctypes.c_void_p(x.ctypes.data), pf, py, pg, pz))
        return y, z

    def exec_host(self, f, out=None):
        out = np.empty(self.M2, dtype=self.np_cdtype) if out is None else out
        _check(self._lib.nnfft_exec_host(self._h, self._host_arr(f, self.M1, "f"),
                                         self._host_arr(out, self.M2, "out")))
        return out

    def adjoint_host(self, g, out=None):
        out = np.empty(self.M1, dtype=self.np_cdtype) if out is None else out
        _check(self._lib.nnfft_adjoint_host(self._h, self._host_arr(g, self.M2, "g"),
                                            self._host_arr(out, self.M1, "out")))
        return out

    def sync(self):
        _check(self._lib.nnfft_sync(self._h))

    def node_order(self, side):
        """(perm, off) of side 0 (v) or 1 (x) after set_nodes: perm[i] = caller index of
        sorted position i, and cell c holds the sorted positions off[c] .. off[c + 1] - 1."""
        ncell = ctypes.c_int64()
        _check(self._lib.nnfft_node_order(self._h, int(side), None, None, ctypes.byref(ncell)))
        M = self.M1 if side == 0 else self.M2
        perm = np.empty(M, dtype=np.int32)
        off = np.empty(ncell.value + 1, dtype=np.int32)
        _check(self._lib.nnfft_node_order(self._h, int(side), perm.ctypes.data, off.ctypes.data,
                                          None))
        return perm, off

    def timing(self, enable=True):
        """Bracket every stage with CUDA events on the plan stream (tracing)."""
        _check(self._lib.nnfft_timing_enable(self._h, int(bool(enable))))

    def timing_read(self, reset=True) -> dict:
        """{stage: (total_ms, count)} accumulated since the last reset (waits for the stream)."""
        t = Timing()
        _check(self._lib.nnfft_timing_read(self._h, ctypes.byref(t), int(bool(reset))))
        return {name: (t.ms[i], int(t.count[i])) for i, name in enumerate(STAGES)}

    def close(self):
        for gr in list(getattr(self, "_graphs", ())):     # graphs first: they use the plan
            gr.close()
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nnfft_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TransformGraph:
    """A captured nnfft_transform or nnfft_transform_host (see Plan.transform_graph and
    Plan.transform_host_graph).  launch() replays it on the plan stream; y and z hold the
    results."""

    def __init__(self, plan, handle, tensors):
        self._plan, self._h = plan, handle
        self._keep = tensors                    # the buffers the graph reads and writes
        self.y, self.z = tensors[4], tensors[5]
        self.kernels = int(plan._lib.nnfft_graph_kernels(handle))
        if not hasattr(plan, "_graphs"):
            plan._graphs = weakref.WeakSet()
        plan._graphs.add(self)

    def launch(self):
        if self._h is None:
            raise NNFFTError(1, "graph closed")
        _check(self._plan._lib.nnfft_graph_launch(self._h))
        return self.y, self.z

    def close(self):
        if self._h is not None and self._h.value:
            self._plan._lib.nnfft_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan(Plan):
    """Many independent NNFFT instances in one plan (one launch per stage for all of them).

    N, M1, M2: sequences of equal length (one entry per instance); sigma, m and dtype are
    shared.  Node, coefficient and output tensors are the instances' arrays concatenated
    in instance order (offsets in `off1` / `off2`); every method of Plan applies.
    """

    def __init__(self, N, M1, M2, sigma1=2.0, sigma2=2.0, m1=8, m2=None, dtype=None,
                 stream=None, window="sinh"):
        import torch
        lib = load_library()
        N, M1, M2 = (np.ascontiguousarray(a, dtype=np.int64).ravel() for a in (N, M1, M2))
        if not (N.size == M1.size == M2.size) or N.size == 0:
            raise ValueError("N, M1 and M2 need one entry per instance (at least one)")
        dtype = torch.complex128 if dtype is None else dtype
        self.dtype = dtype
        self.cdtype = torch.complex128 if _dtype_code(dtype) == NNFFT_C128 else torch.complex64
        self.np_cdtype = np.complex128 if self.cdtype == torch.complex128 else np.complex64
        self.count = int(N.size)
        self.Ns, self.M1s, self.M2s = N.copy(), M1.copy(), M2.copy()
        self.off1 = np.concatenate([[0], np.cumsum(M1)]).astype(np.int64)
        self.off2 = np.concatenate([[0], np.cumsum(M2)]).astype(np.int64)
        self.M1, self.M2, self.N = int(self.off1[-1]), int(self.off2[-1]), int(N.max())
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._h = ctypes.c_void_p()
        m2 = m1 if m2 is None else m2
        pi = ctypes.POINTER(ctypes.c_int64)
        _check(lib.nnfft_batch_plan_window(ctypes.byref(self._h), self.count,
                                           N.ctypes.data_as(pi), M1.ctypes.data_as(pi),
                                           M2.ctypes.data_as(pi), float(sigma1), float(sigma2),
                                           int(m1), int(m2), _dtype_code(dtype),
                                           _window_code(window), _stream_ptr(self.stream)))
        self._lib = lib

    def instance_info(self, i) -> dict:
        info = Info()
        _check(self._lib.nnfft_batch_info(self._h, int(i), ctypes.byref(info)))
        return info.as_dict()


def tolerance_params(tol):
    """(dtype code, m) that the request loop serves a tolerance with."""
    lib = load_library()
    dt, m = ctypes.c_int(), ctypes.c_int()
    _check(lib.nnfft_tolerance_params(float(tol), ctypes.byref(dt), ctypes.byref(m)))
    return dt.value, m.value


class Server:
    """Request loop (continuous batching) for NNFFT and sinc requests on the current GPU.

    Arrays are host numpy arrays (pinned ones copy asynchronously) of the tolerance's type
    (tolerance_params: complex64/float32 for tol >= 1e-6, complex128/float64 otherwise);
    they must stay alive until wait() returns for the request.
    """

    def __init__(self, mem_budget_bytes=64 << 30, slots=4, max_points=1 << 22):
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p()
        self._keep = {}
        _check(lib.nnfft_server_create(ctypes.byref(self._h), int(mem_budget_bytes), int(slots),
                                       int(max_points)))

    @staticmethod
    def _ptr(a, dtypes, n, name):
        if not (isinstance(a, np.ndarray) and a.dtype in dtypes and a.size == n and a.flags.c_contiguous):
            raise TypeError(f"{name} must be a contiguous {'/'.join(map(str, dtypes))} array of {n}")
        return a.ctypes.data if n else None

    def _submit(self, kind, N, v, x, f, y, tol, rule=0, is_complex=1):
        dt, _ = tolerance_params(tol)
        c = np.complex128 if dt == NNFFT_C128 else np.complex64
        r = np.float64 if dt == NNFFT_C128 else np.float32
        vals = (np.dtype(c),) if is_complex else (np.dtype(r),)
        req = Request(kind, int(rule), int(is_complex), 0, int(N), int(v.size), int(x.size), float(tol),
                      self._ptr(v, (np.dtype(np.float64),), v.size, "v"),
                      self._ptr(x, (np.dtype(np.float64),), x.size, "x"),
                      self._ptr(f, vals, v.size, "f"), self._ptr(y, vals, x.size, "y"))
        rid = ctypes.c_int64()
        _check(self._lib.nnfft_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)))
        self._keep[rid.value] = (v, x, f, y)
        return rid.value

    def submit_nnfft(self, N, v, x, f, y, tol):
        """y = sum_k f_k exp(-2 pi i N v_k x); returns the request id."""
        return self._submit(0, N, v, x, f, y, tol)

    def submit_sinc(self, N, a, c, b, h, tol, rule="gl"):
        """h = sum_k c_k sinc(N pi (b - a_k)) (Algorithm 6.1); returns the request id."""
        return self._submit(1, N, a, b, c, h, tol, _rule_code(rule), int(np.iscomplexobj(c)))

    def wait(self, rid):
        """Block until the request is done; returns its latency in ms."""
        lat = ctypes.c_double()
        try:
            _check(self._lib.nnfft_server_wait(self._h, int(rid), ctypes.byref(lat)))
        finally:
            self._keep.pop(rid, None)
        return lat.value

    def wait_device(self, rid):
        """wait() that also returns where the request ran on the device: (latency_ms,
        [before uploads, first kernel, after last kernel, after download]) in ms since the
        server was made."""
        lat = ctypes.c_double()
        t = (ctypes.c_double * 4)()
        try:
            _check(self._lib.nnfft_server_wait_device(self._h, int(rid), ctypes.byref(lat), t))
        finally:
            self._keep.pop(rid, None)
        return lat.value, list(t)

    def stats(self, reset=False) -> dict:
        rep = ServerReport()
        _check(self._lib.nnfft_server_stats(self._h, ctypes.byref(rep), int(bool(reset))))
        return rep.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nnfft_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SINC_RULES = {"gl": 0, "cc": 1}


def _rule_code(rule):
    try:
        return SINC_RULES[rule]
    except KeyError:
        raise ValueError(f"unknown quadrature rule {rule!r} (use 'gl' or 'cc')") from None


def sinc_quadrature(rule, N, n=0):
    """The quadrature rule (t, w) that sinc() uses: 'gl' (n nodes, default 2N) or 'cc'
    (nodes cos(j pi/n)/2, j = 0..n, default n = 4N, weights from the GPU)."""
    lib = load_library()
    cnt = ctypes.c_int64(0)
    _check(lib.sinc_quadrature(_rule_code(rule), int(N), int(n), None, None, ctypes.byref(cnt)))
    t = np.zeros(cnt.value); w = np.zeros(cnt.value)
    _check(lib.sinc_quadrature(_rule_code(rule), int(N), int(n), t.ctypes.data, w.ctypes.data,
                               ctypes.byref(cnt)))
    return t, w


def sinc(N, a, c, b, m=8, out=None, stream=None, rule="gl", n=0):
    """Fast sinc transform (Algorithm 6.1).

    a: L1 float64 CUDA nodes, c: L1 coefficients (float64/float32 real or
    complex128/complex64), b: L2 float64 CUDA targets.  Returns h (L2) of c's type.
    fp64 types use the fp64 path, fp32 types the fp32 path.  rule 'gl': n-point
    Gauss-Legendre (n = 0: 2N); rule 'cc': Clenshaw-Curtis with n + 1 Chebyshev
    nodes (n = 0: 4N, rounded up to 5-smooth).
    """
    import torch
    lib = load_library()
    L1, L2 = a.numel(), b.numel()
    is_complex = c.is_complex()
    dbl = c.dtype in (torch.float64, torch.complex128)
    code = NNFFT_C128 if dbl else NNFFT_C64
    pa = _dev_tensor(a, torch.float64, L1, "a")
    pb = _dev_tensor(b, torch.float64, L2, "b")
    pc = _dev_tensor(c, c.dtype, L1, "c")
    if out is None:
        out = torch.empty(L2, dtype=c.dtype, device=b.device)
    po = _dev_tensor(out, c.dtype, L2, "out")
    _check(lib.sinc_exec_rule(int(N), int(L1), int(L2), int(m), code, _rule_code(rule), int(n),
                              pa, pc, pb, po, int(is_complex), _stream_ptr(stream)))
    return out


def selftest_fixed63(y):
    """Node-kernel conversion check: for an int64 device tensor of fixed-point coordinates
    (value y 2^-63) returns an (n, 4) float32 tensor: the fp32 plans' float, the split
    plans' float pair (h, l), then CUDA's rounding conversion."""
    import torch
    if y.dtype != torch.int64 or not y.is_cuda or not y.is_contiguous():
        raise TypeError("y must be a contiguous int64 CUDA tensor")
    out = torch.empty((y.numel(), 4), dtype=torch.float32, device=y.device)
    _check(load_library().nnfft_selftest_fixed63(ctypes.c_void_p(y.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr()), y.numel()))
    return out


def selftest_bulk_copy(src, arm_only=False, limit_cycles=2_000_000):
    """Bounded-wait check of the bulk (TMA) copy helpers: returns (dst, status) where dst
    is src staged through shared memory (zeros if the wait gave up) and status the bits the
    block set (4: the wait gave up).  arm_only skips the copy, so the wait runs out."""
    import torch
    if src.dtype != torch.float32 or not src.is_cuda or not src.is_contiguous():
        raise TypeError("src must be a contiguous float32 CUDA tensor")
    dst = torch.zeros_like(src)
    status = torch.zeros(1, dtype=torch.int32, device=src.device)
    torch.cuda.synchronize()
    _check(load_library().nnfft_selftest_bulk_copy(
        ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), src.numel(),
        int(bool(arm_only)), int(limit_cycles), ctypes.c_void_p(status.data_ptr())))
    return dst, int(status.item())


def selftest_grid_barrier(blocks=2, extra=0, limit_cycles=2_000_000, words=None):
    """Bounded-wait check of the fused grid stage's grid barrier: a cooperative launch of
    `blocks` blocks passes two barriers expecting blocks + extra arrivals.  Returns (words,
    status): the barrier words after the launch (arrival counter, abort word) and the bits
    the blocks set (4: a wait gave up, which extra > 0 forces).  words: a zeroed int64 CUDA
    tensor of 2 elements to reuse across calls (None: a fresh one)."""
    import torch
    if words is None:
        words = torch.zeros(2, dtype=torch.int64, device="cuda")
    if words.dtype != torch.int64 or words.numel() != 2 or not words.is_cuda:
        raise TypeError("words must be a CUDA int64 tensor of 2 elements")
    status = torch.zeros(1, dtype=torch.int32, device=words.device)
    torch.cuda.synchronize()
    _check(load_library().nnfft_selftest_grid_barrier(
        int(blocks), int(extra), int(limit_cycles), ctypes.c_void_p(words.data_ptr()),
        ctypes.c_void_p(status.data_ptr())))
    return words, int(status.item())


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().nnfft_launch_count())


def sinc_sync(stream=None):
    lib = load_library()
    _check(lib.sinc_sync(_stream_ptr(stream)))


def sinc_release():
    lib = load_library()
    _check(lib.sinc_release())
