"""CPU fp64 oracle for the NNFFT with sinh-type windows and the sinc transform.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2107_02671_gb300``) never imports it, and this package imports nothing
from the product path: the two share no code, helpers or tables.

The arithmetic lives in ``oracle.c`` (plain C, fp64, optional OpenMP over output
rows); this module only compiles it with gcc and marshals numpy arrays.  Each
wrapper names the passage of Kircheis, Potts and Tasche that it follows.

Pinned by ``tests/test_oracle_pins.py``; every function here has at least one pin
that does not reuse its own formula.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

i64 = ctypes.c_longlong
dptr = ctypes.POINTER(ctypes.c_double)
lptr = ctypes.POINTER(ctypes.c_longlong)


class Params(ctypes.Structure):
    """Algorithm 2.2 parameters (Section 2, Section 4), see ``make_params``."""

    _fields_ = [
        ("N", i64), ("Nstar", i64), ("N1", i64), ("K1", i64), ("N2", i64),
        ("m1", ctypes.c_int), ("m2", ctypes.c_int),
        ("sigma1", ctypes.c_double), ("sigma2", ctypes.c_double),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("a", ctypes.c_double),
        ("window", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_expsum.argtypes = [i64, i64, dptr, dptr, i64, dptr, ctypes.c_int, lptr, i64,
                                   dptr, ctypes.c_int]
        lib.orc_sinc_direct.argtypes = [i64, i64, dptr, dptr, i64, dptr, lptr, i64, dptr,
                                        ctypes.c_int]
        lib.orc_sinc_Npi.argtypes = [i64, ctypes.c_double, ctypes.c_double]
        lib.orc_sinc_Npi.restype = ctypes.c_double
        lib.orc_gauss_legendre.argtypes = [i64, dptr, dptr]
        lib.orc_sinc_gl.argtypes = [i64, i64, i64, dptr, dptr, i64, dptr, lptr, i64, dptr,
                                    ctypes.c_int]
        lib.orc_sinc_cc.argtypes = [i64, i64, i64, dptr, dptr, i64, dptr, lptr, i64, dptr,
                                    ctypes.c_int]
        lib.orc_omega_sinh.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_omega_sinh.restype = ctypes.c_double
        lib.orc_omega_sinh_hat.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_omega_sinh_hat.restype = ctypes.c_double
        lib.orc_phi.argtypes = [ctypes.c_double, i64, ctypes.c_int, ctypes.c_double]
        lib.orc_phi.restype = ctypes.c_double
        lib.orc_phi_hat.argtypes = [ctypes.c_double, i64, ctypes.c_int, ctypes.c_double]
        lib.orc_phi_hat.restype = ctypes.c_double
        lib.orc_make_params.argtypes = [i64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(Params)]
        lib.orc_make_params_w.argtypes = [i64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params)]
        lib.orc_omega_w.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.orc_omega_w.restype = ctypes.c_double
        lib.orc_omega_hat_w.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int]
        lib.orc_omega_hat_w.restype = ctypes.c_double
        lib.orc_phi_hat_w.argtypes = [ctypes.c_int, ctypes.c_double, i64, ctypes.c_int,
                                      ctypes.c_double]
        lib.orc_phi_hat_w.restype = ctypes.c_double
        lib.orc_nnfft_alg22.argtypes = [ctypes.POINTER(Params), i64, dptr, dptr, i64, dptr,
                                        dptr, dptr, dptr, ctypes.c_int]
        lib.orc_nnfft_alg22_adjoint.argtypes = [ctypes.POINTER(Params), i64, dptr, i64, dptr,
                                                dptr, dptr, ctypes.c_int]
        lib.orc_bound_sinh.argtypes = [i64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, dptr]
        lib.orc_bound_sinh.restype = ctypes.c_double
        lib.orc_cc_weights.argtypes = [i64, dptr, dptr]
        lib.orc_cc_constant.restype = ctypes.c_double
        lib.orc_cc_bound.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_cc_bound.restype = ctypes.c_double
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(dptr)


def _real(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cplx(a):
    """complex array -> contiguous interleaved float64 view (length 2n)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _rows(rows):
    if rows is None:
        return None, 0
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return r, len(r)


def num_threads() -> int:
    """OpenMP threads the oracle uses by default (1 without OpenMP)."""
    return int(_load().orc_num_threads())


def expsum(N, a, c, b, sign=-1, rows=None, nthreads=0):
    """out_j = sum_k c_k exp(sign 2 pi i N a_k b_j), eq. (1.2) -- a direct O(len(a) len(b)) sum.

    sign=-1, a=v, b=x is the NNFFT; sign=+1, a=x, c=g, b=v its adjoint.
    ``rows`` restricts the evaluation to the listed outputs (in that order).
    """
    lib = _load()
    a = _real(a); b = _real(b); cc = _cplx(c)
    assert cc.size == 2 * a.size
    r, nr = _rows(rows)
    nout = nr if r is not None else b.size
    out = np.zeros(nout, dtype=np.complex128)
    rc = lib.orc_expsum(int(N), a.size, _d(a), _d(cc), b.size, _d(b), int(sign),
                        r.ctypes.data_as(lptr) if r is not None else None, nr,
                        _d(out.view(np.float64)), int(nthreads))
    assert rc == 0
    return out


def nnfft_direct(N, v, f, x, rows=None, nthreads=0):
    """f(x_j) = sum_k f_k exp(-2 pi i N v_k x_j), eq. (1.2), by definition."""
    return expsum(N, v, f, x, -1, rows, nthreads)


def nnfft_adjoint_direct(N, v, x, g, rows=None, nthreads=0):
    """z_k = sum_j g_j exp(+2 pi i N v_k x_j) (the adjoint of eq. (1.2)), by definition."""
    return expsum(N, x, g, v, +1, rows, nthreads)


def sinc_Npi(N, b, a):
    """sinc(N pi (b - a)) of eq. (5.2), with exact argument reduction."""
    return float(_load().orc_sinc_Npi(int(N), float(b), float(a)))


def sinc_direct(N, a, c, b, rows=None, nthreads=0):
    """h(b_l) = sum_k c_k sinc(N pi (b_l - a_k)), eq. (6.2), directly."""
    lib = _load()
    a = _real(a); b = _real(b); cc = _cplx(c)
    r, nr = _rows(rows)
    nout = nr if r is not None else b.size
    out = np.zeros(nout, dtype=np.complex128)
    rc = lib.orc_sinc_direct(int(N), a.size, _d(a), _d(cc), b.size, _d(b),
                             r.ctypes.data_as(lptr) if r is not None else None, nr,
                             _d(out.view(np.float64)), int(nthreads))
    assert rc == 0
    return out


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes (increasing) and weights on [-1/2, 1/2], sum(w) = 1."""
    lib = _load()
    tau = np.zeros(int(n)); w = np.zeros(int(n))
    assert lib.orc_gauss_legendre(int(n), _d(tau), _d(w)) == 0
    return tau, w


def sinc_gl(N, a, c, b, n=None, rows=None, nthreads=0):
    """Eq. (6.3) with an n-point Gauss-Legendre rule on [-1/2,1/2] (n = 2N default)."""
    lib = _load()
    n = 2 * int(N) if n is None else int(n)
    a = _real(a); b = _real(b); cc = _cplx(c)
    r, nr = _rows(rows)
    nout = nr if r is not None else b.size
    out = np.zeros(nout, dtype=np.complex128)
    rc = lib.orc_sinc_gl(int(N), n, a.size, _d(a), _d(cc), b.size, _d(b),
                         r.ctypes.data_as(lptr) if r is not None else None, nr,
                         _d(out.view(np.float64)), int(nthreads))
    assert rc == 0
    return out


def sinc_cc(N, a, c, b, n=None, rows=None, nthreads=0):
    """Algorithm 6.1 with the Clenshaw-Curtis rule (z_j = cos(j pi/n), eq. (5.4) weights,
    n = 4N default), each step a direct sum."""
    lib = _load()
    n = 4 * int(N) if n is None else int(n)
    a = _real(a); b = _real(b); cc = _cplx(c)
    r, nr = _rows(rows)
    nout = nr if r is not None else b.size
    out = np.zeros(nout, dtype=np.complex128)
    rc = lib.orc_sinc_cc(int(N), n, a.size, _d(a), _d(cc), b.size, _d(b),
                         r.ctypes.data_as(lptr) if r is not None else None, nr,
                         _d(out.view(np.float64)), int(nthreads))
    assert rc == 0
    return out


def omega_sinh(x, beta):
    """Sinh-type window of Example 2.1 (vectorised over x)."""
    lib = _load()
    return np.vectorize(lambda t: lib.orc_omega_sinh(float(t), float(beta)))(np.asarray(x, float))


def omega_sinh_hat(v, beta):
    """Eq. (2.1), the Fourier transform of omega_sinh (vectorised over v)."""
    lib = _load()
    return np.vectorize(lambda t: lib.orc_omega_sinh_hat(float(t), float(beta)))(
        np.asarray(v, float))


def phi(t, Nj, m, beta):
    """phi_j(t) = omega(N_j t / m_j), eq. (2.5)."""
    lib = _load()
    return np.vectorize(lambda s: lib.orc_phi(float(s), int(Nj), int(m), float(beta)))(
        np.asarray(t, float))


def phi_hat(v, Nj, m, beta):
    """phihat_j(v) = (m_j/N_j) omegahat(m_j v / N_j) (proof of Theorem 3.4)."""
    lib = _load()
    return np.vectorize(lambda s: lib.orc_phi_hat(float(s), int(Nj), int(m), float(beta)))(
        np.asarray(v, float))


WINDOWS = {"sinh": 0, "kaiser_bessel": 1, "bspline": 2, "algebraic": 3}


def omega(window, x, beta, m):
    """Window omega of the set Omega (Section 2): 'sinh' (Example 2.1 / Section 4),
    'kaiser_bessel', 'bspline' or 'algebraic' (Example 2.1), vectorised over x."""
    lib = _load()
    w = WINDOWS[window]
    return np.vectorize(lambda t: lib.orc_omega_w(w, float(t), float(beta), int(m)))(
        np.asarray(x, float))


def omega_hat(window, v, beta, m):
    """Fourier transform of omega(window, ., beta, m) by its closed form (vectorised)."""
    lib = _load()
    w = WINDOWS[window]
    return np.vectorize(lambda t: lib.orc_omega_hat_w(w, float(t), float(beta), int(m)))(
        np.asarray(v, float))


def phi_hat_w(window, v, Nj, m, beta):
    """phihat_j(v) = (m_j/N_j) omegahat(m_j v / N_j) for any window (vectorised over v)."""
    lib = _load()
    w = WINDOWS[window]
    return np.vectorize(lambda t: lib.orc_phi_hat_w(w, float(t), int(Nj), int(m), float(beta)))(
        np.asarray(v, float))


def make_params(N, sigma1=2.0, sigma2=2.0, m1=4, m2=None, window="sinh"):
    """Parameters of Algorithm 2.2 for nodes in [-1/2,1/2] (Section 2) -> Params or ValueError.
    ``window`` selects the window of both steps (see omega); Algorithm 2.2 then uses it."""
    lib = _load()
    m2 = m1 if m2 is None else m2
    P = Params()
    rc = lib.orc_make_params_w(int(N), float(sigma1), float(sigma2), int(m1), int(m2),
                               WINDOWS[window], ctypes.byref(P))
    if rc != 0:
        raise ValueError("invalid NNFFT parameters")
    return P


def nnfft_alg22(P, v, f, x, nthreads=0, return_stages=False):
    """Algorithm 2.2 step by step (naive DFT in step 3); optionally the step-1 g and step-3 h."""
    lib = _load()
    v = _real(v); x = _real(x); ff = _cplx(f)
    out = np.zeros(x.size, dtype=np.complex128)
    g = np.zeros(P.K1, dtype=np.complex128)
    h = np.zeros(P.N2, dtype=np.complex128)
    rc = lib.orc_nnfft_alg22(ctypes.byref(P), v.size, _d(v), _d(ff), x.size, _d(x),
                             _d(out.view(np.float64)), _d(g.view(np.float64)),
                             _d(h.view(np.float64)), int(nthreads))
    assert rc == 0
    return (out, g, h) if return_stages else out


def nnfft_alg22_adjoint(P, v, x, g, nthreads=0):
    """Exact transpose of Algorithm 2.2 (each step reversed)."""
    lib = _load()
    v = _real(v); x = _real(x); gg = _cplx(g)
    z = np.zeros(v.size, dtype=np.complex128)
    rc = lib.orc_nnfft_alg22_adjoint(ctypes.byref(P), v.size, _d(v), x.size, _d(x), _d(gg),
                                     _d(z.view(np.float64)), int(nthreads))
    assert rc == 0
    return z


def bound_sinh(N1, m1, m2, sigma1, sigma2):
    """Theorem 4.1: (E, term1, term2) of the NNFFT error constant E(phi_sinh)."""
    lib = _load()
    t = np.zeros(2)
    e = lib.orc_bound_sinh(int(N1), int(m1), int(m2), float(sigma1), float(sigma2), _d(t))
    return float(e), float(t[0]), float(t[1])


def cc_weights(n):
    """Chebyshev points z_k = cos(k pi/n) and Clenshaw-Curtis weights of eq. (5.4), k = 0..n."""
    lib = _load()
    z = np.zeros(int(n) + 1); w = np.zeros(int(n) + 1)
    assert lib.orc_cc_weights(int(n), _d(z), _d(w)) == 0
    return z, w


def cc_constant():
    """C = pi (e^2 - 1) / (2 e) of Theorem 5.3."""
    return float(_load().orc_cc_constant())


def cc_bound(N, nu):
    """Right-hand side of Theorem 5.3 for n = nu N."""
    return float(_load().orc_cc_bound(float(N), float(nu)))


def relative_error(approx, exact, coeffs):
    """max_j |approx_j - exact_j| / sum_k |coeffs_k|, eq. (4.5)."""
    approx = np.asarray(approx); exact = np.asarray(exact)
    return float(np.max(np.abs(approx - exact)) / np.sum(np.abs(np.asarray(coeffs))))
