"""CPU tests of the C ABI library: it loads without a GPU, exports every function
include/nnfft.h declares, and its host-side logic (plan parameters, window fits,
Gauss-Legendre rule, error paths) agrees with the oracle.  No compute call is
made on a device."""
import ctypes
import math
from fractions import Fraction
import os
import re

import numpy as np
import pytest

import oracle
from paper_2107_02671_gb300 import nnfft as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                text, flags=re.M)
    return sorted(set(names))


def test_library_loads_and_exports_every_declared_symbol():
    lib = B.load_library()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"missing export {n}"


@pytest.mark.parametrize("N,s1,s2,m1,m2", [(64, 2, 2, 4, 4), (4096, 2, 2, 8, 8), (1024, 2, 2, 8, 8),
                                           (1000, 1.5, 1.25, 6, 3), (77, 1.3, 2.2, 2, 5),
                                           (16384, 2, 2, 8, 8), (4096, 2, 2, 4, 4), (40000, 2, 2, 8, 8)])
def test_plan_parameters_match_oracle(N, s1, s2, m1, m2):
    for dt in ("complex128", "complex64"):
        info = B.params(N, 1000, 999, s1, s2, m1, m2, dt)
        P = oracle.make_params(N, s1, s2, m1, m2)
        for k in ("Nstar", "N1", "K1", "N2"):
            assert info[k] == getattr(P, k), k
        for k in ("sigma1", "sigma2", "beta1", "beta2"):
            assert abs(info[k] - getattr(P, k)) < 1e-12 * abs(getattr(P, k)), k
        assert info["fft_n1"] * info["fft_n2"] == info["N2"]
        assert max(info["fft_n1"], info["fft_n2"]) <= 1024
        # cell counts cover every node in [-1/2, 1/2]: u = v N1 N / N* (exact rational)
        us1 = Fraction(P.N1 * N, P.Nstar)
        assert info["ncell1"] == math.floor(us1 / 2) - math.floor(-us1 / 2) + 1
        us2 = Fraction(P.N2 * P.Nstar, P.N1)
        assert info["ncell2"] == math.floor(us2 / 2) - math.floor(-us2 / 2) + 1


def test_window_fit_is_accurate_against_oracle_window():
    """The library's chosen Chebyshev degree reaches the fit error it reports, and that
    error is far below the window's own error (Theorem 4.1, first term)."""
    for m, dt in [(8, "complex128"), (4, "complex64"), (4, "complex128"), (6, "complex128"), (2, "complex64")]:
        info = B.params(256, 10, 10, 2, 2, m, m, dt)
        E, t1, _ = oracle.bound_sinh(info["N1"], m, m, info["sigma1"], info["sigma2"])
        assert info["fit_err1"] < max(0.05 * t1, 2e-14)
        assert info["D1"] in (8, 10, 12, 14, 16, 20)
    assert B.params(4096, 10, 10, 2, 2, 8, 8, "complex128")["D1"] <= 16
    assert B.params(4096, 10, 10, 2, 2, 4, 4, "complex64")["D1"] <= 10


def test_invalid_parameters_rejected():
    bad = [dict(N=0), dict(m1=1), dict(m2=17), dict(sigma1=1.0), dict(sigma2=0.5), dict(M1=-1),
           dict(N=4, sigma1=1.05, sigma2=1.05, m2=9)]
    for kw in bad:
        args = dict(N=64, M1=10, M2=10, sigma1=2.0, sigma2=2.0, m1=4, m2=4, dtype="complex128")
        args.update(kw)
        with pytest.raises(B.NNFFTError) as ei:
            B.params(**args)
        assert ei.value.code == 1


def test_gauss_legendre_matches_oracle():
    for n in (1, 2, 7, 128, 2048):
        t1, w1 = B.gauss_legendre(n)
        t2, w2 = oracle.gauss_legendre(n)
        assert np.max(np.abs(t1 - t2)) < 1e-15
        assert np.max(np.abs(w1 - w2)) < 1e-15


def test_plan_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = B.load_library()
    h = ctypes.c_void_p()
    rc = lib.nnfft_plan(ctypes.byref(h), 64, 10, 10, 2.0, 2.0, 4, 4, 1, None)
    assert rc == 4 and not h.value
    assert b"CUDA" in lib.nnfft_last_error() or len(lib.nnfft_last_error()) > 0


def test_tolerance_classes():
    """The request loop serves tol >= 1e-6 in fp32 and smaller tolerances in fp64, with the
    smallest m whose Theorem 4.1 first term (sigma = 2) is below tol."""
    assert B.tolerance_params(1e-5) == (B.NNFFT_C64, 4)
    assert B.tolerance_params(1e-9) == (B.NNFFT_C128, 6)
    assert B.tolerance_params(1e-12) == (B.NNFFT_C128, 8)
    for tol in (1e-3, 1e-5, 1e-7, 1e-9, 1e-11, 1e-13):
        _, m = B.tolerance_params(tol)
        term = lambda mm: (24 * mm ** 1.5 + 10) * math.exp(-2 * math.pi * mm * math.sqrt(0.5))  # noqa: E731
        assert term(m) <= tol and (m == 2 or term(m - 1) > tol)


@pytest.mark.parametrize("window", ["sinh", "kaiser_bessel", "bspline", "algebraic"])
def test_library_windows_match_the_oracle(window):
    """The library's host-side windows and Fourier transforms (its own code: C++ special
    functions, a different B-spline recursion) against the oracle's, m = 2..8."""
    import oracle
    worst = 0.0
    for m in (2, 3, 4, 6, 8):
        for sg in (1.25, 1.5, 2.0):
            P = oracle.make_params(64, sg, sg, m, m, window=window)
            beta = {"bspline": 0.0, "algebraic": 3.0 * m}.get(window, 2 * np.pi * m * (1 - 1 / (2 * sg)))
            for x in np.linspace(-1.1, 1.1, 23):
                a, _ = B.window(window, m, sg, x, 0.0)
                worst = max(worst, abs(a - float(oracle.omega(window, x, beta, m))))
            for v in np.linspace(0, m / (2 * sg), 7):
                _, a = B.window(window, m, sg, 0.0, v)
                b = float(oracle.omega_hat(window, v, beta, m))
                worst = max(worst, abs(a - b) / abs(b))
            info = B.params(64, 100, 100, sg, sg, m, m, window=window)
            assert info["window"] == B.WINDOWS[window]
            assert info["beta1"] == pytest.approx(P.beta1, rel=1e-12, abs=0)
    assert worst < 1e-13
    with pytest.raises(B.NNFFTError):
        B.params(300, 10, 10, 1.04, 2.0, 4, 4, window="algebraic")   # sigma <= pi/3
