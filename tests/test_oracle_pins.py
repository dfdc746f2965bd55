"""Pins of the CPU oracle against things other than itself.

Every oracle function is checked against at least one of: a library routine used
as an independent route (numpy FFT, numpy Gauss-Legendre, scipy Bessel functions
and quadrature), a closed form or invariant the paper states, brute force at
higher precision (mpmath), or a number the paper prints (tests/golden/).
A plausible slip in the oracle -- a dropped term, a wrong sign, a swapped index or
a missing scale -- fails at least one test here.  No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2107_02671_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# --------------------------------------------------------------------------------------
# eq. (1.2): the direct exponential sum
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [8, 16, 30])
def test_expsum_equispaced_is_the_dft(N):
    """v_k = k/N, x_j = j/N (k, j in I_N) turn eq. (1.2) into a length-N DFT (numpy FFT)."""
    rng = np.random.default_rng(N)
    k = np.arange(-N // 2, N - N // 2)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = oracle.nnfft_direct(N, k / N, f, k / N)
    # sum_{k in I_N} f_k e^{-2 pi i k j / N} = e^{2 pi i (N//2) j / N} * FFT(f in natural order)[j mod N]
    F = np.fft.fft(f)          # f[i] is the coefficient of k = i - N//2
    ref = np.exp(2j * np.pi * (N // 2) * k / N) * F[np.mod(k, N)]
    assert np.max(np.abs(y - ref)) < 1e-13 * np.sum(np.abs(f))


def test_expsum_single_term_matches_high_precision():
    """One coefficient at large N: exp(-2 pi i N v x) against 50-digit mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(3)
    N = 1 << 22
    v = rng.uniform(-0.5, 0.5, 5)
    x = rng.uniform(-0.5, 0.5, 7)
    for k in range(5):
        f = np.zeros(5, complex); f[k] = 1.0
        y = oracle.nnfft_direct(N, v, f, x)
        for j in range(7):
            ph = -2 * mp.pi * N * mp.mpf(float(v[k])) * mp.mpf(float(x[j]))
            ref = complex(mp.cos(ph), mp.sin(ph))
            assert abs(y[j] - ref) < 5e-15


def test_expsum_linearity_and_rows():
    rng = np.random.default_rng(5)
    v, x, f = W.nnfft_inputs(40, 33, 1)
    g = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    N = 100
    y = oracle.nnfft_direct(N, v, 2.5 * f - 1j * g, x)
    ref = 2.5 * oracle.nnfft_direct(N, v, f, x) - 1j * oracle.nnfft_direct(N, v, g, x)
    assert np.max(np.abs(y - ref)) < 1e-12
    rows = np.array([32, 0, 7])
    assert np.allclose(oracle.nnfft_direct(N, v, f, x, rows=rows), oracle.nnfft_direct(N, v, f, x)[rows],
                       rtol=0, atol=1e-13)


def test_adjoint_identity_of_direct_sums():
    """<A f, g> = <f, A* g> with A from eq. (1.2) and A* its conjugate transpose."""
    v, x, f = W.nnfft_inputs(50, 70, 2)
    g = W.adjoint_inputs(70, 2)
    N = 300
    Af = oracle.nnfft_direct(N, v, f, x)
    Ag = oracle.nnfft_adjoint_direct(N, v, x, g)
    lhs = np.vdot(g, Af)
    rhs = np.vdot(Ag, f)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the adjoint is not the forward with swapped roles and the same sign
    wrong = oracle.expsum(N, x, g, v, -1)
    assert np.max(np.abs(wrong - Ag)) > 1e-3


# --------------------------------------------------------------------------------------
# eq. (6.2) and eq. (6.3)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [16, 64, 127])
def test_sinc_shannon_identity(N):
    """a_k = b_k = k/N: sinc(pi (l - k)) is the identity matrix, so h(l/N) = c_l."""
    rng = np.random.default_rng(N)
    k = np.arange(-(N // 2), N - N // 2) / N
    c = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    h = oracle.sinc_direct(N, k, c, k)
    assert np.max(np.abs(h - c)) < 1e-13


def test_sinc_single_term_matches_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(11)
    for N in (7, 1024, 1 << 20):
        a = rng.uniform(-0.5, 0.5, 4)
        b = np.concatenate([rng.uniform(-0.5, 0.5, 4), a[:1], a[1:2] + 1e-12])
        c = np.eye(4)[0].astype(complex)
        h = oracle.sinc_direct(N, a, c, b)
        for l in range(len(b)):
            d = mp.mpf(float(b[l])) - mp.mpf(float(a[0]))
            ref = mp.mpf(1) if d == 0 else mp.sin(mp.pi * N * d) / (mp.pi * N * d)
            assert abs(h[l] - complex(ref)) < 1e-15


def test_gauss_legendre_rule():
    """Sum of weights 1; exact for monomials up to degree 2n-1; numpy's leggauss as a cross-check."""
    for n in (1, 2, 5, 64, 2048):
        tau, w = oracle.gauss_legendre(n)
        assert abs(w.sum() - 1) < 1e-14
        assert np.all(np.diff(tau) > 0)
        assert np.max(np.abs(tau + tau[::-1])) < 1e-15
        t_np, w_np = np.polynomial.legendre.leggauss(n)
        assert np.max(np.abs(tau - t_np / 2)) < 1e-14
        assert np.max(np.abs(w - w_np / 2)) < 1e-14 * max(1.0, n / 64)
    tau, w = oracle.gauss_legendre(12)
    for p in range(0, 24, 2):   # int_{-1/2}^{1/2} t^p dt = 2 (1/2)^{p+1}/(p+1)
        exact = 2 * 0.5 ** (p + 1) / (p + 1)
        assert abs(np.sum(w * tau ** p) - exact) < 1e-15
    assert abs(np.sum(w * tau ** 25)) < 1e-16


@pytest.mark.parametrize("N", [64, 256])
def test_sinc_gl_definition_approximates_direct(N):
    """The 2N-node Gauss-Legendre factorisation reproduces the direct sinc sum (N >= 64)."""
    a, c, b = W.sinc_inputs(300, 200, 4)
    h = oracle.sinc_direct(N, a, c, b)
    hg = oracle.sinc_gl(N, a, c, b)
    err = np.max(np.abs(h - hg)) / np.sum(np.abs(c))
    assert err < 1e-12
    # far too few nodes must visibly fail: the check has teeth
    hbad = oracle.sinc_gl(N, a, c, b, n=N // 2)
    assert np.max(np.abs(h - hbad)) / np.sum(np.abs(c)) > 1e-6


# --------------------------------------------------------------------------------------
# Example 2.1 / eq. (2.1): the sinh-type window and its Fourier transform
# --------------------------------------------------------------------------------------
def test_omega_sinh_properties():
    beta = 2 * math.pi * 8 * 0.75
    xs = np.linspace(0, 1, 1001)
    w = oracle.omega_sinh(xs, beta)
    assert w[0] == 1.0 and w[-1] == 0.0
    assert np.all(np.diff(w) <= 0)
    assert np.allclose(oracle.omega_sinh(-xs, beta), w, rtol=0, atol=0)
    assert oracle.omega_sinh(1.5, beta) == 0.0
    # the overflow-safe quotient equals sinh(beta sqrt(1-x^2))/sinh(beta) where both are finite
    for beta in (3.0, 18.8, 37.7):
        x = np.linspace(-0.99, 0.99, 37)
        ref = np.sinh(beta * np.sqrt(1 - x ** 2)) / np.sinh(beta)
        assert np.max(np.abs(oracle.omega_sinh(x, beta) - ref) / np.maximum(ref, 1e-300)) < 8e-15


@pytest.mark.parametrize("m,sigma", [(4, 2.0), (8, 2.0), (6, 1.5), (2, 1.25)])
def test_omega_sinh_hat_against_quadrature_and_scipy(m, sigma):
    """eq. (2.1) against 2 int_0^1 omega(x) cos(2 pi v x) dx (Section 2) and scipy's I1, J1."""
    integrate = pytest.importorskip("scipy.integrate")
    special = pytest.importorskip("scipy.special")
    beta = 2 * math.pi * m * (1 - 1 / (2 * sigma))
    vb = beta / (2 * math.pi)                 # = m (1 - 1/(2 sigma)), the branch point
    for v in [0.0, 0.3 * vb, m / (2 * sigma), 0.999 * vb, vb, 1.2 * vb, 2.5 * vb]:
        quad, _ = integrate.quad(lambda t: 2 * oracle.omega_sinh(t, beta) * math.cos(2 * math.pi * v * t),
                                 0, 1, limit=400, epsabs=1e-16, epsrel=1e-13)
        val = oracle.omega_sinh_hat(v, beta)
        assert abs(val - quad) < 1e-11 * max(1.0, abs(quad)) + 1e-15
        q = beta ** 2 - 4 * math.pi ** 2 * v ** 2
        pref = math.pi * beta / math.sinh(beta)
        if q > 0:
            ref = pref * special.i1(math.sqrt(q)) / math.sqrt(q)
        elif q == 0:
            ref = pref * GOLD["sinh_hat_boundary"]["value_over_prefactor"]
        else:
            ref = pref * special.j1(math.sqrt(-q)) / math.sqrt(-q)
        assert abs(val - ref) < 1e-13 * abs(ref) + 1e-16


def test_phi_hat_is_fourier_transform_of_phi():
    """phihat(v) = int phi(t) e^{-2 pi i v t} dt for the scaled window (proof of Theorem 3.4)."""
    integrate = pytest.importorskip("scipy.integrate")
    m, Nj = 5, 300
    beta = 2 * math.pi * m * (1 - 1 / 4)
    for v in (0.0, 17.0, 61.5, 140.0):
        quad, _ = integrate.quad(lambda t: 2 * oracle.phi(t, Nj, m, beta) * math.cos(2 * math.pi * v * t),
                                 0, m / Nj, limit=400, epsabs=1e-18, epsrel=1e-13)
        assert abs(oracle.phi_hat(v, Nj, m, beta) - quad) < 1e-12 * abs(quad)


# --------------------------------------------------------------------------------------
# Section 2: parameters; Algorithm 2.2 and its transpose; Theorem 4.1
# --------------------------------------------------------------------------------------
def test_params_follow_section_2():
    P = oracle.make_params(64, 2, 2, 4, 4)
    assert (P.Nstar, P.N1, P.K1, P.N2) == (68, 136, 144, 288)      # N2 = sigma2 (N1 + 2 m1) already 5-smooth
    P = oracle.make_params(4096, 2, 2, 8, 8)
    assert (P.Nstar, P.N1, P.K1) == (4104, 8208, 8224)
    assert P.N2 >= 2 * P.K1 and P.N2 % 2 == 0 and P.N2 == 17280   # 16448 = 2^6*257 rounded to 2^7*3^3*5
    for N, s1, s2, m1, m2 in [(64, 2, 2, 4, 4), (1000, 1.5, 1.25, 6, 3), (77, 1.3, 2.2, 2, 5)]:
        P = oracle.make_params(N, s1, s2, m1, m2)
        a = 1 + 2 * m1 / P.N1                                        # eq. (2.6)
        assert abs(P.a - a) < 1e-15 and P.K1 == P.N1 + 2 * m1
        assert P.N1 % 2 == 0 and P.N1 >= s1 * P.Nstar - 1e-9
        # eq. (2.7): v in [-1/2, 1/2] rescaled by N/N* lands in [-1/(2a), 1/(2a)]
        assert 0.5 * N / P.Nstar <= 1 / (2 * a) + 1e-15
        assert 2 * m2 <= (1 - 1 / P.sigma1) * P.N2                   # step 4 condition
        assert abs(P.beta1 - 2 * math.pi * m1 * (1 - 1 / (2 * P.sigma1))) < 1e-13
    with pytest.raises(ValueError):
        oracle.make_params(64, 2, 2, 1, 4)
    with pytest.raises(ValueError):
        oracle.make_params(64, 1.0, 2, 4, 4)
    with pytest.raises(ValueError):
        oracle.make_params(4, 1.05, 1.05, 2, 9)     # 2 m2 > (1 - 1/sigma1) N2


@pytest.mark.parametrize("N,M1,M2,m", [(64, 128, 128, 4), (64, 100, 90, 6), (200, 300, 257, 8)])
def test_alg22_within_theorem_4_1(N, M1, M2, m):
    """Algorithm 2.2 approximates the direct sum within the bound of Theorem 4.1."""
    v, x, f = W.nnfft_inputs(M1, M2, 0)
    P = oracle.make_params(N, 2, 2, m, m)
    y = oracle.nnfft_direct(N, v, f, x)
    ya = oracle.nnfft_alg22(P, v, f, x)
    err = oracle.relative_error(ya, y, f)
    E, _, _ = oracle.bound_sinh(P.N1, m, m, P.sigma1, P.sigma2)
    assert err <= E
    if m == 8:
        assert err < 1e-13


def test_alg22_error_decays_exponentially_in_m():
    N, M = 128, 400
    v, x, f = W.nnfft_inputs(M, M, 7, nodes="chebyshev")
    y = oracle.nnfft_direct(N, v, f, x)
    errs = []
    for m in (2, 3, 4, 5, 6, 7):
        P = oracle.make_params(N, 2, 2, m, m)
        errs.append(oracle.relative_error(oracle.nnfft_alg22(P, v, f, x), y, f))
    assert all(e2 < 0.3 * e1 for e1, e2 in zip(errs, errs[1:]))
    # roughly exp(-2 pi m sqrt(1 - 1/sigma)) per step: at least a factor 20 per unit of m
    assert errs[-1] < errs[0] * 20.0 ** -5


def test_alg22_stages():
    """Step 1: sum_l g_l = phi1hat(0) sum_k f_k up to aliasing (Poisson summation);
    step 3: h is the zero-padded DFT of g/phi2hat (numpy FFT)."""
    N, M, m = 64, 50, 6
    v, x, f = W.nnfft_inputs(M, 9, 8)
    P = oracle.make_params(N, 2, 2, m, m)
    out, g, h = oracle.nnfft_alg22(P, v, f, x, return_stages=True)
    ph0 = oracle.phi_hat(0.0, P.N1, m, P.beta1)
    assert abs(g.sum() - ph0 * f.sum()) < 1e-9 * np.sum(np.abs(f))
    K1, N2 = P.K1, P.N2
    ell = np.arange(-K1 // 2, K1 // 2)
    ghat = g / oracle.phi_hat(ell.astype(float), N2, m, P.beta2)
    pad = np.zeros(N2, complex)
    pad[np.mod(ell, N2)] = ghat
    Hs = np.fft.fft(pad) / N2                     # index s mod N2, sign e^{-2 pi i l s / N2}
    s = np.arange(-N2 // 2, N2 // 2)
    assert np.max(np.abs(h - Hs[np.mod(s, N2)])) < 1e-12 * np.max(np.abs(Hs))


def test_alg22_adjoint_is_exact_transpose():
    for (N, M1, M2, m) in [(64, 40, 60, 4), (100, 77, 31, 7)]:
        v, x, f = W.nnfft_inputs(M1, M2, 3)
        g = W.adjoint_inputs(M2, 3)
        P = oracle.make_params(N, 2, 2, m, m)
        Af = oracle.nnfft_alg22(P, v, f, x)
        Ag = oracle.nnfft_alg22_adjoint(P, v, x, g)
        lhs, rhs = np.vdot(g, Af), np.vdot(Ag, f)
        assert abs(lhs - rhs) < 1e-13 * np.sum(np.abs(f)) * np.sum(np.abs(g))
        z = oracle.nnfft_adjoint_direct(N, v, x, g)
        E, _, _ = oracle.bound_sinh(P.N1, m, m, P.sigma1, P.sigma2)
        assert oracle.relative_error(Ag, z, g) <= E


# --------------------------------------------------------------------------------------
# Section 5: Clenshaw-Curtis weights eq. (5.4) and Theorem 5.3
# --------------------------------------------------------------------------------------
def test_cc_weights():
    for n in (1, 2, 3, 8, 16, 33, 256):
        z, w = oracle.cc_weights(n)
        assert abs(w.sum() - GOLD["cc_weights_sum"]["value"]) < 1e-14
        assert np.max(np.abs(w - w[::-1])) < 1e-15 and np.max(np.abs(z + z[::-1])) < 1e-15
        assert np.all(w > 0)
        # (1/2) int_{-1}^{1} t^p dt exact for p <= n
        for p in range(0, n + 1):
            exact = 0.0 if p % 2 else 1.0 / (p + 1)
            assert abs(np.sum(w * z ** p) - exact) < 1e-13
    z, w = oracle.cc_weights(2)                    # Simpson's rule halved: 1/6, 2/3, 1/6
    assert np.max(np.abs(w - np.array([1, 4, 1]) / 6)) < 1e-15


def test_cc_constant_and_worked_example():
    g = GOLD["cc_constant"]
    assert round(oracle.cc_constant(), g["digits"]) == g["value"]
    ex = GOLD["cc_n_ge_4N_for_N_ge_54"]
    assert oracle.cc_bound(ex["N_min"], ex["nu"]) < ex["epsilon"]
    assert oracle.cc_bound(ex["N_min"] - 1, ex["nu"]) > ex["epsilon"]


@pytest.mark.parametrize("N,nu", [(8, 4), (16, 5), (32, 6)])
def test_cc_sinc_error_below_theorem_5_3(N, nu):
    n = nu * N
    z, w = oracle.cc_weights(n)
    x = np.linspace(-1, 1, 2001)
    approx = (w[None, :] * np.exp(-1j * np.pi * N * z[None, :] * x[:, None])).sum(1)
    exact = np.array([oracle.sinc_Npi(N, t, 0.0) for t in x])
    assert np.max(np.abs(approx - exact)) <= oracle.cc_bound(N, nu) + 1e-14


# --------------------------------------------------------------------------------------
# Algorithm 6.1 with the Clenshaw-Curtis rule (steps 1-3 as direct sums)
# --------------------------------------------------------------------------------------
def test_cc_weights_n4_textbook():
    """n = 4: the Clenshaw-Curtis weights on [-1,1] are 1/15, 8/15, 12/15, 8/15, 1/15;
    the rule of eq. (5.4) carries the factor 1/2 of (1/2) int_{-1}^{1}."""
    z, w = oracle.cc_weights(4)
    assert np.max(np.abs(w - np.array([1, 8, 12, 8, 1]) / 30)) < 1e-15
    assert np.max(np.abs(z - np.array([1, np.sqrt(0.5), 0, -np.sqrt(0.5), -1]))) < 1e-15


@pytest.mark.parametrize("N,nu", [(16, 4), (32, 4), (64, 4), (32, 6)])
def test_sinc_cc_within_theorem_5_3(N, nu):
    """|h_CC - h| <= (Theorem 5.3 bound) * sum |c_k| + rounding, with b_l = l/N and
    L1 = N/2 as in the Fig. 6.1 experiment."""
    rng = np.random.default_rng(N + nu)
    a = rng.uniform(-0.5, 0.5, N // 2)
    b = np.arange(-(N // 2), N - N // 2) / N
    c = rng.standard_normal(N // 2) + 1j * rng.standard_normal(N // 2)
    h = oracle.sinc_cc(N, a, c, b, n=nu * N)
    d = oracle.sinc_direct(N, a, c, b)
    err = np.max(np.abs(h - d)) / np.sum(np.abs(c))
    assert err <= oracle.cc_bound(N, nu) + 1e-14


def test_sinc_cc_single_coefficient_and_real_output():
    """c = e_0: h(b) = sinc(N pi (b - a_0)) up to the quadrature error; real c gives a
    real h because z_j = -z_{n-j} and w_j = w_{n-j}."""
    N = 64
    a = np.array([0.1234])
    b = np.linspace(-0.5, 0.5, 101)
    h = oracle.sinc_cc(N, a, np.array([1.0]), b)
    exact = np.array([oracle.sinc_Npi(N, bb, a[0]) for bb in b])
    assert np.max(np.abs(h - exact)) <= oracle.cc_bound(N, 4) + 1e-14
    assert np.max(np.abs(h.imag)) <= 1e-14


def test_sinc_cc_needs_both_steps():
    """A rule with too few nodes (n = N, below Theorem 5.3's nu > C) misses the sinc by
    far more than the n = 4N rule: the test above would catch a dropped weight or a
    node scaled by 2 instead of 1/2."""
    N = 64
    rng = np.random.default_rng(5)
    a = rng.uniform(-0.5, 0.5, 32)
    b = rng.uniform(-0.5, 0.5, 40)
    c = rng.standard_normal(32)
    d = oracle.sinc_direct(N, a, c, b)
    bad = np.max(np.abs(oracle.sinc_cc(N, a, c, b, n=N) - d)) / np.sum(np.abs(c))
    good = np.max(np.abs(oracle.sinc_cc(N, a, c, b, n=4 * N) - d)) / np.sum(np.abs(c))
    assert bad > 1e-3 and good < 1e-14


# --------------------------------------------------------------------------------------
# Theorem 4.1: the constant E(phi_sinh) of eq. (4.2), against the error constants it
# bounds, evaluated from their definitions with scipy's Bessel functions
# --------------------------------------------------------------------------------------
def _omega_hat_sinh(v, m, sigma):
    """eq. (2.1) with scipy's I1 / J1 (exponentially scaled I1, so no overflow); returns
    log(pi beta / sinh beta) and the bracket, i.e. omegahat = exp(logpre) * bracket."""
    sp = pytest.importorskip("scipy.special")
    beta = 2 * np.pi * m * (1 - 1 / (2 * sigma))
    v = np.asarray(v, dtype=float)
    z2 = beta * beta - 4 * np.pi ** 2 * v * v
    br = np.full(v.shape, 0.5)
    lo, hi = z2 > 0, z2 < 0
    s = np.sqrt(z2[lo])
    br[lo] = sp.i1e(s) * np.exp(s) / s
    s = np.sqrt(-z2[hi])
    br[hi] = sp.j1(s) / s
    logpre = math.log(np.pi * beta) - (beta + math.log1p(-math.exp(-2 * beta)) - math.log(2.0))
    return logpre, br


def _error_constant(m, sigma, R=20000, nu=41):
    """eq. (3.7)-(3.8) for the sinh window: max over v in [-N/2, N/2] of the C(T) norm of
    sum_{r != 0} phihat(v + r N1)/phihat(v) e^{2 pi i r N1 .}.  By the scaling of phihat
    the ratio is omegahat(m(u + r))/omegahat(m u) with u = v/N1 in [-1/(2 sigma), 1/(2 sigma)],
    independent of N.  Returns (upper, lower): upper = max_u sum_r |ratio| (>= the norm),
    lower = max_u max over eight points y of |sum_r ratio e^{2 pi i r y}| (<= the norm).
    Terms |r| <= R; the omitted tail is below 1e-3 of the sum (|J1(s)| <= 1.04 (2/(pi s))^{1/2})."""
    r = np.arange(1, R + 1, dtype=float)
    up = lo = 0.0
    for u in np.linspace(-1 / (2 * sigma), 1 / (2 * sigma), nu):
        _, den = _omega_hat_sinh([m * u], m, sigma)
        _, cp = _omega_hat_sinh(m * (u + r), m, sigma)
        _, cm = _omega_hat_sinh(m * (u - r), m, sigma)
        cp, cm = cp / den[0], cm / den[0]
        up = max(up, float(np.sum(np.abs(cp)) + np.sum(np.abs(cm))))
        for y in np.arange(8) / 8.0:
            val = np.sum(cp * np.exp(2j * np.pi * r * y)) + np.sum(cm * np.exp(-2j * np.pi * r * y))
            lo = max(lo, abs(val))
    return up, lo


@pytest.mark.parametrize("sigma", [1.25, 1.5, 2.0])
def test_bound_sinh_term1_bounds_the_error_constant(sigma):
    """Term 1 of eq. (4.2) is the bound eq. (4.3) of E_sigma1(phi1).  It must lie above the
    numerically evaluated constant and within a factor 10 of it (the bound is 2x-4x above
    the constant for sigma in [5/4, 2]), and its decay from m to m + 1 must follow the
    constant's within 25 %: a dropped factor or a wrong exponent fails one of the three."""
    N1 = 2400
    prev = None
    for m in range(2, 9):
        _, t1, _ = oracle.bound_sinh(N1, m, m, sigma, sigma)
        up, lo = _error_constant(m, sigma)
        assert lo <= up
        assert t1 >= 1.001 * up, (m, t1, up)
        assert t1 <= 10.0 * lo, (m, t1, lo)
        if prev is not None:
            q_bound, q_true = t1 / prev[0], up / prev[1]
            assert 0.8 < q_bound / q_true < 1.25, (m, q_bound, q_true)
        prev = (t1, up)


@pytest.mark.parametrize("sigma1,sigma2,N1", [(2.0, 2.0, 8224), (1.5, 2.0, 4800), (1.25, 1.25, 2400)])
def test_bound_sinh_term2_bounds_its_quantity(sigma1, sigma2, N1):
    """Term 2 of eq. (4.2) bounds a / phihat1(N/2) * E_sigma2(phi2) (eq. (3.11) with eq. (4.4)),
    with a = (N1 + 2 m1)/N1 (eq. (2.6)) and phihat1(N/2) = (m1/N1) omegahat1(m1/(2 sigma1))
    evaluated exactly: the term must lie above that product and within a factor 30 of it."""
    for m1 in range(2, 9):
        for m2 in (m1, m1 + 1):
            _, _, t2 = oracle.bound_sinh(N1, m1, m2, sigma1, sigma2)
            logpre, br = _omega_hat_sinh([m1 / (2 * sigma1)], m1, sigma1)
            log_ph = math.log(m1 / N1) + logpre + math.log(br[0])     # log phihat1(N/2)
            a = (N1 + 2 * m1) / N1
            up, lo = _error_constant(m2, sigma2, R=5000, nu=21)
            q_up = a * up * math.exp(-log_ph)
            q_lo = a * lo * math.exp(-log_ph)
            assert t2 >= 1.001 * q_up, (m1, m2, t2, q_up)
            assert t2 <= 30.0 * q_lo, (m1, m2, t2, q_lo)


def test_bessel_envelope_used_for_the_tail():
    """The tail estimate of _error_constant rests on |J1(s)| <= 1.04 (2/(pi s))^{1/2} (the
    envelope's largest excess over the asymptotic amplitude is at the first maximum)."""
    sp = pytest.importorskip("scipy.special")
    s = np.linspace(0.01, 2000.0, 400001)
    assert np.all(np.abs(sp.j1(s)) <= 1.04 * np.sqrt(2 / (np.pi * s)))


# --------------------------------------------------------------------------------------
# The other windows of Section 2 (Example 2.1: B-spline, algebraic; the Kaiser-Bessel window
# of Fig. 4.1(b)) and Algorithm 2.2 with them
# --------------------------------------------------------------------------------------
WINDOWS = ["sinh", "kaiser_bessel", "bspline", "algebraic"]


@pytest.mark.parametrize("window", WINDOWS)
@pytest.mark.parametrize("m,sigma", [(2, 1.5), (4, 2.0), (6, 1.25), (8, 2.0)])
def test_window_belongs_to_omega_and_transform_matches_quadrature(window, m, sigma):
    """Each window is even, 1 at 0, decreasing on [0, 1], zero outside [-1, 1]; its closed-form
    Fourier transform equals 2 int_0^1 omega(x) cos(2 pi v x) dx (scipy quadrature) and is
    positive and decreasing on [0, m/(2 sigma)] (the set Omega of Section 2)."""
    integrate = pytest.importorskip("scipy.integrate")
    P = oracle.make_params(64, sigma, sigma, m, m, window=window)
    beta = P.beta1
    xs = np.linspace(0, 1, 101)
    w = oracle.omega(window, xs, beta, m)
    assert w[0] == 1.0 and np.all(np.diff(w) <= 0)
    assert np.allclose(oracle.omega(window, -xs, beta, m), w, rtol=0, atol=0)
    assert np.all(oracle.omega(window, [1.0001, 1.5, -2.0], beta, m) == 0.0)
    vs = np.linspace(0, m / (2 * P.sigma1), 9)
    wh = oracle.omega_hat(window, vs, beta, m)
    assert np.all(wh > 0) and np.all(np.diff(wh) < 0)
    for v in (0.0, 0.3, m / (4 * P.sigma1), m / (2 * P.sigma1)):
        q, _ = integrate.quad(lambda x: 2 * oracle.omega(window, x, beta, m) * math.cos(2 * math.pi * v * x),
                              0, 1, limit=400, epsabs=1e-15, epsrel=1e-13)
        assert abs(oracle.omega_hat(window, v, beta, m) - q) < 1e-12 * max(1.0, abs(q)), (v, q)


def test_bspline_window_normalisation_from_textbook_values():
    """omegahat_B(0) = 1 / (m B_{2m}(0)) with the centered cardinal B-spline values
    B_4(0) = 2/3, B_6(0) = 11/20, B_8(0) = 151/315, B_10(0) = 15619/36288."""
    for m, b0 in ((2, 2 / 3), (3, 11 / 20), (4, 151 / 315), (5, 15619 / 36288)):
        assert abs(1.0 / (m * float(oracle.omega_hat("bspline", 0.0, 0.0, m))) - b0) < 1e-14
    # omega_B(x) = B_{2m}(m x) / B_{2m}(0): at x = 1/m the value B_4(1)/B_4(0) = (1/6)/(2/3)
    assert abs(float(oracle.omega("bspline", 0.5, 0.0, 2)) - 0.25) < 1e-15


@pytest.mark.parametrize("m", [2, 4, 8])
def test_algebraic_and_kaiser_bessel_against_scipy_bessel(m):
    """The algebraic window's transform against scipy's J_beta (beta = 3m) closed form of
    Example 2.1; the Kaiser-Bessel window against scipy's I0."""
    sp = pytest.importorskip("scipy.special")
    beta = 3 * m
    for v in (0.05, 0.4, m / 4):
        want = (math.pi * math.factorial(2 * beta) / (4 ** beta * math.factorial(beta))
                * (math.pi * v) ** (-beta) * sp.jv(beta, 2 * math.pi * v))
        assert abs(float(oracle.omega_hat("algebraic", v, beta, m)) - want) < 1e-12 * want
    P = oracle.make_params(64, 2.0, 2.0, m, m, window="kaiser_bessel")
    for x in (0.0, 0.3, 0.8, 0.99):
        want = sp.i0(P.beta1 * math.sqrt(1 - x * x)) / sp.i0(P.beta1)
        assert abs(float(oracle.omega("kaiser_bessel", x, P.beta1, m)) - want) < 1e-13


@pytest.mark.parametrize("window", WINDOWS)
def test_alg22_with_each_window_converges_to_the_direct_sum(window):
    """Algorithm 2.2 with each window approximates eq. (1.2); the error falls with m, fastest
    for the sinh-type and Kaiser-Bessel windows (exponential in m), which reach 1e-11 at m = 8."""
    N, M = 128, 300
    v, x, f = W.nnfft_inputs(M, M, 17)
    y = oracle.nnfft_direct(N, v, f, x)
    errs = []
    for m in (2, 4, 6, 8):
        P = oracle.make_params(N, 2.0, 2.0, m, m, window=window)
        errs.append(oracle.relative_error(oracle.nnfft_alg22(P, v, f, x), y, f))
    assert all(e2 < 0.5 * e1 for e1, e2 in zip(errs, errs[1:])), errs
    if window in ("sinh", "kaiser_bessel"):
        assert errs[-1] < 1e-11
    else:
        assert errs[-1] < 1e-4
