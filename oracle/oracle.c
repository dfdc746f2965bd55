/*
 * oracle.c -- plain, slow, fp64 CPU oracle for the NNFFT (type-3 nonuniform FFT)
 * with sinh-type windows and for the discrete / fast sinc transform of
 * Kircheis, Potts and Tasche, "Nonuniform fast Fourier transforms with
 * nonequispaced spatial and frequency data and fast sinc transforms".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg use it.  It shares no code, header, helper or table with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - orc_expsum        the exponential sum of eq. (1.2) (and, with the sign
 *                       flipped and the node roles swapped, its adjoint), by
 *                       its definition: an O(Min*Mout) direct sum.
 *   - orc_sinc_direct   the discrete sinc transform, eq. (6.2), directly.
 *   - orc_gauss_legendre, orc_sinc_gl
 *                       Gauss-Legendre nodes/weights on [-1/2,1/2] and the
 *                       quadrature-factorised sinc transform of eq. (6.3) with
 *                       Gauss-Legendre in place of Clenshaw-Curtis (the variant
 *                       Section 6 attributes to earlier work), by direct sums.
 *   - orc_omega_sinh, orc_omega_sinh_hat
 *                       the sinh-type window of Example 2.1 and its Fourier
 *                       transform, eq. (2.1), with the I1 power series.
 *   - orc_make_params   N*, N1, N2, a, beta_j of Section 2 (eq. (2.6), the
 *                       rescaling after eq. (2.7)) and Section 4, with two
 *                       choices the paper leaves open: N1 rounded up to even and
 *                       N2 rounded up to an even 5-smooth length.
 *   - orc_nnfft_alg22 / orc_nnfft_alg22_adjoint
 *                       Algorithm 2.2 step by step (a naive DFT for step 3) and
 *                       its exact transpose.
 *   - orc_bound_sinh    the error constant E(phi_sinh) of Theorem 4.1.
 *   - orc_omega_kb, orc_omega_bspline, orc_omega_alg (and their transforms)
 *                       the other windows of Section 2 (Example 2.1: B-spline and
 *                       algebraic; the Kaiser-Bessel window of Fig. 4.1(b)), used by
 *                       Algorithm 2.2 through the window id of the parameters.
 *   - orc_cc_weights, orc_cc_bound
 *                       Clenshaw-Curtis weights, eq. (5.4), and the bound of
 *                       Theorem 5.3.
 *   - orc_sinc_cc       Algorithm 6.1 with the Clenshaw-Curtis rule, steps 1-3
 *                       as direct sums.
 *
 * Equations are cited by their printed numbers (numbered within each
 * section), e.g. eq. (2.12) for the grid values g_l of step 1.
 * Complex arrays are interleaved (re, im) doubles.  A centered index set
 * I_M = {-M/2, ..., M/2-1} is stored with array index i = l + M/2.
 *
 * Pins: tests/test_oracle_pins.py (closed forms, library routines used as
 * independent cross-checks, invariants, brute force at higher precision, and
 * the few numbers the paper prints).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef long long i64;

/* ------------------------------------------------------------------------ */
/* compensated (Neumaier) accumulation                                       */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } ksum;
static inline void kadd(ksum *k, double x) {
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else                       k->c += (x - t) + k->s;
    k->s = t;
}
static inline double kval(const ksum *k) { return k->s + k->c; }

/* N*a*b reduced mod 1 to about [-1/2, 1/2].  The products a*b and N*(a*b) are
 * carried exactly with fma-based error-free transformations, so the phase of
 * exp(-2 pi i N a b) is accurate to a few ulps of 1 even when N*a*b is large. */
static double phase_mod1(i64 N, double a, double b) {
    double p  = a * b;
    double pe = fma(a, b, -p);            /* a*b = p + pe exactly            */
    double Nd = (double)N;                /* exact for N < 2^53              */
    double t  = Nd * p;
    double te = fma(Nd, p, -t);           /* Nd*p = t + te exactly           */
    double r  = t - nearbyint(t);         /* exact                           */
    return r + (te + Nd * pe);
}

static int use_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_num_threads(void) { return use_threads(0); }

/* ------------------------------------------------------------------------ */
/* Eq. (1.2): out_j = sum_k c_k exp(sign * 2 pi i N a_k b_j).                */
/* sign = -1 is the NNFFT of eq. (1.2) (a = v frequency nodes, b = x spatial */
/* nodes); sign = +1 with a = x, b = v, c = g is its adjoint                 */
/* z_k = sum_j g_j exp(+2 pi i N v_k x_j).                                   */
/* rows == NULL evaluates every output; otherwise only outputs rows[r],      */
/* r < nrows, written to out[2r], out[2r+1].                                 */
/* ------------------------------------------------------------------------ */
int orc_expsum(i64 N, i64 Min, const double *a, const double *c,
               i64 Mout, const double *b, int sign,
               const i64 *rows, i64 nrows, double *out, int nthreads) {
    if (N < 0 || Min < 0 || Mout < 0 || (sign != 1 && sign != -1)) return 1;
    i64 nr = rows ? nrows : Mout;
    int nt = use_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (i64 r = 0; r < nr; ++r) {
        i64 j = rows ? rows[r] : r;
        ksum sre = {0, 0}, sim = {0, 0};
        if (j >= 0 && j < Mout) {
            double bj = b[j];
            for (i64 k = 0; k < Min; ++k) {
                double fr = phase_mod1(N, a[k], bj);
                double ang = 2.0 * M_PI * fr;
                double cs = cos(ang), sn = sign * sin(ang);
                double cr = c[2 * k], ci = c[2 * k + 1];
                kadd(&sre, cr * cs - ci * sn);
                kadd(&sim, cr * sn + ci * cs);
            }
        }
        out[2 * r]     = kval(&sre);
        out[2 * r + 1] = kval(&sim);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* sinc(pi N (b - a)) of eq. (5.2): sin(pi u)/(pi u), value 1 at u = 0.       */
/* d = b - a is carried as a double-double and u = N d is reduced exactly     */
/* modulo 2 before the sine, so large N*d loses no accuracy.                 */
/* ------------------------------------------------------------------------ */
double orc_sinc_Npi(i64 N, double b, double a) {
    double s  = b - a;                       /* two-sum of b + (-a)          */
    double bp = s - b;
    double ap = s - bp;
    double se = (b - ap) + (-a - bp);        /* b - a = s + se exactly       */
    double Nd = (double)N;
    double t  = Nd * s;
    double te = fma(Nd, s, -t) + Nd * se;    /* N*(b-a) = t + te             */
    double u  = t + te;
    if (fabs(u) < 1e-5) {
        double x2 = (M_PI * u) * (M_PI * u);
        return 1.0 - x2 / 6.0 + x2 * x2 / 120.0;
    }
    double k2 = 2.0 * nearbyint(0.5 * t);    /* even integer nearest t       */
    double r  = (t - k2) + te;               /* u - k2, |r| <= 1 (+tiny)     */
    return sin(M_PI * r) / (M_PI * u);
}

/* Eq. (6.2): h(b_l) = sum_k c_k sinc(N pi (b_l - a_k)), c complex. */
int orc_sinc_direct(i64 N, i64 L1, const double *a, const double *c,
                    i64 L2, const double *b, const i64 *rows, i64 nrows,
                    double *h, int nthreads) {
    if (N < 0 || L1 < 0 || L2 < 0) return 1;
    i64 nr = rows ? nrows : L2;
    int nt = use_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (i64 r = 0; r < nr; ++r) {
        i64 l = rows ? rows[r] : r;
        ksum sre = {0, 0}, sim = {0, 0};
        if (l >= 0 && l < L2) {
            for (i64 k = 0; k < L1; ++k) {
                double s = orc_sinc_Npi(N, b[l], a[k]);
                kadd(&sre, c[2 * k] * s);
                kadd(&sim, c[2 * k + 1] * s);
            }
        }
        h[2 * r]     = kval(&sre);
        h[2 * r + 1] = kval(&sim);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule with n nodes on [-1/2, 1/2] (sum of weights = 1):    */
/* Newton's method on the Legendre three-term recurrence; the weights are    */
/* 2/((1-t^2) P_n'(t)^2) on [-1,1], halved by the map tau = t/2.  Nodes are  */
/* returned in increasing order.                                             */
/* ------------------------------------------------------------------------ */
int orc_gauss_legendre(i64 n, double *tau, double *w) {
    if (n <= 0) return 1;
    for (i64 i = 0; i < (n + 1) / 2; ++i) {
        /* i-th largest root; classical initial guess */
        double t = cos(M_PI * ((double)i + 0.75) / ((double)n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (i64 k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / (double)k;
                p0 = p1; p1 = p2;
            }
            double pn = (n == 1) ? t : p1, pm = (n == 1) ? 1.0 : p0;
            dp = (double)n * (t * pn - pm) / (t * t - 1.0);
            double dt = pn / dp;
            t -= dt;
            if (fabs(dt) < 1e-17) break;
        }
        /* recompute P_n' at the converged node for the weight */
        {
            double p0 = 1.0, p1 = t;
            for (i64 k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / (double)k;
                p0 = p1; p1 = p2;
            }
            double pn = (n == 1) ? t : p1, pm = (n == 1) ? 1.0 : p0;
            dp = (double)n * (t * pn - pm) / (t * t - 1.0);
        }
        double wt = 2.0 / ((1.0 - t * t) * dp * dp);
        /* largest roots first: place symmetric pairs */
        tau[n - 1 - i] = 0.5 * t;
        tau[i]         = -0.5 * t;
        w[n - 1 - i]   = 0.5 * wt;
        w[i]           = 0.5 * wt;
    }
    if (n % 2 == 1) tau[n / 2] = 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (6.3) with a Gauss-Legendre rule (tau_j, w_j), j < n, on [-1/2,1/2]:   */
/*   g_j   = sum_k c_k exp(+2 pi i N tau_j a_k)                              */
/*   h_l   = sum_j w_j g_j exp(-2 pi i N tau_j b_l)                          */
/* which is the quadrature of sinc(N pi (b-a)) = int_{-1/2}^{1/2}             */
/* exp(-2 pi i N tau (b - a)) d tau (proof of Theorem 5.1).  Direct sums.     */
/* ------------------------------------------------------------------------ */
int orc_sinc_gl(i64 N, i64 n, i64 L1, const double *a, const double *c,
                i64 L2, const double *b, const i64 *rows, i64 nrows,
                double *h, int nthreads) {
    if (n <= 0) return 1;
    double *tau = (double *)malloc(sizeof(double) * n);
    double *w   = (double *)malloc(sizeof(double) * n);
    double *g   = (double *)malloc(sizeof(double) * 2 * n);
    if (!tau || !w || !g) { free(tau); free(w); free(g); return 2; }
    orc_gauss_legendre(n, tau, w);
    /* g_j = sum_k c_k exp(+2 pi i N a_k tau_j) */
    orc_expsum(N, L1, a, c, n, tau, +1, NULL, 0, g, nthreads);
    for (i64 j = 0; j < n; ++j) { g[2 * j] *= w[j]; g[2 * j + 1] *= w[j]; }
    /* h_l = sum_j (w_j g_j) exp(-2 pi i N tau_j b_l) */
    orc_expsum(N, n, tau, g, L2, b, -1, rows, nrows, h, nthreads);
    free(tau); free(w); free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sinh-type window, Example 2.1 and Section 4:                                */
/*   omega(x) = sinh(beta sqrt(1-x^2)) / sinh(beta) on [-1,1], 0 outside.    */
/* Evaluated as exp(beta(s-1)) (1-exp(-2 beta s)) / (1-exp(-2 beta)), which  */
/* is the same quotient without overflow.                                    */
/* ------------------------------------------------------------------------ */
double orc_omega_sinh(double x, double beta) {
    if (!(fabs(x) < 1.0)) return 0.0;
    double s = sqrt(1.0 - x * x);
    return exp(beta * (s - 1.0)) * (-expm1(-2.0 * beta * s)) / (-expm1(-2.0 * beta));
}

/* Eq. (2.1): Fourier transform of omega_sinh.
 *   |v| <  beta/(2 pi): (pi beta / sinh beta) * q^{-1/2} I1(sqrt q), q = beta^2 - 4 pi^2 v^2,
 *                       with q^{-1/2} I1(sqrt q) = (1/2) sum_k q^k / (4^k k! (k+1)!)
 *                       (the power series printed after eq. (2.1); all terms positive);
 *   |v| == beta/(2 pi): (pi beta / sinh beta) / 2;
 *   |v| >  beta/(2 pi): (pi beta / sinh beta) * q'^{-1/2} J1(sqrt q'), q' = 4 pi^2 v^2 - beta^2
 *                       (libm j1 used as the Bessel primitive).
 * The threshold m(1 - 1/(2 sigma)) of eq. (2.1) equals beta/(2 pi). */
double orc_omega_sinh_hat(double v, double beta) {
    double pref = M_PI * beta / sinh(beta);
    double q = beta * beta - 4.0 * M_PI * M_PI * v * v;
    if (q > 0.0) {
        double term = 1.0, sum = 1.0;
        for (int k = 0; k < 2000; ++k) {
            term *= q / (4.0 * (k + 1.0) * (k + 2.0));
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        return pref * 0.5 * sum;
    }
    if (q == 0.0) return pref * 0.5;
    double r = sqrt(-q);
    return pref * j1(r) / r;
}

/* ------------------------------------------------------------------------ */
/* The other windows of the set Omega (Section 2).                             */
/* Window ids: 0 sinh-type (above), 1 Kaiser-Bessel, 2 B-spline, 3 algebraic. */
/* ------------------------------------------------------------------------ */

/* I0(z) = sum_k (z/2)^{2k} / (k!)^2 (all terms positive). */
static double orc_i0(double z) {
    double q = 0.25 * z * z, term = 1.0, sum = 1.0;
    for (int k = 1; k < 4000; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* Kaiser-Bessel window on [-1, 1]: omega(x) = I0(beta sqrt(1 - x^2)) / I0(beta) (the standard
 * window the paper's Fig. 4.1(b) uses beside the sinh-type one; shape parameter as there,
 * beta = 2 pi m (1 - 1/(2 sigma))).  Its Fourier transform 2 int_0^1 omega(x) cos(2 pi v x) dx:
 *   q = beta^2 - 4 pi^2 v^2 > 0:  (2 / I0(beta)) sinh(sqrt q) / sqrt q,
 *   q = 0:                         2 / I0(beta),
 *   q < 0:                         (2 / I0(beta)) sin(sqrt(-q)) / sqrt(-q). */
double orc_omega_kb(double x, double beta) {
    if (!(fabs(x) <= 1.0)) return 0.0;
    return orc_i0(beta * sqrt(1.0 - x * x)) / orc_i0(beta);
}
double orc_omega_kb_hat(double v, double beta) {
    double q = beta * beta - 4.0 * M_PI * M_PI * v * v;
    double c = 2.0 / orc_i0(beta);
    if (q > 0.0) { double r = sqrt(q); return c * sinh(r) / r; }
    if (q == 0.0) return c;
    double r = sqrt(-q);
    return c * sin(r) / r;
}

/* Centered cardinal B-spline B_n of order n (degree n - 1, support [-n/2, n/2]) at t, by
 * the Cox-de Boor recursion on the integer knots -n/2, ..., n/2 (positive terms only). */
static double orc_bspline(int n, double t) {
    double N_[64];
    if (n < 1 || n > 63) return 0.0;
    double a = -0.5 * n;                               /* knot i is a + i */
    if (!(t >= a && t < -a)) return 0.0;
    for (int i = 0; i < n; ++i) N_[i] = (t >= a + i && t < a + i + 1) ? 1.0 : 0.0;
    for (int k = 1; k < n; ++k)                        /* degree k */
        for (int i = 0; i + k < n; ++i)
            N_[i] = ((t - (a + i)) * N_[i] + ((a + i + k + 1) - t) * N_[i + 1]) / (double)k;
    return N_[0];
}

/* B-spline window of Example 2.1: omega(x) = B_{2m}(m x) / B_{2m}(0), and its Fourier
 * transform omegahat(v) = (sinc(pi v / m))^{2m} / (m B_{2m}(0)), sinc(y) = sin(y)/y. */
double orc_omega_bspline(double x, int m) {
    return orc_bspline(2 * m, (double)m * x) / orc_bspline(2 * m, 0.0);
}
double orc_omega_bspline_hat(double v, int m) {
    double y = M_PI * v / (double)m;
    double sc = y == 0.0 ? 1.0 : sin(y) / y;
    return pow(sc, 2 * m) / ((double)m * orc_bspline(2 * m, 0.0));
}

/* Algebraic window of Example 2.1 (beta = 3 m, beta integral): omega(x) = (1 - x^2)^{beta - 1/2}
 * on [-1, 1], with omegahat(v) = pi (2 beta)! / (4^beta beta!) (pi v)^{-beta} J_beta(2 pi v), the
 * last factor by its power series sum_k (-1)^k (pi v)^{2k} / (k! (k + beta)!) (value 1/beta!
 * at v = 0).  The alternating series loses accuracy for large pi |v| against beta; the
 * arguments used here (|v| <= m / (2 sigma)) keep pi |v| below about 2 sqrt(beta). */
double orc_omega_alg(double x, double beta) {
    if (!(fabs(x) < 1.0)) return 0.0;
    return pow(1.0 - x * x, beta - 0.5);
}
double orc_omega_alg_hat(double v, double beta) {
    int b = (int)floor(beta + 0.5);
    double x2 = (M_PI * v) * (M_PI * v);
    double term = 1.0, sum = 1.0;                      /* terms scaled by beta! */
    for (int k = 1; k < 2000; ++k) {
        term *= -x2 / ((double)k * (double)(k + b));
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum) && k > 4) break;
    }
    double logc = log(M_PI) + lgamma(2.0 * b + 1.0) - b * log(4.0) - 2.0 * lgamma(b + 1.0);
    return exp(logc) * sum;
}

double orc_omega_w(int window, double x, double beta, int m) {
    switch (window) {
        case 1: return orc_omega_kb(x, beta);
        case 2: return orc_omega_bspline(x, m);
        case 3: return orc_omega_alg(x, beta);
        default: return orc_omega_sinh(x, beta);
    }
}
double orc_omega_hat_w(int window, double v, double beta, int m) {
    switch (window) {
        case 1: return orc_omega_kb_hat(v, beta);
        case 2: return orc_omega_bspline_hat(v, m);
        case 3: return orc_omega_alg_hat(v, beta);
        default: return orc_omega_sinh_hat(v, beta);
    }
}

/* Scaled windows of eq. (2.5): phi(t) = omega(N t / m), phihat(v) = (m/N) omegahat(m v / N). */
double orc_phi_w(int window, double t, i64 Nj, int m, double beta) {
    return orc_omega_w(window, (double)Nj * t / (double)m, beta, m);
}
double orc_phi_hat_w(int window, double v, i64 Nj, int m, double beta) {
    return ((double)m / (double)Nj) * orc_omega_hat_w(window, (double)m * v / (double)Nj, beta, m);
}
double orc_phi(double t, i64 Nj, int m, double beta) { return orc_phi_w(0, t, Nj, m, beta); }
double orc_phi_hat(double v, i64 Nj, int m, double beta) {
    return orc_phi_hat_w(0, v, Nj, m, beta);
}

/* ------------------------------------------------------------------------ */
/* Parameters of Algorithm 2.2 for v_k, x_j in [-1/2, 1/2] (Section 2):       */
/*   N*  = N + ceil(2 m1 / sigma1)   (rescaling after eq. (2.7))              */
/*   N1  = sigma1 N*, rounded up to an even integer; sigma1,eff = N1/N*       */
/*   K1  = N1 + 2 m1 = a N1           (eq. (2.6))                          */
/*   N2  = sigma2 K1, rounded up to an even 2^a 3^b 5^c;                      */
/*         sigma2,eff = N2/K1                                                 */
/*   beta_j = 2 pi m_j (1 - 1/(2 sigma_j,eff))   (Section 4)                  */
/* Returns 0, or 1 when the input violates m_j >= 2, sigma_j > 1, N >= 1 or   */
/* the step-4 condition 2 m2 <= (1 - 1/sigma1) N2.                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    i64 N, Nstar, N1, K1, N2;
    int m1, m2;
    double sigma1, sigma2;   /* effective */
    double beta1, beta2, a;
    int window;              /* 0 sinh-type, 1 Kaiser-Bessel, 2 B-spline, 3 algebraic */
} orc_params;

static int is_5smooth(i64 n) {
    if (n <= 0) return 0;
    const i64 p[3] = {2, 3, 5};
    for (int i = 0; i < 3; ++i) while (n % p[i] == 0) n /= p[i];
    return n == 1;
}

int orc_make_params(i64 N, double sigma1, double sigma2, int m1, int m2, orc_params *P) {
    if (N < 1 || m1 < 2 || m2 < 2 || !(sigma1 > 1.0) || !(sigma2 > 1.0)) return 1;
    memset(P, 0, sizeof(*P));
    P->N = N; P->m1 = m1; P->m2 = m2;
    i64 c = (i64)ceil(2.0 * m1 / sigma1 - 1e-12);
    P->Nstar = N + c;
    i64 n1 = (i64)ceil(sigma1 * (double)P->Nstar - 1e-9);
    if (n1 % 2) n1 += 1;
    P->N1 = n1;
    P->K1 = n1 + 2 * m1;
    i64 n2 = (i64)ceil(sigma2 * (double)P->K1 - 1e-9);
    if (n2 % 2) n2 += 1;
    while (!is_5smooth(n2)) n2 += 2;
    P->N2 = n2;
    P->sigma1 = (double)P->N1 / (double)P->Nstar;
    P->sigma2 = (double)P->N2 / (double)P->K1;
    P->beta1 = 2.0 * M_PI * m1 * (1.0 - 1.0 / (2.0 * P->sigma1));
    P->beta2 = 2.0 * M_PI * m2 * (1.0 - 1.0 / (2.0 * P->sigma2));
    P->a = (double)P->K1 / (double)P->N1;
    if ((double)(2 * m2) > (1.0 - 1.0 / P->sigma1) * (double)P->N2) return 1;
    return 0;
}

/* The same parameters for another window of Omega: Kaiser-Bessel keeps the sinh-type shape
 * parameter, the B-spline has none (beta = 0), the algebraic window takes beta = 3 m and
 * needs sigma > pi / 3 (Example 2.1). */
int orc_make_params_w(i64 N, double sigma1, double sigma2, int m1, int m2, int window,
                      orc_params *P) {
    if (window < 0 || window > 3) return 1;
    if (window == 3 && (!(sigma1 > M_PI / 3.0) || !(sigma2 > M_PI / 3.0))) return 1;
    int rc = orc_make_params(N, sigma1, sigma2, m1, m2, P);
    P->window = window;
    if (window == 2) P->beta1 = P->beta2 = 0.0;
    if (window == 3) { P->beta1 = 3.0 * m1; P->beta2 = 3.0 * m2; }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2.2 (NNFFT), step by step, for v_k, x_j in [-1/2,1/2]:           */
/*   rescale v*_k = (N/N*) v_k so that N v_k = N* v*_k (after eq. (2.7));      */
/*   step 1: g_l = (1/N1) sum_k f_k phi1(l/N1 - v*_k), l in I_{K1} (eq. (2.12)) */
/*   step 2: ghat_l = g_l / phi2hat(l)  (phi2hat at the integer l, as step 2 and  */
/*           the proof of Theorem 3.5 use it; step 0 lists phi2hat(l/a))         */
/*   step 3: h_s = (1/N2) sum_l ghat_l exp(-2 pi i l s / N2), s in I_{N2}      */
/*           (a naive DFT with the index product reduced mod N2 in integers)   */
/*   step 4: s1_j = sum_{s in I''(x_j)} h_s phi2(x_j/sigma1 - s/N2)            */
/*   output: s1_j / phi1hat(N* x_j).                                           */
/* Optional g (K1 complex) and h (N2 complex) receive the step-1 and step-3    */
/* arrays.  Windows are evaluated exactly (no tables, no polynomial).          */
/* ------------------------------------------------------------------------ */
static void alg22_spread_v(const orc_params *P, i64 M1, const double *v, const double *f,
                           double *g) {
    i64 K1 = P->K1, N1 = P->N1;
    int m1 = P->m1;
    memset(g, 0, sizeof(double) * 2 * K1);
    for (i64 k = 0; k < M1; ++k) {
        double vs = ((double)P->N * v[k]) / (double)P->Nstar;   /* v*_k */
        double u = (double)N1 * vs;
        i64 lo = (i64)ceil(u - m1), hi = (i64)floor(u + m1);
        for (i64 l = lo; l <= hi; ++l) {
            if (l < -K1 / 2 || l >= K1 / 2) continue;      /* outside I_{K1} */
            double w = orc_phi_w(P->window, (double)l / (double)N1 - vs, N1, m1, P->beta1);
            g[2 * (l + K1 / 2)]     += f[2 * k] * w / (double)N1;
            g[2 * (l + K1 / 2) + 1] += f[2 * k + 1] * w / (double)N1;
        }
    }
}

static void dft_centered(i64 Nin, i64 Nout, i64 Nmod, int sign, const double *in, double *out,
                         int nthreads) {
    int nt = use_threads(nthreads);
    (void)nt;
#pragma omp parallel for schedule(static) num_threads(nt)
    for (i64 so = 0; so < Nout; ++so) {
        i64 s = so - Nout / 2;
        ksum re = {0, 0}, im = {0, 0};
        for (i64 li = 0; li < Nin; ++li) {
            i64 l = li - Nin / 2;
            i64 r = ((l * s) % Nmod + Nmod) % Nmod;
            double ang = 2.0 * M_PI * (double)r / (double)Nmod;
            double cs = cos(ang), sn = sign * sin(ang);
            double xr = in[2 * li], xi = in[2 * li + 1];
            kadd(&re, xr * cs - xi * sn);
            kadd(&im, xr * sn + xi * cs);
        }
        out[2 * so] = kval(&re);
        out[2 * so + 1] = kval(&im);
    }
}

int orc_nnfft_alg22(const orc_params *P, i64 M1, const double *v, const double *f,
                    i64 M2, const double *x, double *out, double *g_out, double *h_out,
                    int nthreads) {
    i64 K1 = P->K1, N1 = P->N1, N2 = P->N2;
    double *g = (double *)calloc(2 * K1, sizeof(double));
    double *h = (double *)calloc(2 * N2, sizeof(double));
    if (!g || !h) { free(g); free(h); return 2; }
    /* step 1 */
    alg22_spread_v(P, M1, v, f, g);
    if (g_out) memcpy(g_out, g, sizeof(double) * 2 * K1);
    /* step 2: ghat_l = g_l / phi2hat(l) */
    for (i64 li = 0; li < K1; ++li) {
        double ph = orc_phi_hat_w(P->window, (double)(li - K1 / 2), N2, P->m2, P->beta2);
        g[2 * li] /= ph; g[2 * li + 1] /= ph;
    }
    /* step 3: h_s = (1/N2) sum_l ghat_l exp(-2 pi i l s / N2) */
    dft_centered(K1, N2, N2, -1, g, h, nthreads);
    for (i64 i = 0; i < 2 * N2; ++i) h[i] /= (double)N2;
    if (h_out) memcpy(h_out, h, sizeof(double) * 2 * N2);
    /* step 4 and output */
    int m2 = P->m2;
    for (i64 j = 0; j < M2; ++j) {
        double xs = x[j] * (double)P->Nstar / (double)N1;     /* x_j / sigma1 */
        double u = (double)N2 * xs;
        i64 lo = (i64)ceil(u - m2), hi = (i64)floor(u + m2);
        double sr = 0, si = 0;
        for (i64 s = lo; s <= hi; ++s) {
            double w = orc_phi_w(P->window, xs - (double)s / (double)N2, N2, m2, P->beta2);
            i64 si_ = ((s % N2) + N2 + N2 / 2) % N2;          /* centered index of s mod N2 */
            sr += h[2 * si_] * w;
            si += h[2 * si_ + 1] * w;
        }
        double ph1 = orc_phi_hat_w(P->window, (double)P->Nstar * x[j], N1, P->m1, P->beta1);
        out[2 * j] = sr / ph1;
        out[2 * j + 1] = si / ph1;
    }
    free(g); free(h);
    return 0;
}

/* Exact transpose (conjugate transpose; every window and transform is real) of
 * the map f -> out of orc_nnfft_alg22, step by step in reverse order:
 *   g'_j = g_j / phi1hat(N* x_j);  H_s = sum_j g'_j phi2(x_j/sigma1 - s/N2);
 *   G_l = (1/N2) sum_s H_s exp(+2 pi i l s/N2), l in I_{K1};  G_l /= phi2hat(l);
 *   z_k = (1/N1) sum_l G_l phi1(l/N1 - v*_k).
 * It approximates z_k = sum_j g_j exp(+2 pi i N v_k x_j). */
int orc_nnfft_alg22_adjoint(const orc_params *P, i64 M1, const double *v, i64 M2,
                            const double *x, const double *gin, double *z, int nthreads) {
    i64 K1 = P->K1, N1 = P->N1, N2 = P->N2;
    int m1 = P->m1, m2 = P->m2;
    double *H = (double *)calloc(2 * N2, sizeof(double));
    double *G = (double *)calloc(2 * K1, sizeof(double));
    if (!H || !G) { free(H); free(G); return 2; }
    for (i64 j = 0; j < M2; ++j) {
        double ph1 = orc_phi_hat_w(P->window, (double)P->Nstar * x[j], N1, m1, P->beta1);
        double gr = gin[2 * j] / ph1, gi = gin[2 * j + 1] / ph1;
        double xs = x[j] * (double)P->Nstar / (double)N1;
        double u = (double)N2 * xs;
        i64 lo = (i64)ceil(u - m2), hi = (i64)floor(u + m2);
        for (i64 s = lo; s <= hi; ++s) {
            double w = orc_phi_w(P->window, xs - (double)s / (double)N2, N2, m2, P->beta2);
            i64 si_ = ((s % N2) + N2 + N2 / 2) % N2;
            H[2 * si_] += gr * w;
            H[2 * si_ + 1] += gi * w;
        }
    }
    dft_centered(N2, K1, N2, +1, H, G, nthreads);
    for (i64 li = 0; li < K1; ++li) {
        double ph = orc_phi_hat_w(P->window, (double)(li - K1 / 2), N2, m2, P->beta2);
        G[2 * li] /= ((double)N2 * ph);
        G[2 * li + 1] /= ((double)N2 * ph);
    }
    for (i64 k = 0; k < M1; ++k) {
        double vs = ((double)P->N * v[k]) / (double)P->Nstar;
        double u = (double)N1 * vs;
        i64 lo = (i64)ceil(u - m1), hi = (i64)floor(u + m1);
        double zr = 0, zi = 0;
        for (i64 l = lo; l <= hi; ++l) {
            if (l < -K1 / 2 || l >= K1 / 2) continue;
            double w = orc_phi_w(P->window, (double)l / (double)N1 - vs, N1, m1, P->beta1);
            zr += G[2 * (l + K1 / 2)] * w;
            zi += G[2 * (l + K1 / 2) + 1] * w;
        }
        z[2 * k] = zr / (double)N1;
        z[2 * k + 1] = zi / (double)N1;
    }
    free(H); free(G);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Theorem 4.1: E(phi_sinh) =                                                */
/*   (24 m1^{3/2} + 10) exp(-2 pi m1 sqrt(1 - 1/sigma1))                      */
/* + (24 m2^{3/2} + 10) (2 N1 + 4 m1)/sqrt(2 pi m1)                           */
/*     * exp(2 pi m1 (1 - sqrt(1 - 1/sigma1) - 1/(2 sigma1)))                 */
/*     * exp(-2 pi m2 sqrt(1 - 1/sigma2)).                                    */
/* term[0], term[1] receive the two summands when term != NULL.              */
/* ------------------------------------------------------------------------ */
double orc_bound_sinh(i64 N1, int m1, int m2, double sigma1, double sigma2, double *term) {
    double s1 = sqrt(1.0 - 1.0 / sigma1), s2 = sqrt(1.0 - 1.0 / sigma2);
    double t1 = (24.0 * pow(m1, 1.5) + 10.0) * exp(-2.0 * M_PI * m1 * s1);
    double t2 = (24.0 * pow(m2, 1.5) + 10.0) * (2.0 * N1 + 4.0 * m1) / sqrt(2.0 * M_PI * m1)
              * exp(2.0 * M_PI * m1 * (1.0 - s1 - 1.0 / (2.0 * sigma1)))
              * exp(-2.0 * M_PI * m2 * s2);
    if (term) { term[0] = t1; term[1] = t2; }
    return t1 + t2;
}

/* ------------------------------------------------------------------------ */
/* Clenshaw-Curtis weights of eq. (5.4) for the rule                         */
/*   (1/2) int_{-1}^{1} F(t) dt ~ sum_{k=0}^{n} w_k F(z_k), z_k = cos(k pi/n), */
/* w_k = (1/n) eps(k)^2 sum_{j=0}^{floor(n/2)} eps(2j)^2 2/(1-4j^2) cos(2jk pi/n) */
/* with eps(0) = eps(n) = sqrt(2)/2 and eps(j) = 1 otherwise (eps(2j) for    */
/* 2j > n is not used).  Explicit O(n^2) sum.                                */
/* ------------------------------------------------------------------------ */
int orc_cc_weights(i64 n, double *z, double *w) {
    if (n < 1) return 1;
    for (i64 k = 0; k <= n; ++k) {
        double ek2 = (k == 0 || k == n) ? 0.5 : 1.0;
        ksum s = {0, 0};
        for (i64 j = 0; 2 * j <= n; ++j) {
            double ej2 = (2 * j == 0 || 2 * j == n) ? 0.5 : 1.0;
            i64 r = (2 * j * k) % (2 * n);                  /* cos(2 j k pi / n) exactly reduced */
            kadd(&s, ej2 * 2.0 / (1.0 - 4.0 * (double)j * (double)j) * cos(M_PI * (double)r / (double)n));
        }
        w[k] = ek2 * kval(&s) / (double)n;
        z[k] = cos(M_PI * (double)k / (double)n);
    }
    return 0;
}

/* Theorem 5.3: |sinc(N pi x) - sum_k w_k exp(-pi i N z_k x)| <=
 *   36 (1 + exp(-2 C N)) / (35 (e^2 - 1)) * exp(-N (nu - C)),  C = pi (e^2-1)/(2e), n = nu N. */
double orc_cc_constant(void) {
    double e = exp(1.0);
    return M_PI * (e * e - 1.0) / (2.0 * e);
}
double orc_cc_bound(double N, double nu) {
    double e = exp(1.0), C = orc_cc_constant();
    return 36.0 * (1.0 + exp(-2.0 * C * N)) / (35.0 * (e * e - 1.0)) * exp(-N * (nu - C));
}

/* ------------------------------------------------------------------------ */
/* Algorithm 6.1 with the Clenshaw-Curtis rule, every sum taken directly:    */
/*   z_j = cos(j pi/n), w_j of eq. (5.4), j = 0..n;                          */
/*   step 1: g_j     = sum_k c_k exp(-pi i N z_j a_k)                         */
/*   step 2: alpha_j = w_j g_j                                                */
/*   step 3: h_l     = sum_j alpha_j exp(+pi i N z_j b_l)                     */
/* The exponents are written as exp(-+2 pi i N (z_j/2) .), the form of       */
/* orc_expsum.                                                                */
/* ------------------------------------------------------------------------ */
int orc_sinc_cc(i64 N, i64 n, i64 L1, const double *a, const double *c,
                i64 L2, const double *b, const i64 *rows, i64 nrows,
                double *h, int nthreads) {
    if (n < 1) return 1;
    double *z = (double *)malloc(sizeof(double) * (n + 1));
    double *w = (double *)malloc(sizeof(double) * (n + 1));
    double *g = (double *)malloc(sizeof(double) * 2 * (n + 1));
    if (!z || !w || !g) { free(z); free(w); free(g); return 2; }
    orc_cc_weights(n, z, w);
    for (i64 j = 0; j <= n; ++j) z[j] *= 0.5;
    /* g_j = sum_k c_k exp(-2 pi i N a_k (z_j/2)) */
    orc_expsum(N, L1, a, c, n + 1, z, -1, NULL, 0, g, nthreads);
    for (i64 j = 0; j <= n; ++j) { g[2 * j] *= w[j]; g[2 * j + 1] *= w[j]; }
    /* h_l = sum_j alpha_j exp(+2 pi i N (z_j/2) b_l) */
    orc_expsum(N, n + 1, z, g, L2, b, +1, rows, nrows, h, nthreads);
    free(z); free(w); free(g);
    return 0;
}
