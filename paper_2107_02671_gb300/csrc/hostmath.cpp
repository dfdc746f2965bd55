// hostmath.cpp -- see hostmath.h.
#include <algorithm>
#include <thread>

#include "hostmath.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>

namespace nnfft {
namespace hm {

double omega_sinh(double x, double beta) {
    if (!(std::fabs(x) < 1.0)) return 0.0;
    const double s = std::sqrt(1.0 - x * x);
    // sinh(beta s)/sinh(beta) written without overflow
    return std::exp(beta * (s - 1.0)) * (-std::expm1(-2.0 * beta * s)) /
           (-std::expm1(-2.0 * beta));
}

double omega_sinh_hat(double v, double beta) {
    const double pref = PI * beta / std::sinh(beta);
    const double q = beta * beta - 4.0 * PI * PI * v * v;
    if (q > 0.0) {
        // (1/2) sum_k q^k / (4^k k! (k+1)!), positive terms, compensated sum
        double term = 1.0, sum = 1.0, comp = 0.0;
        for (int k = 0; k < 4000; ++k) {
            term *= q / (4.0 * (k + 1) * (k + 2));
            const double t = sum + term;
            comp += (sum - t) + term;
            sum = t;
            if (term < 1e-18 * sum) break;
        }
        return pref * 0.5 * (sum + comp);
    }
    if (q == 0.0) return 0.5 * pref;
    const double r = std::sqrt(-q);
    return pref * ::j1(r) / r;
}

// Centered cardinal B-spline M_n(t) of order n (support [-n/2, n/2]) from the two-sided
// recursion M_k(s) = ((k/2 + s) M_{k-1}(s + 1/2) + (k/2 - s) M_{k-1}(s - 1/2)) / (k - 1):
// level k holds M_k at the offsets t + (j - (n - k)/2), j = 0..n-k, built up from the box
// M_1 (1 on [-1/2, 1/2), 0 elsewhere).
static double cardinal_bspline(int n, double t) {
    if (n < 1 || n > 62 || !(std::fabs(t) < 0.5 * n)) return 0.0;
    std::vector<double> lev((size_t)n);
    for (int j = 0; j < n; ++j) {                 // order 1 at t + j - (n - 1)/2
        const double s = t + j - 0.5 * (n - 1);
        lev[(size_t)j] = (s >= -0.5 && s < 0.5) ? 1.0 : 0.0;
    }
    for (int k = 2; k <= n; ++k) {                // order k at t + j - (n - k)/2, j <= n - k
        for (int j = 0; j + k <= n; ++j) {
            const double s = t + j - 0.5 * (n - k);
            lev[(size_t)j] = ((0.5 * k + s) * lev[(size_t)j + 1] + (0.5 * k - s) * lev[(size_t)j]) /
                             (double)(k - 1);
        }
    }
    return lev[0];
}

double window_beta(int win, int m, double sigma) {
    switch (win) {
        case WIN_BSPLINE: return 0.0;
        case WIN_ALG: return 3.0 * m;
        default: return 2.0 * PI * m * (1.0 - 1.0 / (2.0 * sigma));
    }
}

double omega_w(int win, double x, double beta, int m) {
    switch (win) {
        case WIN_KB: {
            if (!(std::fabs(x) <= 1.0)) return 0.0;
            return std::cyl_bessel_i(0.0, beta * std::sqrt(1.0 - x * x)) / std::cyl_bessel_i(0.0, beta);
        }
        case WIN_BSPLINE:
            return cardinal_bspline(2 * m, m * x) / cardinal_bspline(2 * m, 0.0);
        case WIN_ALG:
            if (!(std::fabs(x) < 1.0)) return 0.0;
            return std::exp((beta - 0.5) * std::log1p(-x * x));
        default:
            return omega_sinh(x, beta);
    }
}

double omega_hat_w(int win, double v, double beta, int m) {
    switch (win) {
        case WIN_KB: {
            // 2 int_0^1 I0(beta sqrt(1-x^2)) cos(2 pi v x) dx / I0(beta)
            const double q = beta * beta - 4.0 * PI * PI * v * v;
            const double c = 2.0 / std::cyl_bessel_i(0.0, beta);
            if (q > 0.0) { const double r = std::sqrt(q); return c * std::sinh(r) / r; }
            if (q == 0.0) return c;
            const double r = std::sqrt(-q);
            return c * std::sin(r) / r;
        }
        case WIN_BSPLINE: {
            const double y = PI * v / m;
            const double sc = y == 0.0 ? 1.0 : std::sin(y) / y;
            return std::pow(sc, 2 * m) / (m * cardinal_bspline(2 * m, 0.0));
        }
        case WIN_ALG: {
            // pi (2 beta)! / (4^beta beta!) (pi v)^{-beta} J_beta(2 pi v), 1/beta! at v = 0
            const double lc = std::log(PI) + std::lgamma(2.0 * beta + 1.0) - beta * std::log(4.0) -
                              std::lgamma(beta + 1.0);
            if (v == 0.0) return std::exp(lc - std::lgamma(beta + 1.0));
            const double a = PI * std::fabs(v);
            return std::exp(lc - beta * std::log(a)) * std::cyl_bessel_j(beta, 2.0 * a);
        }
        default:
            return omega_sinh_hat(v, beta);
    }
}

bool smooth5(int64_t n) {
    if (n <= 0) return false;
    const int64_t p[3] = {2, 3, 5};
    for (int i = 0; i < 3; ++i)
        while (n % p[i] == 0) n /= p[i];
    return n == 1;
}

const char *derive(int64_t N, double sigma1, double sigma2, int m1, int m2, Derived *o,
                   int window) {
    if (N < 1) return "N must be >= 1";
    if (window < WIN_SINH || window > WIN_ALG) return "unknown window";
    if (window == WIN_ALG && (!(sigma1 > PI / 3.0) || !(sigma2 > PI / 3.0)))
        return "the algebraic window needs sigma1, sigma2 > pi/3";
    if (!(sigma1 > 1.0) || !(sigma2 > 1.0)) return "sigma1 and sigma2 must be > 1";
    if (!(sigma1 <= 16.0) || !(sigma2 <= 16.0)) return "sigma1 and sigma2 must be <= 16";
    if (m1 < 2 || m2 < 2) return "m1 and m2 must be >= 2";
    if (m1 > 16 || m2 > 16) return "m1 and m2 must be <= 16";
    if (N > (int64_t(1) << 28)) return "N too large";
    o->N = N;
    o->m1 = m1;
    o->m2 = m2;
    // N* = N + ceil(2 m1 / sigma1): frequencies v in [-1/2,1/2] become v* = N v / N*
    // inside [-1/(2a), 1/(2a)] (rescaling after eq. (2.7)).
    o->Nstar = N + (int64_t)std::ceil(2.0 * m1 / sigma1 - 1e-12);
    int64_t n1 = (int64_t)std::ceil(sigma1 * (double)o->Nstar - 1e-9);
    if (n1 % 2) ++n1;                                   // N1 in 2N
    o->N1 = n1;
    o->K1 = n1 + 2 * m1;                                // a N1 = N1 + 2 m1, eq. (2.6)
    int64_t n2 = (int64_t)std::ceil(sigma2 * (double)o->K1 - 1e-9);
    if (n2 % 2) ++n2;
    while (!smooth5(n2)) n2 += 2;                       // even 2^a 3^b 5^c
    o->N2 = n2;
    o->sigma1 = (double)o->N1 / (double)o->Nstar;
    o->sigma2 = (double)o->N2 / (double)o->K1;
    o->window = window;
    o->beta1 = window_beta(window, m1, o->sigma1);
    o->beta2 = window_beta(window, m2, o->sigma2);
    if (o->N2 > (int64_t(1) << 20)) return "N2 exceeds 2^20 (N too large for the grid FFT)";
    if ((double)(2 * m2) > (1.0 - 1.0 / o->sigma1) * (double)o->N2)
        return "step 4 of Algorithm 2.2 needs 2 m2 <= (1 - 1/sigma1) N2";
    return nullptr;
}

double window_error_term(int m, double sigma) {
    return (24.0 * std::pow((double)m, 1.5) + 10.0) *
           std::exp(-2.0 * PI * m * std::sqrt(1.0 - 1.0 / sigma));
}

double cheb_eval(const double *c, int n, double y) {
    // Clenshaw recurrence
    double b1 = 0.0, b2 = 0.0;
    for (int d = n - 1; d >= 1; --d) {
        const double b0 = 2.0 * y * b1 - b2 + c[d];
        b2 = b1;
        b1 = b0;
    }
    return y * b1 - b2 + c[0];
}

double fit_taps(int m, double beta, int D, std::vector<double> &coef, int win) {
    coef.assign((size_t)2 * m * D, 0.0);
    double err = 0.0;
    constexpr int G = 241;
    for (int t = 0; t < 2 * m; ++t) {
        auto f = [&](double y) {
            const double z = 0.5 * (y + 1.0);
            return omega_w(win, (t - m + 1 - z) / m, beta, m);
        };
        double *c = coef.data() + (size_t)t * D;
        cheb_interp(f, D, c);
        for (int g = 0; g < G; ++g) {
            const double y = -1.0 + 2.0 * g / (G - 1);
            err = std::fmax(err, std::fabs(cheb_eval(c, D, y) - f(y)));
        }
    }
    return err;
}

int choose_degree(int m, double sigma, double beta, bool fp64, double *fit_err,
                  std::vector<double> &coef, int win) {
    static const int cand[] = {8, 10, 12, 14, 16, 20};
    std::vector<double> tmp;
    const double floor_err = fit_taps(m, beta, 24, tmp, win);
    const double e1 = window_error_term(m, sigma);
    const double target = fp64 ? 1e-3 * e1 : std::fmax(1e-2 * e1, 5e-8);
    const double accept = std::fmax(target, 1.5 * floor_err);
    for (int D : cand) {
        const double err = fit_taps(m, beta, D, coef, win);
        if (err <= accept || D == 20) {
            *fit_err = err;
            return D;
        }
    }
    return 20;
}

// One node pair of the n-point rule: Newton on P_n (three-term recurrence) from the
// Chebyshev-like initial guess of node i (from the top), then the weight 2/((1-t^2) P_n'(t)^2),
// halved for [-1/2, 1/2].
static void gl_node(int64_t n, int64_t i, double *tau, double *w) {
    double t = std::cos(PI * ((double)i + 0.75) / ((double)n + 0.5));
    double pn = 0.0, pm = 0.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = t;
        for (int64_t k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / (double)k;
            p0 = p1;
            p1 = p2;
        }
        pn = n == 1 ? t : p1;
        pm = n == 1 ? 1.0 : p0;
        const double dp = (double)n * (t * pn - pm) / (t * t - 1.0);
        const double dt = pn / dp;
        t -= dt;
        if (std::fabs(dt) < 1e-15) break;      // quadratic convergence: t is at ulp level
    }
    double p0 = 1.0, p1 = t;
    for (int64_t k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / (double)k;
        p0 = p1;
        p1 = p2;
    }
    pn = n == 1 ? t : p1;
    pm = n == 1 ? 1.0 : p0;
    const double dp = (double)n * (t * pn - pm) / (t * t - 1.0);
    const double wt = 1.0 / ((1.0 - t * t) * dp * dp);
    tau[n - 1 - i] = 0.5 * t;
    tau[i] = -0.5 * t;
    w[n - 1 - i] = wt;
    w[i] = wt;
}

void gauss_legendre(int64_t n, double *tau, double *w) {
    const int64_t half = (n + 1) / 2;
    // O(n) work per node: large rules are spread over the host's cores
    const int64_t nt = n < 512 ? 1 : std::min<int64_t>(16, std::max<unsigned>(1u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int64_t r = 0; r < nt; ++r)
        th.emplace_back([=] {
            for (int64_t i = r; i < half; i += nt) gl_node(n, i, tau, w);
        });
    for (auto &x : th) x.join();
    if (n % 2 == 1) tau[n / 2] = 0.0;
}

bool cell_map(int64_t num, int64_t den, CellMap *out) {
    if (num <= 0 || den <= 0) return false;
    const unsigned __int128 q = ((unsigned __int128)(uint64_t)num << FX_SB) + (uint64_t)den / 2;
    const unsigned __int128 S = q / (uint64_t)den;
    if (S >> 63) return false;
    out->S = (uint64_t)S;
    const uint64_t half = (uint64_t)1 << (FX_SB + 1);
    const int64_t c_hi = (int64_t)(out->S >> (FX_SB + 1));
    out->c_lo = -(int64_t)((out->S + half - 1) >> (FX_SB + 1));
    out->ncell = c_hi - out->c_lo + 1;
    out->scale = (double)num / (double)den;
    return true;
}

bool split_fft(int64_t N2, int maxf, int *n1, int *n2) {
    int best1 = 0;
    for (int64_t a = 1; a <= maxf; ++a) {
        if (N2 % a) continue;
        const int64_t b = N2 / a;
        if (b > maxf) continue;
        if (!smooth5(a) || !smooth5(b)) continue;
        if (best1 == 0 || std::llabs(a - b) < std::llabs(best1 - N2 / best1)) best1 = (int)a;
    }
    if (best1 == 0) return false;
    *n1 = best1;
    *n2 = (int)(N2 / best1);
    return true;
}

int radices(int n, int *r, int maxr) {
    int k = 0;
    while (n % 4 == 0 && k < maxr) { r[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < maxr) { r[k++] = 2; n /= 2; }
    while (n % 3 == 0 && k < maxr) { r[k++] = 3; n /= 3; }
    while (n % 5 == 0 && k < maxr) { r[k++] = 5; n /= 5; }
    return n == 1 ? k : -1;
}

}  // namespace hm
}  // namespace nnfft
