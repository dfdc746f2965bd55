// hostmath.h -- host-side numerics of the plan: parameter rules, the sinh window
// and its Fourier transform, Chebyshev fits of the window taps and of 1/phihat1,
// the Gauss-Legendre rule and the FFT factorisation.  No GPU calls.
#pragma once

#include <cmath>
#include <cstdint>
#include <vector>

namespace nnfft {
namespace hm {

constexpr double PI = 3.141592653589793238462643383279502884;

// Sinh-type window of Example 2.1 / Section 4 on [-1, 1] (0 outside).
double omega_sinh(double x, double beta);
// Its Fourier transform, eq. (2.1), for |v| <= beta/(2 pi) via the I1 power
// series (all terms positive); beyond the branch point via J1.
double omega_sinh_hat(double v, double beta);

// Windows of the set Omega (Section 2): 0 sinh-type, 1 Kaiser-Bessel (I0(beta sqrt(1-x^2)) /
// I0(beta), shape parameter as for sinh), 2 B-spline B_{2m}(m x) / B_{2m}(0) (Example 2.1, no
// shape parameter), 3 algebraic (1 - x^2)^{beta - 1/2} with beta = 3m (Example 2.1, needs
// sigma > pi/3).  omega_w and omega_hat_w evaluate any of them and its Fourier transform.
enum { WIN_SINH = 0, WIN_KB = 1, WIN_BSPLINE = 2, WIN_ALG = 3 };
double omega_w(int win, double x, double beta, int m);
double omega_hat_w(int win, double v, double beta, int m);
// The window's shape parameter for truncation m and oversampling sigma.
double window_beta(int win, int m, double sigma);

struct Derived {
    int64_t N, Nstar, N1, K1, N2;
    int m1, m2;
    double sigma1, sigma2, beta1, beta2;
    int window;
};
// Section 2 / Section 4 parameter rules; returns an error message or nullptr.
const char *derive(int64_t N, double sigma1, double sigma2, int m1, int m2, Derived *out,
                   int window = WIN_SINH);

// Theorem 4.1's first term (24 m^{3/2} + 10) exp(-2 pi m sqrt(1 - 1/sigma)).
double window_error_term(int m, double sigma);

// Chebyshev interpolation of f at n first-kind points on [-1, 1]:
// coefficients c[0..n-1] with f(y) ~ sum_d c[d] T_d(y).
template <class F> void cheb_interp(const F &f, int n, double *c) {
    const double pi = 3.141592653589793238462643383279502884;
    std::vector<double> fy(n);
    for (int i = 0; i < n; ++i) fy[i] = f(std::cos(pi * (i + 0.5) / n));
    for (int d = 0; d < n; ++d) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fy[i] * std::cos(pi * d * (i + 0.5) / n);
        c[d] = s * 2.0 / n;
    }
    c[0] *= 0.5;
}
double cheb_eval(const double *c, int n, double y);

// Fit the 2m tap functions w_t(y) = omega((t - m + 1 - (y+1)/2)/m) with D
// coefficients each (row-major [t][d]); returns the max abs error on a test grid.
double fit_taps(int m, double beta, int D, std::vector<double> &coef, int win = WIN_SINH);
// Pick the coefficient count D for a window: the smallest supported D whose fit
// error is below the target for the dtype (or at the window's floor).
int choose_degree(int m, double sigma, double beta, bool fp64, double *fit_err,
                  std::vector<double> &coef, int win = WIN_SINH);

// n-point Gauss-Legendre rule on [-1/2, 1/2] (Newton on the Legendre recurrence).
void gauss_legendre(int64_t n, double *tau, double *w);

// Cells of one node side.  A node t in [-1/2, 1/2] has u = t * num / den (the rational
// scale N1 N / N* on the v side, N2 N* / N1 on the x side); the kernels compute u in
// fixed point with the scale rounded to S = round(num / den * 2^FX_SB).  Cell c = floor(u)
// runs from c_lo = floor(-S / 2^(FX_SB+1)) to floor(S / 2^(FX_SB+1)), exactly as the
// kernels' fixed-point floor does at t = -1/2 and t = 1/2.
constexpr int FX_SB = 44;
struct CellMap {
    uint64_t S;        // scale in units of 2^-FX_SB (< 2^63: scale < 2^19)
    int64_t c_lo;
    int64_t ncell;
    double scale;      // num / den as a double (host-side fits only)
};
bool cell_map(int64_t num, int64_t den, CellMap *out);

// n has no prime factor above 5.
bool smooth5(int64_t n);
// N2 = n1 * n2 with n1, n2 <= maxf and 5-smooth, as square as possible; radix lists.
bool split_fft(int64_t N2, int maxf, int *n1, int *n2);
int radices(int n, int *r, int maxr);

}  // namespace hm
}  // namespace nnfft
