// nnfft_host.cu -- the C ABI of include/nnfft.h: plan construction (parameters,
// window fits, deconvolution tables, FFT tables, device buffers), the step-0
// node preprocessing, and the launch sequences of Algorithm 2.2 (forward), its
// transpose (adjoint) and Algorithm 6.1 (fast sinc transform).
//
// Launch sequence of nnfft_exec (all on the plan stream, no host sync):
//   k_moments(v side)      cell moments of f over the sorted v nodes      step 1
//   k_spread_conv(v side)  g_l / (N1 N2 phihat2(l)) into the N2 buffer     steps 1-2
//   k_fft_pass1/2          h_s = sum_l ghat_l e^{-2 pi i l s/N2}           step 3
//   k_gather_conv(x side)  per-cell window sums of h                       step 4
//   k_eval(x side)         s1(N x_j) / phihat1(N* x_j), scattered to y     step 4 + output
// nnfft_adjoint runs the transposes in reverse order with the +sign FFT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hostmath.h"
#include "internal.h"
#include "nnfft.h"

using namespace nnfft;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(NNFFT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define NN_CUDA(call, where)                                     \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);      \
    } while (0)

struct Side {
    // plan-time
    int m = 0, D = 0;
    double beta = 0, sigma = 0, uscale = 0, fit_err = 0;
    long long c_lo = 0;
    int ncell = 0, M = 0, max_items = 0, key_bits = 8;
    bool has_r = false;
    void *coef = nullptr, *rfit = nullptr;
    // node-time
    uint32_t *keys = nullptr, *keys_alt = nullptr;
    int *vals = nullptr, *vals_alt = nullptr, *hist = nullptr;
    int *perm = nullptr;
    uint32_t *keys_sorted = nullptr;
    void *ys = nullptr;
    void *y_user = nullptr;        // coordinates in caller order (step-0 scratch)
    int *cell_off = nullptr, *item_cnt = nullptr, *item_off = nullptr;
    int *item_cell = nullptr, *item_pb = nullptr, *item_pe = nullptr, *nitems = nullptr;
    bool set = false;
};

}  // namespace

struct nnfft_plan_s {
    nnfft_info info{};
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;              // second stream: the two node sides sort concurrently
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool dbl = true;
    bool split = false;          // fp64 plan using the split-precision kernels
    std::vector<double> rfit_host;   // x-side 1/phihat1 fits (plan construction only)
    bool split_ok = false;       // the window fits allow them (see kern_spread_df.cu)
    Side side[2];   // 0: v (frequency) side, 1: x (spatial) side
    void *dec2 = nullptr;
    FftPlanDev fft{};
    // split-precision tables (fp64 plans)
    void *coef_df[2] = {nullptr, nullptr};
    void *rfit_df = nullptr, *dec2_df = nullptr;
    FftDf fftdf{};
    void *bufA = nullptr, *bufB = nullptr, *bufC = nullptr;
    void *P = nullptr;   // per-item moments
    void *Q = nullptr;   // per-cell moments (spread) and per-cell window sums (gather)
    int *status = nullptr;
    int *status_host = nullptr;   // pinned
    // host-API staging (allocated on first use)
    double *st_v = nullptr, *st_x = nullptr;
    void *st_f = nullptr, *st_y = nullptr;
    std::vector<void *> allocs;
    // per-stage timing (nnfft_timing_enable)
    bool timing = false;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double acc_ms[16] = {0};
    int64_t acc_n[16] = {0};
};

namespace {

size_t real_size(bool dbl) { return dbl ? sizeof(double) : sizeof(float); }

int dalloc(nnfft_plan_s *p, void **ptr, size_t bytes, const char *what) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NNFFT_ENOMEM : NNFFT_ECUDA,
                    std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
    }
    p->allocs.push_back(*ptr);
    return NNFFT_OK;
}

template <class T> int dalloc_n(nnfft_plan_s *p, T **ptr, size_t n, const char *what) {
    void *v = nullptr;
    int rc = dalloc(p, &v, n * sizeof(T), what);
    *ptr = static_cast<T *>(v);
    return rc;
}

// Upload a host double array as the plan's real type.
int upload_real(nnfft_plan_s *p, void **dst, const std::vector<double> &src, const char *what) {
    int rc = dalloc(p, dst, src.size() * real_size(p->dbl), what);
    if (rc) return rc;
    if (p->dbl) {
        NN_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice),
                what);
    } else {
        std::vector<float> f(src.begin(), src.end());
        NN_CUDA(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice),
                what);
    }
    return NNFFT_OK;
}

// Upload doubles as (hi, lo) float pairs: hi = fl(x), lo = fl(x - hi); scale multiplies x.
int upload_df2(nnfft_plan_s *p, void **dst, const std::vector<double> &src, double scale,
               const char *what) {
    std::vector<float> f(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        const double x = src[i] * scale;
        const float h = (float)x;
        f[2 * i] = h;
        f[2 * i + 1] = (float)(x - (double)h);
    }
    int rc = dalloc(p, dst, f.size() * sizeof(float), what);
    if (rc) return rc;
    NN_CUDA(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice), what);
    return NNFFT_OK;
}

// Complex table exp(-2 pi i k / n), k < n, computed in long double and rounded.
std::vector<double> twiddles(int64_t n) {
    std::vector<double> t(2 * (size_t)n);
    const long double twopi = 6.283185307179586476925286766559005768L;
    for (int64_t k = 0; k < n; ++k) {
        // reduce k/n to [-1/2, 1/2] before the trig calls
        int64_t kk = k <= n / 2 ? k : k - n;
        long double a = -twopi * (long double)kk / (long double)n;
        t[2 * k] = (double)cosl(a);
        t[2 * k + 1] = (double)sinl(a);
    }
    return t;
}

int fill_info(int64_t N, int64_t M1, int64_t M2, double sigma1, double sigma2, int m1, int m2,
              nnfft_dtype dtype, nnfft_info *info, hm::Derived *d, std::vector<double> *coef1,
              std::vector<double> *coef2) {
    if (!info) return fail(NNFFT_EINVAL, "null output pointer");
    if (M1 < 0 || M2 < 0) return fail(NNFFT_EINVAL, "M1 and M2 must be >= 0");
    if (M1 > (int64_t(1) << 30) || M2 > (int64_t(1) << 30))
        return fail(NNFFT_EINVAL, "M1 and M2 must be <= 2^30");
    if (dtype != NNFFT_C64 && dtype != NNFFT_C128) return fail(NNFFT_EINVAL, "unknown dtype");
    const char *msg = hm::derive(N, sigma1, sigma2, m1, m2, d);
    if (msg) return fail(NNFFT_EINVAL, msg);
    memset(info, 0, sizeof(*info));
    info->N = d->N;
    info->Nstar = d->Nstar;
    info->N1 = d->N1;
    info->K1 = d->K1;
    info->N2 = d->N2;
    info->M1 = M1;
    info->M2 = M2;
    info->m1 = m1;
    info->m2 = m2;
    info->sigma1 = d->sigma1;
    info->sigma2 = d->sigma2;
    info->beta1 = d->beta1;
    info->beta2 = d->beta2;
    info->dtype = (int)dtype;
    const bool fp64 = dtype == NNFFT_C128;
    std::vector<double> tmp1, tmp2;
    info->D1 = hm::choose_degree(m1, d->sigma1, d->beta1, fp64, &info->fit_err1,
                                 coef1 ? *coef1 : tmp1);
    info->D2 = hm::choose_degree(m2, d->sigma2, d->beta2, fp64, &info->fit_err2,
                                 coef2 ? *coef2 : tmp2);
    // cells: v side u = v * N1 N / N*, x side u = x * N2 N* / N1; |node| <= 1/2
    const double us1 = (double)d->N1 * (double)d->N / (double)d->Nstar;
    const double us2 = (double)d->N2 * (double)d->Nstar / (double)d->N1;
    info->ncell1 = (int64_t)std::floor(0.5 * us1) - (int64_t)std::floor(-0.5 * us1) + 1;
    info->ncell2 = (int64_t)std::floor(0.5 * us2) - (int64_t)std::floor(-0.5 * us2) + 1;
    int n1 = 0, n2 = 0;
    if (!hm::split_fft(d->N2, FFT_MAX_FACTOR, &n1, &n2))
        return fail(NNFFT_EINVAL, "N2 has no factorisation n1*n2 with n1, n2 <= 1024");
    info->fft_n1 = n1;
    info->fft_n2 = n2;
    return NNFFT_OK;
}

bool split_weights_ok(const std::vector<double> &coef, int ntap, int D) {
    for (int d = D / 2; d < D; ++d) {
        double k = 0.0;
        for (int t = 0; t < ntap; ++t) k = std::max(k, std::fabs(coef[(size_t)t * D + d]));
        if (k > 2e-7) return false;
    }
    return true;
}

int key_bits_for(int ncell) {
    int b = 1;
    while ((1LL << b) < ncell) ++b;
    return ((b + 7) / 8) * 8;
}

int setup_side(nnfft_plan_s *p, int s, const hm::Derived &d, const std::vector<double> &coef) {
    Side &S = p->side[s];
    const nnfft_info &I = p->info;
    S.m = s == 0 ? d.m1 : d.m2;
    S.D = s == 0 ? I.D1 : I.D2;
    S.beta = s == 0 ? d.beta1 : d.beta2;
    S.sigma = s == 0 ? d.sigma1 : d.sigma2;
    S.fit_err = s == 0 ? I.fit_err1 : I.fit_err2;
    S.uscale = s == 0 ? (double)d.N1 * (double)d.N / (double)d.Nstar
                      : (double)d.N2 * (double)d.Nstar / (double)d.N1;
    S.c_lo = (long long)std::floor(-0.5 * S.uscale);
    S.ncell = (int)(s == 0 ? I.ncell1 : I.ncell2);
    S.M = (int)(s == 0 ? I.M1 : I.M2);
    S.max_items = S.ncell + (S.M + ITEM_CAP - 1) / ITEM_CAP;
    S.key_bits = key_bits_for(S.ncell);
    S.has_r = s == 1;
    if (!supported_degree(S.D)) return fail(NNFFT_EINVAL, "unsupported window degree");
    int rc = upload_real(p, &S.coef, coef, "window coefficients");
    if (rc) return rc;
    if (S.has_r) {
        // Per x cell c: Chebyshev fit in y of 1/phihat1(N* x), x = (c + (y+1)/2)/uscale,
        // phihat1(v) = (m1/N1) omegahat1(m1 v / N1) (scaling in the proof of Theorem 3.4).
        std::vector<double> r((size_t)S.ncell * NR);
        for (int ic = 0; ic < S.ncell; ++ic) {
            const double c = (double)(S.c_lo + ic);
            auto f = [&](double y) {
                const double x = (c + 0.5 * (y + 1.0)) / S.uscale;
                const double w = (double)d.m1 * (double)d.Nstar * x / (double)d.N1;
                return (double)d.N1 / ((double)d.m1 * hm::omega_sinh_hat(w, d.beta1));
            };
            hm::cheb_interp(f, NR, r.data() + (size_t)ic * NR);
        }
        rc = upload_real(p, &S.rfit, r, "phihat1 fit");
        if (rc) return rc;
        p->rfit_host = r;
    }
    const size_t M = (size_t)S.M;
    const size_t rs = real_size(p->dbl);
    if ((rc = dalloc_n(p, &S.keys, M, "keys")) || (rc = dalloc_n(p, &S.keys_alt, M, "keys")) ||
        (rc = dalloc_n(p, &S.vals, M, "perm")) || (rc = dalloc_n(p, &S.vals_alt, M, "perm")) ||
        (rc = dalloc_n(p, &S.hist, radix_sort_hist_len(S.M), "sort histogram")) ||
        (rc = dalloc(p, &S.ys, M * rs, "sorted coordinates")) ||
        (rc = dalloc(p, &S.y_user, M * rs, "coordinates")) ||
        (rc = dalloc_n(p, &S.cell_off, (size_t)S.ncell + 1, "cell offsets")) ||
        (rc = dalloc_n(p, &S.item_cnt, (size_t)S.ncell + 1, "item counts")) ||
        (rc = dalloc_n(p, &S.item_off, (size_t)S.ncell + 1, "item offsets")) ||
        (rc = dalloc_n(p, &S.item_cell, (size_t)S.max_items, "items")) ||
        (rc = dalloc_n(p, &S.item_pb, (size_t)S.max_items, "items")) ||
        (rc = dalloc_n(p, &S.item_pe, (size_t)S.max_items, "items")) ||
        (rc = dalloc_n(p, &S.nitems, 1, "item count")))
        return rc;
    NN_CUDA(cudaMemset(S.item_off, 0, sizeof(int) * ((size_t)S.ncell + 1)), "memset");
    NN_CUDA(cudaMemset(S.nitems, 0, sizeof(int)), "memset");
    return NNFFT_OK;
}

// Brackets one stage with CUDA events on the plan stream when timing is enabled.
struct StageTimer {
    nnfft_plan_s *p;
    int stage;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    StageTimer(nnfft_plan_s *p_, int stage_, cudaStream_t st_ = nullptr)
        : p(p_), stage(stage_), st(st_ ? st_ : p_->stream) {
        if (!p->timing) return;
        cudaEvent_t a = take();
        b = take();
        if (a && b) {
            cudaEventRecord(a, st);
            p->recs.push_back({stage, a, b});
        } else {
            b = nullptr;
        }
    }
    ~StageTimer() {
        if (b) cudaEventRecord(b, st);
    }
    cudaEvent_t take() {
        if (!p->pool.empty()) {
            cudaEvent_t e = p->pool.back();
            p->pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
};

template <typename Real> SideK<Real> side_args(const Side &S, bool with_r) {
    SideK<Real> k;
    k.m = S.m;
    k.D = S.D;
    k.ncell = S.ncell;
    k.c_lo = S.c_lo;
    k.coef = static_cast<const Real *>(S.coef);
    k.rfit = with_r ? static_cast<const Real *>(S.rfit) : nullptr;
    k.perm = S.perm;
    k.ys = static_cast<const Real *>(S.ys);
    k.item_off = S.item_off;
    k.item_cell = S.item_cell;
    k.item_pb = S.item_pb;
    k.item_pe = S.item_pe;
    k.nitems = S.nitems;
    k.max_items = S.max_items;
    return k;
}

int set_side_nodes(nnfft_plan_s *p, int s, const double *nodes, cudaStream_t st) {
    Side &S = p->side[s];
    StageTimer timer(p, s, st);
    if (S.M == 0) {
        NN_CUDA(cudaMemsetAsync(S.item_off, 0, sizeof(int) * ((size_t)S.ncell + 1), st), "memset");
        NN_CUDA(cudaMemsetAsync(S.nitems, 0, sizeof(int), st), "memset");
        S.perm = S.vals;
        S.set = true;
        return NNFFT_OK;
    }
    const int yfmt = !p->dbl ? 0 : (p->split ? 2 : 1);
    const int ybytes = p->dbl ? 8 : 4;
    NN_CUDA(launch_node_keys_y(nodes, S.M, S.uscale, S.c_lo, S.ncell, S.keys, S.y_user, yfmt,
                               S.hist, p->status, st),
            "node keys");
    uint32_t *ks = nullptr;
    int *vs = nullptr;
    NN_CUDA(radix_sort_cells(S.keys, S.vals, S.keys_alt, S.vals_alt, S.hist, S.M, S.key_bits,
                             S.y_user, S.ys, ybytes, st, &ks, &vs),
            "radix sort");
    S.perm = vs;
    S.keys_sorted = ks;
    NN_CUDA(launch_cell_offsets(ks, S.M, S.ncell, S.cell_off, st), "cell offsets");
    NN_CUDA(launch_build_items_fused(S.cell_off, S.ncell, S.item_off, S.item_cell, S.item_pb,
                                     S.item_pe, S.nitems, st),
            "work items");
    S.set = true;
    return NNFFT_OK;
}

int run_forward_split(nnfft_plan_s *p, const void *f, void *y) {
    const Side &V = p->side[0], &X = p->side[1];
    cudaStream_t st = p->stream;
    if (X.M == 0) return NNFFT_OK;
    const SideK<double> sv = side_args<double>(V, false);
    const SideK<double> sx = side_args<double>(X, true);
    const SideDf tv{static_cast<const float2 *>(p->coef_df[0]), nullptr};
    const SideDf tx{static_cast<const float2 *>(p->coef_df[1]), static_cast<const float2 *>(p->rfit_df)};
    const long long K1 = p->info.K1;
    const int N2 = (int)p->info.N2;
    {
        StageTimer t(p, 2);
        NN_CUDA(launch_moments_df(sv, f, p->P, st), "spread moments");
    }
    {
        StageTimer t(p, 12);
        NN_CUDA(launch_cell_fold_df(sv, tv, p->P, p->Q, st), "cell fold");
    }
    {
        StageTimer t(p, 3);
        NN_CUDA(launch_spread_conv_df(sv, tv, p->Q, static_cast<const float2 *>(p->dec2_df), K1 / 2,
                                      K1, N2, p->bufA, st),
                "spread convolution");
    }
    {
        StageTimer t(p, 4);
        NN_CUDA(launch_fft_df(p->fftdf, p->bufA, p->bufB, p->bufC, -1, st), "fft");
    }
    {
        StageTimer t(p, 5);
        NN_CUDA(launch_gather_conv_df(sx, tx, p->bufC, nullptr, 0, 0, N2, p->Q, st),
                "gather convolution");
    }
    {
        StageTimer t(p, 6);
        NN_CUDA(launch_eval_df(sx, p->Q, y, st), "gather evaluation");
    }
    return NNFFT_OK;
}

int run_adjoint_split(nnfft_plan_s *p, const void *g, void *z) {
    const Side &V = p->side[0], &X = p->side[1];
    cudaStream_t st = p->stream;
    if (V.M == 0) return NNFFT_OK;
    const SideK<double> sv = side_args<double>(V, false);
    const SideK<double> sx = side_args<double>(X, true);
    const SideDf tv{static_cast<const float2 *>(p->coef_df[0]), nullptr};
    const SideDf tx{static_cast<const float2 *>(p->coef_df[1]), static_cast<const float2 *>(p->rfit_df)};
    const SideDf tx_nofold{static_cast<const float2 *>(p->coef_df[1]), nullptr};
    const long long K1 = p->info.K1;
    const int N2 = (int)p->info.N2;
    {
        StageTimer t(p, 7);
        NN_CUDA(launch_moments_df(sx, g, p->P, st), "adjoint spread moments");
    }
    {
        StageTimer t(p, 13);
        NN_CUDA(launch_cell_fold_df(sx, tx, p->P, p->Q, st), "adjoint cell fold");
    }
    {
        StageTimer t(p, 8);
        NN_CUDA(launch_spread_conv_df(sx, tx_nofold, p->Q, nullptr, 0, 0, N2, p->bufA, st),
                "adjoint spread convolution");
    }
    {
        StageTimer t(p, 9);
        NN_CUDA(launch_fft_df(p->fftdf, p->bufA, p->bufB, p->bufC, +1, st), "adjoint fft");
    }
    {
        StageTimer t(p, 10);
        NN_CUDA(launch_gather_conv_df(sv, tv, p->bufC, static_cast<const float2 *>(p->dec2_df),
                                      K1 / 2, K1, N2, p->Q, st),
                "adjoint gather convolution");
    }
    {
        StageTimer t(p, 11);
        NN_CUDA(launch_eval_df(sv, p->Q, z, st), "adjoint gather evaluation");
    }
    return NNFFT_OK;
}

template <typename Real> int run_forward(nnfft_plan_s *p, const void *f, void *y) {
    const Side &V = p->side[0], &X = p->side[1];
    cudaStream_t st = p->stream;
    if (X.M == 0) return NNFFT_OK;
    const SideK<Real> sv = side_args<Real>(V, false);
    const SideK<Real> sx = side_args<Real>(X, true);
    const long long K1 = p->info.K1;
    const int N2 = (int)p->info.N2;
    {
        StageTimer t(p, 2);
        NN_CUDA(launch_moments<Real>(sv, f, p->P, st), "spread moments");
    }
    {
        StageTimer t(p, 12);
        NN_CUDA(launch_cell_fold<Real>(sv, p->P, p->Q, st), "cell fold");
    }
    {
        StageTimer t(p, 3);
        NN_CUDA(launch_spread_conv<Real>(sv, p->Q, static_cast<const Real *>(p->dec2), K1 / 2, K1,
                                         N2, p->bufA, st),
                "spread convolution");
    }
    {
        StageTimer t(p, 4);
        NN_CUDA(launch_fft<Real>(p->fft, p->bufA, p->bufB, p->bufC, -1, st), "fft");
    }
    {
        StageTimer t(p, 5);
        NN_CUDA(launch_gather_conv<Real>(sx, p->bufC, nullptr, 0, 0, N2, p->Q, st),
                "gather convolution");
    }
    {
        StageTimer t(p, 6);
        NN_CUDA(launch_eval<Real>(sx, p->Q, y, st), "gather evaluation");
    }
    return NNFFT_OK;
}

template <typename Real> int run_adjoint(nnfft_plan_s *p, const void *g, void *z) {
    const Side &V = p->side[0], &X = p->side[1];
    cudaStream_t st = p->stream;
    if (V.M == 0) return NNFFT_OK;
    const SideK<Real> sv = side_args<Real>(V, false);
    const SideK<Real> sx = side_args<Real>(X, true);
    const long long K1 = p->info.K1;
    const int N2 = (int)p->info.N2;
    {
        StageTimer t(p, 7);
        NN_CUDA(launch_moments<Real>(sx, g, p->P, st), "adjoint spread moments");
    }
    {
        StageTimer t(p, 13);
        NN_CUDA(launch_cell_fold<Real>(sx, p->P, p->Q, st), "adjoint cell fold");
    }
    {
        StageTimer t(p, 8);
        NN_CUDA(launch_spread_conv<Real>(sx, p->Q, nullptr, 0, 0, N2, p->bufA, st),
                "adjoint spread convolution");
    }
    {
        StageTimer t(p, 9);
        NN_CUDA(launch_fft<Real>(p->fft, p->bufA, p->bufB, p->bufC, +1, st), "adjoint fft");
    }
    {
        StageTimer t(p, 10);
        NN_CUDA(launch_gather_conv<Real>(sv, p->bufC, static_cast<const Real *>(p->dec2), K1 / 2,
                                         K1, N2, p->Q, st),
                "adjoint gather convolution");
    }
    {
        StageTimer t(p, 11);
        NN_CUDA(launch_eval<Real>(sv, p->Q, z, st), "adjoint gather evaluation");
    }
    return NNFFT_OK;
}

int collect_status(nnfft_plan_s *p) {
    NN_CUDA(cudaMemcpyAsync(p->status_host, p->status, sizeof(int), cudaMemcpyDeviceToHost,
                            p->stream),
            "status read");
    NN_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream), "status reset");
    NN_CUDA(cudaStreamSynchronize(p->stream), "stream synchronize");
    const int st = *p->status_host;
    if (st & STATUS_RANGE) return fail(NNFFT_ERANGE, "a node is outside [-1/2, 1/2] or NaN");
    if (st & STATUS_INTERNAL)
        return fail(NNFFT_ECUDA, "internal error: inconsistent node cell assignment");
    return NNFFT_OK;
}

void free_plan(nnfft_plan_s *p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    if (p->aux) {
        cudaStreamSynchronize(p->aux);
        cudaStreamDestroy(p->aux);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    for (auto &r : p->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
    for (void *a : p->allocs) cudaFree(a);
    if (p->status_host) cudaFreeHost(p->status_host);
    delete p;
}

}  // namespace

namespace nnfft {
int report_error(int code, const std::string &msg) { return fail(code, msg); }
cudaStream_t plan_stream(nnfft_plan_t p) { return p->stream; }
}  // namespace nnfft

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

const char *nnfft_last_error(void) { return g_last_error.c_str(); }

int nnfft_params(int64_t N, int64_t M1, int64_t M2, double sigma1, double sigma2, int m1, int m2,
                 nnfft_dtype dtype, nnfft_info *out) {
    hm::Derived d;
    return fill_info(N, M1, M2, sigma1, sigma2, m1, m2, dtype, out, &d, nullptr, nullptr);
}

int nnfft_gauss_legendre(int64_t n, double *tau_host, double *w_host) {
    if (n < 1 || !tau_host || !w_host) return fail(NNFFT_EINVAL, "invalid Gauss-Legendre request");
    hm::gauss_legendre(n, tau_host, w_host);
    return NNFFT_OK;
}

int nnfft_plan(nnfft_plan_t *out, int64_t N, int64_t M1, int64_t M2, double sigma1,
               double sigma2, int m1, int m2, nnfft_dtype dtype, void *stream) {
    if (!out) return fail(NNFFT_EINVAL, "null plan pointer");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(NNFFT_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    nnfft_plan_s *p = new nnfft_plan_s();
    p->stream = static_cast<cudaStream_t>(stream);
    p->dbl = dtype == NNFFT_C128;
    hm::Derived d;
    std::vector<double> coef1, coef2;
    int rc = fill_info(N, M1, M2, sigma1, sigma2, m1, m2, dtype, &p->info, &d, &coef1, &coef2);
    if (rc) { delete p; return rc; }
    const nnfft_info &I = p->info;
    const size_t rs = real_size(p->dbl), cs = 2 * rs;
    auto bail = [&](int code) { free_plan(p); return code; };

    if (cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "stream/event creation"));
    if ((rc = dalloc_n(p, &p->status, 1, "status"))) return bail(rc);
    if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    if (cudaMallocHost(&p->status_host, sizeof(int)) != cudaSuccess) {
        p->status_host = nullptr;
        cudaGetLastError();
        return bail(fail(NNFFT_ENOMEM, "cudaMallocHost(status)"));
    }
    if ((rc = setup_side(p, 0, d, coef1))) return bail(rc);
    if ((rc = setup_side(p, 1, d, coef2))) return bail(rc);
    // Split precision (fp64 plans): degrees >= D/2 run in FP32, so their weights
    // kappa_d = max_t |coef[t][d]| must be small enough that an FP32 error there stays
    // near 1e-13 of ||f||_1 in the worst case.
    p->split_ok = p->dbl && df_supported_degree(I.D1) && df_supported_degree(I.D2) &&
                  split_weights_ok(coef1, 2 * d.m1, I.D1) && split_weights_ok(coef2, 2 * d.m2, I.D2);
    p->split = p->split_ok;
    p->info.arith = !p->dbl ? NNFFT_ARITH_FP32 : (p->split ? NNFFT_ARITH_FP64_SPLIT : NNFFT_ARITH_FP64);
    if (p->split_ok) {
        if ((rc = upload_df2(p, &p->coef_df[0], coef1, 1.0, "window coefficients (df)")) ||
            (rc = upload_df2(p, &p->coef_df[1], coef2, 1.0, "window coefficients (df)")))
            return bail(rc);
    }

    // dec2[l] = 1 / (N1 N2 phihat2(l)), l in I_{K1}: the 1/N1 of eq. (gell), the division
    // of step 2 and the 1/N2 of step 3, with phihat2(l) = (m2/N2) omegahat2(m2 l / N2).
    {
        std::vector<double> dec((size_t)I.K1);
        for (int64_t i = 0; i < I.K1; ++i) {
            const double l = (double)(i - I.K1 / 2);
            dec[(size_t)i] = 1.0 / ((double)I.N1 * (double)d.m2 *
                                    hm::omega_sinh_hat((double)d.m2 * l / (double)I.N2, d.beta2));
        }
        if ((rc = upload_real(p, &p->dec2, dec, "deconvolution table"))) return bail(rc);
        if (p->split_ok && (rc = upload_df2(p, &p->dec2_df, dec, 1.0, "deconvolution table (df)")))
            return bail(rc);
        if (p->split_ok && (rc = upload_df2(p, &p->rfit_df, p->rfit_host, 0.5, "phihat1 fit (df)")))
            return bail(rc);
    }
    // FFT tables
    {
        FftPlanDev &F = p->fft;
        F.N2 = (int)I.N2;
        F.n1 = (int)I.fft_n1;
        F.n2 = (int)I.fft_n2;
        F.nr1 = hm::radices(F.n1, F.r1, FFT_MAX_STAGES);
        F.nr2 = hm::radices(F.n2, F.r2, FFT_MAX_STAGES);
        if (F.nr1 < 0 || F.nr2 < 0) return bail(fail(NNFFT_EINVAL, "FFT factorisation failed"));
        void *t1 = nullptr, *t2 = nullptr, *tN = nullptr;
        if ((rc = upload_real(p, &t1, twiddles(F.n1), "twiddles")) ||
            (rc = upload_real(p, &t2, twiddles(F.n2), "twiddles")) ||
            (rc = upload_real(p, &tN, twiddles(F.N2), "twiddles")))
            return bail(rc);
        F.tw1 = t1;
        F.tw2 = t2;
        F.twN = tN;
        if (p->split_ok) {
            FftDf &G = p->fftdf;
            G.N2 = F.N2;
            G.n1 = F.n1;
            G.n2 = F.n2;
            G.nr1 = F.nr1;
            G.nr2 = F.nr2;
            for (int i = 0; i < FFT_MAX_STAGES; ++i) {
                G.r1[i] = F.r1[i];
                G.r2[i] = F.r2[i];
            }
            void *u1 = nullptr, *u2 = nullptr, *uN = nullptr;
            if ((rc = upload_df2(p, &u1, twiddles(F.n1), 1.0, "twiddles (df)")) ||
                (rc = upload_df2(p, &u2, twiddles(F.n2), 1.0, "twiddles (df)")) ||
                (rc = upload_df2(p, &uN, twiddles(F.N2), 1.0, "twiddles (df)")))
                return bail(rc);
            G.tw1 = static_cast<const float4 *>(u1);
            G.tw2 = static_cast<const float4 *>(u2);
            G.twN = static_cast<const float4 *>(uN);
        }
    }
    // work buffers
    {
        const size_t N2 = (size_t)I.N2;
        size_t pmax = 0, qmax = 0;
        for (int s = 0; s < 2; ++s) {
            pmax = std::max(pmax, (size_t)p->side[s].max_items * p->side[s].D);
            qmax = std::max(qmax, (size_t)p->side[s].ncell * p->side[s].D);
        }
        if ((rc = dalloc(p, &p->bufA, N2 * cs, "grid")) || (rc = dalloc(p, &p->bufB, N2 * cs, "grid")) ||
            (rc = dalloc(p, &p->bufC, N2 * cs, "grid")) || (rc = dalloc(p, &p->P, pmax * cs, "moments")) ||
            (rc = dalloc(p, &p->Q, qmax * cs, "cell windows")))
            return bail(rc);
    }
    *out = p;
    return NNFFT_OK;
}

int nnfft_plan_info(nnfft_plan_t p, nnfft_info *out) {
    if (!p || !out) return fail(NNFFT_EINVAL, "null argument");
    *out = p->info;
    return NNFFT_OK;
}

int nnfft_set_nodes(nnfft_plan_t p, const double *v_dev, const double *x_dev) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (v_dev == nullptr && p->side[0].M > 0 && !p->side[0].set && x_dev == nullptr)
        return fail(NNFFT_EINVAL, "no nodes given");
    int rc;
    const bool do_v = v_dev || p->side[0].M == 0, do_x = x_dev || p->side[1].M == 0;
    if (do_v && do_x) {
        // fork: the x side runs on the auxiliary stream, concurrently with the v side
        NN_CUDA(cudaEventRecord(p->ev_fork, p->stream), "fork");
        NN_CUDA(cudaStreamWaitEvent(p->aux, p->ev_fork, 0), "fork");
        rc = set_side_nodes(p, 1, x_dev, p->aux);
        int rc0 = set_side_nodes(p, 0, v_dev, p->stream);
        NN_CUDA(cudaEventRecord(p->ev_join, p->aux), "join");
        NN_CUDA(cudaStreamWaitEvent(p->stream, p->ev_join, 0), "join");
        if (rc) return rc;
        if (rc0) return rc0;
        return NNFFT_OK;
    }
    if (do_v && (rc = set_side_nodes(p, 0, v_dev, p->stream))) return rc;
    if (do_x && (rc = set_side_nodes(p, 1, x_dev, p->stream))) return rc;
    return NNFFT_OK;
}

int nnfft_exec(nnfft_plan_t p, const void *f_dev, void *y_dev) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (!p->side[0].set || !p->side[1].set) return fail(NNFFT_ESTATE, "nnfft_set_nodes first");
    if ((p->info.M1 > 0 && !f_dev) || (p->info.M2 > 0 && !y_dev))
        return fail(NNFFT_EINVAL, "null data pointer");
    if (p->dbl && p->split) return run_forward_split(p, f_dev, y_dev);
    return p->dbl ? run_forward<double>(p, f_dev, y_dev) : run_forward<float>(p, f_dev, y_dev);
}

int nnfft_adjoint(nnfft_plan_t p, const void *g_dev, void *z_dev) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (!p->side[0].set || !p->side[1].set) return fail(NNFFT_ESTATE, "nnfft_set_nodes first");
    if ((p->info.M2 > 0 && !g_dev) || (p->info.M1 > 0 && !z_dev))
        return fail(NNFFT_EINVAL, "null data pointer");
    if (p->dbl && p->split) return run_adjoint_split(p, g_dev, z_dev);
    return p->dbl ? run_adjoint<double>(p, g_dev, z_dev) : run_adjoint<float>(p, g_dev, z_dev);
}

int nnfft_set_arith(nnfft_plan_t p, int arith) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (!p->dbl) {
        if (arith != NNFFT_ARITH_FP32) return fail(NNFFT_EINVAL, "complex64 plans compute in fp32");
        return NNFFT_OK;
    }
    if (arith == NNFFT_ARITH_FP64_SPLIT && !p->split_ok)
        return fail(NNFFT_EINVAL, "split precision not available for these window parameters");
    if (arith != NNFFT_ARITH_FP64 && arith != NNFFT_ARITH_FP64_SPLIT)
        return fail(NNFFT_EINVAL, "unknown arithmetic mode for a complex128 plan");
    const bool want = arith == NNFFT_ARITH_FP64_SPLIT;
    if (want != p->split) {
        NN_CUDA(cudaStreamSynchronize(p->stream), "stream synchronize");
        p->split = want;
        p->side[0].set = p->side[1].set = false;     // coordinates are stored per mode
    }
    p->info.arith = want ? NNFFT_ARITH_FP64_SPLIT : NNFFT_ARITH_FP64;
    return NNFFT_OK;
}

int nnfft_timing_enable(nnfft_plan_t p, int enable) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    p->timing = enable != 0;
    return NNFFT_OK;
}

int nnfft_timing_read(nnfft_plan_t p, nnfft_timing *out, int reset) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    NN_CUDA(cudaStreamSynchronize(p->stream), "stream synchronize");
    for (auto &r : p->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            p->acc_ms[r.stage] += ms;
            p->acc_n[r.stage] += 1;
        } else {
            cudaGetLastError();
        }
        p->pool.push_back(r.a);
        p->pool.push_back(r.b);
    }
    p->recs.clear();
    if (out) {
        memset(out, 0, sizeof(*out));
        for (int i = 0; i < 16; ++i) {
            out->ms[i] = p->acc_ms[i];
            out->count[i] = p->acc_n[i];
        }
    }
    if (reset) {
        for (int i = 0; i < 16; ++i) {
            p->acc_ms[i] = 0;
            p->acc_n[i] = 0;
        }
    }
    return NNFFT_OK;
}

int64_t nnfft_launch_count(void) { return launches_so_far(); }

int nnfft_sync(nnfft_plan_t p) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    return collect_status(p);
}

int nnfft_destroy(nnfft_plan_t p) {
    free_plan(p);
    return NNFFT_OK;
}

static int ensure_staging(nnfft_plan_s *p) {
    const size_t cs = 2 * real_size(p->dbl);
    int rc;
    if (!p->st_v && (rc = dalloc_n(p, &p->st_v, (size_t)p->info.M1, "staging"))) return rc;
    if (!p->st_x && (rc = dalloc_n(p, &p->st_x, (size_t)p->info.M2, "staging"))) return rc;
    if (!p->st_f && (rc = dalloc(p, &p->st_f, (size_t)p->info.M1 * cs, "staging"))) return rc;
    if (!p->st_y && (rc = dalloc(p, &p->st_y, (size_t)p->info.M2 * cs, "staging"))) return rc;
    return NNFFT_OK;
}

int nnfft_set_nodes_host(nnfft_plan_t p, const double *v_host, const double *x_host) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    int rc = ensure_staging(p);
    if (rc) return rc;
    if (v_host && p->info.M1 > 0)
        NN_CUDA(cudaMemcpyAsync(p->st_v, v_host, sizeof(double) * p->info.M1,
                                cudaMemcpyHostToDevice, p->stream), "copy v");
    if (x_host && p->info.M2 > 0)
        NN_CUDA(cudaMemcpyAsync(p->st_x, x_host, sizeof(double) * p->info.M2,
                                cudaMemcpyHostToDevice, p->stream), "copy x");
    rc = nnfft_set_nodes(p, v_host ? p->st_v : nullptr, x_host ? p->st_x : nullptr);
    if (rc) return rc;
    return collect_status(p);
}

int nnfft_exec_host(nnfft_plan_t p, const void *f_host, void *y_host) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    int rc = ensure_staging(p);
    if (rc) return rc;
    const size_t cs = 2 * real_size(p->dbl);
    if (p->info.M1 > 0)
        NN_CUDA(cudaMemcpyAsync(p->st_f, f_host, cs * p->info.M1, cudaMemcpyHostToDevice,
                                p->stream), "copy f");
    if ((rc = nnfft_exec(p, p->st_f, p->st_y))) return rc;
    if (p->info.M2 > 0)
        NN_CUDA(cudaMemcpyAsync(y_host, p->st_y, cs * p->info.M2, cudaMemcpyDeviceToHost,
                                p->stream), "copy y");
    return collect_status(p);
}

int nnfft_adjoint_host(nnfft_plan_t p, const void *g_host, void *z_host) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    int rc = ensure_staging(p);
    if (rc) return rc;
    const size_t cs = 2 * real_size(p->dbl);
    if (p->info.M2 > 0)
        NN_CUDA(cudaMemcpyAsync(p->st_y, g_host, cs * p->info.M2, cudaMemcpyHostToDevice,
                                p->stream), "copy g");
    if ((rc = nnfft_adjoint(p, p->st_y, p->st_f))) return rc;
    if (p->info.M1 > 0)
        NN_CUDA(cudaMemcpyAsync(z_host, p->st_f, cs * p->info.M1, cudaMemcpyDeviceToHost,
                                p->stream), "copy z");
    return collect_status(p);
}

}  // extern "C"

// =====================================================================================
// Fast sinc transform (Algorithm 6.1) with a Gauss-Legendre or a Clenshaw-Curtis rule
// =====================================================================================
namespace {

// One quadrature rule (t_j, w_j) with sum_j w_j exp(-2 pi i N t_j x) ~ sinc(N pi x):
//   GL: the n-point Gauss-Legendre rule on [-1/2, 1/2];
//   CC: t_j = cos(j pi / n) / 2, j = 0..n, with the weights of eq. (wk=) (Section 5).
// NNFFT #1 evaluates g_j at the nodes x1 (= -t for GL, +t for CC) and NNFFT #2 sums
// alpha_j = w_j g_j from the nodes v2 (= +t for GL, -t for CC); for CC this is the
// sign convention of Algorithm 6.1, for the symmetric GL rule both conventions agree.
struct SincPlan {
    nnfft_plan_t p1 = nullptr, p2 = nullptr;
    int64_t nq = 0;                           // number of quadrature nodes
    double *x1 = nullptr, *v2 = nullptr, *w = nullptr;
    void *cbuf = nullptr, *gbuf = nullptr, *hbuf = nullptr;
    bool nodes_fixed = false;
    cudaStream_t stream = nullptr;
};

using SincKey = std::tuple<int64_t, int64_t, int64_t, int, int, int, int64_t, uintptr_t>;
std::mutex g_sinc_mu;
std::map<SincKey, SincPlan *> g_sinc;

void sinc_free(SincPlan *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    nnfft_destroy(s->p1);
    nnfft_destroy(s->p2);
    cudaFree(s->x1);
    cudaFree(s->v2);
    cudaFree(s->w);
    cudaFree(s->cbuf);
    cudaFree(s->gbuf);
    cudaFree(s->hbuf);
    delete s;
}

// Number of quadrature intervals / nodes of a rule: GL n nodes (default 2N); CC n
// intervals (default 4N, Algorithm 6.1's n >= 4N) rounded up to a 5-smooth n so that
// the DCT-I runs as one FFT of length 2n; n + 1 nodes.
int sinc_rule_size(int rule, int64_t N, int64_t n_req, int64_t *n_out, int64_t *nodes_out) {
    if (rule == SINC_RULE_GL) {
        const int64_t n = n_req > 0 ? n_req : 2 * N;
        *n_out = n;
        *nodes_out = n;
        return NNFFT_OK;
    }
    if (rule != SINC_RULE_CC) return fail(NNFFT_EINVAL, "unknown quadrature rule");
    int64_t n = n_req > 0 ? n_req : 4 * N;
    if (n < 2) n = 2;
    while (!hm::smooth5(n)) ++n;
    if (2 * n > (int64_t)FFT_MAX_FACTOR * FFT_MAX_FACTOR)
        return fail(NNFFT_EINVAL, "Clenshaw-Curtis rule too long (2n > 2^20)");
    *n_out = n;
    *nodes_out = n + 1;
    return NNFFT_OK;
}

// Clenshaw-Curtis weights and nodes on the device (Algorithm 5.4 with the DCT-I taken
// from a length-2n FFT of the even extension).  w, half_z, neg_half_z: n + 1 doubles.
int cc_rule_device(int64_t n, double *w, double *half_z, double *neg_half_z, cudaStream_t st) {
    const int64_t L = 2 * n;
    FftPlanDev F{};
    int n1 = 0, n2 = 0;
    if (!hm::split_fft(L, FFT_MAX_FACTOR, &n1, &n2))
        return fail(NNFFT_EINVAL, "Clenshaw-Curtis FFT length not factorable");
    F.N2 = (int)L;
    F.n1 = n1;
    F.n2 = n2;
    F.nr1 = hm::radices(n1, F.r1, FFT_MAX_STAGES);
    F.nr2 = hm::radices(n2, F.r2, FFT_MAX_STAGES);
    if (F.nr1 < 0 || F.nr2 < 0) return fail(NNFFT_EINVAL, "FFT factorisation failed");
    void *t1 = nullptr, *t2 = nullptr, *tN = nullptr, *x = nullptr, *y = nullptr, *X = nullptr;
    auto release = [&]() {
        cudaFree(t1); cudaFree(t2); cudaFree(tN); cudaFree(x); cudaFree(y); cudaFree(X);
    };
    cudaError_t e = cudaSuccess;
    const std::vector<double> w1 = twiddles(n1), w2 = twiddles(n2), wN = twiddles(L);
    if (e == cudaSuccess) e = cudaMalloc(&t1, w1.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&t2, w2.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&tN, wN.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&x, (size_t)L * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&y, (size_t)L * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&X, (size_t)L * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpyAsync(t1, w1.data(), w1.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t2, w2.data(), w2.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tN, wN.data(), wN.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    F.tw1 = t1;
    F.tw2 = t2;
    F.twN = tN;
    if (e == cudaSuccess) e = launch_cc_extend(n, x, st);
    if (e == cudaSuccess) e = launch_fft<double>(F, x, y, X, -1, st);
    if (e == cudaSuccess) e = launch_cc_finish(n, X, w, half_z, neg_half_z, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NNFFT_ENOMEM : NNFFT_ECUDA,
                    std::string("Clenshaw-Curtis weights: ") + cudaGetErrorString(e));
    }
    return NNFFT_OK;
}

int sinc_make(int64_t N, int64_t L1, int64_t L2, int m, nnfft_dtype dtype, int rule, int64_t n_req,
              cudaStream_t st, SincPlan **out) {
    int64_t n = 0, nq = 0;
    int rc = sinc_rule_size(rule, N, n_req, &n, &nq);
    if (rc) return rc;
    SincPlan *s = new SincPlan();
    s->stream = st;
    s->nq = nq;
    rc = nnfft_plan(&s->p1, N, L1, nq, 2.0, 2.0, m, m, dtype, st);
    if (!rc) rc = nnfft_plan(&s->p2, N, nq, L2, 2.0, 2.0, m, m, dtype, st);
    if (rc) { sinc_free(s); return rc; }
    const size_t cs = 2 * (dtype == NNFFT_C128 ? sizeof(double) : sizeof(float));
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&s->x1, sizeof(double) * nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->v2, sizeof(double) * nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->w, sizeof(double) * nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->cbuf, cs * (size_t)std::max<int64_t>(L1, 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->gbuf, cs * (size_t)nq);
    if (e == cudaSuccess) e = cudaMalloc(&s->hbuf, cs * (size_t)std::max<int64_t>(L2, 1));
    if (e == cudaSuccess && rule == SINC_RULE_GL) {
        std::vector<double> tau((size_t)nq), w((size_t)nq), neg((size_t)nq);
        hm::gauss_legendre(nq, tau.data(), w.data());
        for (int64_t j = 0; j < nq; ++j) neg[(size_t)j] = -tau[(size_t)j];
        e = cudaMemcpy(s->x1, neg.data(), sizeof(double) * nq, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->v2, tau.data(), sizeof(double) * nq, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->w, w.data(), sizeof(double) * nq, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        sinc_free(s);
        return fail(e == cudaErrorMemoryAllocation ? NNFFT_ENOMEM : NNFFT_ECUDA,
                    std::string("sinc plan: ") + cudaGetErrorString(e));
    }
    if (rule == SINC_RULE_CC && (rc = cc_rule_device(n, s->w, s->x1, s->v2, st))) {
        sinc_free(s);
        return rc;
    }
    *out = s;
    return NNFFT_OK;
}

template <typename Real>
int sinc_run(SincPlan *s, int64_t L1, int64_t L2, const double *a, const void *c, const double *b,
             void *h, int is_complex) {
    cudaStream_t st = s->stream;
    const int nq = (int)s->nq;
    int rc;
    // step 1, NNFFT #1: g_j = sum_k c_k e^{-2 pi i N a_k x1_j}
    if ((rc = nnfft_set_nodes(s->p1, a, s->nodes_fixed ? nullptr : s->x1))) return rc;
    const void *cin = c;
    if (!is_complex) {
        NN_CUDA(launch_real_to_complex<Real>(static_cast<const Real *>(c), (int)L1, s->cbuf, st),
                "sinc pack");
        cin = s->cbuf;
    }
    if ((rc = nnfft_exec(s->p1, cin, s->gbuf))) return rc;
    // step 2: alpha_j = w_j g_j
    NN_CUDA(launch_scale_by_weights<Real>(s->gbuf, s->w, nq, st), "sinc weights");
    // step 3, NNFFT #2: h_l = sum_j alpha_j e^{-2 pi i N v2_j b_l}
    if ((rc = nnfft_set_nodes(s->p2, s->nodes_fixed ? nullptr : s->v2, b))) return rc;
    s->nodes_fixed = true;
    if (is_complex) {
        if ((rc = nnfft_exec(s->p2, s->gbuf, h))) return rc;
    } else {
        if ((rc = nnfft_exec(s->p2, s->gbuf, s->hbuf))) return rc;
        NN_CUDA(launch_complex_to_real<Real>(s->hbuf, (int)L2, static_cast<Real *>(h), st),
                "sinc real part");
    }
    return NNFFT_OK;
}

int sinc_get(int64_t N, int64_t L1, int64_t L2, int m, nnfft_dtype dtype, int rule, int64_t n,
             cudaStream_t st, SincPlan **out) {
    std::lock_guard<std::mutex> lk(g_sinc_mu);
    SincKey key{N, L1, L2, m, (int)dtype, rule, n, reinterpret_cast<uintptr_t>(st)};
    auto it = g_sinc.find(key);
    if (it != g_sinc.end()) {
        *out = it->second;
        return NNFFT_OK;
    }
    SincPlan *s = nullptr;
    const int rc = sinc_make(N, L1, L2, m, dtype, rule, n, st, &s);
    if (rc) return rc;
    g_sinc[key] = s;
    *out = s;
    return NNFFT_OK;
}

}  // namespace

extern "C" {

int sinc_exec_rule(int64_t N, int64_t L1, int64_t L2, int m, nnfft_dtype dtype, int rule,
                   int64_t n, const double *a_dev, const void *c_dev, const double *b_dev,
                   void *h_dev, int is_complex, void *stream) {
    if (N < 1 || L1 < 0 || L2 < 0 || n < 0) return fail(NNFFT_EINVAL, "invalid sinc sizes");
    if ((L1 > 0 && (!a_dev || !c_dev)) || (L2 > 0 && (!b_dev || !h_dev)))
        return fail(NNFFT_EINVAL, "null data pointer");
    if (dtype != NNFFT_C64 && dtype != NNFFT_C128) return fail(NNFFT_EINVAL, "unknown dtype");
    if (rule != SINC_RULE_GL && rule != SINC_RULE_CC) return fail(NNFFT_EINVAL, "unknown quadrature rule");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SincPlan *s = nullptr;
    int rc = sinc_get(N, L1, L2, m, dtype, rule, n, st, &s);
    if (rc) return rc;
    if (L2 == 0) return NNFFT_OK;
    return dtype == NNFFT_C128 ? sinc_run<double>(s, L1, L2, a_dev, c_dev, b_dev, h_dev, is_complex)
                               : sinc_run<float>(s, L1, L2, a_dev, c_dev, b_dev, h_dev, is_complex);
}

int sinc_exec(int64_t N, int64_t L1, int64_t L2, int m, nnfft_dtype dtype, const double *a_dev,
              const void *c_dev, const double *b_dev, void *h_dev, int is_complex, void *stream) {
    return sinc_exec_rule(N, L1, L2, m, dtype, SINC_RULE_GL, 0, a_dev, c_dev, b_dev, h_dev,
                          is_complex, stream);
}

int sinc_quadrature(int rule, int64_t N, int64_t n, double *t_host, double *w_host,
                    int64_t *nodes_out) {
    if (N < 1 || n < 0) return fail(NNFFT_EINVAL, "invalid sizes");
    int64_t nn = 0, nq = 0;
    int rc = sinc_rule_size(rule, N, n, &nn, &nq);
    if (rc) return rc;
    if (nodes_out) *nodes_out = nq;
    if (!t_host || !w_host) return NNFFT_OK;
    if (rule == SINC_RULE_GL) {
        hm::gauss_legendre(nq, t_host, w_host);
        return NNFFT_OK;
    }
    int dev = 0;
    if (cudaGetDeviceCount(&dev) != cudaSuccess || dev == 0) {
        cudaGetLastError();
        return fail(NNFFT_ECUDA, "no CUDA device (the Clenshaw-Curtis weights are computed on the GPU)");
    }
    double *d = nullptr;
    NN_CUDA(cudaMalloc(&d, sizeof(double) * 3 * (size_t)nq), "quadrature buffers");
    rc = cc_rule_device(nn, d, d + nq, d + 2 * nq, nullptr);
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpy(t_host, d + nq, sizeof(double) * nq, cudaMemcpyDeviceToHost);
    if (!rc && e == cudaSuccess) e = cudaMemcpy(w_host, d, sizeof(double) * nq, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (rc) return rc;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NNFFT_ECUDA, std::string("quadrature copy: ") + cudaGetErrorString(e));
    }
    return NNFFT_OK;
}

int sinc_sync(void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<SincPlan *> mine;
    {
        std::lock_guard<std::mutex> lk(g_sinc_mu);
        for (auto &kv : g_sinc)
            if (kv.second->stream == st) mine.push_back(kv.second);
    }
    NN_CUDA(cudaStreamSynchronize(st), "stream synchronize");
    int worst = NNFFT_OK;
    for (SincPlan *s : mine) {
        int rc = nnfft_sync(s->p1);
        if (rc && !worst) worst = rc;
        rc = nnfft_sync(s->p2);
        if (rc && !worst) worst = rc;
    }
    return worst;
}

int sinc_release(void) {
    std::lock_guard<std::mutex> lk(g_sinc_mu);
    for (auto &kv : g_sinc) sinc_free(kv.second);
    g_sinc.clear();
    return NNFFT_OK;
}

}  // extern "C"
