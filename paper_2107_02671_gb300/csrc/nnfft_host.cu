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
#include <new>
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
    // plan-time (all instances of the plan concatenated)
    int m = 0, D = 0;
    int ncell = 0, M = 0, max_items = 0, key_bits = 8;
    int max_items_alloc = 0;               // item buffers: enough for the smallest item cap
    int M_cap = 0;                         // points the buffers hold (M <= M_cap)
    bool has_r = false;
    NodeInst one{};                        // binning of a single-instance plan
    long long *pt_off = nullptr;           // [ninst + 1] device, batches only
    NodeInst *node_tab = nullptr;          // [ninst] device, batches only
    // batches: instance-aligned sort tiles; keys are sorted by the local cell within each
    // instance (sort_bits: the largest instance's cells) instead of over all cells
    SortTiles tiles{};
    int sort_bits = 8;
    // batches with 9- to 16-bit local keys: first block of each instance in the two-stage
    // sort's second stage (one block per bucket of 2^(sort_bits - 8) cells)
    int *local_blk = nullptr;
    int local_blocks = 0;
    void *coef = nullptr;                  // [ninst][2m][D] real tap coefficients
    void *coef_df = nullptr;               // same as (hi, lo) float pairs
    void *rfit = nullptr;                  // x side: [ncell][NR] real 1/phihat1 fits
    void *rfit_df = nullptr;               // x side: (hi, lo) of r_j / 2
    void *grid_real = nullptr;             // [ninst] GridInst<Real>
    void *grid_df = nullptr;               // [ninst] GridInst<float2>
    int *blk_sn = nullptr, *blk_gn = nullptr, *blk_sd = nullptr, *blk_gd = nullptr;
    int nb_sn = 0, nb_gn = 0, nb_sd = 0, nb_gd = 0;   // spread/gather x native/df blocks
    // node-time
    uint32_t *keys = nullptr, *keys_alt = nullptr;
    int *vals = nullptr, *vals_alt = nullptr, *hist = nullptr;
    int *perm = nullptr;
    uint32_t *keys_sorted = nullptr;
    void *ys = nullptr;
    void *y_user = nullptr;        // coordinates in caller order (step-0 scratch)
    void *y_tmp = nullptr;         // coordinates between radix passes
    int *cell_off = nullptr, *item_off = nullptr, *items_scratch = nullptr;
    int *item_cell = nullptr, *item_pb = nullptr, *item_pe = nullptr, *nitems = nullptr;
    // small-item split (sides where some instance has few points per cell)
    bool split_items = false;     // for the current node set
    bool split_rule = false;      // batches: some instance has few points per cell
    int *list_small = nullptr, *list_big = nullptr, *n2 = nullptr;
    bool set = false;
};

// Work buffers of one transform direction.
struct Work {
    void *bufA = nullptr, *bufB = nullptr, *bufC = nullptr;   // grids (all instances)
    void *P = nullptr;   // per-item moments
    void *Q = nullptr;   // per-cell moments (spread) and per-cell window sums (gather)
    unsigned long long *gbar = nullptr;   // the fused grid stage's barrier words (2, zeroed)
};

}  // namespace

struct nnfft_plan_s {
    nnfft_info info{};                       // the instance (or, for batches, totals)
    int64_t ninst = 1;
    int64_t N_built = 0;                     // N the plan was made for (single instance)
    std::vector<nnfft_info> inst_info;       // per instance
    int device = 0;                          // the device current when the plan was made
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;              // second stream: the two node sides sort concurrently
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool dbl = true;
    bool split = false;          // fp64 plan using the split-precision kernels
    bool split_ok = false;       // the window fits allow them (see kern_spread_df.cu)
    Side side[2];   // 0: v (frequency) side, 1: x (spatial) side
    // FFT of every instance (four-step tables), all-real and double-float forms
    FftLaunch<FftPlanDev> fft[2]{};   // two column packings (see build_plan)
    FftLaunch<FftDf> fftdf[2]{};
    // tuning (nnfft_autotune): moments kernel lanes per item per side, FFT packing variant
    int mom_lanes[2] = {32, 32};     // moments: 32, 16 (split precision only) or 8 lanes per item
    int eval_lanes[2] = {32, 32};    // evaluation: 32 or 8 per item, EVAL_FLAT per point,
                                     // EVAL_FLAT_TMA per point with TMA-staged cells,
                                     // EVAL_GATHER 32 per item with the gather convolution
    int fft_variant = 0;         // 0, 1: column packings of the two-pass FFT; 2: cluster FFT;
                                 // 3: the split-precision grid stage as one cooperative launch
    bool fft_cluster_ok = false; // the cluster FFT applies (single instance, split precision,
                                 // shared memory within FFT_CLUSTER_SMEM_MAX)
    bool grid_fused_ok = false;  // the fused grid stage applies (split precision, D1 = D2,
                                 // two blocks per SM resident)
    int fused_blocks = 0;        // its cooperative grid: half the resident blocks
    size_t fused_smem = 0;       // its dynamic shared memory per block
    int item_cap = ITEM_CAP;     // points per work item at most (ITEM_CAP_MIN .. ITEM_CAP)
    int sort_lsd = 0;            // 1: LSD radix passes even where the two-stage sort applies
                                 // (the default for batches, where it measured faster)
    int item_split = 0;          // 1: split small work items where the size rule says so
                                 // (off by default: the warp-per-item kernels measured faster
                                 // on the batched workload; the autotuner may turn it on)
    nnfft_tuning tuning{};
    long long grid_total = 0;    // sum of the instances' N2
    // work buffers of a transform: [0] for exec / adjoint, [1] (allocated on first use) for
    // the adjoint when nnfft_exec_adjoint runs both directions concurrently
    Work work[2];
    size_t work_bytes[3] = {0, 0, 0};   // grid, moments, cell buffer sizes
    int *status = nullptr;
    int *status_host = nullptr;   // pinned
    // host-API staging (allocated on first use)
    double *st_v = nullptr, *st_x = nullptr;
    void *st_f = nullptr, *st_y = nullptr;
    void *st_g = nullptr, *st_z = nullptr;     // nnfft_transform_host: adjoint in / out
    cudaStream_t copy = nullptr;               // nnfft_transform_host: value uploads
    cudaEvent_t ev_v = nullptr, ev_x = nullptr, ev_up = nullptr;
    cudaEvent_t ev_up_v = nullptr, ev_up_x = nullptr, ev_up_f = nullptr;   // host uploads
    std::vector<void *> allocs;
    size_t bytes = 0;            // device bytes the plan holds
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
    p->bytes += bytes;
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

// Complex table exp(-2 pi i k / n), k < n.  k/n is split exactly into a quarter turn q
// and a remainder, so the library sin / cos calls see angles in [0, pi/2) (error about one
// ulp), and exp(-2 pi i k/n) = (-i)^q exp(-i theta).
std::vector<double> twiddles(int64_t n) {
    std::vector<double> t(2 * (size_t)n);
    const double half_pi = 1.57079632679489661923;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t q = (4 * k) / n, rem = 4 * k - q * n;
        const double th = half_pi * ((double)rem / (double)n);
        const double c = std::cos(th), sn = std::sin(th);
        double re = c, im = -sn;                       // exp(-i theta)
        for (int64_t j = 0; j < q; ++j) {              // times -i per quarter turn
            const double r2 = im, i2 = -re;
            re = r2;
            im = i2;
        }
        t[2 * k] = re;
        t[2 * k + 1] = im;
    }
    return t;
}

int fill_info(int64_t N, int64_t M1, int64_t M2, double sigma1, double sigma2, int m1, int m2,
              nnfft_dtype dtype, nnfft_info *info, hm::Derived *d, std::vector<double> *coef1,
              std::vector<double> *coef2, int window = NNFFT_WINDOW_SINH) {
    if (!info) return fail(NNFFT_EINVAL, "null output pointer");
    if (M1 < 0 || M2 < 0) return fail(NNFFT_EINVAL, "M1 and M2 must be >= 0");
    if (M1 > (int64_t(1) << 30) || M2 > (int64_t(1) << 30))
        return fail(NNFFT_EINVAL, "M1 and M2 must be <= 2^30");
    if (dtype != NNFFT_C64 && dtype != NNFFT_C128) return fail(NNFFT_EINVAL, "unknown dtype");
    const char *msg = hm::derive(N, sigma1, sigma2, m1, m2, d, window);
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
    info->window = window;
    const bool fp64 = dtype == NNFFT_C128;
    std::vector<double> tmp1, tmp2;
    info->D1 = hm::choose_degree(m1, d->sigma1, d->beta1, fp64, &info->fit_err1,
                                 coef1 ? *coef1 : tmp1, window);
    info->D2 = hm::choose_degree(m2, d->sigma2, d->beta2, fp64, &info->fit_err2,
                                 coef2 ? *coef2 : tmp2, window);
    // cells: v side u = v * N1 N / N*, x side u = x * N2 N* / N1; |node| <= 1/2
    hm::CellMap c1, c2;
    if (!hm::cell_map(d->N1 * d->N, d->Nstar, &c1) || !hm::cell_map(d->N2 * d->Nstar, d->N1, &c2))
        return fail(NNFFT_EINVAL, "grid too large for the node binning (scale >= 2^19)");
    info->ncell1 = c1.ncell;
    info->ncell2 = c2.ncell;
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
    return b;
}

template <class T>
int upload_vec(nnfft_plan_s *p, T **dst, const std::vector<T> &v, const char *what) {
    int rc = dalloc_n(p, dst, v.size(), what);
    if (rc) return rc;
    if (!v.empty())
        NN_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return NNFFT_OK;
}

// Cell map of side s of an instance: v side u = v N1 N / N*, x side u = x N2 N* / N1.
hm::CellMap side_map(const nnfft_info &I, int s) {
    hm::CellMap c{};
    if (s == 0) hm::cell_map(I.N1 * I.N, I.Nstar, &c);
    else hm::cell_map(I.N2 * I.Nstar, I.N1, &c);
    return c;
}

// Prefix sums of per-instance block counts: blk[i] = first block of instance i.
std::vector<int> prefix(const std::vector<int> &cnt, int *total) {
    std::vector<int> off(cnt.size() + 1, 0);
    for (size_t i = 0; i < cnt.size(); ++i) off[i + 1] = off[i] + cnt[i];
    *total = off.back();
    return off;
}

int alloc_work(nnfft_plan_s *p, Work &W) {
    int rc;
    if ((rc = dalloc(p, &W.bufA, p->work_bytes[0], "grid")) ||
        (rc = dalloc(p, &W.bufB, p->work_bytes[0], "grid")) ||
        (rc = dalloc(p, &W.bufC, p->work_bytes[0], "grid")) ||
        (rc = dalloc(p, &W.P, p->work_bytes[1], "moments")) ||
        (rc = dalloc(p, &W.Q, p->work_bytes[2], "cell windows")) ||
        (rc = dalloc_n(p, &W.gbar, 2, "grid barrier")))
        return rc;
    if (cudaMemset(W.gbar, 0, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "memset");
    return NNFFT_OK;
}

// Per-instance host data gathered while the plan is built.
struct InstHost {
    hm::Derived d;
    std::vector<double> coef[2];
};

// Grid-stage descriptor tables of one side for one real/coefficient type.
template <typename CoefT>
int upload_grid_tables(nnfft_plan_s *p, Side &S, int s, const void *coef_base, const void *dec_base,
                       const std::vector<long long> &dec_off, const void *rfit_base,
                       const std::vector<long long> &cell_base, const std::vector<long long> &grid_base,
                       void **dst) {
    const int64_t n = p->ninst;
    std::vector<GridInst<CoefT>> tab((size_t)n);
    const size_t per = (size_t)2 * S.m * S.D;
    for (int64_t i = 0; i < n; ++i) {
        const nnfft_info &I = p->inst_info[(size_t)i];
        GridInst<CoefT> &G = tab[(size_t)i];
        memset(&G, 0, sizeof(G));
        G.c_lo = side_map(I, s).c_lo;
        G.ncell = (int)(s == 0 ? I.ncell1 : I.ncell2);
        G.cell_base = (int)cell_base[(size_t)i];
        G.N2 = (int)I.N2;
        G.grid_base = grid_base[(size_t)i];
        G.coef = static_cast<const CoefT *>(coef_base) + per * (size_t)i;
        if (s == 0) {
            G.scale = static_cast<const CoefT *>(dec_base) + dec_off[(size_t)i];
            G.scale_off = I.K1 / 2;
            G.scale_len = I.K1;
        }
        if (s == 1 && rfit_base)
            G.rfit = static_cast<const CoefT *>(rfit_base) + (size_t)cell_base[(size_t)i] * NR;
    }
    GridInst<CoefT> *d = nullptr;
    int rc = upload_vec(p, &d, tab, "grid tables");
    *dst = d;
    return rc;
}

// Step 0 (i) for every instance and both sides: window fits at a common degree per side,
// binning tables, 1/phihat1 fits, deconvolution tables, FFT tables, the grid-stage
// descriptors and block maps, and all device buffers.
int build_plan(nnfft_plan_s *p, int64_t count, const int64_t *Ns, const int64_t *M1s,
               const int64_t *M2s, double sigma1, double sigma2, int m1, int m2,
               nnfft_dtype dtype, int window) {
    int rc;
    p->ninst = count;
    p->sort_lsd = count > 1 ? 1 : 0;
    p->dbl = dtype == NNFFT_C128;
    p->inst_info.assign((size_t)count, nnfft_info{});
    std::vector<InstHost> H((size_t)count);
    int D[2] = {0, 0};
    long long Mtot[2] = {0, 0};
    for (int64_t i = 0; i < count; ++i) {
        rc = fill_info(Ns[i], M1s[i], M2s[i], sigma1, sigma2, m1, m2, dtype, &p->inst_info[(size_t)i],
                       &H[(size_t)i].d, &H[(size_t)i].coef[0], &H[(size_t)i].coef[1], window);
        if (rc) return count > 1 ? fail(rc, "instance " + std::to_string(i) + ": " + g_last_error) : rc;
        D[0] = std::max(D[0], (int)p->inst_info[(size_t)i].D1);
        D[1] = std::max(D[1], (int)p->inst_info[(size_t)i].D2);
        Mtot[0] += M1s[i];
        Mtot[1] += M2s[i];
    }
    if (Mtot[0] > (1LL << 30) || Mtot[1] > (1LL << 30))
        return fail(NNFFT_EINVAL, "total M1 and M2 of a plan must be <= 2^30");
    // one degree per side for all instances: refit the instances that chose fewer terms
    for (int64_t i = 0; i < count; ++i) {
        nnfft_info &I = p->inst_info[(size_t)i];
        if (I.D1 != D[0]) { I.fit_err1 = hm::fit_taps(m1, I.beta1, D[0], H[(size_t)i].coef[0], window); I.D1 = D[0]; }
        if (I.D2 != D[1]) { I.fit_err2 = hm::fit_taps(m2, I.beta2, D[1], H[(size_t)i].coef[1], window); I.D2 = D[1]; }
    }
    if (!supported_degree(D[0]) || !supported_degree(D[1]))
        return fail(NNFFT_EINVAL, "unsupported window degree");
    // Split precision (fp64 plans): degrees >= D/2 run in FP32, so their weights
    // kappa_d = max_t |coef[t][d]| must be small enough that an FP32 error there stays
    // near 1e-13 of ||f||_1 in the worst case.
    p->split_ok = p->dbl && df_supported_degree(D[0]) && df_supported_degree(D[1]);
    for (int64_t i = 0; i < count && p->split_ok; ++i)
        p->split_ok = split_weights_ok(H[(size_t)i].coef[0], 2 * m1, D[0]) &&
                      split_weights_ok(H[(size_t)i].coef[1], 2 * m2, D[1]);
    p->split = p->split_ok;

    // grid layout: instance i's grid buffer [grid_base, grid_base + N2)
    std::vector<long long> grid_base((size_t)count);
    long long gtot = 0;
    for (int64_t i = 0; i < count; ++i) {
        grid_base[(size_t)i] = gtot;
        gtot += p->inst_info[(size_t)i].N2;
    }
    p->grid_total = gtot;

    // aggregate info: the instance itself, or totals / maxima for a batch
    p->info = p->inst_info[0];
    p->N_built = p->inst_info[0].N;
    if (count > 1) {
        nnfft_info &A = p->info;
        A.M1 = Mtot[0];
        A.M2 = Mtot[1];
        A.N = A.Nstar = A.N1 = A.K1 = 0;
        A.N2 = gtot;
        A.ncell1 = A.ncell2 = 0;
        A.fit_err1 = A.fit_err2 = 0;
        A.fft_n1 = A.fft_n2 = 0;
        for (const nnfft_info &I : p->inst_info) {
            A.N = std::max(A.N, I.N);
            A.Nstar = std::max(A.Nstar, I.Nstar);
            A.N1 += I.N1;
            A.K1 += I.K1;
            A.ncell1 += I.ncell1;
            A.ncell2 += I.ncell2;
            A.fit_err1 = std::max(A.fit_err1, I.fit_err1);
            A.fit_err2 = std::max(A.fit_err2, I.fit_err2);
            A.fft_n1 = std::max(A.fft_n1, I.fft_n1);
            A.fft_n2 = std::max(A.fft_n2, I.fft_n2);
        }
    }
    const int arith = !p->dbl ? NNFFT_ARITH_FP32 : (p->split ? NNFFT_ARITH_FP64_SPLIT : NNFFT_ARITH_FP64);
    p->info.arith = arith;
    for (nnfft_info &I : p->inst_info) I.arith = arith;

    // deconvolution tables dec2[l] = 1 / (N1 N2 phihat2(l)), l in I_{K1}: the 1/N1 of
    // eq. (2.12), the division of step 2 and the 1/N2 of step 3, with
    // phihat2(l) = (m2/N2) omegahat2(m2 l / N2); concatenated over instances.
    std::vector<double> dec;
    std::vector<long long> dec_off((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const nnfft_info &I = p->inst_info[(size_t)i];
        dec_off[(size_t)i] = (long long)dec.size();
        for (int64_t k = 0; k < I.K1; ++k) {
            const double l = (double)(k - I.K1 / 2);
            dec.push_back(1.0 / ((double)I.N1 * (double)m2 *
                                 hm::omega_hat_w(window, (double)m2 * l / (double)I.N2, I.beta2, m2)));
        }
    }
    void *dec_real = nullptr, *dec_df = nullptr;
    if ((rc = upload_real(p, &dec_real, dec, "deconvolution table"))) return rc;
    if (p->split_ok && (rc = upload_df2(p, &dec_df, dec, 1.0, "deconvolution table (df)"))) return rc;

    const size_t rs = real_size(p->dbl);
    for (int s = 0; s < 2; ++s) {
        Side &S = p->side[s];
        S.m = s == 0 ? m1 : m2;
        S.D = D[s];
        S.has_r = s == 1;
        std::vector<NodeInst> tab((size_t)count);
        std::vector<long long> pt_off((size_t)count + 1, 0), cell_base((size_t)count);
        std::vector<double> coef_all, rfit_all;
        long long cells = 0;
        for (int64_t i = 0; i < count; ++i) {
            const nnfft_info &I = p->inst_info[(size_t)i];
            const hm::Derived &d = H[(size_t)i].d;
            NodeInst &T = tab[(size_t)i];
            const hm::CellMap cm = side_map(I, s);
            T.S = cm.S;
            T.c_lo = cm.c_lo;
            T.ncell = (int)cm.ncell;
            T.cell_base = (int)cells;
            cell_base[(size_t)i] = cells;
            cells += T.ncell;
            pt_off[(size_t)i + 1] = pt_off[(size_t)i] + (s == 0 ? I.M1 : I.M2);
            const std::vector<double> &c = H[(size_t)i].coef[s];
            coef_all.insert(coef_all.end(), c.begin(), c.end());
            if (S.has_r) {
                // Per x cell c: Chebyshev fit in y of 1/phihat1(N* x), x = (c + (y+1)/2)/uscale,
                // phihat1(v) = (m1/N1) omegahat1(m1 v / N1) (scaling in the proof of Theorem 3.4).
                const size_t r0 = rfit_all.size();
                rfit_all.resize(r0 + (size_t)T.ncell * NR);
                for (int ic = 0; ic < T.ncell; ++ic) {
                    const double cc = (double)(T.c_lo + ic);
                    auto f = [&](double y) {
                        const double x = (cc + 0.5 * (y + 1.0)) / cm.scale;
                        const double w = (double)d.m1 * (double)d.Nstar * x / (double)d.N1;
                        return (double)d.N1 / ((double)d.m1 * hm::omega_hat_w(window, w, d.beta1, d.m1));
                    };
                    hm::cheb_interp(f, NR, rfit_all.data() + r0 + (size_t)ic * NR);
                }
            }
        }
        if (cells > (1LL << 30)) return fail(NNFFT_EINVAL, "too many grid cells in one plan");
        S.ncell = (int)cells;
        S.M = (int)pt_off.back();
        S.M_cap = S.M;
        S.max_items = S.ncell + (S.M + ITEM_CAP - 1) / ITEM_CAP + (int)count;
        S.max_items_alloc = S.ncell + (S.M + ITEM_CAP_MIN - 1) / ITEM_CAP_MIN + (int)count;
        S.key_bits = key_bits_for(S.ncell);
        S.one = tab[0];
        S.sort_bits = S.key_bits;
        if (count > 1) {
            if ((rc = upload_vec(p, &S.node_tab, tab, "binning tables")) ||
                (rc = upload_vec(p, &S.pt_off, pt_off, "instance offsets")))
                return rc;
            std::vector<int> tinst, tile0((size_t)count + 1, 0);
            std::vector<long long> tstart;
            int max_cells = 1;
            for (int64_t i = 0; i < count; ++i) {
                tile0[(size_t)i] = (int)tinst.size();
                for (long long q = pt_off[(size_t)i]; q < pt_off[(size_t)i + 1]; q += SORT_TILE) {
                    tinst.push_back((int)i);
                    tstart.push_back(q);
                }
                max_cells = std::max(max_cells, tab[(size_t)i].ncell);
            }
            tile0[(size_t)count] = (int)tinst.size();
            int *d_inst = nullptr, *d_tile0 = nullptr;
            long long *d_start = nullptr;
            if (!tinst.empty() && ((rc = upload_vec(p, &d_inst, tinst, "sort tiles")) ||
                                   (rc = upload_vec(p, &d_start, tstart, "sort tiles"))))
                return rc;
            if ((rc = upload_vec(p, &d_tile0, tile0, "sort tiles"))) return rc;
            S.tiles.inst = d_inst;
            S.tiles.start = d_start;
            S.tiles.inst_tile0 = d_tile0;
            S.tiles.pt_off = S.pt_off;
            S.tiles.tab = S.node_tab;
            S.tiles.ntiles = (int)tinst.size();
            S.tiles.ninst = (int)count;
            S.sort_bits = key_bits_for(max_cells);
            if (local_sort_ok(S.sort_bits)) {     // two-stage sort: blocks per (instance, bucket)
                const int lb = local_sort_low_bits(S.sort_bits);
                std::vector<int> bf((size_t)count + 1, 0);
                for (int64_t i = 0; i < count; ++i)
                    bf[(size_t)i + 1] = bf[(size_t)i] + ((tab[(size_t)i].ncell - 1) >> lb) + 1;
                S.local_blocks = bf.back();
                if ((rc = upload_vec(p, &S.local_blk, bf, "sort buckets"))) return rc;
            }
        }
        if ((rc = upload_real(p, &S.coef, coef_all, "window coefficients"))) return rc;
        if (p->split_ok && (rc = upload_df2(p, &S.coef_df, coef_all, 1.0, "window coefficients (df)")))
            return rc;
        if (S.has_r) {
            if ((rc = upload_real(p, &S.rfit, rfit_all, "phihat1 fit"))) return rc;
            if (p->split_ok && (rc = upload_df2(p, &S.rfit_df, rfit_all, 0.5, "phihat1 fit (df)")))
                return rc;
        }
        // grid-stage descriptors and block maps
        rc = p->dbl ? upload_grid_tables<double>(p, S, s, S.coef, dec_real, dec_off, S.rfit,
                                                 cell_base, grid_base, &S.grid_real)
                    : upload_grid_tables<float>(p, S, s, S.coef, dec_real, dec_off, S.rfit,
                                                cell_base, grid_base, &S.grid_real);
        if (rc) return rc;
        if (p->split_ok &&
            (rc = upload_grid_tables<float2>(p, S, s, S.coef_df, dec_df, dec_off, S.rfit_df,
                                             cell_base, grid_base, &S.grid_df)))
            return rc;
        std::vector<int> sn((size_t)count), gn((size_t)count), sd((size_t)count), gd((size_t)count);
        for (int64_t i = 0; i < count; ++i) {
            const int N2 = (int)p->inst_info[(size_t)i].N2, nc = tab[(size_t)i].ncell;
            sn[(size_t)i] = spread_blocks_native(N2, S.D);
            gn[(size_t)i] = gather_blocks_native(nc, S.D);
            sd[(size_t)i] = p->split_ok ? spread_blocks_df(N2, S.D) : 0;
            gd[(size_t)i] = p->split_ok ? gather_blocks_df(nc, S.D) : 0;
        }
        if ((rc = upload_vec(p, &S.blk_sn, prefix(sn, &S.nb_sn), "block map")) ||
            (rc = upload_vec(p, &S.blk_gn, prefix(gn, &S.nb_gn), "block map")) ||
            (rc = upload_vec(p, &S.blk_sd, prefix(sd, &S.nb_sd), "block map")) ||
            (rc = upload_vec(p, &S.blk_gd, prefix(gd, &S.nb_gd), "block map")))
            return rc;
        // node-time buffers
        const size_t M = (size_t)S.M;
        if ((rc = dalloc_n(p, &S.keys, M, "keys")) || (rc = dalloc_n(p, &S.keys_alt, M, "keys")) ||
            (rc = dalloc_n(p, &S.vals, M, "perm")) || (rc = dalloc_n(p, &S.vals_alt, M, "perm")) ||
            (rc = dalloc_n(p, &S.hist,
                           count > 1 ? radix_sort_hist_len(S.tiles.ntiles, (int)count)
                                     : radix_sort_hist_len((S.M + SORT_TILE - 1) / SORT_TILE, 1),
                           "sort histogram")) ||
            (rc = dalloc(p, &S.ys, M * rs, "sorted coordinates")) ||
            (rc = dalloc(p, &S.y_user, M * rs, "coordinates")) ||
            (!p->dbl && (rc = dalloc(p, &S.y_tmp, M * rs, "coordinates (sort scratch)"))) ||
            (rc = dalloc_n(p, &S.cell_off, (size_t)S.ncell + 1, "cell offsets")) ||
            (rc = dalloc_n(p, &S.item_off, (size_t)S.ncell + 1, "item offsets")) ||
            (rc = dalloc_n(p, &S.items_scratch, build_items_scratch_len(S.ncell), "item scratch")) ||
            (rc = dalloc_n(p, &S.item_cell, (size_t)S.max_items_alloc, "items")) ||
            (rc = dalloc_n(p, &S.item_pb, (size_t)S.max_items_alloc, "items")) ||
            (rc = dalloc_n(p, &S.item_pe, (size_t)S.max_items_alloc, "items")) ||
            (rc = dalloc_n(p, &S.nitems, 1, "item count")))
            return rc;
        NN_CUDA(cudaMemset(S.item_off, 0, sizeof(int) * ((size_t)S.ncell + 1)), "memset");
        NN_CUDA(cudaMemset(S.nitems, 0, sizeof(int)), "memset");
        // Small-item split when some instance expects few points per cell (a warp per item
        // would idle most of its lanes and pay a full reduction per item); single plans
        // decide again at every node set from their current size (nnfft_set_sizes).
        for (int64_t i = 0; i < count && !S.split_rule; ++i) {
            const int64_t Mi = pt_off[(size_t)i + 1] - pt_off[(size_t)i];
            S.split_rule = Mi > 0 && Mi < 4LL * SMALL_ITEM * tab[(size_t)i].ncell;
        }
        if ((rc = dalloc_n(p, &S.list_small, (size_t)S.max_items_alloc, "item lists")) ||
            (rc = dalloc_n(p, &S.list_big, (size_t)S.max_items_alloc, "item lists")) ||
            (rc = dalloc_n(p, &S.n2, 2, "item lists")))
            return rc;
        NN_CUDA(cudaMemset(S.n2, 0, 2 * sizeof(int)), "memset");
    }

    // FFT tables: twiddles exp(-2 pi i k/n) for every distinct length, concatenated
    {
        std::map<int64_t, size_t> at;          // length -> first complex entry
        std::vector<double> tw;
        auto twid_of = [&](int64_t n) {
            auto it = at.find(n);
            if (it != at.end()) return it->second;
            const size_t off = tw.size() / 2;
            const std::vector<double> t = twiddles(n);
            tw.insert(tw.end(), t.begin(), t.end());
            at[n] = off;
            return off;
        };
        std::vector<FftPlanDev> F((size_t)count);
        std::vector<size_t> o1((size_t)count), o2((size_t)count), oN((size_t)count);
        for (int64_t i = 0; i < count; ++i) {
            const nnfft_info &I = p->inst_info[(size_t)i];
            FftPlanDev &f = F[(size_t)i];
            memset(&f, 0, sizeof(f));
            f.N2 = (int)I.N2;
            f.n1 = (int)I.fft_n1;
            f.n2 = (int)I.fft_n2;
            f.nr1 = hm::radices(f.n1, f.r1, FFT_MAX_STAGES);
            f.nr2 = hm::radices(f.n2, f.r2, FFT_MAX_STAGES);
            if (f.nr1 < 0 || f.nr2 < 0) return fail(NNFFT_EINVAL, "FFT factorisation failed");
            f.grid_base = grid_base[(size_t)i];
            o1[(size_t)i] = twid_of(f.n1);
            o2[(size_t)i] = twid_of(f.n2);
            oN[(size_t)i] = twid_of(f.N2);
        }
        void *tw_real = nullptr, *tw_df = nullptr;
        if ((rc = upload_real(p, &tw_real, tw, "twiddles"))) return rc;
        if (p->split_ok && (rc = upload_df2(p, &tw_df, tw, 1.0, "twiddles (df)"))) return rc;
        const size_t cs = 2 * rs;
        for (int64_t i = 0; i < count; ++i) {
            FftPlanDev &f = F[(size_t)i];
            f.tw1 = static_cast<const char *>(tw_real) + cs * o1[(size_t)i];
            f.tw2 = static_cast<const char *>(tw_real) + cs * o2[(size_t)i];
            f.twN = static_cast<const char *>(tw_real) + cs * oN[(size_t)i];
        }
        // Two packings of short columns into blocks: variant 0 by rule (packed when the
        // plan's grids fill the GPU anyway, about 4 blocks of FFT_TILE elements per SM),
        // variant 1 the other extreme (one column per block, or as many as fit FFT_TILE);
        // the autotuner may switch.
        auto rule = [&](int n) {
            const long long c = gtot / (4LL * 152 * n);
            return (int)std::max(1LL, std::min(c, (long long)std::max(1, FFT_TILE / n)));
        };
        bool rule_packs = false;
        for (const FftPlanDev &f : F) rule_packs = rule_packs || rule(f.n1) > 1 || rule(f.n2) > 1;
        for (int variant = 0; variant < 2; ++variant) {
            std::vector<int> c1((size_t)count), c2((size_t)count);
            std::vector<FftDf> G((size_t)count);
            int sm1 = 0, sm2 = 0;
            for (int64_t i = 0; i < count; ++i) {
                FftPlanDev &f = F[(size_t)i];
                auto cols = [&](int n) {
                    if (variant == 0) return rule(n);
                    return rule_packs ? 1 : std::max(1, FFT_TILE / n);
                };
                f.cols1 = cols(f.n1);
                f.cols2 = cols(f.n2);
                c1[(size_t)i] = (f.n2 + f.cols1 - 1) / f.cols1;    // pass 1: columns of length n1
                c2[(size_t)i] = (f.n1 + f.cols2 - 1) / f.cols2;    // pass 2: rows of length n2
                sm1 = std::max(sm1, (2 * f.cols1 + 1) * f.n1);
                sm2 = std::max(sm2, (2 * f.cols2 + 1) * f.n2);
                FftDf &g = G[(size_t)i];
                memset(&g, 0, sizeof(g));
                g.N2 = f.N2;
                g.n1 = f.n1;
                g.n2 = f.n2;
                g.nr1 = f.nr1;
                g.nr2 = f.nr2;
                for (int k = 0; k < FFT_MAX_STAGES; ++k) {
                    g.r1[k] = f.r1[k];
                    g.r2[k] = f.r2[k];
                }
                g.grid_base = f.grid_base;
                g.cols1 = f.cols1;
                g.cols2 = f.cols2;
                if (tw_df) {
                    g.tw1 = static_cast<const float4 *>(tw_df) + o1[(size_t)i];
                    g.tw2 = static_cast<const float4 *>(tw_df) + o2[(size_t)i];
                    g.twN = static_cast<const float4 *>(tw_df) + oN[(size_t)i];
                }
            }
            int n1tot = 0, n2tot = 0;
            int *b1 = nullptr, *b2 = nullptr;
            FftPlanDev *fd = nullptr;
            if ((rc = upload_vec(p, &b1, prefix(c1, &n1tot), "FFT block map")) ||
                (rc = upload_vec(p, &b2, prefix(c2, &n2tot), "FFT block map")) ||
                (rc = upload_vec(p, &fd, F, "FFT tables")))
                return rc;
            p->fft[variant] = FftLaunch<FftPlanDev>{fd, b1, b2, (int)count, n1tot, n2tot, sm1, sm2};
            if (p->split_ok) {
                FftDf *gd = nullptr;
                if ((rc = upload_vec(p, &gd, G, "FFT tables (df)"))) return rc;
                p->fftdf[variant] = FftLaunch<FftDf>{gd, b1, b2, (int)count, n1tot, n2tot, sm1, sm2};
            }
        }
    }
    // work buffers
    {
        const size_t cs = 2 * rs;
        size_t pmax = 0, qmax = 0;
        for (int s = 0; s < 2; ++s) {
            pmax = std::max(pmax, (size_t)p->side[s].max_items_alloc * p->side[s].D);
            qmax = std::max(qmax, (size_t)p->side[s].ncell * p->side[s].D);
        }
        p->work_bytes[0] = (size_t)gtot * cs;
        p->work_bytes[1] = pmax * cs;
        p->work_bytes[2] = qmax * cs;
        if ((rc = alloc_work(p, p->work[0]))) return rc;
    }
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

}  // namespace

namespace nnfft {
int device_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}
}  // namespace nnfft

namespace {

template <typename Real> SideK<Real> side_args(const Side &S, bool with_r, int *status) {
    SideK<Real> k;
    k.m = S.m;
    k.D = S.D;
    k.ncell = S.ncell;
    k.c_lo = 0;
    k.coef = nullptr;
    k.rfit = with_r ? static_cast<const Real *>(S.rfit) : nullptr;
    k.perm = S.perm;
    k.ys = static_cast<const Real *>(S.ys);
    k.item_off = S.item_off;
    k.item_cell = S.item_cell;
    k.item_pb = S.item_pb;
    k.item_pe = S.item_pe;
    k.nitems = S.nitems;
    k.max_items = S.max_items;
    k.list_small = S.split_items ? S.list_small : nullptr;
    k.list_big = S.split_items ? S.list_big : nullptr;
    k.n_small = S.split_items ? S.n2 : nullptr;
    k.n_big = S.split_items ? S.n2 + 1 : nullptr;
    k.keys = S.keys_sorted;
    k.M = (int)S.M;
    k.status = status;
    return k;
}

// Grid-stage launch over all instances of one side.
template <typename CoefT>
GridLaunch<CoefT> grid_launch(const nnfft_plan_s *p, int s, bool spread, bool fold) {
    const Side &S = p->side[s];
    constexpr bool df = std::is_same<CoefT, float2>::value;
    GridLaunch<CoefT> L;
    L.inst = static_cast<const GridInst<CoefT> *>(df ? S.grid_df : S.grid_real);
    L.blk = spread ? (df ? S.blk_sd : S.blk_sn) : (df ? S.blk_gd : S.blk_gn);
    L.nblocks = spread ? (df ? S.nb_sd : S.nb_sn) : (df ? S.nb_gd : S.nb_gn);
    L.ninst = (int)p->ninst;
    L.m = S.m;
    L.D = S.D;
    L.fold = fold;
    return L;
}

int set_side_nodes(nnfft_plan_s *p, int s, const double *nodes, cudaStream_t st) {
    Side &S = p->side[s];
    StageTimer timer(p, s, st);
    if (p->ninst == 1) S.split_items = S.M > 0 && (int64_t)S.M < 4LL * SMALL_ITEM * S.ncell;
    else S.split_items = S.split_rule;
    S.split_items = S.split_items && p->item_split;
    S.max_items = S.ncell + (S.M + p->item_cap - 1) / p->item_cap + (int)p->ninst;
    if (S.M == 0) {
        NN_CUDA(cudaMemsetAsync(S.item_off, 0, sizeof(int) * ((size_t)S.ncell + 1), st), "memset");
        NN_CUDA(cudaMemsetAsync(S.nitems, 0, sizeof(int), st), "memset");
        NN_CUDA(cudaMemsetAsync(S.n2, 0, 2 * sizeof(int), st), "memset");
        S.perm = S.vals;
        S.set = true;
        return NNFFT_OK;
    }
    const int yfmt = !p->dbl ? 0 : (p->split ? 2 : 1);
    const int ybytes = p->dbl ? 8 : 4;
    const SortTiles *tiles = p->ninst > 1 ? &S.tiles : nullptr;
    // one instance with 9- to 16-bit cell keys: the two-stage sort (high-digit scatter, then
    // a shared-memory sort of each bucket that also writes the cell offsets and items)
    const bool two_stage = !p->sort_lsd && S.M >= 2 && local_sort_ok(S.sort_bits) &&
                           (p->ninst == 1 || S.local_blk != nullptr);
    NN_CUDA(launch_node_keys_y(nodes, S.M, S.one, tiles, S.tiles.ntiles, S.keys, S.y_user, yfmt,
                               S.sort_bits, ybytes, S.hist, p->status, st, two_stage),
            "node keys");
    uint32_t *ks = nullptr;
    int *vs = nullptr;
    if (two_stage) {
        const bool per_cell = p->ninst == 1 && (int64_t)S.M >= 2LL * S.ncell;
        NN_CUDA(radix_sort_cells_local(S.keys, S.vals, S.keys_alt, S.vals_alt, S.hist, tiles,
                                       S.tiles.ntiles, S.local_blk, S.local_blocks, S.M, S.ncell,
                                       S.sort_bits, S.y_user, S.ys, S.y_tmp, ybytes, p->item_cap,
                                       per_cell, S.cell_off, S.item_off, S.item_cell, S.item_pb,
                                       S.item_pe, S.nitems, S.items_scratch, st, &ks, &vs),
                "two-stage sort");
        S.perm = vs;
        S.keys_sorted = ks;
        if (S.split_items) {
            NN_CUDA(cudaMemsetAsync(S.n2, 0, 2 * sizeof(int), st), "memset");
            NN_CUDA(launch_split_items(S.nitems, S.item_pb, S.item_pe, S.max_items, S.list_small,
                                       S.list_big, S.n2, st),
                    "item split");
        }
        S.set = true;
        return NNFFT_OK;
    }
    NN_CUDA(radix_sort_cells(S.keys, S.vals, S.keys_alt, S.vals_alt, S.hist, tiles, S.tiles.ntiles,
                             S.M, S.sort_bits, S.y_user, S.ys, S.y_tmp, ybytes, st, &ks, &vs),
            "radix sort");
    S.perm = vs;
    S.keys_sorted = ks;
    // one item per cell first where cells are dense (a single instance with at least two
    // points per cell on average): empty items would cost a reduction and a zero row each
    const bool per_cell = p->ninst == 1 && (int64_t)S.M >= 2LL * S.ncell;
    NN_CUDA(launch_cells_and_items(ks, S.M, S.ncell, p->item_cap, per_cell, S.cell_off, S.item_off,
                                   S.item_cell, S.item_pb, S.item_pe, S.nitems, S.items_scratch, st),
            "cell offsets and work items");
    if (S.split_items) {
        NN_CUDA(cudaMemsetAsync(S.n2, 0, 2 * sizeof(int), st), "memset");
        NN_CUDA(launch_split_items(S.nitems, S.item_pb, S.item_pe, S.max_items, S.list_small,
                                   S.list_big, S.n2, st),
                "item split");
    }
    S.set = true;
    return NNFFT_OK;
}

// Step 3 of a split-precision plan, grid bufA -> bufC: the two-pass four-step FFT (column
// packing fft_variant 0 or 1), or (FFT_CLUSTER_VARIANT) one launch of the cluster FFT.
cudaError_t fft_df(const nnfft_plan_s *p, const Work &W, int sign, cudaStream_t st) {
    if (p->fft_variant == FFT_CLUSTER_VARIANT)
        return launch_fft_cluster_df(p->fftdf[0], (int)p->info.fft_n1, (int)p->info.fft_n2, W.bufA,
                                     W.bufC, sign, st);
    return launch_fft_df(p->fftdf[p->fft_variant == 1 ? 1 : 0], W.bufA, W.bufB, W.bufC, sign, st);
}

// Step 3 of an all-real (fp32 or all-FP64) plan: the two-pass FFT or the cluster FFT.
template <typename Real>
cudaError_t fft_native(const nnfft_plan_s *p, const Work &W, int sign, cudaStream_t st) {
    if (p->fft_variant == FFT_CLUSTER_VARIANT)
        return launch_fft_cluster<Real>(p->fft[0], (int)p->info.fft_n1, (int)p->info.fft_n2,
                                        W.bufA, W.bufC, sign, st);
    return launch_fft<Real>(p->fft[p->fft_variant == 1 ? 1 : 0], W.bufA, W.bufB, W.bufC, sign, st);
}

// The fused grid stage runs when the tuning selects it, the plan supports it and the work
// buffers carry barrier words.
bool use_grid_fused(const nnfft_plan_s *p, const Work &W) {
    return p->fft_variant == GRID_FUSED_VARIANT && p->grid_fused_ok && W.gbar != nullptr;
}

// Arguments of the fused grid stage: spreading side s (0: v, forward; 1: x, adjoint) with its
// kernel descriptor S and fit tables T, the other side gathering; FFT sign.
GridStageDf grid_stage_args(const nnfft_plan_s *p, const Work &W, const SideK<double> &S,
                            const SideDf &T, int s, int sign) {
    GridStageDf A;
    A.fold_side = S;
    A.fold_tab = T;
    A.P4 = static_cast<const float4 *>(W.P);
    A.Q4 = static_cast<float4 *>(W.Q);
    A.spread = grid_launch<float2>(p, s, true, false);
    A.gather = grid_launch<float2>(p, 1 - s, false, s == 0);
    A.fft = p->fftdf[0];
    A.bufA = static_cast<float4 *>(W.bufA);
    A.bufB = static_cast<float4 *>(W.bufB);
    A.bufC = static_cast<float4 *>(W.bufC);
    A.sign = sign;
    A.bar = W.gbar;
    A.status = p->status;
    A.limit = GRID_WAIT_LIMIT_CYCLES;
    return A;
}

int run_forward_split(nnfft_plan_s *p, const void *f, void *y, cudaStream_t st, const Work &W,
                      cudaEvent_t mid = nullptr, int part = 3) {
    const Side &V = p->side[0], &X = p->side[1];
    // part 1: steps 1-2 (spread into the grid buffer); part 2: steps 3-4 from it
    if (X.M == 0 && part == 3) return NNFFT_OK;
    const SideK<double> sv = side_args<double>(V, false, p->status);
    const SideK<double> sx = side_args<double>(X, true, p->status);
    const SideDf tv{nullptr, nullptr};
    if (part == 3 && use_grid_fused(p, W) && X.M > 0) {
        {
            StageTimer t(p, 2, st);
            NN_CUDA(launch_moments_df(sv, f, W.P, p->mom_lanes[0], st), "spread moments");
        }
        {   // cell fold, spread convolution, FFT and gather convolution in one launch
            StageTimer t(p, 4, st);
            NN_CUDA(launch_grid_stage_df(grid_stage_args(p, W, sv, tv, 0, -1), sv.D, p->fused_blocks,
                                         p->fused_smem, st),
                    "fused grid stage");
        }
        if (mid) NN_CUDA(cudaStreamWaitEvent(st, mid, 0), "wait for the other side");
        {
            StageTimer t(p, 6, st);
            NN_CUDA(launch_eval_df(sx, W.Q, y, p->eval_lanes[1], st), "gather evaluation");
        }
        return NNFFT_OK;
    }
    if (part & 1) {
        {
            StageTimer t(p, 2, st);
            NN_CUDA(launch_moments_df(sv, f, W.P, p->mom_lanes[0], st), "spread moments");
        }
        // the degree-major spread convolution folds the cells' items itself
        const GridLaunch<float2> Ls = grid_launch<float2>(p, 0, true, false);
        const bool fold_in = spread_df_folds(Ls);
        if (!fold_in) {
            StageTimer t(p, 12, st);
            NN_CUDA(launch_cell_fold_df(sv, tv, W.P, W.Q, st), "cell fold");
        }
        {
            StageTimer t(p, 3, st);
            SpreadFoldDf F;
            if (fold_in) {
                F.item_off = sv.item_off;
                F.P4 = static_cast<const float4 *>(W.P);
            }
            NN_CUDA(launch_spread_conv_df(Ls, W.Q, W.bufA, st, F), "spread convolution");
        }
    }
    if ((part & 2) && !(X.M == 0)) {
        {
            StageTimer t(p, 4, st);
            NN_CUDA(fft_df(p, W, -1, st), "fft");
        }
        // EVAL_GATHER: the evaluation computes each item's window sums from the grid itself
        const GridLaunch<float2> Lg = grid_launch<float2>(p, 1, false, true);
        const bool gather_in = p->eval_lanes[1] == EVAL_GATHER && sx.list_small == nullptr &&
                               eval_gather_df_ok(Lg);
        if (!gather_in) {
            StageTimer t(p, 5, st);
            NN_CUDA(launch_gather_conv_df(Lg, W.bufC, W.Q, st), "gather convolution");
        }
        // the gather side's sorted nodes (sorted on another stream) are needed from here on;
        // the gather convolution reads only the plan's grid geometry
        if (mid) NN_CUDA(cudaStreamWaitEvent(st, mid, 0), "wait for the other side");
        {
            StageTimer t(p, 6, st);
            NN_CUDA(gather_in ? launch_eval_gather_df(sx, Lg, W.bufC, y, st)
                              : launch_eval_df(sx, W.Q, y, p->eval_lanes[1], st),
                    "gather evaluation");
        }
    }
    return NNFFT_OK;
}

int run_adjoint_split(nnfft_plan_s *p, const void *g, void *z, cudaStream_t st, const Work &W,
                      cudaEvent_t mid = nullptr, int part = 3) {
    const Side &V = p->side[0], &X = p->side[1];
    // part 1: steps 1-2 (spread into the grid buffer); part 2: steps 3-4 from it
    if (V.M == 0 && part == 3) return NNFFT_OK;
    const SideK<double> sv = side_args<double>(V, false, p->status);
    const SideK<double> sx = side_args<double>(X, true, p->status);
    const SideDf tx{nullptr, static_cast<const float2 *>(X.rfit_df)};
    if (part == 3 && use_grid_fused(p, W) && V.M > 0) {
        {
            StageTimer t(p, 7, st);
            NN_CUDA(launch_moments_df(sx, g, W.P, p->mom_lanes[1], st), "adjoint spread moments");
        }
        {
            StageTimer t(p, 9, st);
            NN_CUDA(launch_grid_stage_df(grid_stage_args(p, W, sx, tx, 1, +1), sx.D, p->fused_blocks,
                                         p->fused_smem, st),
                    "adjoint fused grid stage");
        }
        if (mid) NN_CUDA(cudaStreamWaitEvent(st, mid, 0), "wait for the other side");
        {
            StageTimer t(p, 11, st);
            NN_CUDA(launch_eval_df(sv, W.Q, z, p->eval_lanes[0], st), "adjoint gather evaluation");
        }
        return NNFFT_OK;
    }
    if (part & 1) {
        {
            StageTimer t(p, 7, st);
            NN_CUDA(launch_moments_df(sx, g, W.P, p->mom_lanes[1], st), "adjoint spread moments");
        }
        const GridLaunch<float2> Ls = grid_launch<float2>(p, 1, true, false);
        const bool fold_in = spread_df_folds(Ls);
        if (!fold_in) {
            StageTimer t(p, 13, st);
            NN_CUDA(launch_cell_fold_df(sx, tx, W.P, W.Q, st), "adjoint cell fold");
        }
        {
            StageTimer t(p, 8, st);
            SpreadFoldDf F;
            if (fold_in) {
                F.item_off = sx.item_off;
                F.P4 = static_cast<const float4 *>(W.P);
                F.rfit = tx.rfit;
            }
            NN_CUDA(launch_spread_conv_df(Ls, W.Q, W.bufA, st, F), "adjoint spread convolution");
        }
    }
    if ((part & 2) && !(V.M == 0)) {
        {
            StageTimer t(p, 9, st);
            NN_CUDA(fft_df(p, W, +1, st), "adjoint fft");
        }
        const GridLaunch<float2> Lg = grid_launch<float2>(p, 0, false, false);
        const bool gather_in = p->eval_lanes[0] == EVAL_GATHER && sv.list_small == nullptr &&
                               eval_gather_df_ok(Lg);
        if (!gather_in) {
            StageTimer t(p, 10, st);
            NN_CUDA(launch_gather_conv_df(Lg, W.bufC, W.Q, st), "adjoint gather convolution");
        }
        if (mid) NN_CUDA(cudaStreamWaitEvent(st, mid, 0), "wait for the other side");
        {
            StageTimer t(p, 11, st);
            NN_CUDA(gather_in ? launch_eval_gather_df(sv, Lg, W.bufC, z, st)
                              : launch_eval_df(sv, W.Q, z, p->eval_lanes[0], st),
                    "adjoint gather evaluation");
        }
    }
    return NNFFT_OK;
}

template <typename Real>
int run_forward(nnfft_plan_s *p, const void *f, void *y, cudaStream_t st, const Work &W,
                cudaEvent_t mid = nullptr, int part = 3) {
    const Side &V = p->side[0], &X = p->side[1];
    // part 1: steps 1-2 (spread into the grid buffer); part 2: steps 3-4 from it
    if (X.M == 0 && part == 3) return NNFFT_OK;
    const SideK<Real> sv = side_args<Real>(V, false, p->status);
    const SideK<Real> sx = side_args<Real>(X, true, p->status);
    if (part & 1) {
        {
            StageTimer t(p, 2, st);
            NN_CUDA(launch_moments<Real>(sv, f, W.P, p->mom_lanes[0], st), "spread moments");
        }
        {
            StageTimer t(p, 12, st);
            NN_CUDA(launch_cell_fold<Real>(sv, W.P, W.Q, st), "cell fold");
        }
        {
            StageTimer t(p, 3, st);
            NN_CUDA(launch_spread_conv<Real>(grid_launch<Real>(p, 0, true, false), W.Q, W.bufA, st),
                    "spread convolution");
        }
    }
    if ((part & 2) && !(X.M == 0)) {
        {
            StageTimer t(p, 4, st);
            NN_CUDA(fft_native<Real>(p, W, -1, st), "fft");
        }
        {
            StageTimer t(p, 5, st);
            NN_CUDA(launch_gather_conv<Real>(grid_launch<Real>(p, 1, false, true), W.bufC, W.Q, st),
                    "gather convolution");
        }
        // the gather side's sorted nodes (sorted on another stream) are needed from here on;
        // the gather convolution reads only the plan's grid geometry
        if (mid) NN_CUDA(cudaStreamWaitEvent(st, mid, 0), "wait for the other side");
        {
            StageTimer t(p, 6, st);
            NN_CUDA(launch_eval<Real>(sx, W.Q, y, p->eval_lanes[1], st), "gather evaluation");
        }
    }
    return NNFFT_OK;
}

template <typename Real>
int run_adjoint(nnfft_plan_s *p, const void *g, void *z, cudaStream_t st, const Work &W,
                cudaEvent_t mid = nullptr, int part = 3) {
    const Side &V = p->side[0], &X = p->side[1];
    // part 1: steps 1-2 (spread into the grid buffer); part 2: steps 3-4 from it
    if (V.M == 0 && part == 3) return NNFFT_OK;
    const SideK<Real> sv = side_args<Real>(V, false, p->status);
    const SideK<Real> sx = side_args<Real>(X, true, p->status);
    if (part & 1) {
        {
            StageTimer t(p, 7, st);
            NN_CUDA(launch_moments<Real>(sx, g, W.P, p->mom_lanes[1], st), "adjoint spread moments");
        }
        {
            StageTimer t(p, 13, st);
            NN_CUDA(launch_cell_fold<Real>(sx, W.P, W.Q, st), "adjoint cell fold");
        }
        {
            StageTimer t(p, 8, st);
            NN_CUDA(launch_spread_conv<Real>(grid_launch<Real>(p, 1, true, false), W.Q, W.bufA, st),
                    "adjoint spread convolution");
        }
    }
    if ((part & 2) && !(V.M == 0)) {
        {
            StageTimer t(p, 9, st);
            NN_CUDA(fft_native<Real>(p, W, +1, st), "adjoint fft");
        }
        {
            StageTimer t(p, 10, st);
            NN_CUDA(launch_gather_conv<Real>(grid_launch<Real>(p, 0, false, false), W.bufC, W.Q, st),
                    "adjoint gather convolution");
        }
        if (mid) NN_CUDA(cudaStreamWaitEvent(st, mid, 0), "wait for the other side");
        {
            StageTimer t(p, 11, st);
            NN_CUDA(launch_eval<Real>(sv, W.Q, z, p->eval_lanes[0], st), "adjoint gather evaluation");
        }
    }
    return NNFFT_OK;
}

// mid: an event the evaluation (the gather half's point kernel) waits for, or nullptr.
// part: 1 the spread half only (into the grid buffer W.bufA), 2 the rest only (from W.bufA:
// FFT, gather convolution, evaluation), 3 both.
int forward(nnfft_plan_s *p, const void *f, void *y, cudaStream_t st, const Work &W,
            cudaEvent_t mid = nullptr, int part = 3) {
    if (p->dbl && p->split) return run_forward_split(p, f, y, st, W, mid, part);
    return p->dbl ? run_forward<double>(p, f, y, st, W, mid, part)
                  : run_forward<float>(p, f, y, st, W, mid, part);
}

int adjoint(nnfft_plan_s *p, const void *g, void *z, cudaStream_t st, const Work &W,
            cudaEvent_t mid = nullptr, int part = 3) {
    if (p->dbl && p->split) return run_adjoint_split(p, g, z, st, W, mid, part);
    return p->dbl ? run_adjoint<double>(p, g, z, st, W, mid, part)
                  : run_adjoint<float>(p, g, z, st, W, mid, part);
}

// Element format of the plan's grid buffers (launch_grid_export / launch_grid_import).
int grid_format(const nnfft_plan_s *p) { return !p->dbl ? 0 : (p->split ? 2 : 1); }

// Checks shared by the four sharded-transform calls.
int shard_check(nnfft_plan_s *p, const void *grid) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (p->ninst != 1) return fail(NNFFT_EINVAL, "the sharded calls take single-instance plans");
    if (!p->side[0].set || !p->side[1].set) return fail(NNFFT_ESTATE, "nnfft_set_nodes first");
    if (!grid) return fail(NNFFT_EINVAL, "null grid pointer");
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
    if (st & STATUS_TIMEOUT) {
        // a fused grid stage that gave up leaves its barrier counter off a multiple of the
        // block count: start both directions' counters afresh
        for (const Work &W : p->work)
            if (W.gbar) cudaMemset(W.gbar, 0, 2 * sizeof(unsigned long long));
        return fail(NNFFT_ETIMEOUT,
                    "a bounded device-side wait (bulk copy or grid barrier) gave up");
    }
    if (st & STATUS_INTERNAL)
        return fail(NNFFT_ECUDA, "internal error: inconsistent node cell assignment");
    return NNFFT_OK;
}

void free_plan(nnfft_plan_s *p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    if (p->copy) {
        cudaStreamSynchronize(p->copy);
        cudaStreamDestroy(p->copy);
    }
    if (p->ev_v) cudaEventDestroy(p->ev_v);
    if (p->ev_x) cudaEventDestroy(p->ev_x);
    if (p->ev_up) cudaEventDestroy(p->ev_up);
    if (p->ev_up_v) cudaEventDestroy(p->ev_up_v);
    if (p->ev_up_x) cudaEventDestroy(p->ev_up_x);
    if (p->ev_up_f) cudaEventDestroy(p->ev_up_f);
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
int plan_device(nnfft_plan_t p) { return p->device; }
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

int nnfft_params_window(int64_t N, int64_t M1, int64_t M2, double sigma1, double sigma2, int m1,
                        int m2, int dtype, int window, nnfft_info *out) {
    hm::Derived d;
    return fill_info(N, M1, M2, sigma1, sigma2, m1, m2, (nnfft_dtype)dtype, out, &d, nullptr,
                     nullptr, window);
}

int nnfft_window(int window, int m, double sigma, double x, double v, double *omega_x,
                 double *omega_hat_v) {
    if (window < NNFFT_WINDOW_SINH || window > NNFFT_WINDOW_ALGEBRAIC || m < 2 || m > 16 ||
        !(sigma > 1.0) || !omega_x || !omega_hat_v)
        return fail(NNFFT_EINVAL, "invalid window arguments");
    const double beta = hm::window_beta(window, m, sigma);
    *omega_x = hm::omega_w(window, x, beta, m);
    *omega_hat_v = hm::omega_hat_w(window, v, beta, m);
    return NNFFT_OK;
}

int nnfft_gauss_legendre(int64_t n, double *tau_host, double *w_host) {
    if (n < 1 || !tau_host || !w_host) return fail(NNFFT_EINVAL, "invalid Gauss-Legendre request");
    hm::gauss_legendre(n, tau_host, w_host);
    return NNFFT_OK;
}

int nnfft_batch_plan_window(nnfft_plan_t *out, int64_t count, const int64_t *N, const int64_t *M1,
                            const int64_t *M2, double sigma1, double sigma2, int m1, int m2,
                            nnfft_dtype dtype, int window, void *stream) {
    if (!out) return fail(NNFFT_EINVAL, "null plan pointer");
    *out = nullptr;
    if (count < 1 || !N || !M1 || !M2) return fail(NNFFT_EINVAL, "a plan needs >= 1 instance");
    if (count > (1 << 20)) return fail(NNFFT_EINVAL, "too many instances in one plan");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(NNFFT_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    int cur = 0;
    if ((e = cudaGetDevice(&cur)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NNFFT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    nnfft_plan_s *p = new nnfft_plan_s();
    p->device = cur;
    p->stream = static_cast<cudaStream_t>(stream);
    auto bail = [&](int code) { free_plan(p); return code; };
    if (cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "stream/event creation"));
    int rc;
    if ((rc = dalloc_n(p, &p->status, 1, "status"))) return bail(rc);
    if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    if (cudaMallocHost(&p->status_host, sizeof(int)) != cudaSuccess) {
        p->status_host = nullptr;
        cudaGetLastError();
        return bail(fail(NNFFT_ENOMEM, "cudaMallocHost(status)"));
    }
    if ((rc = build_plan(p, count, N, M1, M2, sigma1, sigma2, m1, m2, dtype, window))) return bail(rc);
    if (prepare_local_sort() != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "sort setup"));
    if (p->dbl && p->split_ok && p->side[0].D == p->side[1].D && df_supported_degree(p->side[0].D)) {
        // the fused grid stage: two blocks per SM must be resident, the launch takes one
        const int D = p->side[0].D;
        const int mm = std::max(p->side[0].m, p->side[1].m);
        const size_t sm = grid_stage_df_smem(D, mm, mm, p->fftdf[0].smem1, p->fftdf[0].smem2);
        const int bps = prepare_grid_stage_df(D, sm);
        if (bps >= 2) {
            p->grid_fused_ok = true;
            p->fused_blocks = device_sm_count() * (bps / 2);
            p->fused_smem = sm;
        }
    }
    if (count == 1) {        // the cluster FFT: every arithmetic mode of the plan must fit
        const int n1 = (int)p->info.fft_n1, n2 = (int)p->info.fft_n2;
        const size_t need = p->dbl ? std::max(fft_cluster_smem(n1, n2), fft_cluster_smem_real<double>(n1, n2))
                                   : fft_cluster_smem_real<float>(n1, n2);
        if (need <= FFT_CLUSTER_SMEM_MAX) {
            cudaError_t ce = p->dbl ? prepare_fft_cluster<double>() : prepare_fft_cluster<float>();
            if (ce == cudaSuccess && p->dbl && p->split_ok) ce = prepare_fft_cluster_df();
            if (ce != cudaSuccess) return bail(cuda_fail(ce, "cluster FFT setup"));
            p->fft_cluster_ok = true;
        }
    }
    *out = p;
    return NNFFT_OK;
}

int nnfft_batch_plan(nnfft_plan_t *out, int64_t count, const int64_t *N, const int64_t *M1,
                     const int64_t *M2, double sigma1, double sigma2, int m1, int m2,
                     nnfft_dtype dtype, void *stream) {
    return nnfft_batch_plan_window(out, count, N, M1, M2, sigma1, sigma2, m1, m2, dtype,
                                   NNFFT_WINDOW_SINH, stream);
}

int nnfft_plan(nnfft_plan_t *out, int64_t N, int64_t M1, int64_t M2, double sigma1,
               double sigma2, int m1, int m2, nnfft_dtype dtype, void *stream) {
    return nnfft_batch_plan_window(out, 1, &N, &M1, &M2, sigma1, sigma2, m1, m2, dtype,
                                   NNFFT_WINDOW_SINH, stream);
}

int nnfft_plan_window(nnfft_plan_t *out, int64_t N, int64_t M1, int64_t M2, double sigma1,
                      double sigma2, int m1, int m2, nnfft_dtype dtype, int window, void *stream) {
    return nnfft_batch_plan_window(out, 1, &N, &M1, &M2, sigma1, sigma2, m1, m2, dtype, window,
                                   stream);
}

int nnfft_set_sizes(nnfft_plan_t p, int64_t M1, int64_t M2) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (p->ninst != 1) return fail(NNFFT_EINVAL, "nnfft_set_sizes applies to single-instance plans");
    if (M1 < 0 || M2 < 0 || M1 > p->side[0].M_cap || M2 > p->side[1].M_cap)
        return fail(NNFFT_EINVAL, "sizes exceed the plan's capacity");
    p->side[0].M = (int)M1;
    p->side[1].M = (int)M2;
    p->side[0].set = p->side[1].set = false;
    p->info.M1 = p->inst_info[0].M1 = M1;
    p->info.M2 = p->inst_info[0].M2 = M2;
    return NNFFT_OK;
}

int nnfft_set_bandwidth(nnfft_plan_t p, int64_t N) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (p->ninst != 1) return fail(NNFFT_EINVAL, "nnfft_set_bandwidth applies to single-instance plans");
    nnfft_info &I = p->inst_info[0];
    if (N < 1 || N > p->N_built) return fail(NNFFT_EINVAL, "bandwidth above the plan's N");
    hm::CellMap cm{};
    if (!hm::cell_map(I.N1 * N, I.Nstar, &cm)) return fail(NNFFT_EINVAL, "invalid bandwidth");
    p->side[0].one.S = cm.S;      // u = v N1 N / N*: the cells of the plan's N cover it
    p->side[0].set = false;
    I.N = N;
    p->info.N = N;
    return NNFFT_OK;
}

int nnfft_set_stream(nnfft_plan_t p, void *stream) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    p->stream = static_cast<cudaStream_t>(stream);
    return NNFFT_OK;
}

int nnfft_batch_count(nnfft_plan_t p, int64_t *count) {
    if (!p || !count) return fail(NNFFT_EINVAL, "null argument");
    *count = p->ninst;
    return NNFFT_OK;
}

int nnfft_batch_info(nnfft_plan_t p, int64_t i, nnfft_info *out) {
    if (!p || !out) return fail(NNFFT_EINVAL, "null argument");
    if (i < 0 || i >= p->ninst) return fail(NNFFT_EINVAL, "instance index out of range");
    *out = p->inst_info[(size_t)i];
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
    return forward(p, f_dev, y_dev, p->stream, p->work[0]);
}

int nnfft_adjoint(nnfft_plan_t p, const void *g_dev, void *z_dev) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (!p->side[0].set || !p->side[1].set) return fail(NNFFT_ESTATE, "nnfft_set_nodes first");
    if ((p->info.M2 > 0 && !g_dev) || (p->info.M1 > 0 && !z_dev))
        return fail(NNFFT_EINVAL, "null data pointer");
    return adjoint(p, g_dev, z_dev, p->stream, p->work[0]);
}

int nnfft_spread_grid(nnfft_plan_t p, const void *f_dev, void *grid_dev) {
    int rc = shard_check(p, grid_dev);
    if (rc) return rc;
    if (p->info.M1 > 0 && !f_dev) return fail(NNFFT_EINVAL, "null data pointer");
    if ((rc = forward(p, f_dev, nullptr, p->stream, p->work[0], nullptr, 1))) return rc;
    NN_CUDA(launch_grid_export(grid_format(p), p->work[0].bufA, (int)p->info.N2,
                               (int)p->info.K1, grid_dev, p->stream),
            "grid export");
    return NNFFT_OK;
}

int nnfft_exec_grid(nnfft_plan_t p, const void *grid_dev, void *y_dev) {
    int rc = shard_check(p, grid_dev);
    if (rc) return rc;
    if (p->info.M2 > 0 && !y_dev) return fail(NNFFT_EINVAL, "null data pointer");
    if (p->info.M2 == 0) return NNFFT_OK;
    NN_CUDA(launch_grid_import(grid_format(p), grid_dev, (int)p->info.N2, (int)p->info.K1,
                               p->work[0].bufA, p->stream),
            "grid import");
    return forward(p, nullptr, y_dev, p->stream, p->work[0], nullptr, 2);
}

int nnfft_adjoint_spread_grid(nnfft_plan_t p, const void *g_dev, void *grid_dev) {
    int rc = shard_check(p, grid_dev);
    if (rc) return rc;
    if (p->info.M2 > 0 && !g_dev) return fail(NNFFT_EINVAL, "null data pointer");
    if ((rc = adjoint(p, g_dev, nullptr, p->stream, p->work[0], nullptr, 1))) return rc;
    NN_CUDA(launch_grid_export(grid_format(p), p->work[0].bufA, (int)p->info.N2,
                               (int)p->info.N2, grid_dev, p->stream),
            "grid export");
    return NNFFT_OK;
}

int nnfft_adjoint_grid(nnfft_plan_t p, const void *grid_dev, void *z_dev) {
    int rc = shard_check(p, grid_dev);
    if (rc) return rc;
    if (p->info.M1 > 0 && !z_dev) return fail(NNFFT_EINVAL, "null data pointer");
    if (p->info.M1 == 0) return NNFFT_OK;
    NN_CUDA(launch_grid_import(grid_format(p), grid_dev, (int)p->info.N2, (int)p->info.N2,
                               p->work[0].bufA, p->stream),
            "grid import");
    return adjoint(p, nullptr, z_dev, p->stream, p->work[0], nullptr, 2);
}

int nnfft_exec_adjoint(nnfft_plan_t p, const void *f_dev, void *y_dev, const void *g_dev,
                       void *z_dev) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (!p->side[0].set || !p->side[1].set) return fail(NNFFT_ESTATE, "nnfft_set_nodes first");
    if ((p->info.M1 > 0 && (!f_dev || !z_dev)) || (p->info.M2 > 0 && (!y_dev || !g_dev)))
        return fail(NNFFT_EINVAL, "null data pointer");
    int rc;
    if (!p->work[1].P && (rc = alloc_work(p, p->work[1]))) return rc;
    // fork: the adjoint runs on the auxiliary stream with its own work buffers
    NN_CUDA(cudaEventRecord(p->ev_fork, p->stream), "fork");
    NN_CUDA(cudaStreamWaitEvent(p->aux, p->ev_fork, 0), "fork");
    const int ra = adjoint(p, g_dev, z_dev, p->aux, p->work[1]);
    const int rf = forward(p, f_dev, y_dev, p->stream, p->work[0]);
    NN_CUDA(cudaEventRecord(p->ev_join, p->aux), "join");
    NN_CUDA(cudaStreamWaitEvent(p->stream, p->ev_join, 0), "join");
    return ra ? ra : rf;
}

int nnfft_autotune(nnfft_plan_t p, const double *v_dev, const double *x_dev, const void *f_dev,
                   void *y_dev, const void *g_dev, void *z_dev, int reps, int flags) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    const bool with_nodes = v_dev || x_dev;
    if (with_nodes && ((p->info.M1 > 0 && !v_dev) || (p->info.M2 > 0 && !x_dev)))
        return fail(NNFFT_EINVAL, "give both node arrays or neither");
    if (!with_nodes && (!p->side[0].set || !p->side[1].set))
        return fail(NNFFT_ESTATE, "nnfft_set_nodes first (or pass the nodes)");
    if (reps < 1) reps = 1;
    // moments lanes per item: 32/16/8 for the split-precision kernels, 32/8 for the all-real
    // ones (D <= 16); evaluation: 32 or 8 lanes per item, or flat (one thread per point)
    const bool dfk = p->dbl && p->split;
    const bool small_d = p->side[0].D <= 16 && p->side[1].D <= 16;
    std::vector<int> lanes = dfk ? std::vector<int>{32, 16, 8, MOM_TEAM_PF}
                                 : (small_d ? std::vector<int>{32, 8} : std::vector<int>{32});
    std::vector<int> elanes{32, 8, EVAL_FLAT, EVAL_FLAT_TMA};
    if (dfk && p->ninst == 1) elanes.push_back(EVAL_GATHER);
    // splitting small items changes the node-time work lists: only with the nodes given,
    // and only where the size rule would split somewhere
    bool split_possible = false;
    for (int s = 0; s < 2; ++s) {
        const Side &S = p->side[s];
        split_possible = split_possible || S.split_rule ||
                         (p->ninst == 1 && S.M > 0 && (int64_t)S.M < 4LL * SMALL_ITEM * S.ncell);
    }
    std::vector<int> splits = with_nodes && split_possible ? std::vector<int>{0, 1} : std::vector<int>{p->item_split};
    void *flush = nullptr;
    const size_t flush_bytes = (size_t)192 << 20;         // larger than GB300's L2
    if ((flags & NNFFT_TUNE_FLUSH_L2) && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;
    }
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    int rc = NNFFT_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "event");
    auto run = [&]() {
        return with_nodes ? nnfft_transform(p, v_dev, x_dev, f_dev, y_dev, g_dev, z_dev)
                          : nnfft_exec_adjoint(p, f_dev, y_dev, g_dev, z_dev);
    };
    // Coordinate descent from the defaults: the dimensions (moments lanes, evaluation form,
    // FFT packing, item split, item cap) are searched one at a time with the others held at
    // their current best, in two sweeps.  Within a dimension every value is timed in ROUNDS
    // interleaved rounds (best time kept) and the incumbent stays unless another value is
    // more than 3 % faster.  The item split and cap change the node-time work lists, so they
    // are searched only with the nodes given (every run is then a full transform).
    struct Cfg { int lv, lx, el, fv, sp, cap, lsd; };
    const std::vector<int> caps = with_nodes ? std::vector<int>{ITEM_CAP, 128, 64, ITEM_CAP_MIN}
                                             : std::vector<int>{p->item_cap};
    // the node sort (two-stage or LSD passes) only matters where the nodes are sorted
    const std::vector<int> sorts = with_nodes ? std::vector<int>{p->sort_lsd, 1 - p->sort_lsd}
                                              : std::vector<int>{p->sort_lsd};
    std::vector<int> ffts{0, 1};
    if (p->fft_cluster_ok) ffts.push_back(FFT_CLUSTER_VARIANT);
    if (p->grid_fused_ok && dfk) ffts.push_back(GRID_FUSED_VARIANT);
    const std::vector<std::vector<int>> dims{lanes, elanes, ffts, splits, caps, sorts};
    auto set_dim = [](Cfg c, size_t d, int v) {
        switch (d) {
            case 0: c.lv = c.lx = v; break;
            case 1: c.el = v; break;
            case 2: c.fv = v; break;
            case 3: c.sp = v; break;
            case 4: c.cap = v; break;
            default: c.lsd = v; break;
        }
        return c;
    };
    auto apply = [&](const Cfg &c) {
        p->fft_variant = c.fv;
        p->mom_lanes[0] = c.lv;
        p->mom_lanes[1] = c.lx;
        p->eval_lanes[0] = p->eval_lanes[1] = c.el;
        p->item_split = c.sp;
        p->item_cap = c.cap;
        p->sort_lsd = c.lsd;
    };
    auto time_cfg = [&](const Cfg &c, double &ms) -> int {
        apply(c);
        int r = run();                                  // warm-up (and work lists)
        for (int k = 0; k < reps && !r; ++k) {
            if (flush) cudaMemsetAsync(flush, k & 1, flush_bytes, p->stream);
            cudaEventRecord(ev[2 * k], p->stream);
            r = run();
            cudaEventRecord(ev[2 * k + 1], p->stream);
        }
        if (r) return r;
        if (cudaEventSynchronize(ev.back()) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune timing");
        double tot = 0;
        for (int k = 0; k < reps; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]);
            tot += t;
        }
        ms = tot / reps;
        return NNFFT_OK;
    };
    constexpr int ROUNDS = 3;
    const bool timing = p->timing;
    p->timing = false;
    Cfg cur{lanes[0], lanes[0], elanes[0], 0, splits[0], with_nodes ? ITEM_CAP : p->item_cap,
            sorts[0]};
    double cur_ms = 1e300, default_ms = -1.0;
    for (int sweep = 0; sweep < 2 && !rc; ++sweep)
        for (size_t d = 0; d < dims.size() && !rc; ++d) {
            const std::vector<int> &vals = dims[d];
            if (vals.size() < 2) continue;
            std::vector<double> best(vals.size(), 1e300);
            for (int round = 0; round < ROUNDS && !rc; ++round)
                for (size_t i = 0; i < vals.size() && !rc; ++i) {
                    const size_t vi = round % 2 ? vals.size() - 1 - i : i;
                    double ms = 0;
                    if ((rc = time_cfg(set_dim(cur, d, vals[vi]), ms))) break;
                    best[vi] = std::min(best[vi], ms);
                }
            if (rc) break;
            int inc = 0;                                   // the incumbent's value index
            int curv = d == 0 ? cur.lv : d == 1 ? cur.el : d == 2 ? cur.fv : d == 3 ? cur.sp
                     : d == 4 ? cur.cap : cur.lsd;
            for (size_t i = 0; i < vals.size(); ++i)
                if (vals[i] == curv) inc = (int)i;
            if (default_ms < 0) default_ms = best[inc];
            size_t bi = inc;
            for (size_t i = 0; i < vals.size(); ++i)
                if (best[i] < best[bi]) bi = i;
            if (best[bi] < 0.97 * best[inc]) {
                cur = set_dim(cur, d, vals[bi]);
                cur_ms = best[bi];
            } else {
                cur_ms = best[inc];
            }
        }
    p->timing = timing;
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (flush) {
        cudaStreamSynchronize(p->stream);
        cudaFree(flush);
    }
    apply(cur);
    if (rc) return rc;
    if (default_ms < 0) {                      // nothing to choose between: time the one config
        double ms = 0;
        if ((rc = time_cfg(cur, ms))) return rc;
        default_ms = cur_ms = ms;
    }
    p->tuning = nnfft_tuning{cur.lv, cur.lx, cur.fv, 1, default_ms, cur_ms, cur.sp,
                             with_nodes ? 1 : 0, cur.el, cur.el, cur.cap, cur.lsd};
    // the work lists of the current node set follow the chosen split and cap
    if (with_nodes && (rc = run())) return rc;
    return collect_status(p);
}

int nnfft_get_tuning(nnfft_plan_t p, nnfft_tuning *out) {
    if (!p || !out) return fail(NNFFT_EINVAL, "null argument");
    *out = p->tuning;
    out->moments_lanes_v = p->mom_lanes[0];
    out->moments_lanes_x = p->mom_lanes[1];
    out->fft_variant = p->fft_variant;
    out->item_split = p->item_split;
    out->eval_lanes_v = p->eval_lanes[0];
    out->eval_lanes_x = p->eval_lanes[1];
    out->item_cap = p->item_cap;
    out->sort_lsd = p->sort_lsd;
    return NNFFT_OK;
}

int nnfft_set_tuning(nnfft_plan_t p, const nnfft_tuning *t) {
    if (!p || !t) return fail(NNFFT_EINVAL, "null argument");
    auto ok_lanes = [](int l) { return l == MOM_TEAM_PF || l == 8 || l == 16 || l == 32; };
    auto ok_elanes = [](int l) {
        return l == 0 || l == EVAL_FLAT || l == EVAL_FLAT_TMA || l == EVAL_GATHER || l == 8 ||
               l == 32;
    };
    if (!ok_lanes(t->moments_lanes_v) || !ok_lanes(t->moments_lanes_x) ||
        !ok_elanes(t->eval_lanes_v) || !ok_elanes(t->eval_lanes_x) ||
        (t->fft_variant != 0 && t->fft_variant != 1 &&
         !(t->fft_variant == FFT_CLUSTER_VARIANT && p->fft_cluster_ok) &&
         !(t->fft_variant == GRID_FUSED_VARIANT && p->grid_fused_ok)) ||
        (t->item_split != 0 && t->item_split != 1) ||
        (t->item_cap != 0 && t->item_cap != 32 && t->item_cap != 64 && t->item_cap != 128 &&
         t->item_cap != ITEM_CAP) || (t->sort_lsd != 0 && t->sort_lsd != 1))
        return fail(NNFFT_EINVAL, "invalid tuning values");
    p->mom_lanes[0] = t->moments_lanes_v;
    p->mom_lanes[1] = t->moments_lanes_x;
    p->eval_lanes[0] = t->eval_lanes_v ? t->eval_lanes_v : 32;
    p->eval_lanes[1] = t->eval_lanes_x ? t->eval_lanes_x : 32;
    p->fft_variant = t->fft_variant;
    const int cap = t->item_cap ? t->item_cap : ITEM_CAP;
    if (t->item_split != p->item_split || cap != p->item_cap || t->sort_lsd != p->sort_lsd) {
        p->item_split = t->item_split;   // work lists and sorted nodes: built with the nodes
        p->item_cap = cap;
        p->sort_lsd = t->sort_lsd;
        p->side[0].set = p->side[1].set = false;
    }
    return NNFFT_OK;
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
    for (nnfft_info &I : p->inst_info) I.arith = p->info.arith;
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

int nnfft_selftest_fixed63(const int64_t *in_dev, float *out_dev, int64_t n) {
    if (n < 0 || n > (1LL << 28) || (n > 0 && (!in_dev || !out_dev)))
        return fail(NNFFT_EINVAL, "invalid self-test arguments");
    NN_CUDA(selftest_fixed63(reinterpret_cast<const long long *>(in_dev), out_dev, (int)n, nullptr),
            "self-test launch");
    NN_CUDA(cudaStreamSynchronize(nullptr), "self-test");
    return NNFFT_OK;
}

int nnfft_selftest_bulk_copy(const float *src_dev, float *dst_dev, int n, int arm_only,
                             int64_t limit_cycles, int *status_dev) {
    if (!dst_dev || !status_dev || (!src_dev && !arm_only) || n <= 0 || n > 4096 || (n & 3) ||
        limit_cycles <= 0)
        return fail(NNFFT_EINVAL, "invalid self-test arguments");
    NN_CUDA(selftest_bulk_copy(src_dev, dst_dev, n, arm_only, (long long)limit_cycles, status_dev,
                               nullptr),
            "bulk-copy self-test");
    NN_CUDA(cudaStreamSynchronize(nullptr), "bulk-copy self-test");
    return NNFFT_OK;
}

int nnfft_selftest_grid_barrier(int blocks, int extra, int64_t limit_cycles,
                                uint64_t *words_dev, int *status_dev) {
    if (!words_dev || !status_dev || blocks <= 0 || blocks > device_sm_count() || extra < 0 ||
        limit_cycles <= 0)
        return fail(NNFFT_EINVAL, "invalid self-test arguments");
    NN_CUDA(selftest_grid_barrier(blocks, extra, (long long)limit_cycles,
                                  reinterpret_cast<unsigned long long *>(words_dev), status_dev,
                                  nullptr),
            "grid-barrier self-test");
    NN_CUDA(cudaStreamSynchronize(nullptr), "grid-barrier self-test");
    return NNFFT_OK;
}

int64_t nnfft_launch_count(void) { return launches_so_far(); }

int nnfft_sync(nnfft_plan_t p) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    return collect_status(p);
}

int nnfft_node_order(nnfft_plan_t p, int side, int32_t *perm_host, int32_t *off_host,
                     int64_t *ncell_out) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    if (side != 0 && side != 1) return fail(NNFFT_EINVAL, "node order: side must be 0 or 1");
    if (p->ninst != 1) return fail(NNFFT_EINVAL, "node order: single-instance plans only");
    const Side &S = p->side[side];
    if (ncell_out) *ncell_out = S.ncell;
    if (!perm_host && !off_host) return NNFFT_OK;
    if (!S.set || !S.perm || !S.cell_off)
        return fail(NNFFT_ESTATE, "node order: nnfft_set_nodes first");
    NN_CUDA(cudaStreamSynchronize(p->stream), "stream synchronize");
    if (perm_host && S.M > 0)
        NN_CUDA(cudaMemcpy(perm_host, S.perm, (size_t)S.M * sizeof(int), cudaMemcpyDeviceToHost),
                "node order copy");
    if (off_host)
        NN_CUDA(cudaMemcpy(off_host, S.cell_off, ((size_t)S.ncell + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost),
                "cell offsets copy");
    return NNFFT_OK;
}

int nnfft_destroy(nnfft_plan_t p) {
    free_plan(p);
    return NNFFT_OK;
}

static int ensure_staging(nnfft_plan_s *p) {
    const size_t cs = 2 * real_size(p->dbl);
    int rc;
    const size_t c1 = (size_t)p->side[0].M_cap, c2 = (size_t)p->side[1].M_cap;
    if (!p->st_v && (rc = dalloc_n(p, &p->st_v, c1, "staging"))) return rc;
    if (!p->st_x && (rc = dalloc_n(p, &p->st_x, c2, "staging"))) return rc;
    if (!p->st_f && (rc = dalloc(p, &p->st_f, c1 * cs, "staging"))) return rc;
    if (!p->st_y && (rc = dalloc(p, &p->st_y, c2 * cs, "staging"))) return rc;
    return NNFFT_OK;
}

// Events of host uploads that the transform's work waits for (nullptr: already there).
struct Uploads {
    cudaEvent_t v = nullptr, x = nullptr, f = nullptr, g = nullptr;
};

// Both node sides sorted concurrently (v on the plan stream, x on the second stream); each
// direction starts on the stream of the side its spread needs and waits for the other side
// only before its gather half.  Nodes are in st_v / st_x style device arrays v, x.  Each
// node sort waits only for its own nodes' upload, each direction only for its own values.
static int transform_dag(nnfft_plan_s *p, const double *v, const double *x, const void *f,
                         void *y, const void *g, void *z, const Uploads &up) {
    cudaStream_t A = p->stream, Bs = p->aux;
    int rc;
    if (up.x) NN_CUDA(cudaStreamWaitEvent(Bs, up.x, 0), "wait for the x upload");
    if ((rc = set_side_nodes(p, 1, x, Bs))) return rc;
    NN_CUDA(cudaEventRecord(p->ev_x, Bs), "event");
    if (up.v) NN_CUDA(cudaStreamWaitEvent(A, up.v, 0), "wait for the v upload");
    if ((rc = set_side_nodes(p, 0, v, A))) return rc;
    NN_CUDA(cudaEventRecord(p->ev_v, A), "event");
    if (up.g) NN_CUDA(cudaStreamWaitEvent(Bs, up.g, 0), "wait for the g upload");
    if (up.f) NN_CUDA(cudaStreamWaitEvent(A, up.f, 0), "wait for the f upload");
    // adjoint: spread from x (on Bs), gather to v; forward: spread from v (on A), gather to x
    if (g && (rc = adjoint(p, g, z, Bs, p->work[1], p->ev_v))) return rc;
    if (f && (rc = forward(p, f, y, A, p->work[0], p->ev_x))) return rc;
    return NNFFT_OK;
}

static int ensure_dag(nnfft_plan_s *p, bool adj) {
    int rc;
    if (adj && !p->work[1].P && (rc = alloc_work(p, p->work[1]))) return rc;
    if (!p->copy) {
        NN_CUDA(cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking), "stream");
        NN_CUDA(cudaEventCreateWithFlags(&p->ev_v, cudaEventDisableTiming), "event");
        NN_CUDA(cudaEventCreateWithFlags(&p->ev_x, cudaEventDisableTiming), "event");
        NN_CUDA(cudaEventCreateWithFlags(&p->ev_up, cudaEventDisableTiming), "event");
        NN_CUDA(cudaEventCreateWithFlags(&p->ev_up_v, cudaEventDisableTiming), "event");
        NN_CUDA(cudaEventCreateWithFlags(&p->ev_up_x, cudaEventDisableTiming), "event");
        NN_CUDA(cudaEventCreateWithFlags(&p->ev_up_f, cudaEventDisableTiming), "event");
    }
    return NNFFT_OK;
}

int nnfft_transform(nnfft_plan_t p, const double *v_dev, const double *x_dev, const void *f_dev,
                    void *y_dev, const void *g_dev, void *z_dev) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    const int64_t M1 = p->info.M1, M2 = p->info.M2;
    if ((M1 > 0 && !v_dev) || (M2 > 0 && !x_dev)) return fail(NNFFT_EINVAL, "null node pointer");
    const bool fwd = f_dev && y_dev, adj = g_dev && z_dev;
    int rc = ensure_dag(p, adj);
    if (rc) return rc;
    NN_CUDA(cudaEventRecord(p->ev_fork, p->stream), "fork");
    NN_CUDA(cudaStreamWaitEvent(p->aux, p->ev_fork, 0), "fork");
    if ((rc = transform_dag(p, v_dev, x_dev, fwd ? f_dev : nullptr, y_dev, adj ? g_dev : nullptr,
                            z_dev, Uploads{})))
        return rc;
    NN_CUDA(cudaEventRecord(p->ev_join, p->aux), "join");
    NN_CUDA(cudaStreamWaitEvent(p->stream, p->ev_join, 0), "join");
    return NNFFT_OK;
}

struct nnfft_graph_s {
    nnfft_plan_t plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;       // library kernels one replay runs
};

}  // extern "C"

// Capture the work enqueue(p) puts on the plan's streams into a CUDA graph.  The capture
// runs on a stream of its own (the plan stream may be the legacy default stream, which
// cannot be captured); replays go to the plan stream.
template <class F>
static int capture_graph(nnfft_plan_s *p, F &&enqueue, nnfft_graph_t *out) {
    cudaStream_t cs = nullptr;
    NN_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    cudaStream_t saved = p->stream;
    const bool timing = p->timing;
    p->stream = cs;
    p->timing = false;
    const long long l0 = launches_so_far();
    cudaGraph_t graph = nullptr;
    int rc = NNFFT_OK;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        rc = enqueue();
        const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (!rc && ee != cudaSuccess) rc = cuda_fail(ee, "end capture");
    } else {
        rc = cuda_fail(ce, "begin capture");
    }
    const int64_t kernels = launches_so_far() - l0;
    p->stream = saved;
    p->timing = timing;
    cudaGetLastError();
    cudaStreamDestroy(cs);
    count_launches(-(int)kernels);          // captured, not run
    cudaGraphExec_t exec = nullptr;
    if (!rc && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "graph instantiate");
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    nnfft_graph_s *gr = new (std::nothrow) nnfft_graph_s;
    if (!gr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(NNFFT_ENOMEM, "graph handle");
    }
    gr->plan = p;
    gr->graph = graph;
    gr->exec = exec;
    gr->kernels = kernels;
    *out = gr;
    return NNFFT_OK;
}

static int transform_host_enqueue(nnfft_plan_s *p, const double *v_host, const double *x_host,
                                  const void *f_host, void *y_host, const void *g_host,
                                  void *z_host);

// staging buffers, streams and events of the host-buffer transform (allocated once)
static int transform_host_prepare(nnfft_plan_s *p, bool adj) {
    int rc = ensure_staging(p);
    if (rc) return rc;
    const size_t cs = 2 * real_size(p->dbl);
    if (adj && !p->st_g && (rc = dalloc(p, &p->st_g, (size_t)p->side[1].M_cap * cs, "staging"))) return rc;
    if (adj && !p->st_z && (rc = dalloc(p, &p->st_z, (size_t)p->side[0].M_cap * cs, "staging"))) return rc;
    return ensure_dag(p, adj);
}

extern "C" {

int nnfft_transform_graph(nnfft_plan_t p, const double *v_dev, const double *x_dev,
                          const void *f_dev, void *y_dev, const void *g_dev, void *z_dev,
                          nnfft_graph_t *out) {
    if (!p || !out) return fail(NNFFT_EINVAL, "null argument");
    *out = nullptr;
    const int64_t M1 = p->info.M1, M2 = p->info.M2;
    if ((M1 > 0 && !v_dev) || (M2 > 0 && !x_dev)) return fail(NNFFT_EINVAL, "null node pointer");
    const bool adj = g_dev && z_dev;
    int rc = ensure_dag(p, adj);        // every buffer and stream exists before the capture
    if (rc) return rc;
    return capture_graph(
        p, [&]() { return nnfft_transform(p, v_dev, x_dev, f_dev, y_dev, g_dev, z_dev); }, out);
}

int nnfft_transform_host_graph(nnfft_plan_t p, const double *v_host, const double *x_host,
                               const void *f_host, void *y_host, const void *g_host,
                               void *z_host, nnfft_graph_t *out) {
    if (!p || !out) return fail(NNFFT_EINVAL, "null argument");
    *out = nullptr;
    const int64_t M1 = p->info.M1, M2 = p->info.M2;
    if ((M1 > 0 && !v_host) || (M2 > 0 && !x_host))
        return fail(NNFFT_EINVAL, "null node pointer");
    // copies into a graph must come from page-locked memory (a pageable copy cannot be
    // captured): check every host buffer first
    const void *bufs[6] = {v_host, x_host, f_host, y_host, g_host, z_host};
    for (const void *b : bufs) {
        if (!b) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, b) != cudaSuccess || a.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return fail(NNFFT_EINVAL, "host buffers of a graph must be page-locked");
        }
    }
    int rc = transform_host_prepare(p, g_host && z_host);   // allocations before the capture
    if (rc) return rc;
    return capture_graph(
        p,
        [&]() { return transform_host_enqueue(p, v_host, x_host, f_host, y_host, g_host, z_host); },
        out);
}

int nnfft_graph_launch(nnfft_graph_t gr) {
    if (!gr) return fail(NNFFT_EINVAL, "null graph");
    NN_CUDA(cudaGraphLaunch(gr->exec, gr->plan->stream), "graph launch");
    count_launches((int)gr->kernels);
    return NNFFT_OK;
}

int64_t nnfft_graph_kernels(nnfft_graph_t gr) { return gr ? gr->kernels : -1; }

int nnfft_graph_destroy(nnfft_graph_t gr) {
    if (!gr) return NNFFT_OK;
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
    return NNFFT_OK;
}

int nnfft_transform_host(nnfft_plan_t p, const double *v_host, const double *x_host,
                         const void *f_host, void *y_host, const void *g_host, void *z_host) {
    if (!p) return fail(NNFFT_EINVAL, "null plan");
    const int rc = transform_host_enqueue(p, v_host, x_host, f_host, y_host, g_host, z_host);
    if (rc) return rc;
    return collect_status(p);
}

}  // extern "C"

// the work of nnfft_transform_host, queued (uploads, transform, downloads) without waiting
static int transform_host_enqueue(nnfft_plan_s *p, const double *v_host, const double *x_host,
                                  const void *f_host, void *y_host, const void *g_host,
                                  void *z_host) {
    const int64_t M1 = p->info.M1, M2 = p->info.M2;
    if ((M1 > 0 && !v_host) || (M2 > 0 && !x_host))
        return fail(NNFFT_EINVAL, "null node pointer");
    const bool fwd = f_host && y_host, adj = g_host && z_host;
    int rc = transform_host_prepare(p, adj);
    if (rc) return rc;
    const size_t cs = 2 * real_size(p->dbl);
    cudaStream_t A = p->stream, Bs = p->aux, C = p->copy;
    // All uploads in one queue on the copy stream, in the order they are needed: v, x, f,
    // g.  Host-to-device copies share one link (~205 GB/s measured on GB300; two concurrent
    // ones add nothing), so queued copies finish one after another instead of all at the end:
    // each node sort starts once its own nodes are up, each direction once its own values are.
    NN_CUDA(cudaEventRecord(p->ev_fork, A), "fork");
    NN_CUDA(cudaStreamWaitEvent(Bs, p->ev_fork, 0), "fork");
    NN_CUDA(cudaStreamWaitEvent(C, p->ev_fork, 0), "fork");
    Uploads up;
    if (M1) NN_CUDA(cudaMemcpyAsync(p->st_v, v_host, 8 * (size_t)M1, cudaMemcpyHostToDevice, C), "copy v");
    NN_CUDA(cudaEventRecord(up.v = p->ev_up_v, C), "event");
    if (M2) NN_CUDA(cudaMemcpyAsync(p->st_x, x_host, 8 * (size_t)M2, cudaMemcpyHostToDevice, C), "copy x");
    NN_CUDA(cudaEventRecord(up.x = p->ev_up_x, C), "event");
    if (fwd && M1) NN_CUDA(cudaMemcpyAsync(p->st_f, f_host, cs * (size_t)M1, cudaMemcpyHostToDevice, C), "copy f");
    NN_CUDA(cudaEventRecord(up.f = p->ev_up_f, C), "event");
    if (adj && M2) NN_CUDA(cudaMemcpyAsync(p->st_g, g_host, cs * (size_t)M2, cudaMemcpyHostToDevice, C), "copy g");
    NN_CUDA(cudaEventRecord(up.g = p->ev_up, C), "event");
    if ((rc = transform_dag(p, p->st_v, p->st_x, fwd ? p->st_f : nullptr, p->st_y,
                            adj ? p->st_g : nullptr, p->st_z, up)))
        return rc;
    if (adj && M1) NN_CUDA(cudaMemcpyAsync(z_host, p->st_z, cs * (size_t)M1, cudaMemcpyDeviceToHost, Bs), "copy z");
    if (fwd && M2) NN_CUDA(cudaMemcpyAsync(y_host, p->st_y, cs * (size_t)M2, cudaMemcpyDeviceToHost, A), "copy y");
    NN_CUDA(cudaEventRecord(p->ev_join, Bs), "join");
    NN_CUDA(cudaStreamWaitEvent(A, p->ev_join, 0), "join");
    return NNFFT_OK;
}

extern "C" {

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
//   CC: t_j = cos(j pi / n) / 2, j = 0..n, with the weights of eq. (5.4) (Section 5).
// NNFFT #1 evaluates g_j at the nodes x1 (= -t for GL, +t for CC) and NNFFT #2 sums
// alpha_j = w_j g_j from the nodes v2 (= +t for GL, -t for CC); for CC this is the
// sign convention of Algorithm 6.1, for the symmetric GL rule both conventions agree.
struct SincPlan {
    nnfft_plan_t p1 = nullptr, p2 = nullptr;
    int64_t nq = 0;                           // number of quadrature nodes
    int64_t L1 = 0, L2 = 0;                   // current sizes (<= the plans' capacities)
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
    void *tab = nullptr;     // the FftPlanDev, then the two block maps {0, n2} and {0, n1}
    auto release = [&]() {
        cudaFree(t1); cudaFree(t2); cudaFree(tN); cudaFree(x); cudaFree(y); cudaFree(X);
        cudaFree(tab);
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
    F.grid_base = 0;
    F.cols1 = F.cols2 = 1;
    const size_t fb = (sizeof(FftPlanDev) + 15) / 16 * 16;
    const int blk[4] = {0, n2, 0, n1};
    if (e == cudaSuccess) e = cudaMalloc(&tab, fb + sizeof(blk));
    if (e == cudaSuccess) e = cudaMemcpyAsync(tab, &F, sizeof(F), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char *>(tab) + fb, blk, sizeof(blk), cudaMemcpyHostToDevice, st);
    const int *blk_dev = reinterpret_cast<const int *>(static_cast<char *>(tab) + fb);
    const FftLaunch<FftPlanDev> FL{static_cast<const FftPlanDev *>(tab), blk_dev, blk_dev + 2, 1,
                                   n2, n1, 3 * n1, 3 * n2};
    if (e == cudaSuccess) e = launch_cc_extend(n, x, st);
    if (e == cudaSuccess) e = launch_fft<double>(FL, x, y, X, -1, st);
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
    s->L1 = L1;
    s->L2 = L2;
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
    if (L1 != s->L1 || L2 != s->L2) {         // a plan made for larger sizes serves this call
        if ((rc = nnfft_set_sizes(s->p1, L1, nq)) || (rc = nnfft_set_sizes(s->p2, nq, L2))) return rc;
        s->L1 = L1;
        s->L2 = L2;
        s->nodes_fixed = false;
    }
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

}  // extern "C"

namespace nnfft {
// Algorithm 6.1 through plans cached for capacities (L1cap, L2cap) >= (L1, L2) on `stream`
// (the request loop's slots): the cache key holds the capacities, the call the sizes.
int sinc_exec_capacity(int64_t N, int64_t L1, int64_t L2, int64_t L1cap, int64_t L2cap, int m,
                       nnfft_dtype dtype, int rule, int64_t n, const double *a_dev,
                       const void *c_dev, const double *b_dev, void *h_dev, int is_complex,
                       cudaStream_t stream, size_t *plan_bytes) {
    if (L1 > L1cap || L2 > L2cap) return fail(NNFFT_EINVAL, "sizes above the capacity");
    SincPlan *s = nullptr;
    int rc = sinc_get(N, L1cap, L2cap, m, dtype, rule, n, stream, &s);
    if (rc) return rc;
    if (plan_bytes) *plan_bytes = s->p1->bytes + s->p2->bytes;
    if (L2 == 0) return NNFFT_OK;
    return dtype == NNFFT_C128 ? sinc_run<double>(s, L1, L2, a_dev, c_dev, b_dev, h_dev, is_complex)
                               : sinc_run<float>(s, L1, L2, a_dev, c_dev, b_dev, h_dev, is_complex);
}
// Free the cached sinc plans of one stream; returns the device bytes released.
size_t sinc_release_stream(cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g_sinc_mu);
    size_t freed = 0;
    for (auto it = g_sinc.begin(); it != g_sinc.end();) {
        if (it->second->stream == stream) {
            freed += it->second->p1->bytes + it->second->p2->bytes;
            sinc_free(it->second);
            it = g_sinc.erase(it);
        } else {
            ++it;
        }
    }
    return freed;
}
size_t plan_bytes(nnfft_plan_t p) { return p ? p->bytes : 0; }
}  // namespace nnfft

extern "C" {

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
