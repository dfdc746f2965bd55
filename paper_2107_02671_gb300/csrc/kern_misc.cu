// kern_misc.cu -- small elementwise kernels of the fast sinc transform
// (Algorithm 6.1): real <-> complex packing, the step-2 product alpha_j = w_j g_j,
// and the two ends of the Clenshaw-Curtis weight
// computation (Algorithm 5.4) around a length-2n FFT; and the grid export / import
// of the sharded transform (Algorithm 2.2 split at its grid).
#include "internal.h"
#include "gridsync.cuh"
#include "tma.cuh"

namespace nnfft {

namespace {

template <typename Real>
__global__ void k_real_to_complex(const Real *__restrict__ in, int n, C2<Real> *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    C2<Real> v;
    v.x = in[i];
    v.y = Real(0);
    out[i] = v;
}

template <typename Real>
__global__ void k_scale_by_weights(C2<Real> *__restrict__ v, const double *__restrict__ w, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Real s = (Real)w[i];
    C2<Real> a = v[i];
    a.x *= s;
    a.y *= s;
    v[i] = a;
}

template <typename Real>
__global__ void k_complex_to_real(const C2<Real> *__restrict__ in, int n, Real *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = in[i].x;
}

// Clenshaw-Curtis weights, eq. (5.4), through Algorithm 5.4's DCT-I: with
//   x_j = eps(j)^2 * 2/(1 - j^2)  for even j <= n,  x_j = 0 for odd j
// (eps(0)^2 = eps(n)^2 = 1/2, else 1), w_k = eps(k)^2/n * sum_{j=0}^{n} x_j cos(j k pi/n).
// The sum is the DCT-I of x; it is read off the FFT of the even extension of
// length 2n, X_k = x_0 + (-1)^k x_n + 2 sum_{0<j<n} x_j cos(pi j k / n).
__device__ __forceinline__ double cc_x(long long j, long long n) {
    if (j & 1) return 0.0;
    const double h = (double)(j / 2);
    const double e2 = (j == 0 || j == n) ? 0.5 : 1.0;
    return e2 * 2.0 / (1.0 - 4.0 * h * h);
}

__global__ void k_cc_extend(long long n, double2 *__restrict__ x) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= 2 * n) return;
    const long long jj = j <= n ? j : 2 * n - j;
    x[j] = make_double2(cc_x(jj, n), 0.0);
}

// w_k, k = 0..n, and the nodes z_k / 2 = cos(k pi / n) / 2 (exactly antisymmetric)
__global__ void k_cc_finish(long long n, const double2 *__restrict__ X, double *__restrict__ w,
                            double *__restrict__ half_z, double *__restrict__ neg_half_z) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k > n) return;
    const double ek2 = (k == 0 || k == n) ? 0.5 : 1.0;
    const double xn = cc_x(n, n);
    const double dct = 0.5 * (X[k].x + cc_x(0, n) + ((k & 1) ? -xn : xn));
    w[k] = ek2 * dct / (double)n;
    // cos(k pi / n) from the half of the range nearer to zero, mirrored for k > n/2
    const long long kk = 2 * k <= n ? k : n - k;
    double z = 0.5 * cospi((double)kk / (double)n);
    if (2 * k == n) z = 0.0;
    if (kk != k) z = -z;
    half_z[k] = z;
    neg_half_z[k] = -z;
}

// ---------------------------------------------------------------------------------
// Sharded transform: the grid exchanged between the two halves of a direction.  The
// plan's N2 grid buffer holds position p (centered) at p mod N2; the exchanged array
// holds the n positions l in I_n = {-n/2, ..., n/2 - 1} at index l + n/2 as complex
// values of the plan's type (complex64 for fp32 plans, complex128 for fp64 plans).
// Buffer element formats: 0 float2, 1 double2, 2 float4 (double-float re.h, re.l, im.h,
// im.l).  Export reads the n positions; import writes all N2 buffer elements (the n
// positions, zero elsewhere).
// ---------------------------------------------------------------------------------
template <int FMT> struct GridElem;
template <> struct GridElem<0> {
    using B = float2;
    using X = float2;
    __device__ static X out(B b) { return b; }
    __device__ static B in(X x) { return x; }
    __device__ static B zero() { return make_float2(0.f, 0.f); }
};
template <> struct GridElem<1> {
    using B = double2;
    using X = double2;
    __device__ static X out(B b) { return b; }
    __device__ static B in(X x) { return x; }
    __device__ static B zero() { return make_double2(0.0, 0.0); }
};
template <> struct GridElem<2> {
    using B = float4;
    using X = double2;
    __device__ static X out(B b) {
        return make_double2((double)b.x + (double)b.y, (double)b.z + (double)b.w);
    }
    __device__ static B in(X x) {
        const float rh = (float)x.x, ih = (float)x.y;
        return make_float4(rh, (float)(x.x - (double)rh), ih, (float)(x.y - (double)ih));
    }
    __device__ static B zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};

template <int FMT>
__global__ void k_grid_export(const typename GridElem<FMT>::B *__restrict__ buf, int N2, int n,
                              typename GridElem<FMT>::X *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = i - n / 2;
    out[i] = GridElem<FMT>::out(buf[l < 0 ? l + N2 : l]);
}

template <int FMT>
__global__ void k_grid_import(const typename GridElem<FMT>::X *__restrict__ in, int N2, int n,
                              typename GridElem<FMT>::B *__restrict__ buf) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N2) return;
    // the position l in I_n with l = q mod N2, if any (n <= N2, both even)
    const int l = q < n / 2 ? q : (q >= N2 - n / 2 ? q - N2 : N2);
    buf[q] = l < N2 ? GridElem<FMT>::in(in[l + n / 2]) : GridElem<FMT>::zero();
}

// Self-test of the bulk-copy helpers: one block stages n floats (n % 4 == 0, n <= 4096)
// in shared memory with one bulk copy and writes them back to dst.  arm_only announces
// the bytes on the barrier but issues no copy, so the bounded wait runs out: the block
// sets STATUS_TIMEOUT in *status, waits once more and returns without writing dst.
__global__ void k_selftest_bulk_copy(const float *__restrict__ src, float *__restrict__ dst,
                                     int n, int arm_only, long long limit, int *status) {
    __shared__ __align__(128) float buf[4096];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tma::bar_init(&bar);
        tma::bar_expect(&bar, (unsigned)n * 4u);
        if (!arm_only) tma::copy_g2s(buf, src, (unsigned)n * 4u, &bar);
    }
    __syncthreads();
    if (!tma::bar_wait(&bar, 0, limit)) {
        if (threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
        tma::bar_wait(&bar, 0, limit);
        return;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = buf[i];
}

// two grid barriers that expect gridDim.x + extra arrivals each
__global__ void k_selftest_grid_barrier(int extra, long long limit, unsigned long long *words,
                                        int *status) {
    const unsigned expect = gridDim.x + (unsigned)extra;
    if (!gsync::grid_barrier(words, expect, limit, status)) return;
    gsync::grid_barrier(words, expect, limit, status);
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

std::atomic<long long> g_launches{0};

}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

template <typename Real>
cudaError_t launch_real_to_complex(const Real *in, int n, void *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_real_to_complex<Real><<<cdiv(n, 256), 256, 0, s>>>(in, n, static_cast<C2<Real> *>(out));
    count_launches(1);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_scale_by_weights(void *vals, const double *w, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_scale_by_weights<Real><<<cdiv(n, 256), 256, 0, s>>>(static_cast<C2<Real> *>(vals), w, n);
    count_launches(1);
    return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_complex_to_real(const void *in, int n, Real *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_complex_to_real<Real><<<cdiv(n, 256), 256, 0, s>>>(static_cast<const C2<Real> *>(in), n,
                                                         out);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_cc_extend(long long n, void *x, cudaStream_t s) {
    k_cc_extend<<<cdiv(2 * n, 256), 256, 0, s>>>(n, static_cast<double2 *>(x));
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_cc_finish(long long n, const void *X, double *w, double *half_z,
                             double *neg_half_z, cudaStream_t s) {
    k_cc_finish<<<cdiv(n + 1, 256), 256, 0, s>>>(n, static_cast<const double2 *>(X), w, half_z,
                                                  neg_half_z);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t selftest_bulk_copy(const float *src, float *dst, int n, int arm_only,
                               long long limit, int *status, cudaStream_t s) {
    if (n <= 0 || n > 4096 || (n & 3) || limit <= 0) return cudaErrorInvalidValue;
    k_selftest_bulk_copy<<<1, 256, 0, s>>>(src, dst, n, arm_only, limit, status);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t selftest_grid_barrier(int blocks, int extra, long long limit,
                                  unsigned long long *words, int *status, cudaStream_t s) {
    if (blocks <= 0 || extra < 0 || limit <= 0) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(64);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_selftest_grid_barrier, extra, limit, words, status);
    count_launches(1);
    return e;
}

cudaError_t launch_grid_export(int fmt, const void *buf, int N2, int n, void *out,
                               cudaStream_t s) {
    if (n <= 0 || n > N2 || (n & 1) || (N2 & 1) || fmt < 0 || fmt > 2)
        return cudaErrorInvalidValue;
    const int nb = cdiv(n, 256);
    if (fmt == 0)
        k_grid_export<0><<<nb, 256, 0, s>>>(static_cast<const float2 *>(buf), N2, n,
                                            static_cast<float2 *>(out));
    else if (fmt == 1)
        k_grid_export<1><<<nb, 256, 0, s>>>(static_cast<const double2 *>(buf), N2, n,
                                            static_cast<double2 *>(out));
    else
        k_grid_export<2><<<nb, 256, 0, s>>>(static_cast<const float4 *>(buf), N2, n,
                                            static_cast<double2 *>(out));
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_grid_import(int fmt, const void *in, int N2, int n, void *buf,
                               cudaStream_t s) {
    if (n <= 0 || n > N2 || (n & 1) || (N2 & 1) || fmt < 0 || fmt > 2)
        return cudaErrorInvalidValue;
    const int nb = cdiv(N2, 256);
    if (fmt == 0)
        k_grid_import<0><<<nb, 256, 0, s>>>(static_cast<const float2 *>(in), N2, n,
                                            static_cast<float2 *>(buf));
    else if (fmt == 1)
        k_grid_import<1><<<nb, 256, 0, s>>>(static_cast<const double2 *>(in), N2, n,
                                            static_cast<double2 *>(buf));
    else
        k_grid_import<2><<<nb, 256, 0, s>>>(static_cast<const double2 *>(in), N2, n,
                                            static_cast<float4 *>(buf));
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_real_to_complex<double>(const double *, int, void *, cudaStream_t);
template cudaError_t launch_real_to_complex<float>(const float *, int, void *, cudaStream_t);
template cudaError_t launch_scale_by_weights<double>(void *, const double *, int, cudaStream_t);
template cudaError_t launch_scale_by_weights<float>(void *, const double *, int, cudaStream_t);
template cudaError_t launch_complex_to_real<double>(const void *, int, double *, cudaStream_t);
template cudaError_t launch_complex_to_real<float>(const void *, int, float *, cudaStream_t);

}  // namespace nnfft
