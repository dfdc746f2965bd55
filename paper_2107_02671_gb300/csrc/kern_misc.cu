// kern_misc.cu -- small elementwise kernels of the fast sinc transform
// (Algorithm 6.1): real <-> complex packing, the step-2 product alpha_j = w_j g_j,
// and the node reflection tau -> -tau of NNFFT #1.
#include "internal.h"

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

__global__ void k_negate(const double *__restrict__ in, int n, double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = -in[i];
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
cudaError_t launch_negate(const double *in, int n, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_negate<<<cdiv(n, 256), 256, 0, s>>>(in, n, out);
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
