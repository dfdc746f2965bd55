// kern_fft.cu -- step 3 of Algorithm 2.2: the length-N2 FFT on the oversampled
// grid, h_s = sum_l ghat_l exp(sign 2 pi i l s / N2), written as a four-step
// transform N2 = n1 * n2 with index maps n = n2 a + b, k = c + n1 d:
//   pass 1 (one CTA per column b):  Z[b][c] = w_N2^{b c} * sum_a X[n2 a + b] w_n1^{a c}
//   pass 2 (one CTA per column c):  Y[c + n1 d] = sum_b Z[b][c] w_n2^{b d}
// Each column transform is a Stockham autosort FFT in shared memory with radices
// 2, 3, 4, 5, so no bit reversal is needed.  Twiddles come from
// host-computed tables exp(-2 pi i k / n); sign = +1 uses their conjugates.
// The whole grid (N2 <= 2^20 points) stays resident in L2 between the passes.
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.h"

namespace nnfft {

namespace {

template <typename Real>
__device__ __forceinline__ C2<Real> cadd(C2<Real> a, C2<Real> b) {
    C2<Real> r; r.x = a.x + b.x; r.y = a.y + b.y; return r;
}
template <typename Real>
__device__ __forceinline__ C2<Real> csub(C2<Real> a, C2<Real> b) {
    C2<Real> r; r.x = a.x - b.x; r.y = a.y - b.y; return r;
}
template <typename Real>
__device__ __forceinline__ C2<Real> cmul(C2<Real> a, C2<Real> b) {
    C2<Real> r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// twiddle exp(sign 2 pi i idx / n) from the table of exp(-2 pi i idx / n)
template <typename Real>
__device__ __forceinline__ C2<Real> twid(const C2<Real> *tw, int idx, int sign) {
    C2<Real> w = tw[idx];
    if (sign > 0) w.y = -w.y;
    return w;
}
// multiply by exp(sign * i pi/2) = i*sign
template <typename Real>
__device__ __forceinline__ C2<Real> mul_isign(C2<Real> a, int sign) {
    C2<Real> r;
    r.x = sign > 0 ? -a.y : a.y;
    r.y = sign > 0 ? a.x : -a.x;
    return r;
}

// cos and sin of 2 pi / 3, 2 pi / 5 and 4 pi / 5 (the radix-3 and radix-5 butterflies)
constexpr double SB_S3 = 0.866025403784438646763723170753;    // sin(2 pi / 3)
constexpr double SB_C51 = 0.309016994374947424102293417183;   // cos(2 pi / 5)
constexpr double SB_C52 = -0.809016994374947424102293417183;  // cos(4 pi / 5)
constexpr double SB_S51 = 0.951056516295153572116439333379;   // sin(2 pi / 5)
constexpr double SB_S52 = 0.587785252292473129168705954639;   // sin(4 pi / 5)
template <typename Real>
__device__ __forceinline__ C2<Real> cscl(C2<Real> a, Real c) {
    C2<Real> r;
    r.x = a.x * c;
    r.y = a.y * c;
    return r;
}

// One Stockham stage of radix R over `cols` length-n sequences held back to back in
// shared memory: butterfly j (0 <= j < n/R) of each sequence, k = j mod L,
//   a_q = src[j + q n/R] * w_{L R}^{q k},  b_p = sum_q a_q w_R^{p q} (radices 3 and 5 through
//   the symmetric forms above: cosine sums shared by b_p and b_(R-p), sine sums with opposite signs),
//   dst[(j - k) R + k + p L] = b_p,
// where L is the product of the radices of the earlier stages.
template <typename Real, int R>
__device__ __forceinline__ void stage(const C2<Real> *src, C2<Real> *dst, int n, int cols, int L,
                                      const C2<Real> *tw, int sign) {
    const int nr = n / R;
    const int tstep = n / (L * R);
    for (int jj = threadIdx.x; jj < cols * nr; jj += blockDim.x) {
        const int col = jj / nr, j = jj - col * nr;
        const C2<Real> *s0 = src + col * n;
        C2<Real> *d0 = dst + col * n;
        const int k = j % L;
        C2<Real> a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            a[q] = s0[j + q * nr];
            if (q > 0 && k > 0) a[q] = cmul<Real>(a[q], twid<Real>(tw, q * k * tstep, sign));
        }
        C2<Real> b[R];
        if (R == 2) {
            b[0] = cadd<Real>(a[0], a[1]);
            b[1] = csub<Real>(a[0], a[1]);
        } else if (R == 4) {
            const C2<Real> s02 = cadd<Real>(a[0], a[2]), d02 = csub<Real>(a[0], a[2]);
            const C2<Real> s13 = cadd<Real>(a[1], a[3]);
            const C2<Real> d13 = mul_isign<Real>(csub<Real>(a[1], a[3]), sign);
            b[0] = cadd<Real>(s02, s13);
            b[1] = cadd<Real>(d02, d13);
            b[2] = csub<Real>(s02, s13);
            b[3] = csub<Real>(d02, d13);
        } else if (R == 3) {
            // w = exp(sign 2 pi i / 3): b1, b2 = a0 - (a1 + a2) / 2 +- i sign sin(2 pi / 3) (a1 - a2)
            const C2<Real> s12 = cadd<Real>(a[1], a[2]);
            const C2<Real> t = csub<Real>(a[0], cscl<Real>(s12, Real(0.5)));
            const C2<Real> u = mul_isign<Real>(cscl<Real>(csub<Real>(a[1], a[2]), Real(SB_S3)), sign);
            b[0] = cadd<Real>(a[0], s12);
            b[1] = cadd<Real>(t, u);
            b[2] = csub<Real>(t, u);
        } else {
            // R == 5, w = exp(sign 2 pi i / 5): b_p and b_(5-p) share the cosine sums and
            // differ in the sign of the sine sums
            const C2<Real> s1 = cadd<Real>(a[1], a[4]), d1 = csub<Real>(a[1], a[4]);
            const C2<Real> s2 = cadd<Real>(a[2], a[3]), d2 = csub<Real>(a[2], a[3]);
            const Real c1 = Real(SB_C51), c2 = Real(SB_C52), n1 = Real(SB_S51), n2 = Real(SB_S52);
            const C2<Real> t1 = cadd<Real>(a[0], cadd<Real>(cscl<Real>(s1, c1), cscl<Real>(s2, c2)));
            const C2<Real> t2 = cadd<Real>(a[0], cadd<Real>(cscl<Real>(s1, c2), cscl<Real>(s2, c1)));
            const C2<Real> u1 = mul_isign<Real>(cadd<Real>(cscl<Real>(d1, n1), cscl<Real>(d2, n2)), sign);
            const C2<Real> u2 = mul_isign<Real>(csub<Real>(cscl<Real>(d1, n2), cscl<Real>(d2, n1)), sign);
            b[0] = cadd<Real>(a[0], cadd<Real>(s1, s2));
            b[1] = cadd<Real>(t1, u1);
            b[4] = csub<Real>(t1, u1);
            b[2] = cadd<Real>(t2, u2);
            b[3] = csub<Real>(t2, u2);
        }
#pragma unroll
        for (int p = 0; p < R; ++p) d0[(j - k) * R + k + p * L] = b[p];
    }
}

// Stockham FFTs of `cols` sequences of length n (= product of radices) in shared
// memory; returns the buffer that holds the natural-order results (A or B).
template <typename Real>
__device__ C2<Real> *stockham(C2<Real> *A, C2<Real> *B, int n, int cols, const int *radices,
                              int nr, const C2<Real> *tw, int sign) {
    int L = 1;
    C2<Real> *src = A, *dst = B;
    for (int s = 0; s < nr; ++s) {
        const int R = radices[s];
        switch (R) {
            case 2: stage<Real, 2>(src, dst, n, cols, L, tw, sign); break;
            case 3: stage<Real, 3>(src, dst, n, cols, L, tw, sign); break;
            case 4: stage<Real, 4>(src, dst, n, cols, L, tw, sign); break;
            case 5: stage<Real, 5>(src, dst, n, cols, L, tw, sign); break;
            default: break;
        }
        __syncthreads();
        L *= R;
        C2<Real> *t = src; src = dst; dst = t;
    }
    return src;
}

// Block b of pass 1 holds columns [b0, b0 + cols1) of instance i (b0 = (b - blk1[i]) cols1),
// block c of pass 2 rows [c0, c0 + cols2); each instance works on its own grid_base.
// Shared memory: A and B (cols x n each), then the length-n twiddles.
template <typename Real>
__global__ void __launch_bounds__(256)
k_fft_pass1(const C2<Real> *__restrict__ X_all, C2<Real> *__restrict__ Z_all,
            FftLaunch<FftPlanDev> L, int sign) {
    extern __shared__ unsigned char smem_raw[];
    const int inst = block_instance(L.blk1, L.ninst, blockIdx.x);
    const FftPlanDev &F = L.inst[inst];
    const C2<Real> *__restrict__ X = X_all + F.grid_base;
    C2<Real> *__restrict__ Z = Z_all + F.grid_base;
    const int n = F.n1, n2 = F.n2;
    const int b0 = (blockIdx.x - L.blk1[inst]) * F.cols1;
    const int cols = min(F.cols1, n2 - b0);
    C2<Real> *A = reinterpret_cast<C2<Real> *>(smem_raw);
    C2<Real> *B = A + cols * n;
    C2<Real> *tw = B + cols * n;
    const C2<Real> *tw1 = static_cast<const C2<Real> *>(F.tw1);
    const C2<Real> *twN = static_cast<const C2<Real> *>(F.twN);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {   // element (a, b0 + bb)
        const int a = e / cols, bb = e - a * cols;
        A[bb * n + a] = X[(long long)n2 * a + b0 + bb];
    }
    for (int a = threadIdx.x; a < n; a += blockDim.x) tw[a] = tw1[a];
    __syncthreads();
    const C2<Real> *res = stockham<Real>(A, B, n, cols, F.r1, F.nr1, tw, sign);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int bb = e / n, c = e - bb * n, b = b0 + bb;
        Z[(long long)b * n + c] = cmul<Real>(res[e], twid<Real>(twN, b * c, sign));
    }
}

template <typename Real>
__global__ void __launch_bounds__(256)
k_fft_pass2(const C2<Real> *__restrict__ Z_all, C2<Real> *__restrict__ Y_all,
            FftLaunch<FftPlanDev> L, int sign) {
    extern __shared__ unsigned char smem_raw[];
    const int inst = block_instance(L.blk2, L.ninst, blockIdx.x);
    const FftPlanDev &F = L.inst[inst];
    const C2<Real> *__restrict__ Z = Z_all + F.grid_base;
    C2<Real> *__restrict__ Y = Y_all + F.grid_base;
    const int n = F.n2, n1 = F.n1;
    const int c0 = (blockIdx.x - L.blk2[inst]) * F.cols2;
    const int cols = min(F.cols2, n1 - c0);
    C2<Real> *A = reinterpret_cast<C2<Real> *>(smem_raw);
    C2<Real> *B = A + cols * n;
    C2<Real> *tw = B + cols * n;
    const C2<Real> *tw2 = static_cast<const C2<Real> *>(F.tw2);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {   // element (b, c0 + cc)
        const int b = e / cols, cc = e - b * cols;
        A[cc * n + b] = Z[(long long)b * n1 + c0 + cc];
    }
    for (int b = threadIdx.x; b < n; b += blockDim.x) tw[b] = tw2[b];
    __syncthreads();
    const C2<Real> *res = stockham<Real>(A, B, n, cols, F.r2, F.nr2, tw, sign);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {   // element (d, c0 + cc)
        const int d = e / cols, cc = e - d * cols;
        Y[c0 + cc + (long long)n1 * d] = res[cc * n + d];
    }
}

// The FFT of a single instance as one launch of a thread-block cluster, the grid in
// distributed shared memory (the structure of k_fft_cluster_df in kern_grid_df.cu): pass 1
// on CTA r's columns into its own shared memory, a cluster barrier, the rows gathered from
// every CTA's shared memory, a second barrier, pass 2 on the rows, written out.
template <typename Real>
__global__ void __cluster_dims__(FFT_CLUSTER, 1, 1) __launch_bounds__(FFT_CLUSTER_THREADS)
k_fft_cluster(const C2<Real> *__restrict__ X, C2<Real> *__restrict__ Y, FftLaunch<FftPlanDev> L,
              int sign) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ unsigned char smem_raw[];
    const int r = (int)cl.block_rank();
    const FftPlanDev &F = L.inst[0];
    const int n1 = F.n1, n2 = F.n2;
    const int per1 = (n2 + FFT_CLUSTER - 1) / FFT_CLUSTER, per2 = (n1 + FFT_CLUSTER - 1) / FFT_CLUSTER;
    const int cap = max(per1 * n1, per2 * n2);
    C2<Real> *buf0 = reinterpret_cast<C2<Real> *>(smem_raw);
    C2<Real> *buf1 = buf0 + cap, *buf2 = buf0 + 2 * cap;
    C2<Real> *tw1 = buf0 + 3 * cap, *tw2 = tw1 + n1;
    const C2<Real> *gtw1 = static_cast<const C2<Real> *>(F.tw1);
    const C2<Real> *gtw2 = static_cast<const C2<Real> *>(F.tw2);
    const C2<Real> *twN = static_cast<const C2<Real> *>(F.twN);
    const int b0 = r * per1, cols1 = max(0, min(per1, n2 - b0));
    for (int e = threadIdx.x; e < cols1 * n1; e += blockDim.x) {     // columns b0 + bb
        const int a = e / cols1, bb = e - a * cols1;
        buf0[bb * n1 + a] = X[(long long)n2 * a + b0 + bb];
    }
    for (int a = threadIdx.x; a < n1; a += blockDim.x) tw1[a] = gtw1[a];
    for (int b = threadIdx.x; b < n2; b += blockDim.x) tw2[b] = gtw2[b];
    __syncthreads();
    C2<Real> *res1 = stockham<Real>(buf0, buf1, n1, cols1, F.r1, F.nr1, tw1, sign);
    for (int e = threadIdx.x; e < cols1 * n1; e += blockDim.x) {
        const int bb = e / n1, c = e - bb * n1;
        res1[e] = cmul<Real>(res1[e], twid<Real>(twN, (b0 + bb) * c, sign));
    }
    cl.sync();                                   // every CTA's pass 1 is in its shared memory
    C2<Real> *A2 = res1 == buf0 ? buf1 : buf0;   // the same buffer in every CTA
    const int c0 = r * per2, cols2 = max(0, min(per2, n1 - c0));
    for (int e = threadIdx.x; e < cols2 * n2; e += blockDim.x) {     // rows c0 + cc
        const int b = e / cols2, cc = e - b * cols2;
        const int owner = b / per1;
        const C2<Real> *rem = cl.map_shared_rank(res1, owner);
        A2[cc * n2 + b] = rem[(b - owner * per1) * n1 + c0 + cc];
    }
    cl.sync();                                   // no CTA leaves while its memory is read
    const C2<Real> *res2 = stockham<Real>(A2, buf2, n2, cols2, F.r2, F.nr2, tw2, sign);
    for (int e = threadIdx.x; e < cols2 * n2; e += blockDim.x) {
        const int d = e / cols2, cc = e - d * cols2;
        Y[c0 + cc + (long long)n1 * d] = res2[cc * n2 + d];
    }
}

}  // namespace

template <typename Real>
size_t fft_cluster_smem_real(int n1, int n2) {
    const int per1 = (n2 + FFT_CLUSTER - 1) / FFT_CLUSTER, per2 = (n1 + FFT_CLUSTER - 1) / FFT_CLUSTER;
    const size_t cap = (size_t)std::max(per1 * n1, per2 * n2);
    return sizeof(C2<Real>) * (3 * cap + (size_t)n1 + (size_t)n2);
}

template <typename Real>
cudaError_t prepare_fft_cluster() {
    return cudaFuncSetAttribute(k_fft_cluster<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FFT_CLUSTER_SMEM_MAX);
}

template <typename Real>
cudaError_t launch_fft_cluster(const FftLaunch<FftPlanDev> &F, int n1, int n2, const void *in,
                               void *out, int sign, cudaStream_t s) {
    const size_t sm = fft_cluster_smem_real<Real>(n1, n2);
    if (F.ninst != 1 || sm > FFT_CLUSTER_SMEM_MAX) return cudaErrorInvalidValue;
    k_fft_cluster<Real><<<FFT_CLUSTER, FFT_CLUSTER_THREADS, sm, s>>>(
        static_cast<const C2<Real> *>(in), static_cast<C2<Real> *>(out), F, sign);
    count_launches(1);
    return cudaGetLastError();
}

template size_t fft_cluster_smem_real<double>(int, int);
template size_t fft_cluster_smem_real<float>(int, int);
template cudaError_t prepare_fft_cluster<double>();
template cudaError_t prepare_fft_cluster<float>();
template cudaError_t launch_fft_cluster<double>(const FftLaunch<FftPlanDev> &, int, int,
                                                const void *, void *, int, cudaStream_t);
template cudaError_t launch_fft_cluster<float>(const FftLaunch<FftPlanDev> &, int, int,
                                               const void *, void *, int, cudaStream_t);

template <typename Real>
cudaError_t launch_fft(const FftLaunch<FftPlanDev> &F, const void *in, void *tmp, void *out,
                       int sign, cudaStream_t s) {
    if (F.nblk1 <= 0) return cudaSuccess;
    const size_t sm1 = sizeof(C2<Real>) * F.smem1;
    const size_t sm2 = sizeof(C2<Real>) * F.smem2;
    if (sm1 > 48 * 1024)
        cudaFuncSetAttribute(k_fft_pass1<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm1);
    if (sm2 > 48 * 1024)
        cudaFuncSetAttribute(k_fft_pass2<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm2);
    k_fft_pass1<Real><<<F.nblk1, 256, sm1, s>>>(static_cast<const C2<Real> *>(in),
                                                static_cast<C2<Real> *>(tmp), F, sign);
    k_fft_pass2<Real><<<F.nblk2, 256, sm2, s>>>(static_cast<const C2<Real> *>(tmp),
                                                static_cast<C2<Real> *>(out), F, sign);
    count_launches(2);
    return cudaGetLastError();
}

template cudaError_t launch_fft<double>(const FftLaunch<FftPlanDev> &, const void *, void *,
                                        void *, int, cudaStream_t);
template cudaError_t launch_fft<float>(const FftLaunch<FftPlanDev> &, const void *, void *,
                                       void *, int, cudaStream_t);

}  // namespace nnfft
