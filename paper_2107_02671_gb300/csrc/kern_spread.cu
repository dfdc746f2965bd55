// kern_spread.cu -- the point-sized hot loops of Algorithm 2.2 (step 1, the spread,
// and step 4, the gather) and the grid-sized cell convolutions that connect them
// to the FFT grid.
//
// Window representation.  For a node with u = N_j * node (cell c = floor(u),
// z = u - c) the 2m taps of Algorithm 2.2 step 0 (ii)/(iii) are the window
// values w_t(z) = omega((t - m + 1 - z)/m), t = 0..2m-1, on grid positions
// p = c - m + 1 + t.  Each w_t is stored as a degree D-1 Chebyshev series in
// y = 2z - 1 (fitted at plan time to the sinh window's own accuracy floor).
// Then
//   spread (step 1):  g_p = sum_t sum_d coef[t][d] * P_{p+m-1-t}[d],
//                     P_c[d] = sum_{k in cell c} f_k T_d(y_k)   ("cell moments")
//   gather (step 4):  s_j = sum_d T_d(y_j) * Q_{c_j}[d],
//                     Q_c[d] = sum_t coef[t][d] * h_{c-m+1+t}    ("cell windows")
// so the per-point work is O(D) instead of O(m * D): the point kernels only
// accumulate or evaluate one Chebyshev series per point, and the O(m D) tap
// algebra happens once per cell on the small grid.
#include "internal.h"

namespace nnfft {

namespace {

template <typename Real>
__device__ __forceinline__ C2<Real> mk2(Real a, Real b) {
    C2<Real> r;
    r.x = a;
    r.y = b;
    return r;
}

__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// T_0..T_{D-1} at y (three-term recurrence T_{d+1} = 2y T_d - T_{d-1}).
template <typename Real, int D>
__device__ __forceinline__ void cheb(Real y, Real (&T)[D]) {
    T[0] = Real(1);
    if (D > 1) T[1] = y;
    const Real y2 = y + y;
#pragma unroll
    for (int d = 2; d < D; ++d) T[d] = fma(y2, T[d - 1], -T[d - 2]);
}

// ---------------------------------------------------------------------------------
// Cell moments (spread, step 1).  One warp per work item (<= ITEM_CAP sorted
// points of one cell): lanes stride over the points, accumulate
// sum_k val_k * T_d(y_k) in registers, and the warp reduces the D complex sums.
// HAS_R: the values are first multiplied by the cell's fit of 1/phihat1
// (adjoint: the division by phihat1(N* x_j) that precedes the transposed gather).
// ---------------------------------------------------------------------------------
template <typename Real, int D, bool HAS_R>
__global__ void __launch_bounds__(256)
k_moments(SideK<Real> S, const C2<Real> *__restrict__ vals, C2<Real> *__restrict__ P) {
    const int item = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= *S.nitems) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    Real r[NR];
    if (HAS_R) {
#pragma unroll
        for (int e = 0; e < NR; ++e) r[e] = S.rfit[(long long)c * NR + e];
    }
    Real ar[D], ai[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { ar[d] = Real(0); ai[d] = Real(0); }
    for (int p = pb + lane; p < pe; p += 32) {
        const Real y = S.ys[p];
        C2<Real> v = vals[S.perm[p]];
        Real T[D];
        cheb<Real, D>(y, T);
        if (HAS_R) {
            Real sc = Real(0);
#pragma unroll
            for (int e = 0; e < NR; ++e) sc = fma(r[e], T[e], sc);
            v.x *= sc;
            v.y *= sc;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
            ar[d] = fma(v.x, T[d], ar[d]);
            ai[d] = fma(v.y, T[d], ai[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
        ar[d] = warp_sum(ar[d]);
        ai[d] = warp_sum(ai[d]);
    }
#pragma unroll
    for (int d = 0; d < D; ++d)
        if (lane == d) P[(long long)item * D + d] = mk2<Real>(ar[d], ai[d]);
}

// ---------------------------------------------------------------------------------
// Spread convolution: one thread per FFT-buffer index q in [0, N2).  Sums the
// taps of every cell whose support covers a grid position p == q (mod N2):
//   g_p = scale(p) * sum_t sum_d coef[t][d] * sum_{items of cell p+m-1-t} P[item][d].
// v side (forward): scale = 1/(N1 N2 phihat2(l)) (steps 2-3 factors folded in).
// x side (adjoint): scale = 1.  Positions outside every support give 0, which
// is the zero padding of step 3.
// ---------------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(128)
k_spread_conv(SideK<Real> S, const C2<Real> *__restrict__ P, const Real *__restrict__ scale,
              long long scale_off, long long scale_len, int N2, C2<Real> *__restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    Real *coef = reinterpret_cast<Real *>(smem_raw);
    const int m = S.m, D = S.D, ntap = 2 * S.m;
    for (int i = threadIdx.x; i < ntap * D; i += blockDim.x) coef[i] = S.coef[i];
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N2) return;
    const long long qc = q < N2 / 2 ? q : (long long)q - N2;
    const long long p_lo = S.c_lo - m + 1, p_hi = S.c_lo + S.ncell - 1 + m;
    Real accr = Real(0), acci = Real(0);
    for (int wrap = -1; wrap <= 1; ++wrap) {
        const long long p = qc + (long long)wrap * N2;
        if (p < p_lo || p > p_hi) continue;
        Real gr = Real(0), gi = Real(0);
        for (int t = 0; t < ntap; ++t) {
            const long long ic = p + m - 1 - t - S.c_lo;
            if (ic < 0 || ic >= S.ncell) continue;
            const int i0 = S.item_off[ic], i1 = S.item_off[ic + 1];
            const Real *ct = coef + t * D;
            for (int it = i0; it < i1; ++it) {
                const C2<Real> *Pi = P + (long long)it * D;
                for (int d = 0; d < D; ++d) {
                    const C2<Real> pv = Pi[d];
                    gr = fma(ct[d], pv.x, gr);
                    gi = fma(ct[d], pv.y, gi);
                }
            }
        }
        if (scale != nullptr) {
            const long long si = p + scale_off;
            const Real sc = (si >= 0 && si < scale_len) ? scale[si] : Real(0);
            gr *= sc;
            gi *= sc;
        }
        accr += gr;
        acci += gi;
    }
    out[q] = mk2<Real>(accr, acci);
}

// ---------------------------------------------------------------------------------
// Gather convolution: one thread per cell c of the gathering side,
//   Q_c[d] = sum_t coef[t][d] * scale(p) * buf[p mod N2],  p = c - m + 1 + t.
// x side (forward): buf = h of step 3, scale = 1.
// v side (adjoint): buf = the +sign FFT of the x-side spread, scale = 1/(N1 N2 phihat2(l)).
// ---------------------------------------------------------------------------------
template <typename Real, int D>
__global__ void __launch_bounds__(128)
k_gather_conv(SideK<Real> S, const C2<Real> *__restrict__ buf, const Real *__restrict__ scale,
              long long scale_off, long long scale_len, int N2, C2<Real> *__restrict__ Q) {
    extern __shared__ unsigned char smem_raw[];
    Real *coef = reinterpret_cast<Real *>(smem_raw);
    const int m = S.m, ntap = 2 * S.m;
    for (int i = threadIdx.x; i < ntap * D; i += blockDim.x) coef[i] = S.coef[i];
    __syncthreads();
    const int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic >= S.ncell) return;
    const long long c = S.c_lo + ic;
    Real qr[D], qi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { qr[d] = Real(0); qi[d] = Real(0); }
    for (int t = 0; t < ntap; ++t) {
        const long long p = c - m + 1 + t;
        long long qidx = p % N2;
        if (qidx < 0) qidx += N2;
        C2<Real> h = buf[qidx];
        if (scale != nullptr) {
            const long long si = p + scale_off;
            const Real sc = (si >= 0 && si < scale_len) ? scale[si] : Real(0);
            h.x *= sc;
            h.y *= sc;
        }
        const Real *ct = coef + t * D;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            qr[d] = fma(ct[d], h.x, qr[d]);
            qi[d] = fma(ct[d], h.y, qi[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) Q[(long long)ic * D + d] = mk2<Real>(qr[d], qi[d]);
}

// ---------------------------------------------------------------------------------
// Point evaluation (gather, step 4 and the output division).  One warp per work
// item; the cell's D complex window coefficients are loaded once (uniform loads)
// and every lane evaluates sum_d T_d(y) Q_c[d] for its points.  HAS_R: multiply by
// the cell's fit of 1/phihat1(N* x) (forward output division).
// ---------------------------------------------------------------------------------
template <typename Real, int D, bool HAS_R>
__global__ void __launch_bounds__(256)
k_eval(SideK<Real> S, const C2<Real> *__restrict__ Q, C2<Real> *__restrict__ out) {
    const int item = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= *S.nitems) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    Real qr[D], qi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const C2<Real> q = Q[(long long)c * D + d];
        qr[d] = q.x;
        qi[d] = q.y;
    }
    Real r[NR];
    if (HAS_R) {
#pragma unroll
        for (int e = 0; e < NR; ++e) r[e] = S.rfit[(long long)c * NR + e];
    }
    for (int p = pb + lane; p < pe; p += 32) {
        const Real y = S.ys[p];
        Real T[D];
        cheb<Real, D>(y, T);
        Real sr = Real(0), si = Real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            sr = fma(qr[d], T[d], sr);
            si = fma(qi[d], T[d], si);
        }
        if (HAS_R) {
            Real sc = Real(0);
#pragma unroll
            for (int e = 0; e < NR; ++e) sc = fma(r[e], T[e], sc);
            sr *= sc;
            si *= sc;
        }
        out[S.perm[p]] = mk2<Real>(sr, si);
    }
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

// D >= NR is required: the 1/phihat1 fit reuses T_0..T_{NR-1} of the window series.
bool supported_degree(int D) {
    return D == 8 || D == 10 || D == 12 || D == 14 || D == 16 || D == 20;
}

#define NNFFT_DISPATCH_D(D_, ...)                         \
    switch (D_) {                                         \
        case 8: { constexpr int DD = 8; __VA_ARGS__; } break;   \
        case 10: { constexpr int DD = 10; __VA_ARGS__; } break; \
        case 12: { constexpr int DD = 12; __VA_ARGS__; } break; \
        case 14: { constexpr int DD = 14; __VA_ARGS__; } break; \
        case 16: { constexpr int DD = 16; __VA_ARGS__; } break; \
        case 20: { constexpr int DD = 20; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;            \
    }

template <typename Real>
cudaError_t launch_moments(const SideK<Real> &S, const void *vals, void *P, cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    const int blocks = cdiv((long long)S.max_items * 32, 256);
    const C2<Real> *v = static_cast<const C2<Real> *>(vals);
    C2<Real> *Pp = static_cast<C2<Real> *>(P);
    if (S.rfit) {
        NNFFT_DISPATCH_D(S.D, (k_moments<Real, DD, true><<<blocks, 256, 0, s>>>(S, v, Pp)));
    } else {
        NNFFT_DISPATCH_D(S.D, (k_moments<Real, DD, false><<<blocks, 256, 0, s>>>(S, v, Pp)));
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_spread_conv(const SideK<Real> &S, const void *P, const Real *scale,
                               long long scale_off, long long scale_len, int N2, void *out,
                               cudaStream_t s) {
    const size_t sm = sizeof(Real) * 2 * S.m * S.D;
    k_spread_conv<Real><<<cdiv(N2, 128), 128, sm, s>>>(
        S, static_cast<const C2<Real> *>(P), scale, scale_off, scale_len, N2,
        static_cast<C2<Real> *>(out));
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_gather_conv(const SideK<Real> &S, const void *buf, const Real *scale,
                               long long scale_off, long long scale_len, int N2, void *Q,
                               cudaStream_t s) {
    if (S.ncell <= 0) return cudaSuccess;
    const size_t sm = sizeof(Real) * 2 * S.m * S.D;
    const C2<Real> *b = static_cast<const C2<Real> *>(buf);
    C2<Real> *q = static_cast<C2<Real> *>(Q);
    NNFFT_DISPATCH_D(S.D, (k_gather_conv<Real, DD><<<cdiv(S.ncell, 128), 128, sm, s>>>(
                              S, b, scale, scale_off, scale_len, N2, q)));
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_eval(const SideK<Real> &S, const void *Q, void *out, cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    const int blocks = cdiv((long long)S.max_items * 32, 256);
    const C2<Real> *q = static_cast<const C2<Real> *>(Q);
    C2<Real> *o = static_cast<C2<Real> *>(out);
    if (S.rfit) {
        NNFFT_DISPATCH_D(S.D, (k_eval<Real, DD, true><<<blocks, 256, 0, s>>>(S, q, o)));
    } else {
        NNFFT_DISPATCH_D(S.D, (k_eval<Real, DD, false><<<blocks, 256, 0, s>>>(S, q, o)));
    }
    count_launches(1);
    return cudaGetLastError();
}

#define NNFFT_INST(R)                                                                      \
    template cudaError_t launch_moments<R>(const SideK<R> &, const void *, void *,         \
                                           cudaStream_t);                                  \
    template cudaError_t launch_spread_conv<R>(const SideK<R> &, const void *, const R *,  \
                                               long long, long long, int, void *,         \
                                               cudaStream_t);                              \
    template cudaError_t launch_gather_conv<R>(const SideK<R> &, const void *, const R *,  \
                                               long long, long long, int, void *,         \
                                               cudaStream_t);                              \
    template cudaError_t launch_eval<R>(const SideK<R> &, const void *, void *, cudaStream_t);

NNFFT_INST(double)
NNFFT_INST(float)

}  // namespace nnfft
