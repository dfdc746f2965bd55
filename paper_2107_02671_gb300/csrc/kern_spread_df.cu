// kern_spread_df.cu -- the fp64 path's point kernels (cell moments of step 1 and
// point evaluation of step 4) in split precision for GB300, whose FP64 pipe runs
// at 1/64 of the FP32 rate.
//
// The Chebyshev degrees of the window series carry geometrically decreasing
// weights kappa_d = max_t |coef[t][d]| (at m = 8: 0.9, 0.2, 3e-2, 2e-3, 2e-4, 2e-5,
// 1e-6, 1e-7, 6e-9, ...).  An error u in the degree-d term of a point costs at most
// kappa_d * u relative to ||f||_1, so
//   * degrees d < B = D/2 are computed in double-float arithmetic (unevaluated sums
//     hi + lo of two floats, about 48 bits: FMA-based exact products and TwoSum
//     accumulation), and
//   * degrees d >= B in plain FP32,
// which keeps the worst-case error near 1e-13 and the typical error near 1e-16
// (the plan checks kappa_d <= 2e-7 for d >= B before choosing these kernels).
// The complex128 inputs are split into float pairs with integer bit operations and
// the results are assembled into doubles with integer bit operations plus one FP64
// add, so a point costs ~2 FP64 instructions instead of ~40.
#include "internal.h"

namespace nnfft {

namespace {

struct df {
    float h, l;
};

// exact product a*b as an unevaluated pair (a.l*b.l dropped: below 2^-48 |a b|)
__device__ __forceinline__ df df_mul(df a, df b) {
    df r;
    r.h = a.h * b.h;
    float e = fmaf(a.h, b.h, -r.h);
    e = fmaf(a.h, b.l, e);
    r.l = fmaf(a.l, b.h, e);
    return r;
}

// s += p: TwoSum on the high parts, low parts accumulated
__device__ __forceinline__ void df_acc(df &s, df p) {
    const float t = s.h + p.h;
    const float bp = t - s.h;
    const float e = (s.h - (t - bp)) + (p.h - bp);
    s.l = s.l + (e + p.l);
    s.h = t;
}

// renormalise so that |l| <= ulp(h)/2 (Fast2Sum, |h| >= |l|)
__device__ __forceinline__ df df_norm(df a) {
    df r;
    r.h = a.h + a.l;
    r.l = a.l - (r.h - a.h);
    return r;
}

// Chebyshev recurrence T_{d+1} = (2y) T_d - T_{d-1} in double-float
__device__ __forceinline__ df df_rec(df y2, df t1, df t0) {
    const df p = df_mul(y2, t1);
    const float s = p.h - t0.h;
    const float bp = s - p.h;
    const float e = (p.h - (s - bp)) + (-t0.h - bp);
    df r;
    r.h = s;
    r.l = (p.l - t0.l) + e;
    return df_norm(r);
}

// double -> (hi, lo) floats with integer operations only: hi keeps the top 24
// significant bits (truncated), lo the next 24 (rounded), so hi + lo = x to 2^-48.
// Values below 2^-100 in magnitude become 0 (their contribution is far below the
// result's rounding); inputs are finite.
__device__ __forceinline__ df split_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int ex = (int)((hi >> 20) & 0x7ffu);
    const unsigned mh = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const bool ok = ex > 1023 - 100 && ex < 1023 + 127;
    df r;
    r.h = ok ? __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | mh) : 0.0f;
    // remainder: 29 low mantissa bits, weight 2^(ex - 1075)
    const float rem = __uint2float_rn(lo & 0x1fffffffu);
    const int se = ex - 1075 + 127;                 // biased float exponent of 2^(ex-1075)
    const float scale = se > 0 ? __uint_as_float((unsigned)se << 23) : 0.0f;
    const float lv = rem * scale;
    r.l = ok ? (sign ? -lv : lv) : 0.0f;
    return r;
}

// float -> double with integer operations (exact; zero and subnormals -> signed 0)
__device__ __forceinline__ double float_to_double_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned ex = (u >> 23) & 0xffu;
    const unsigned man = u & 0x7fffffu;
    const unsigned hi = ex ? (sign | ((ex + 896u) << 20) | (man >> 3)) : sign;
    const unsigned lo = ex ? ((man & 7u) << 29) : 0u;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

__device__ __forceinline__ double df_to_double(df a) {
    return float_to_double_bits(a.h) + float_to_double_bits(a.l);
}

// reduce-scatter of 32 double-float values per lane: afterwards lane L holds the
// warp sum of value L
template <int O>
__device__ __forceinline__ void rs_step_df(df (&v)[32], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const df send = up ? v[i] : v[O + i];
        df keep = up ? v[O + i] : v[i];
        df other;
        other.h = __shfl_xor_sync(0xffffffffu, send.h, O);
        other.l = __shfl_xor_sync(0xffffffffu, send.l, O);
        df_acc(keep, other);
        v[i] = df_norm(keep);
    }
}

// ---------------------------------------------------------------------------------
// Cell moments, split precision.  Same work decomposition as the fp64 kernel: one
// warp per work item, lanes stride over the item's points, reduce-scatter.
// ys2 holds each sorted local coordinate y as a float pair (hi, lo).
// ---------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256)
k_moments_df(SideK<double> S, const float2 *__restrict__ ys2, const double2 *__restrict__ vals,
             double2 *__restrict__ P) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int item = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= *S.nitems) return;
    const int pb = S.item_pb[item], pe = S.item_pe[item];
    df ar[B], ai[B];
    float br[F], bi[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = {0.f, 0.f}; ai[d] = {0.f, 0.f}; }
#pragma unroll
    for (int d = 0; d < F; ++d) { br[d] = 0.f; bi[d] = 0.f; }
    for (int p = pb + lane; p < pe; p += 32) {
        const float2 yy = ys2[p];
        const double2 v = vals[S.perm[p]];
        const df fr = split_double(v.x), fi = split_double(v.y);
        const df y = {yy.x, yy.y};
        const df y2 = {2.f * yy.x, 2.f * yy.y};
        df_acc(ar[0], fr);
        df_acc(ai[0], fi);
        df_acc(ar[1], df_mul(fr, y));
        df_acc(ai[1], df_mul(fi, y));
        df t0 = {1.f, 0.f}, t1 = y;
#pragma unroll
        for (int d = 2; d < B; ++d) {
            const df t = df_rec(y2, t1, t0);
            df_acc(ar[d], df_mul(fr, t));
            df_acc(ai[d], df_mul(fi, t));
            t0 = t1;
            t1 = t;
        }
        float g0 = t0.h, g1 = t1.h;
        const float yf2 = y2.h;
#pragma unroll
        for (int d = 0; d < F; ++d) {
            const float t = fmaf(yf2, g1, -g0);
            br[d] = fmaf(fr.h, t, br[d]);
            bi[d] = fmaf(fi.h, t, bi[d]);
            g0 = g1;
            g1 = t;
        }
    }
    static_assert(2 * D <= 32, "split-precision moments need 2D <= 32");
    df vv[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) vv[i] = {0.f, 0.f};
#pragma unroll
    for (int d = 0; d < B; ++d) {
        vv[d] = df_norm(ar[d]);
        vv[D + d] = df_norm(ai[d]);
    }
#pragma unroll
    for (int d = 0; d < F; ++d) {
        vv[B + d] = {br[d], 0.f};
        vv[D + B + d] = {bi[d], 0.f};
    }
    rs_step_df<16>(vv, lane);
    rs_step_df<8>(vv, lane);
    rs_step_df<4>(vv, lane);
    rs_step_df<2>(vv, lane);
    rs_step_df<1>(vv, lane);
    double *Pr = reinterpret_cast<double *>(P + (long long)item * D);
    if (lane < D) Pr[2 * lane] = df_to_double(vv[0]);
    else if (lane < 2 * D) Pr[2 * (lane - D) + 1] = df_to_double(vv[0]);
}

// ---------------------------------------------------------------------------------
// Point evaluation, split precision.  Q2 holds each cell's D complex coefficients as
// float4 (re.hi, re.lo, im.hi, im.lo); the degree-d < B part is summed in
// double-float, the rest in FP32, and the pair is assembled into a double.
// ---------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256)
k_eval_df(SideK<double> S, const float2 *__restrict__ ys2, const float4 *__restrict__ Q2,
          double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int item = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item >= *S.nitems) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = Q2[(long long)c * D + d];
        if (d < B) {
            qr[d < B ? d : 0] = {q.x, q.y};
            qi[d < B ? d : 0] = {q.z, q.w};
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
    for (int p = pb + lane; p < pe; p += 32) {
        const float2 yy = ys2[p];
        const df y = {yy.x, yy.y};
        const df y2 = {2.f * yy.x, 2.f * yy.y};
        df sr = qr[0], si = qi[0];
        df_acc(sr, df_mul(qr[1], y));
        df_acc(si, df_mul(qi[1], y));
        df t0 = {1.f, 0.f}, t1 = y;
#pragma unroll
        for (int d = 2; d < B; ++d) {
            const df t = df_rec(y2, t1, t0);
            df_acc(sr, df_mul(qr[d], t));
            df_acc(si, df_mul(qi[d], t));
            t0 = t1;
            t1 = t;
        }
        float g0 = t0.h, g1 = t1.h, ur = 0.f, ui = 0.f;
        const float yf2 = y2.h;
#pragma unroll
        for (int d = 0; d < F; ++d) {
            const float t = fmaf(yf2, g1, -g0);
            ur = fmaf(fr[d], t, ur);
            ui = fmaf(fi[d], t, ui);
            g0 = g1;
            g1 = t;
        }
        df_acc(sr, {ur, 0.f});
        df_acc(si, {ui, 0.f});
        double2 o;
        o.x = df_to_double(df_norm(sr));
        o.y = df_to_double(df_norm(si));
        out[S.perm[p]] = o;
    }
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

bool df_supported_degree(int D) { return D == 8 || D == 10 || D == 12 || D == 14 || D == 16; }

#define NNFFT_DISPATCH_DF(D_, ...)                              \
    switch (D_) {                                               \
        case 8: { constexpr int DD = 8; __VA_ARGS__; } break;   \
        case 10: { constexpr int DD = 10; __VA_ARGS__; } break; \
        case 12: { constexpr int DD = 12; __VA_ARGS__; } break; \
        case 14: { constexpr int DD = 14; __VA_ARGS__; } break; \
        case 16: { constexpr int DD = 16; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                  \
    }

cudaError_t launch_moments_df(const SideK<double> &S, const void *vals, void *P, void *Pc,
                              cudaStream_t s) {
    if (S.max_items > 0) {
        const int blocks = cdiv((long long)S.max_items * 32, 256);
        NNFFT_DISPATCH_DF(S.D, (k_moments_df<DD><<<blocks, 256, 0, s>>>(
                                   S, reinterpret_cast<const float2 *>(S.ys),
                                   static_cast<const double2 *>(vals), static_cast<double2 *>(P))));
        count_launches(1);
    }
    return launch_cell_fold<double>(S, P, Pc, s);
}

cudaError_t launch_eval_df(const SideK<double> &S, const void *Q2, void *out, cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    const int blocks = cdiv((long long)S.max_items * 32, 256);
    NNFFT_DISPATCH_DF(S.D, (k_eval_df<DD><<<blocks, 256, 0, s>>>(
                               S, reinterpret_cast<const float2 *>(S.ys),
                               static_cast<const float4 *>(Q2), static_cast<double2 *>(out))));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnfft
