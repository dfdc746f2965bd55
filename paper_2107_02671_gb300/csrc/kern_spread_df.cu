// kern_spread_df.cu -- the fp64 path's point kernels (cell moments of step 1 and
// point evaluation of step 4) in split precision for GB300, whose FP64 pipe runs
// at 1/64 of the FP32 rate.
//
// The Chebyshev degrees of the window series carry geometrically decreasing
// weights kappa_d = max_t |coef[t][d]| (at m = 8: 0.9, 0.2, 3e-2, 2e-3, 2e-4, 2e-5,
// 1e-6, 1e-7, 6e-9, ...).  An error u in the degree-d term of a point costs at most
// kappa_d * u relative to ||f||_1, so
//   * degrees d < B = D/2 are computed in double-float arithmetic (df.cuh), and
//   * degrees d >= B in plain FP32,
// which keeps the worst-case error near 1e-13 and the typical error near 1e-16
// (the plan checks kappa_d <= 2e-7 for d >= B before choosing these kernels).
// The complex128 inputs are split into float pairs with integer bit operations and
// the outputs assembled into doubles with integer operations plus one FP64 add, so a
// point costs ~2 FP64 instructions instead of ~40.  Per-item moments leave as
// double-float complex values (float4) for the double-float grid stage.
#include "df.cuh"
#include "internal.h"
#include "tma.cuh"

namespace nnfft {

namespace {

using namespace dfa;

constexpr int PPL = ITEM_CAP / 32;   // points per lane of a work item

// Chebyshev recurrence T_{d+1} = (2y) T_d - T_{d-1} in double-float, TwoSum on the high
// parts, the result not renormalised: its low part is a sum of rounding errors of O(1)
// quantities (|T_d| <= 1), so it stays within a few 2^-24 in absolute terms, and the next
// product and the accumulations take unnormalised pairs at the same 2^-48 absolute accuracy.
// (Measured against a Fast2Sum renormalisation per step: graph step 155.0 -> 154.2-154.5 us
// with the two-set 8-lane moments, 159.9 -> 156.2-156.5 us with the 8-lane team kernel.)
__device__ __forceinline__ df df_rec(df y2, df t1, df t0) {
    const df p = mul_u(y2, t1);
    const float s = p.h - t0.h;
    const float bp = s - p.h;
    const float e = (p.h - (s - bp)) + (-t0.h - bp);
    return mk(s, (p.l - t0.l) + e);
}

// reduce-scatter of 32 double-float values per lane: afterwards lane L holds the
// warp sum of value L
template <int O>
__device__ __forceinline__ void rs_step_df(df (&v)[32], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const df send = up ? v[i] : v[O + i];
        const df keep = up ? v[O + i] : v[i];
        df other;
        other.h = __shfl_xor_sync(0xffffffffu, send.h, O);
        other.l = __shfl_xor_sync(0xffffffffu, send.l, O);
        v[i] = add_lazy(keep, other);
    }
}

// One point's contribution to the moments: degrees d < B in double-float, the rest in
// FP32 from the high parts (the arithmetic of every moments kernel below).
template <int B, int F>
__device__ __forceinline__ void moments_point(float2 yy, double2 v, df (&ar)[B], df (&ai)[B],
                                              float (&br)[F], float (&bi)[F]) {
    const df fr = split_double(v.x), fi = split_double(v.y);
    const df y = mk(yy.x, yy.y);
    const df y2 = mk(2.f * yy.x, 2.f * yy.y);
    acc(ar[0], fr);
    acc(ai[0], fi);
    acc(ar[1], mul_u(fr, y));
    acc(ai[1], mul_u(fi, y));
    df t0 = mk(1.f), t1 = y;
#pragma unroll
    for (int d = 2; d < B; ++d) {
        const df t = df_rec(y2, t1, t0);
        acc(ar[d], mul_u(fr, t));
        acc(ai[d], mul_u(fi, t));
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

// One point's value sum_d Q[d] T_d(y) (double-float for d < B, FP32 above), as a double pair.
template <int B, int F>
__device__ __forceinline__ double2 eval_point(float2 yy, const df (&qr)[B], const df (&qi)[B],
                                              const float (&fr)[F], const float (&fi)[F]) {
    const df y = mk(yy.x, yy.y);
    const df y2 = mk(2.f * yy.x, 2.f * yy.y);
    df sr = qr[0], si = qi[0];
    acc(sr, mul_u(qr[1], y));
    acc(si, mul_u(qi[1], y));
    df t0 = mk(1.f), t1 = y;
#pragma unroll
    for (int d = 2; d < B; ++d) {
        const df t = df_rec(y2, t1, t0);
        acc(sr, mul_u(qr[d], t));
        acc(si, mul_u(qi[d], t));
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
    acc(sr, mk(ur));
    acc(si, mk(ui));
    double2 o;
    o.x = to_double(norm(sr));
    o.y = to_double(norm(si));
    return o;
}

// Work item of warp w (or of half-warp w): w itself, or the w-th big item; -1 past the end.
__device__ __forceinline__ int big_item(const SideK<double> &S, int w) {
    if (S.list_big) return w < *S.n_big ? S.list_big[w] : -1;
    return w < *S.nitems ? w : -1;
}

// ---------------------------------------------------------------------------------
// Cell moments, split precision, one warp per work item: lanes stride over the item's
// points (up to 8 each, all loads issued first), then a 32-lane reduce-scatter of the 2D
// double-float moments.  Fewer serial points per lane than the half-warp form below
// (shorter accumulation chains), more exchange work per point; which is faster depends on
// the cell sizes and occupancy, so the plan's autotuner picks.
// P4[item*D + d] = moment d as (re.h, re.l, im.h, im.l).
// ---------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256)
k_moments_df_warp(SideK<double> S, const float2 *__restrict__ ys2, const double2 *__restrict__ vals,
             float4 *__restrict__ P4) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int item = big_item(S, (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5));
    const int lane = threadIdx.x & 31;
    if (item < 0) return;
    const int pb = S.item_pb[item], pe = S.item_pe[item];
    df ar[B], ai[B];
    float br[F], bi[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = mk(0.f); ai[d] = mk(0.f); }
#pragma unroll
    for (int d = 0; d < F; ++d) { br[d] = 0.f; bi[d] = 0.f; }
    // issue every load of the item first (coordinates and indices, then the gathers)
    float2 yv[PPL];
    int jv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int p = pb + lane + 32 * k;
        yv[k] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
        jv[k] = p < pe ? S.perm[p] : -1;
    }
    double2 vv2[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) vv2[k] = jv[k] >= 0 ? vals[jv[k]] : make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        if (pb + 32 * k >= pe) break;                 // warp-uniform: no point in this round
        moments_point<B, F>(yv[k], vv2[k], ar, ai, br, bi);
    }
    static_assert(2 * D <= 32, "split-precision moments need 2D <= 32");
    df vv[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) vv[i] = mk(0.f);
#pragma unroll
    for (int d = 0; d < B; ++d) {
        vv[d] = ar[d];
        vv[D + d] = ai[d];
    }
#pragma unroll
    for (int d = 0; d < F; ++d) {
        vv[B + d] = mk(br[d]);
        vv[D + B + d] = mk(bi[d]);
    }
    rs_step_df<16>(vv, lane);
    rs_step_df<8>(vv, lane);
    rs_step_df<4>(vv, lane);
    rs_step_df<2>(vv, lane);
    rs_step_df<1>(vv, lane);
    float2 *P2 = reinterpret_cast<float2 *>(P4 + (long long)item * D);
    const df r = norm_any(vv[0]);
    if (lane < D) P2[2 * lane] = make_float2(r.h, r.l);
    else if (lane < 2 * D) P2[2 * (lane - D) + 1] = make_float2(r.h, r.l);
}

// ---------------------------------------------------------------------------------
// Cell moments, split precision.  Half a warp (16 lanes) per work item, lanes stride over
// the item's points (up to 16 each, loaded 8 at a time), then a reduce-scatter over the
// 16 lanes.  The 2D moments sit in 16 double-float slots (re of degree d < B at j = d, im
// at j = 8 + d) and 16 FP32 slots (re of degree B + d at j = d, im at 8 + d); each
// exchange step pairs slots that differ in one bit of j, so double-float meets
// double-float and FP32 meets FP32, and after four steps lane s of the half holds slot
// j = s of each kind.  P4[item*D + d] = moment d as (re.h, re.l, im.h, im.l).
// ys2 holds each sorted local coordinate y as a float pair (hi, lo).
// ---------------------------------------------------------------------------------
template <int O>
__device__ __forceinline__ void rs_step_mixed(df (&vd)[16], float (&vf)[16], int sub) {
    const bool up = (sub & O) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const df send = up ? vd[i] : vd[O + i];
        const df keep = up ? vd[O + i] : vd[i];
        df other;
        other.h = __shfl_xor_sync(0xffffffffu, send.h, O);
        other.l = __shfl_xor_sync(0xffffffffu, send.l, O);
        vd[i] = add_lazy(keep, other);
        const float fs = up ? vf[i] : vf[O + i];
        const float fk = up ? vf[O + i] : vf[i];
        vf[i] = fk + __shfl_xor_sync(0xffffffffu, fs, O);
    }
}

constexpr int MOM_LANES = 16;                       // lanes per work item
// points per lane loaded at a time, threads per block (measured at 2^20 points, graph step:
// 4 points and 64-thread blocks 167 us, 8 points and 256-thread blocks 175 us)
constexpr int MOM_CHUNK = 4;
constexpr int MOM_BLOCK = 64;

template <int D>
__global__ void __launch_bounds__(MOM_BLOCK, 2 * 256 / MOM_BLOCK)
k_moments_df_half(SideK<double> S, const float2 *__restrict__ ys2, const double2 *__restrict__ vals,
                  float4 *__restrict__ P4) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    static_assert(B <= 8 && F <= 8, "the slot layout holds at most 8 degrees of each kind");
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int item = big_item(S, gt / MOM_LANES);
    const int sub = threadIdx.x & (MOM_LANES - 1);
    const bool live = item >= 0;                    // both halves of a warp stay for the shuffles
    int pb = 0, pe = 0;
    if (live) {
        pb = S.item_pb[item];
        pe = S.item_pe[item];
    }
    df ar[B], ai[B];
    float br[F], bi[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = mk(0.f); ai[d] = mk(0.f); }
#pragma unroll
    for (int d = 0; d < F; ++d) { br[d] = 0.f; bi[d] = 0.f; }
    for (int c0 = pb; c0 < pe; c0 += MOM_LANES * MOM_CHUNK) {
        float2 yv[MOM_CHUNK];
        int jv[MOM_CHUNK];
#pragma unroll
        for (int k = 0; k < MOM_CHUNK; ++k) {
            const int p = c0 + sub + MOM_LANES * k;
            yv[k] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
        double2 vv2[MOM_CHUNK];
#pragma unroll
        for (int k = 0; k < MOM_CHUNK; ++k) vv2[k] = jv[k] >= 0 ? vals[jv[k]] : make_double2(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < MOM_CHUNK; ++k) {
            if (jv[k] < 0) continue;
            moments_point<B, F>(yv[k], vv2[k], ar, ai, br, bi);
        }
    }
    df vd[16];
    float vf[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) { vd[j] = mk(0.f); vf[j] = 0.f; }
#pragma unroll
    for (int d = 0; d < B; ++d) {
        vd[d] = ar[d];
        vd[8 + d] = ai[d];
    }
#pragma unroll
    for (int d = 0; d < F; ++d) {
        vf[d] = br[d];
        vf[8 + d] = bi[d];
    }
    rs_step_mixed<8>(vd, vf, sub);
    rs_step_mixed<4>(vd, vf, sub);
    rs_step_mixed<2>(vd, vf, sub);
    rs_step_mixed<1>(vd, vf, sub);
    if (!live) return;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + (long long)item * D);
    const int j = sub & 7, part = sub >> 3;          // part 0: real, 1: imaginary
    const df r = norm_any(vd[0]);
    if (j < B) P2[2 * j + part] = make_float2(r.h, r.l);
    if (j < F) P2[2 * (B + j) + part] = make_float2(vf[0], 0.f);
}

// ---------------------------------------------------------------------------------
// Point evaluation, split precision.  Q4 holds each cell's D complex coefficients as
// float4 (re.h, re.l, im.h, im.l); the degree-d < B part is summed in double-float,
// the rest in FP32, and the pair is assembled into a double.
// ---------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256, 3)
k_eval_df(SideK<double> S, const float2 *__restrict__ ys2, const float4 *__restrict__ Q4,
          double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int item = big_item(S, (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5));
    const int lane = threadIdx.x & 31;
    if (item < 0) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = Q4[(long long)c * D + d];
        if (d < B) {
            qr[d < B ? d : 0] = mk(q.x, q.y);
            qi[d < B ? d : 0] = mk(q.z, q.w);
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
    float2 yv[PPL];
    int jv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int p = pb + lane + 32 * k;
        yv[k] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
        jv[k] = p < pe ? S.perm[p] : -1;
    }
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        if (pb + 32 * k >= pe) break;
        const double2 o = eval_point<B, F>(yv[k], qr, qi, fr, fi);
        if (jv[k] >= 0) out[jv[k]] = o;
    }
}

// One warp per work item with the gather convolution of the item's cell done in the warp
// (evaluation lanes value EVAL_GATHER, single instances): lanes t < 2m load and scale the grid
// values h_{c-m+1+t}, lane d < D forms the window sum Q_c[d] = sum_t coef[t][d] h_t and, on
// the x side, lane n the 1/phihat1 fold of the sums -- the arithmetic of k_gather_conv_df
// for one cell, in the same order, so the results are bitwise those of the gather kernel
// followed by k_eval_df -- then the warp evaluates its points as k_eval_df does.  The
// separate gather launch and its per-cell output disappear; a cell with several items is
// convolved once per item.
constexpr int EG_HS = 32;   // grid values a warp stages (2m <= 32)
template <int D>
__global__ void __launch_bounds__(256, 3)
k_eval_gather_df(SideK<double> S, const float2 *__restrict__ ys2, GridLaunch<float2> L,
                 const float4 *__restrict__ buf_all, double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    __shared__ float4 wsm[8][EG_HS + 2 * 16];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = big_item(S, (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5));
    if (item < 0) return;                                        // warp-uniform
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    float2 yv[PPL];
    int jv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {                              // the points' loads first
        const int p = pb + lane + 32 * k;
        yv[k] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
        jv[k] = p < pe ? S.perm[p] : -1;
    }
    const GridInst<float2> G = L.inst[0];
    const float4 *__restrict__ buf = buf_all + G.grid_base;
    const int m = L.m, ntap = 2 * L.m, N2 = G.N2;
    const long long icl = (long long)c - G.cell_base;            // the instance's cell
    float4 *hs = wsm[w], *qa = hs + EG_HS, *qq = qa + 16;
    if (lane < ntap) {
        const long long p = G.c_lo + icl - m + 1 + lane;
        cdf h = ld(buf + wrap_index(p, N2));
        if (G.scale != nullptr) {
            const long long si = p + G.scale_off;
            const float2 sc = (si >= 0 && si < G.scale_len) ? G.scale[si] : make_float2(0.f, 0.f);
            h = cscale(h, mk(sc.x, sc.y));
        }
        st(hs + lane, h);
    }
    __syncwarp();
    const float2 *__restrict__ rfit = L.fold ? G.rfit : nullptr;
    if (lane < D) {
        const int d = lane;
        cdf q;
        if (d < B) {
            df qr = mk(0.f), qi = mk(0.f);
            for (int t = 0; t < ntap; ++t) {
                const cdf h = ld(hs + t);
                const float2 c2 = G.coef[t * D + d];
                const df cd = mk(c2.x, c2.y);
                acc(qr, mul_u(cd, h.re));
                acc(qi, mul_u(cd, h.im));
            }
            q.re = norm(qr);
            q.im = norm(qi);
        } else {
            float fr = 0.f, fi = 0.f;
            for (int t = 0; t < ntap; ++t) {
                const float4 hv = hs[t];
                const float cc = G.coef[t * D + d].x;
                fr = fmaf(cc, hv.x, fr);
                fi = fmaf(cc, hv.z, fi);
            }
            q.re = mk(fr);
            q.im = mk(fi);
        }
        st((rfit == nullptr ? qq : qa) + d, q);
    }
    __syncwarp();
    if (rfit != nullptr) {
        if (lane < D) {
            const int n = lane;
            df ar = mk(0.f), ai = mk(0.f);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const float2 rv = rfit[icl * NR + j];
                const df r = mk(rv.x, rv.y);
                if (j <= n) {
                    const cdf v = ld(qa + (n - j));
                    acc(ar, mul_u(r, v.re));
                    acc(ai, mul_u(r, v.im));
                }
                if (n + j < D) {
                    const cdf v = ld(qa + (n + j));
                    acc(ar, mul_u(r, v.re));
                    acc(ai, mul_u(r, v.im));
                }
                if (n > 0 && j >= n && j - n < D) {
                    const cdf v = ld(qa + (j - n));
                    acc(ar, mul_u(r, v.re));
                    acc(ai, mul_u(r, v.im));
                }
            }
            cdf o;
            o.re = norm(ar);
            o.im = norm(ai);
            st(qq + n, o);
        }
        __syncwarp();
    }
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = qq[d];
        if (d < B) {
            qr[d < B ? d : 0] = mk(q.x, q.y);
            qi[d < B ? d : 0] = mk(q.z, q.w);
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        if (pb + 32 * k >= pe) break;
        const double2 o = eval_point<B, F>(yv[k], qr, qi, fr, fi);
        if (jv[k] >= 0) out[jv[k]] = o;
    }
}

// Flat split-precision evaluation: one thread per sorted point, its cell from the sorted
// cell keys (no work-item indirection; threads of one cell share Q4 through L1).
template <int D>
__global__ void __launch_bounds__(256)
k_eval_df_flat(SideK<double> S, const float2 *__restrict__ ys2, const float4 *__restrict__ Q4,
               double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.M) return;
    const int c = (int)S.keys[p];
    const float2 yv = ys2[p];
    const int j = S.perm[p];
    const float4 *q4 = Q4 + (long long)c * D;
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = q4[d];
        if (d < B) {
            qr[d < B ? d : 0] = mk(q.x, q.y);
            qi[d < B ? d : 0] = mk(q.z, q.w);
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
    out[j] = eval_point<B, F>(yv, qr, qi, fr, fi);
}

// The flat evaluation with the block's cells staged by the Tensor Memory Accelerator.
// The block's 256 sorted points lie in the cells [c0, c1] (keys ascending); their window
// sums Q4[c0*D .. (c1+1)*D) are one contiguous run, which thread 0 copies into shared
// memory with one bulk copy while every thread loads its own point.  A block spanning more
// than TMA_MAX_CELLS cells (sparse plans) reads Q4 from global memory instead.  A copy
// that does not complete within the wait limit sets STATUS_TIMEOUT and the block returns
// (after a second bounded wait so that no copy is left writing its shared memory).
template <int D>
__global__ void __launch_bounds__(256)
k_eval_df_flat_tma(SideK<double> S, const float2 *__restrict__ ys2, const float4 *__restrict__ Q4,
                   double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    __shared__ __align__(128) float4 qs[TMA_MAX_CELLS * D];
    __shared__ __align__(8) uint64_t bar;
    const int p0 = blockIdx.x * blockDim.x;
    const int p = p0 + threadIdx.x;
    const int plast = min(p0 + (int)blockDim.x, S.M) - 1;
    const int c0 = (int)S.keys[p0], c1 = (int)S.keys[plast];
    const int nc = c1 - c0 + 1;
    const bool staged = nc <= TMA_MAX_CELLS;          // block-uniform
    if (staged) {
        if (threadIdx.x == 0) {
            tma::bar_init(&bar);
            const unsigned bytes = (unsigned)nc * D * (unsigned)sizeof(float4);
            tma::bar_expect(&bar, bytes);
            tma::copy_g2s(qs, Q4 + (long long)c0 * D, bytes, &bar);
        }
        __syncthreads();
    }
    int c = 0, j = -1;
    float2 yv = make_float2(0.f, 0.f);
    if (p < S.M) {
        c = (int)S.keys[p];
        yv = ys2[p];
        j = S.perm[p];
    }
    const float4 *q4 = Q4 + (long long)c * D;
    if (staged) {
        if (!tma::bar_wait(&bar, 0, tma::WAIT_LIMIT_CYCLES)) {
            if (threadIdx.x == 0) atomicOr(S.status, STATUS_TIMEOUT);
            tma::bar_wait(&bar, 0, tma::WAIT_LIMIT_CYCLES);
            return;
        }
        q4 = qs + (c - c0) * D;
    }
    if (p >= S.M) return;
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = q4[d];
        if (d < B) {
            qr[d < B ? d : 0] = mk(q.x, q.y);
            qi[d < B ? d : 0] = mk(q.z, q.w);
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
    out[j] = eval_point<B, F>(yv, qr, qi, fr, fi);
}

// ---------------------------------------------------------------------------------
// Team kernels: DTEAM = 8 lanes per work item, four items per warp (sparse cells).
// Moments use the slot layout of the half-warp kernel; three exchange steps over slot
// bits 3..1 leave lane s with slots j = 2s and 2s+1 of each kind.
// ---------------------------------------------------------------------------------
constexpr int DTEAM = 8;
// team moments: points per lane loaded at a time and the register bound in 256-thread
// blocks per SM (4 and 2: up to 128 registers; one item per cell at 2^20 points gives only
// ~13 warps per SM, so occupancy is not what the registers limit.  Measured: the 80-register
// bound of three blocks 1-3 % slower per step, 8 points per lane at a time 4-10 % slower)
constexpr int TEAM_CH = 4;
constexpr int TEAM_MINB = 2;
// Threads per block of the team moments kernels.  One item per cell at 2^20 points puts
// 8224 x 8 lanes = 257 blocks of 256 threads on 152 SMs: half the SMs ran two blocks, the
// rest one, and the kernel lasted as long as the loaded half.  Blocks of TEAM_BLOCK threads
// spread the same warps evenly.
constexpr int TEAM_BLOCK = 64;

template <int O, int LB>
__device__ __forceinline__ void rs_mixed_team(df (&vd)[16], float (&vf)[16], int sub) {
    const bool up = (sub & LB) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const df send = up ? vd[i] : vd[O + i];
        const df keep = up ? vd[O + i] : vd[i];
        df other;
        other.h = __shfl_xor_sync(0xffffffffu, send.h, LB);
        other.l = __shfl_xor_sync(0xffffffffu, send.l, LB);
        vd[i] = add_lazy(keep, other);
        const float fs = up ? vf[i] : vf[O + i];
        const float fk = up ? vf[O + i] : vf[i];
        vf[i] = fk + __shfl_xor_sync(0xffffffffu, fs, LB);
    }
}

template <int D, int CH, int MINB>
__global__ void __launch_bounds__(TEAM_BLOCK, MINB * 256 / TEAM_BLOCK)
k_moments_df_team(SideK<double> S, const float2 *__restrict__ ys2, const double2 *__restrict__ vals,
                  float4 *__restrict__ P4) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    static_assert(B <= 8 && F <= 8, "the slot layout holds at most 8 degrees of each kind");
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int item = big_item(S, gt / DTEAM);
    const int sub = threadIdx.x & (DTEAM - 1);
    int pb = 0, pe = 0;
    if (item >= 0) {                                 // every lane stays for the exchanges
        pb = S.item_pb[item];
        pe = S.item_pe[item];
    }
    df ar[B], ai[B];
    float br[F], bi[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = mk(0.f); ai[d] = mk(0.f); }
#pragma unroll
    for (int d = 0; d < F; ++d) { br[d] = 0.f; bi[d] = 0.f; }
    for (int c0 = pb; c0 < pe; c0 += DTEAM * CH) {
        float2 yv[CH];
        int jv[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int p = c0 + sub + DTEAM * k;
            yv[k] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
        double2 vv2[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) vv2[k] = jv[k] >= 0 ? vals[jv[k]] : make_double2(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < CH; ++k)
            if (jv[k] >= 0) moments_point<B, F>(yv[k], vv2[k], ar, ai, br, bi);
    }
    df vd[16];
    float vf[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) { vd[j] = mk(0.f); vf[j] = 0.f; }
#pragma unroll
    for (int d = 0; d < B; ++d) {
        vd[d] = ar[d];
        vd[8 + d] = ai[d];
    }
#pragma unroll
    for (int d = 0; d < F; ++d) {
        vf[d] = br[d];
        vf[8 + d] = bi[d];
    }
    rs_mixed_team<8, 4>(vd, vf, sub);
    rs_mixed_team<4, 2>(vd, vf, sub);
    rs_mixed_team<2, 1>(vd, vf, sub);
    if (item < 0) return;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + (long long)item * D);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int j = 2 * sub + t, deg = j & 7, part = j >> 3;   // part 0: real, 1: imaginary
        const df r = norm_any(vd[t]);
        if (deg < B) P2[2 * deg + part] = make_float2(r.h, r.l);
        if (deg < F) P2[2 * (B + deg) + part] = make_float2(vf[t], 0.f);
    }
}

// The same per-item moments as k_moments_df_team with more independent work per lane: the
// points of a chunk alternate between two sets of accumulators, so that consecutive points
// do not wait on each other's compensated sums (the sets are added before the exchange).
// More registers (two blocks of 256 per SM), for launches whose work items are too few to
// fill the SMs anyway.
template <int D, int CH>
__global__ void __launch_bounds__(TEAM_BLOCK, 2 * 256 / TEAM_BLOCK)
k_moments_df_team_pf(SideK<double> S, const float2 *__restrict__ ys2,
                     const double2 *__restrict__ vals, float4 *__restrict__ P4) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    static_assert(B <= 8 && F <= 8, "the slot layout holds at most 8 degrees of each kind");
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int item = big_item(S, gt / DTEAM);
    const int sub = threadIdx.x & (DTEAM - 1);
    int pb = 0, pe = 0;
    if (item >= 0) {                                 // every lane stays for the exchanges
        pb = S.item_pb[item];
        pe = S.item_pe[item];
    }
    df ar[B], ai[B], ar2[B], ai2[B];
    float br[F], bi[F], br2[F], bi2[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = mk(0.f); ai[d] = mk(0.f); ar2[d] = mk(0.f); ai2[d] = mk(0.f); }
#pragma unroll
    for (int d = 0; d < F; ++d) { br[d] = 0.f; bi[d] = 0.f; br2[d] = 0.f; bi2[d] = 0.f; }
    for (int c0 = pb; c0 < pe; c0 += DTEAM * CH) {
        float2 yv[CH];
        int jv[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int p = c0 + sub + DTEAM * q;
            yv[q] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
            jv[q] = p < pe ? S.perm[p] : -1;
        }
        double2 vv2[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) vv2[q] = jv[q] >= 0 ? vals[jv[q]] : make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < CH; q += 2) {
            if (jv[q] >= 0) moments_point<B, F>(yv[q], vv2[q], ar, ai, br, bi);
            if (q + 1 < CH && jv[q + 1] >= 0)
                moments_point<B, F>(yv[q + 1], vv2[q + 1], ar2, ai2, br2, bi2);
        }
    }
#pragma unroll
    for (int d = 0; d < B; ++d) {              // the two accumulator sets
        ar[d] = add_lazy(ar[d], ar2[d]);
        ai[d] = add_lazy(ai[d], ai2[d]);
    }
#pragma unroll
    for (int d = 0; d < F; ++d) {
        br[d] += br2[d];
        bi[d] += bi2[d];
    }
    df vd[16];
    float vf[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) { vd[j] = mk(0.f); vf[j] = 0.f; }
#pragma unroll
    for (int d = 0; d < B; ++d) {
        vd[d] = ar[d];
        vd[8 + d] = ai[d];
    }
#pragma unroll
    for (int d = 0; d < F; ++d) {
        vf[d] = br[d];
        vf[8 + d] = bi[d];
    }
    rs_mixed_team<8, 4>(vd, vf, sub);
    rs_mixed_team<4, 2>(vd, vf, sub);
    rs_mixed_team<2, 1>(vd, vf, sub);
    if (item < 0) return;
    float2 *P2 = reinterpret_cast<float2 *>(P4 + (long long)item * D);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int j = 2 * sub + t, deg = j & 7, part = j >> 3;   // part 0: real, 1: imaginary
        const df r = norm_any(vd[t]);
        if (deg < B) P2[2 * deg + part] = make_float2(r.h, r.l);
        if (deg < F) P2[2 * (B + deg) + part] = make_float2(vf[t], 0.f);
    }
}

template <int D>
__global__ void __launch_bounds__(256)
k_eval_df_team(SideK<double> S, const float2 *__restrict__ ys2, const float4 *__restrict__ Q4,
               double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int item = big_item(S, gt / DTEAM);
    const int sub = threadIdx.x & (DTEAM - 1);
    if (item < 0) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = Q4[(long long)c * D + d];
        if (d < B) {
            qr[d < B ? d : 0] = mk(q.x, q.y);
            qi[d < B ? d : 0] = mk(q.z, q.w);
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
    for (int c0 = pb; c0 < pe; c0 += DTEAM * MOM_CHUNK) {
        float2 yv[MOM_CHUNK];
        int jv[MOM_CHUNK];
#pragma unroll
        for (int k = 0; k < MOM_CHUNK; ++k) {
            const int p = c0 + sub + DTEAM * k;
            yv[k] = p < pe ? ys2[p] : make_float2(0.f, 0.f);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
#pragma unroll
        for (int k = 0; k < MOM_CHUNK; ++k)
            if (jv[k] >= 0) out[jv[k]] = eval_point<B, F>(yv[k], qr, qi, fr, fi);
    }
}

// ---------------------------------------------------------------------------------
// Small work items (<= SMALL_ITEM points): one thread per item walks its points in
// order; moments go out without any reduction, values straight to the caller's order.
// ---------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256)
k_moments_df_small(SideK<double> S, const float2 *__restrict__ ys2,
                   const double2 *__restrict__ vals, float4 *__restrict__ P4) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= *S.n_small) return;
    const int item = S.list_small[idx];
    const int pb = S.item_pb[item], pe = S.item_pe[item];
    df ar[B], ai[B];
    float br[F], bi[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = mk(0.f); ai[d] = mk(0.f); }
#pragma unroll
    for (int d = 0; d < F; ++d) { br[d] = 0.f; bi[d] = 0.f; }
    for (int p0 = pb; p0 < pe; p0 += 4) {             // loads of 4 points first
        float2 yv[4];
        int jv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            yv[k] = p0 + k < pe ? ys2[p0 + k] : make_float2(0.f, 0.f);
            jv[k] = p0 + k < pe ? S.perm[p0 + k] : -1;
        }
        double2 vv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) vv[k] = jv[k] >= 0 ? vals[jv[k]] : make_double2(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (jv[k] >= 0) moments_point<B, F>(yv[k], vv[k], ar, ai, br, bi);
    }
    float4 *o = P4 + (long long)item * D;
#pragma unroll
    for (int d = 0; d < B; ++d) {
        const df r = norm(ar[d]), i = norm(ai[d]);
        o[d] = make_float4(r.h, r.l, i.h, i.l);
    }
#pragma unroll
    for (int d = 0; d < F; ++d) o[B + d] = make_float4(br[d], 0.f, bi[d], 0.f);
}

template <int D>
__global__ void __launch_bounds__(256)
k_eval_df_small(SideK<double> S, const float2 *__restrict__ ys2, const float4 *__restrict__ Q4,
                double2 *__restrict__ out) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= *S.n_small) return;
    const int item = S.list_small[idx];
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    df qr[B], qi[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 q = Q4[(long long)c * D + d];
        if (d < B) {
            qr[d < B ? d : 0] = mk(q.x, q.y);
            qi[d < B ? d : 0] = mk(q.z, q.w);
        } else {
            fr[d >= B ? d - B : 0] = q.x;
            fi[d >= B ? d - B : 0] = q.z;
        }
    }
    for (int p0 = pb; p0 < pe; p0 += 4) {
        float2 yv[4];
        int jv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            yv[k] = p0 + k < pe ? ys2[p0 + k] : make_float2(0.f, 0.f);
            jv[k] = p0 + k < pe ? S.perm[p0 + k] : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (jv[k] >= 0) out[jv[k]] = eval_point<B, F>(yv[k], qr, qi, fr, fi);
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

cudaError_t launch_moments_df(const SideK<double> &S, const void *vals, void *P4, int lanes,
                              cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    const float2 *y2 = reinterpret_cast<const float2 *>(S.ys);
    const double2 *v = static_cast<const double2 *>(vals);
    float4 *o = static_cast<float4 *>(P4);
    if (lanes == MOM_LANES) {
        const int blocks = cdiv((long long)S.max_items * MOM_LANES, MOM_BLOCK);
        NNFFT_DISPATCH_DF(S.D, (k_moments_df_half<DD><<<blocks, MOM_BLOCK, 0, s>>>(S, y2, v, o)));
    } else if (lanes == DTEAM) {
        const int blocks = cdiv((long long)S.max_items * DTEAM, TEAM_BLOCK);
        NNFFT_DISPATCH_DF(S.D, (k_moments_df_team<DD, TEAM_CH, TEAM_MINB><<<blocks, TEAM_BLOCK, 0, s>>>(S, y2, v, o)));
    } else if (lanes == MOM_TEAM_PF) {
        const int blocks = cdiv((long long)S.max_items * DTEAM, TEAM_BLOCK);
        NNFFT_DISPATCH_DF(S.D, (k_moments_df_team_pf<DD, TEAM_CH><<<blocks, TEAM_BLOCK, 0, s>>>(S, y2, v, o)));
    } else {
        const int blocks = cdiv((long long)S.max_items * 32, 256);
        NNFFT_DISPATCH_DF(S.D, (k_moments_df_warp<DD><<<blocks, 256, 0, s>>>(S, y2, v, o)));
    }
    count_launches(1);
    if (S.list_small) {
        NNFFT_DISPATCH_DF(S.D, (k_moments_df_small<DD><<<cdiv(S.max_items, 256), 256, 0, s>>>(S, y2, v, o)));
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_eval_df(const SideK<double> &S, const void *Q4, void *out, int lanes,
                           cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    if (lanes == EVAL_FLAT) {                       // covers every point: no small-item pass
        if (S.M <= 0) return cudaSuccess;
        NNFFT_DISPATCH_DF(S.D, (k_eval_df_flat<DD><<<cdiv(S.M, 256), 256, 0, s>>>(
                                   S, reinterpret_cast<const float2 *>(S.ys),
                                   static_cast<const float4 *>(Q4), static_cast<double2 *>(out))));
        count_launches(1);
        return cudaGetLastError();
    }
    if (lanes == EVAL_FLAT_TMA) {
        if (S.M <= 0) return cudaSuccess;
        NNFFT_DISPATCH_DF(S.D, (k_eval_df_flat_tma<DD><<<cdiv(S.M, 256), 256, 0, s>>>(
                                   S, reinterpret_cast<const float2 *>(S.ys),
                                   static_cast<const float4 *>(Q4), static_cast<double2 *>(out))));
        count_launches(1);
        return cudaGetLastError();
    }
    if (lanes == DTEAM) {
        const int blocks = cdiv((long long)S.max_items * DTEAM, 256);
        NNFFT_DISPATCH_DF(S.D, (k_eval_df_team<DD><<<blocks, 256, 0, s>>>(
                                   S, reinterpret_cast<const float2 *>(S.ys),
                                   static_cast<const float4 *>(Q4), static_cast<double2 *>(out))));
    } else {
        const int blocks = cdiv((long long)S.max_items * 32, 256);
        NNFFT_DISPATCH_DF(S.D, (k_eval_df<DD><<<blocks, 256, 0, s>>>(
                                   S, reinterpret_cast<const float2 *>(S.ys),
                                   static_cast<const float4 *>(Q4), static_cast<double2 *>(out))));
    }
    count_launches(1);
    if (S.list_small) {
        NNFFT_DISPATCH_DF(S.D, (k_eval_df_small<DD><<<cdiv(S.max_items, 256), 256, 0, s>>>(
                                   S, reinterpret_cast<const float2 *>(S.ys),
                                   static_cast<const float4 *>(Q4), static_cast<double2 *>(out))));
        count_launches(1);
    }
    return cudaGetLastError();
}

bool eval_gather_df_ok(const GridLaunch<float2> &L) {
    return L.ninst == 1 && 2 * L.m <= EG_HS && L.D <= 16 && df_supported_degree(L.D);
}

cudaError_t launch_eval_gather_df(const SideK<double> &S, const GridLaunch<float2> &L,
                                  const void *grid, void *out, cudaStream_t s) {
    // every item runs one warp: not with small-item splitting (the callers fall back)
    if (S.list_small || !eval_gather_df_ok(L) || L.D != S.D) return cudaErrorInvalidValue;
    if (S.max_items <= 0) return cudaSuccess;
    const int blocks = cdiv((long long)S.max_items * 32, 256);
    NNFFT_DISPATCH_DF(S.D, (k_eval_gather_df<DD><<<blocks, 256, 0, s>>>(
                               S, reinterpret_cast<const float2 *>(S.ys), L,
                               static_cast<const float4 *>(grid), static_cast<double2 *>(out))));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnfft
