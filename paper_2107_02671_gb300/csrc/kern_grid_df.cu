// kern_grid_df.cu -- the grid stage of Algorithm 2.2 (cell fold, spread convolution
// with the step-2 deconvolution, the step-3 FFT and the step-4 gather convolution)
// in double-float arithmetic (df.cuh) for fp64 plans in split precision.
//
// Same decompositions as the FP64 kernels in kern_spread.cu / kern_fft.cu; every
// complex value is a float4 (re.h, re.l, im.h, im.l).  Window degrees d >= B = D/2
// (weights <= 2e-7) are accumulated in FP32 from the high parts, as in the point
// kernels.  The FFT butterflies run fully in double-float.
#include <cooperative_groups.h>

#include <algorithm>

#include "df.cuh"
#include "gridsync.cuh"
#include "internal.h"

namespace nnfft {

namespace {

using namespace dfa;

// ---------------------------------------------------------------------------------
// Cell fold: sum of the items' moments per cell; with a 1/phihat1 fit (x side,
// adjoint) the factor R(y) = sum_j r_j T_j(y) is applied in the Chebyshev basis,
// out_d = sum_j (r_j/2) (M_{d+j} + M_{|d-j|}), truncated at degree D.
// rh holds r_j / 2 as (hi, lo) floats.
// ---------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ cdf item_sum(const float4 *__restrict__ P4, int i0, int i1, int e) {
    cdf m = ld(P4 + (long long)i0 * D + e);
    for (int it = i0 + 1; it < i1; ++it) m = cadd(m, ld(P4 + (long long)it * D + e));
    return m;
}

// one thread per (cell, degree d): element idx = cell * D + d
template <int D>
__device__ __forceinline__ void cell_fold_df_elem(const SideK<double> &S, const SideDf &T,
                                                  const float4 *__restrict__ P4,
                                                  float4 *__restrict__ Pc4, long long idx) {
    const int ic = (int)(idx / D), d = (int)(idx - (long long)ic * D);
    if (ic >= S.ncell) return;
    const int i0 = S.item_off[ic], i1 = S.item_off[ic + 1];
    cdf o = czero();
    if (i1 > i0) {
        if (T.rfit == nullptr) {
            o = item_sum<D>(P4, i0, i1, d);
        } else {
            df ar = mk(0.f), ai = mk(0.f);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const float2 rv = T.rfit[(long long)ic * NR + j];
                const df r = mk(rv.x, rv.y);
                const int hi = d + j, lo = d > j ? d - j : j - d;
                if (hi < D) {
                    const cdf m = item_sum<D>(P4, i0, i1, hi);
                    acc(ar, mul_u(r, m.re));
                    acc(ai, mul_u(r, m.im));
                }
                if (lo < D) {
                    const cdf m = item_sum<D>(P4, i0, i1, lo);
                    acc(ar, mul_u(r, m.re));
                    acc(ai, mul_u(r, m.im));
                }
            }
            o.re = norm(ar);
            o.im = norm(ai);
        }
    }
    st(Pc4 + (long long)ic * D + d, o);
}

template <int D>
__global__ void __launch_bounds__(128)
k_cell_fold_df(SideK<double> S, SideDf T, const float4 *__restrict__ P4,
               float4 *__restrict__ Pc4) {
    cell_fold_df_elem<D>(S, T, P4, Pc4, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// With the fit (x side, adjoint): a block of CFP = 32 cells and one warp per degree
// (lane = cell).  The item sums M_d are formed once per (cell, degree) into shared memory,
// the fold reads them there (the per-thread form above re-sums up to 2 NR of them), and
// the outputs leave as coalesced rows.  Same sums in the same order.
constexpr int CFP = 32;

// block vb of D * CFP threads: cells [vb CFP, vb CFP + CFP)
template <int D>
__device__ __forceinline__ void cell_fold_df_fit_block(const SideK<double> &S, const SideDf &T,
                                                       const float4 *__restrict__ P4,
                                                       float4 *__restrict__ Pc4, int vb) {
    __shared__ float4 ms[D][CFP];
    __shared__ float4 os[CFP * D];
    const int k = threadIdx.x & (CFP - 1), d = threadIdx.x / CFP;
    const int c0 = vb * CFP;
    const int ic = c0 + k;
    int i0 = 0, i1 = 0;
    if (ic < S.ncell) {
        i0 = S.item_off[ic];
        i1 = S.item_off[ic + 1];
    }
    st(&ms[d][k], i1 > i0 ? item_sum<D>(P4, i0, i1, d) : czero());
    __syncthreads();
    cdf o = czero();
    if (i1 > i0) {
        df ar = mk(0.f), ai = mk(0.f);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const float2 rv = T.rfit[(long long)ic * NR + j];
            const df r = mk(rv.x, rv.y);
            const int hi = d + j, lo = d > j ? d - j : j - d;
            if (hi < D) {
                const cdf m = ld(&ms[hi][k]);
                acc(ar, mul_u(r, m.re));
                acc(ai, mul_u(r, m.im));
            }
            if (lo < D) {
                const cdf m = ld(&ms[lo][k]);
                acc(ar, mul_u(r, m.re));
                acc(ai, mul_u(r, m.im));
            }
        }
        o.re = norm(ar);
        o.im = norm(ai);
    }
    st(os + k * D + d, o);
    __syncthreads();
    const int nc = min(CFP, S.ncell - c0);
    float4 *dst = Pc4 + (long long)c0 * D;
    for (int e = threadIdx.x; e < nc * D; e += D * CFP) dst[e] = os[e];
}

template <int D>
__global__ void __launch_bounds__(512)
k_cell_fold_df_fit(SideK<double> S, SideDf T, const float4 *__restrict__ P4,
                   float4 *__restrict__ Pc4) {
    cell_fold_df_fit_block<D>(S, T, P4, Pc4, blockIdx.x);
}

// ---------------------------------------------------------------------------------
// Spread convolution.  Grid position p = p_lo + i (centered; the taps of all cells
// cover [p_lo, p_hi], never wider than N2) goes to buffer index p mod N2:
//   g_p = scale(p) * sum_t sum_d coef[t][d] * Pc_{p+m-1-t}[d],  0 beyond p_hi.
// A block handles SCP = 32 consecutive positions of one instance with one warp per
// Chebyshev degree d (lane = position): every warp takes one arithmetic path
// (double-float for d < D/2, FP32 above), reads its tap coefficients as broadcasts and
// consecutive staged cells ([D][SCP + 2m - 1] in shared memory), and there are D warps
// per 32 positions to hide the latency of the accumulation chains.  Warp 0 then adds
// the D partial sums of its position in the order d = D-1, ..., 0 and applies the
// deconvolution factor.
// ---------------------------------------------------------------------------------
constexpr int SCP = 32;

// Shared memory of a degree-major spread block: Ps [D][ncl] float4, part [D][SCP] float4,
// coef [ntap][D] float2, then (cell fold with the fit) Ms [D][ncl] float4.
template <int D>
__device__ __forceinline__ float4 *coef_end_df(float4 *part, int ntap) {
    return reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(part + D * SCP) + ntap * D);
}

// block vb of D * SCP threads; smem4: the block's dynamic shared memory.  With F.P4 the
// block forms the cell moments of its staged cells itself from the work items (the cell
// fold, k_cell_fold_df / k_cell_fold_df_fit, same sums in the same order) instead of
// reading them from Pc_all.
template <int D>
__device__ __forceinline__ void spread_conv_df_block(const GridLaunch<float2> &L,
                                                     const float4 *__restrict__ Pc_all,
                                                     float4 *__restrict__ out_all, int vb,
                                                     float4 *smem4, const SpreadFoldDf &F) {
    constexpr int B = D / 2;
    constexpr int NT = D * SCP;
    const int inst = block_instance(L.blk, L.ninst, vb);
    const GridInst<float2> G = L.inst[inst];
    const float4 *__restrict__ Pc4 = Pc_all + (long long)G.cell_base * D;
    float4 *__restrict__ out = out_all + G.grid_base;
    const int N2 = G.N2;
    const int m = L.m, ntap = 2 * L.m;
    const int ncl = SCP + ntap - 1;
    float4 *Ps = smem4;                                          // [D][ncl] staged cells
    float4 *part = Ps + D * ncl;                                 // [D][SCP] partial sums
    float2 *coef = reinterpret_cast<float2 *>(part + D * SCP);  // [ntap][D]
    const long long p_lo = G.c_lo - m + 1, p_hi = G.c_lo + G.ncell - 1 + m;
    const long long i0 = (long long)(vb - L.blk[inst]) * SCP;
    const long long p0 = p_lo + i0;
    const int k = threadIdx.x & (SCP - 1), d = threadIdx.x / SCP;   // position, degree
    const long long i = i0 + k;
    if (p0 > p_hi) {                                             // zero padding only
        if (d == 0 && i < N2) out[wrap_index(p_lo + i, N2)] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const long long cbase = p0 - m;
    for (int e = threadIdx.x; e < ntap * D; e += NT) coef[e] = G.coef[e];
    if (F.P4 == nullptr) {
        for (int e = threadIdx.x; e < ncl * D; e += NT) {
            const int lc = e / D, dd = e - lc * D;
            const long long ic = cbase + lc - G.c_lo;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ic >= 0 && ic < G.ncell) v = Pc4[ic * D + dd];
            Ps[dd * ncl + lc] = v;
        }
    } else {
        // item sums of the staged cells (into Ms with the 1/phihat1 fit, else straight into Ps)
        float4 *Ms = F.rfit != nullptr ? coef_end_df<D>(part, ntap) : Ps;
        for (int e = threadIdx.x; e < ncl * D; e += NT) {
            const int lc = e / D, dd = e - lc * D;
            const long long ic = cbase + lc - G.c_lo;
            cdf mv = czero();
            if (ic >= 0 && ic < G.ncell) {
                const long long gc = G.cell_base + ic;
                const int i0 = F.item_off[gc], i1 = F.item_off[gc + 1];
                if (i1 > i0) mv = item_sum<D>(F.P4, i0, i1, dd);
            }
            st(Ms + dd * ncl + lc, mv);
        }
        if (F.rfit != nullptr) {
            __syncthreads();
            for (int e = threadIdx.x; e < ncl * D; e += NT) {
                const int lc = e / D, dd = e - lc * D;
                const long long ic = cbase + lc - G.c_lo;
                cdf o = czero();
                if (ic >= 0 && ic < G.ncell) {
                    const long long gc = G.cell_base + ic;
                    if (F.item_off[gc + 1] > F.item_off[gc]) {
                        df ar = mk(0.f), ai = mk(0.f);
#pragma unroll
                        for (int j = 0; j < NR; ++j) {
                            const float2 rv = F.rfit[gc * NR + j];
                            const df r = mk(rv.x, rv.y);
                            const int hi = dd + j, lo = dd > j ? dd - j : j - dd;
                            if (hi < D) {
                                const cdf mm = ld(Ms + hi * ncl + lc);
                                acc(ar, mul_u(r, mm.re));
                                acc(ai, mul_u(r, mm.im));
                            }
                            if (lo < D) {
                                const cdf mm = ld(Ms + lo * ncl + lc);
                                acc(ar, mul_u(r, mm.re));
                                acc(ai, mul_u(r, mm.im));
                            }
                        }
                        o.re = norm(ar);
                        o.im = norm(ai);
                    }
                }
                st(Ps + dd * ncl + lc, o);
            }
        }
    }
    __syncthreads();
    const int lbase = k + ntap - 1;
    const float4 *Pd = Ps + d * ncl + lbase;
    cdf g;
    if (d < B) {                                                 // warp-uniform branch
        df ar = mk(0.f), ai = mk(0.f);
        for (int t = 0; t < ntap; ++t) {
            const float4 pv = Pd[-t];
            const float2 c2 = coef[t * D + d];
            const df cd = mk(c2.x, c2.y);
            acc(ar, mul_u(cd, mk(pv.x, pv.y)));
            acc(ai, mul_u(cd, mk(pv.z, pv.w)));
        }
        g.re = norm(ar);
        g.im = norm(ai);
    } else {
        float fr = 0.f, fi = 0.f;
        for (int t = 0; t < ntap; ++t) {
            const float4 pv = Pd[-t];
            const float c = coef[t * D + d].x;
            fr = fmaf(c, pv.x, fr);
            fi = fmaf(c, pv.z, fi);
        }
        g.re = mk(fr);
        g.im = mk(fi);
    }
    st(part + d * SCP + k, g);
    __syncthreads();
    if (d != 0 || i >= N2) return;
    const long long p = p_lo + i;
    const int q = wrap_index(p, N2);
    if (p > p_hi) {
        out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    g = ld(part + (D - 1) * SCP + k);
#pragma unroll
    for (int e = D - 2; e >= 0; --e) g = cadd(g, ld(part + e * SCP + k));
    if (G.scale != nullptr) {
        const long long si = p + G.scale_off;
        const float2 sc = (si >= 0 && si < G.scale_len) ? G.scale[si] : make_float2(0.f, 0.f);
        g = cscale(g, mk(sc.x, sc.y));
    }
    st(out + q, g);
}

template <int D>
__global__ void __launch_bounds__(512)
k_spread_conv_df(GridLaunch<float2> L, const float4 *__restrict__ Pc_all,
                 float4 *__restrict__ out_all, SpreadFoldDf F) {
    extern __shared__ float4 smem4[];
    spread_conv_df_block<D>(L, Pc_all, out_all, blockIdx.x, smem4, F);
}

// Position-major form of the same sum for launches with many blocks (batches): one
// thread per position with all D degrees in registers (fewer instructions per position,
// one warp per block); the degree partials meet in the same order.
template <int D>
__global__ void __launch_bounds__(SCP)
k_spread_conv_df_pos(GridLaunch<float2> L, const float4 *__restrict__ Pc_all,
                     float4 *__restrict__ out_all) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    extern __shared__ float4 smem4[];
    const int inst = block_instance(L.blk, L.ninst, blockIdx.x);
    const GridInst<float2> G = L.inst[inst];
    const float4 *__restrict__ Pc4 = Pc_all + (long long)G.cell_base * D;
    float4 *__restrict__ out = out_all + G.grid_base;
    const int N2 = G.N2;
    const int m = L.m, ntap = 2 * L.m;
    const int ncl = SCP + ntap - 1;
    float4 *Ps = smem4;                                          // [D][ncl] staged cells
    float2 *coef = reinterpret_cast<float2 *>(Ps + D * ncl);    // [ntap][D]
    const long long p_lo = G.c_lo - m + 1, p_hi = G.c_lo + G.ncell - 1 + m;
    const long long i0 = (long long)(blockIdx.x - L.blk[inst]) * SCP;
    const long long p0 = p_lo + i0;
    const int k = threadIdx.x;
    const long long i = i0 + k;
    if (p0 > p_hi) {                                             // zero padding only
        if (i < N2) out[wrap_index(p_lo + i, N2)] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const long long cbase = p0 - m;
    for (int e = k; e < ntap * D; e += SCP) coef[e] = G.coef[e];
    for (int e = k; e < ncl * D; e += SCP) {
        const int lc = e / D, d = e - lc * D;
        const long long ic = cbase + lc - G.c_lo;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ic >= 0 && ic < G.ncell) v = Pc4[ic * D + d];
        Ps[d * ncl + lc] = v;
    }
    __syncthreads();
    if (i >= N2) return;
    const long long p = p_lo + i;
    const int q = wrap_index(p, N2);
    if (p > p_hi) {
        out[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    df ar[B], ai[B];
    float fr[F], fi[F];
#pragma unroll
    for (int d = 0; d < B; ++d) { ar[d] = mk(0.f); ai[d] = mk(0.f); }
#pragma unroll
    for (int d = 0; d < F; ++d) { fr[d] = 0.f; fi[d] = 0.f; }
    const int lbase = k + ntap - 1;
    for (int t = 0; t < ntap; ++t) {
        const int lc = lbase - t;
#pragma unroll
        for (int d = 0; d < B; ++d) {
            const float4 pv = Ps[d * ncl + lc];
            const float2 c2 = coef[t * D + d];
            const df cd = mk(c2.x, c2.y);
            acc(ar[d], mul_u(cd, mk(pv.x, pv.y)));
            acc(ai[d], mul_u(cd, mk(pv.z, pv.w)));
        }
#pragma unroll
        for (int d = 0; d < F; ++d) {
            const float4 pv = Ps[(B + d) * ncl + lc];
            const float c = coef[t * D + B + d].x;
            fr[d] = fmaf(c, pv.x, fr[d]);
            fi[d] = fmaf(c, pv.z, fi[d]);
        }
    }
    cdf g;
    g.re = mk(fr[F - 1]);
    g.im = mk(fi[F - 1]);
#pragma unroll
    for (int d = F - 2; d >= 0; --d) {
        g.re = add(g.re, mk(fr[d]));
        g.im = add(g.im, mk(fi[d]));
    }
#pragma unroll
    for (int d = B - 1; d >= 0; --d) {
        g.re = add(g.re, norm(ar[d]));
        g.im = add(g.im, norm(ai[d]));
    }
    if (G.scale != nullptr) {
        const long long si = p + G.scale_off;
        const float2 sc = (si >= 0 && si < G.scale_len) ? G.scale[si] : make_float2(0.f, 0.f);
        g = cscale(g, mk(sc.x, sc.y));
    }
    st(out + q, g);
}

// ---------------------------------------------------------------------------------
// FFT (step 3), four-step N2 = n1 * n2 as in kern_fft.cu, Stockham stages in
// double-float.  Twiddle tables hold exp(-2 pi i k/n) as float4; sign = +1 conjugates.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ cdf twd(const float4 *tw, int idx, int sign) {
    return conj_if(ld(tw + idx), sign > 0);
}

// cos and sin of 2 pi / 3, 2 pi / 5 and 4 pi / 5 as float pairs (the radix-3 and radix-5
// butterflies below)
constexpr double BF_S3 = 0.866025403784438646763723170753;    // sin(2 pi / 3)
constexpr double BF_C51 = 0.309016994374947424102293417183;   // cos(2 pi / 5)
constexpr double BF_C52 = -0.809016994374947424102293417183;  // cos(4 pi / 5)
constexpr double BF_S51 = 0.951056516295153572116439333379;   // sin(2 pi / 5)
constexpr double BF_S52 = 0.587785252292473129168705954639;   // sin(4 pi / 5)
// float pairs (hi, lo) of those constants, computed at compile time
constexpr float bf_hi(double c) { return (float)c; }
constexpr float bf_lo(double c) { return (float)(c - (double)(float)c); }
constexpr float BF_S3_H = bf_hi(BF_S3), BF_S3_L = bf_lo(BF_S3);
constexpr float BF_C51_H = bf_hi(BF_C51), BF_C51_L = bf_lo(BF_C51);
constexpr float BF_C52_H = bf_hi(BF_C52), BF_C52_L = bf_lo(BF_C52);
constexpr float BF_S51_H = bf_hi(BF_S51), BF_S51_L = bf_lo(BF_S51);
constexpr float BF_S52_H = bf_hi(BF_S52), BF_S52_L = bf_lo(BF_S52);
__device__ __forceinline__ cdf chalf(cdf a) {                  // a / 2, exact
    a.re = mk(0.5f * a.re.h, 0.5f * a.re.l);
    a.im = mk(0.5f * a.im.h, 0.5f * a.im.l);
    return a;
}

template <int R>
__device__ __forceinline__ void stage_df(const float4 *src, float4 *dst, int n, int cols, int L,
                                         const float4 *tw, int sign) {
    const int nr = n / R;
    const int tstep = n / (L * R);
    for (int jj = threadIdx.x; jj < cols * nr; jj += blockDim.x) {
        const int col = jj / nr, j = jj - col * nr;
        const float4 *s0 = src + col * n;
        float4 *d0 = dst + col * n;
        const int k = j % L;
        cdf a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            a[q] = ld(s0 + j + q * nr);
            if (q > 0 && k > 0) a[q] = cmul(a[q], twd(tw, q * k * tstep, sign));
        }
        cdf b[R];
        if (R == 2) {
            b[0] = cadd(a[0], a[1]);
            b[1] = csub(a[0], a[1]);
        } else if (R == 4) {
            const cdf s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
            const cdf s13 = cadd(a[1], a[3]);
            const cdf d13 = cmul_isign(csub(a[1], a[3]), sign);
            b[0] = cadd(s02, s13);
            b[1] = cadd(d02, d13);
            b[2] = csub(s02, s13);
            b[3] = csub(d02, d13);
        } else if (R == 3) {
            // with w = exp(sign 2 pi i / 3) = -1/2 + i sign sin(2 pi / 3):
            // b1, b2 = a0 - (a1 + a2) / 2 +- i sign sin(2 pi / 3) (a1 - a2)
            const cdf s12 = cadd(a[1], a[2]);
            const cdf t = csub(a[0], chalf(s12));
            const cdf u = cmul_isign(cscale(csub(a[1], a[2]), mk(BF_S3_H, BF_S3_L)), sign);
            b[0] = cadd(a[0], s12);
            b[1] = cadd(t, u);
            b[2] = csub(t, u);
        } else {
            // R == 5, w = exp(sign 2 pi i / 5): b_p and b_(5-p) share the cosine sums and
            // differ in the sign of the sine sums (a_q w^(pq) + a_(5-q) w^(-pq))
            const cdf s1 = cadd(a[1], a[4]), d1 = csub(a[1], a[4]);
            const cdf s2 = cadd(a[2], a[3]), d2 = csub(a[2], a[3]);
            const df c1 = mk(BF_C51_H, BF_C51_L), c2 = mk(BF_C52_H, BF_C52_L);
            const df n1 = mk(BF_S51_H, BF_S51_L), n2 = mk(BF_S52_H, BF_S52_L);
            const cdf t1 = cadd(a[0], cadd(cscale(s1, c1), cscale(s2, c2)));
            const cdf t2 = cadd(a[0], cadd(cscale(s1, c2), cscale(s2, c1)));
            const cdf u1 = cmul_isign(cadd(cscale(d1, n1), cscale(d2, n2)), sign);
            const cdf u2 = cmul_isign(csub(cscale(d1, n2), cscale(d2, n1)), sign);
            b[0] = cadd(a[0], cadd(s1, s2));
            b[1] = cadd(t1, u1);
            b[4] = csub(t1, u1);
            b[2] = cadd(t2, u2);
            b[3] = csub(t2, u2);
        }
#pragma unroll
        for (int p = 0; p < R; ++p) st(d0 + (j - k) * R + k + p * L, b[p]);
    }
}

__device__ float4 *stockham_df(float4 *A, float4 *Bf, int n, int cols, const int *radices,
                               int nrad, const float4 *tw, int sign) {
    int L = 1;
    float4 *src = A, *dst = Bf;
    for (int s = 0; s < nrad; ++s) {
        const int R = radices[s];
        switch (R) {
            case 2: stage_df<2>(src, dst, n, cols, L, tw, sign); break;
            case 3: stage_df<3>(src, dst, n, cols, L, tw, sign); break;
            case 4: stage_df<4>(src, dst, n, cols, L, tw, sign); break;
            case 5: stage_df<5>(src, dst, n, cols, L, tw, sign); break;
            default: break;
        }
        __syncthreads();
        L *= R;
        float4 *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Block b of pass 1 holds columns [b0, b0 + cols1) of instance i (b0 = (b - blk1[i]) cols1),
// block c of pass 2 rows [c0, c0 + cols2); shared memory A, B (cols x n) and twiddles (n).
__device__ __forceinline__ void fft_pass1_df_block(const float4 *__restrict__ X_all,
                                                   float4 *__restrict__ Z_all,
                                                   const FftLaunch<FftDf> &L, int sign, int vb,
                                                   float4 *smem4) {
    const int inst = block_instance(L.blk1, L.ninst, vb);
    const FftDf &F = L.inst[inst];
    const float4 *__restrict__ X = X_all + F.grid_base;
    float4 *__restrict__ Z = Z_all + F.grid_base;
    const int n = F.n1, n2 = F.n2;
    const int b0 = (vb - L.blk1[inst]) * F.cols1;
    const int cols = min(F.cols1, n2 - b0);
    float4 *A = smem4, *Bf = smem4 + cols * n, *tw = smem4 + 2 * cols * n;
    // the four-step twiddles of this thread's first outputs, loaded now so that their latency
    // overlaps the column loads and the butterflies instead of following them
    constexpr int PF = 2;
    float4 twp[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e < cols * n) {
            const int bb = e / n, c = e - bb * n;
            twp[q] = F.twN[(b0 + bb) * c];
        }
    }
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int a = e / cols, bb = e - a * cols;
        A[bb * n + a] = X[(long long)n2 * a + b0 + bb];
    }
    for (int a = threadIdx.x; a < n; a += blockDim.x) tw[a] = F.tw1[a];
    __syncthreads();
    const float4 *res = stockham_df(A, Bf, n, cols, F.r1, F.nr1, tw, sign);
    int q = 0;
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x, ++q) {
        const int bb = e / n, c = e - bb * n, b = b0 + bb;
        cdf w;
        if (q < PF) {
            float4 t4 = twp[0];
#pragma unroll
            for (int r = 1; r < PF; ++r)
                if (q == r) t4 = twp[r];
            w = conj_if(ld(&t4), sign > 0);
        } else {
            w = twd(F.twN, b * c, sign);
        }
        st(Z + (long long)b * n + c, cmul(ld(res + e), w));
    }
}

__device__ __forceinline__ void fft_pass2_df_block(const float4 *__restrict__ Z_all,
                                                   float4 *__restrict__ Y_all,
                                                   const FftLaunch<FftDf> &L, int sign, int vb,
                                                   float4 *smem4) {
    const int inst = block_instance(L.blk2, L.ninst, vb);
    const FftDf &F = L.inst[inst];
    const float4 *__restrict__ Z = Z_all + F.grid_base;
    float4 *__restrict__ Y = Y_all + F.grid_base;
    const int n = F.n2, n1 = F.n1;
    const int c0 = (vb - L.blk2[inst]) * F.cols2;
    const int cols = min(F.cols2, n1 - c0);
    float4 *A = smem4, *Bf = smem4 + cols * n, *tw = smem4 + 2 * cols * n;
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int b = e / cols, cc = e - b * cols;
        A[cc * n + b] = Z[(long long)b * n1 + c0 + cc];
    }
    for (int b = threadIdx.x; b < n; b += blockDim.x) tw[b] = F.tw2[b];
    __syncthreads();
    const float4 *res = stockham_df(A, Bf, n, cols, F.r2, F.nr2, tw, sign);
    for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
        const int d = e / cols, cc = e - d * cols;
        Y[c0 + cc + (long long)n1 * d] = res[cc * n + d];
    }
}

__global__ void __launch_bounds__(128)
k_fft_pass1_df(const float4 *__restrict__ X_all, float4 *__restrict__ Z_all, FftLaunch<FftDf> L,
               int sign) {
    extern __shared__ float4 smem4[];
    fft_pass1_df_block(X_all, Z_all, L, sign, blockIdx.x, smem4);
}

__global__ void __launch_bounds__(128)
k_fft_pass2_df(const float4 *__restrict__ Z_all, float4 *__restrict__ Y_all, FftLaunch<FftDf> L,
               int sign) {
    extern __shared__ float4 smem4[];
    fft_pass2_df_block(Z_all, Y_all, L, sign, blockIdx.x, smem4);
}

// ---------------------------------------------------------------------------------
// The same four-step FFT of one instance in one launch: a cluster of FFT_CLUSTER CTAs keeps
// the whole grid in distributed shared memory.  CTA r transforms the columns [r P1, (r+1) P1)
// (pass 1, with the twiddles) into its own shared memory; after a cluster barrier it gathers
// the rows [r P2, (r+1) P2) of the intermediate from every CTA's shared memory (DSMEM loads,
// consecutive threads reading consecutive addresses of one CTA), waits for the cluster again
// (no CTA may leave while others read its memory), transforms the rows (pass 2) and writes
// them.  No intermediate goes through global memory and there is one launch instead of two.
// Shared memory per CTA: three buffers of max(P1 n1, P2 n2) elements and both twiddle
// tables (fft_cluster_smem).
// ---------------------------------------------------------------------------------
__global__ void __cluster_dims__(FFT_CLUSTER, 1, 1) __launch_bounds__(FFT_CLUSTER_THREADS)
k_fft_cluster_df(const float4 *__restrict__ X, float4 *__restrict__ Y, FftLaunch<FftDf> L,
                 int sign) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smem4[];
    const int r = (int)cl.block_rank();
    const FftDf &F = L.inst[0];
    const int n1 = F.n1, n2 = F.n2;
    const int per1 = (n2 + FFT_CLUSTER - 1) / FFT_CLUSTER, per2 = (n1 + FFT_CLUSTER - 1) / FFT_CLUSTER;
    const int cap = max(per1 * n1, per2 * n2);
    float4 *buf0 = smem4, *buf1 = smem4 + cap, *buf2 = smem4 + 2 * cap;
    float4 *tw1 = smem4 + 3 * cap, *tw2 = tw1 + n1;
    const int b0 = r * per1, cols1 = max(0, min(per1, n2 - b0));
    for (int e = threadIdx.x; e < cols1 * n1; e += blockDim.x) {     // columns b0 + bb
        const int a = e / cols1, bb = e - a * cols1;
        buf0[bb * n1 + a] = X[(long long)n2 * a + b0 + bb];
    }
    for (int a = threadIdx.x; a < n1; a += blockDim.x) tw1[a] = F.tw1[a];
    for (int b = threadIdx.x; b < n2; b += blockDim.x) tw2[b] = F.tw2[b];
    __syncthreads();
    float4 *res1 = stockham_df(buf0, buf1, n1, cols1, F.r1, F.nr1, tw1, sign);
    for (int e = threadIdx.x; e < cols1 * n1; e += blockDim.x) {
        const int bb = e / n1, c = e - bb * n1;
        st(res1 + e, cmul(ld(res1 + e), twd(F.twN, (b0 + bb) * c, sign)));
    }
    cl.sync();                                   // every CTA's pass 1 is in its shared memory
    float4 *A2 = res1 == buf0 ? buf1 : buf0;     // the same buffer in every CTA
    const int c0 = r * per2, cols2 = max(0, min(per2, n1 - c0));
    for (int e = threadIdx.x; e < cols2 * n2; e += blockDim.x) {     // rows c0 + cc
        const int b = e / cols2, cc = e - b * cols2;
        const int owner = b / per1;
        const float4 *rem = cl.map_shared_rank(res1, owner);
        A2[cc * n2 + b] = rem[(b - owner * per1) * n1 + c0 + cc];
    }
    cl.sync();                                   // no CTA leaves while its memory is read
    const float4 *res2 = stockham_df(A2, buf2, n2, cols2, F.r2, F.nr2, tw2, sign);
    for (int e = threadIdx.x; e < cols2 * n2; e += blockDim.x) {
        const int d = e / cols2, cc = e - d * cols2;
        Y[c0 + cc + (long long)n1 * d] = res2[cc * n2 + d];
    }
}

// ---------------------------------------------------------------------------------
// Gather convolution:
//   Q_c[d] = sum_t coef[t][d] * scale(p) * h[p mod N2],  p = c - m + 1 + t,
// then (x side) the 1/phihat1 fold in the Chebyshev basis: the coefficients of
// R(y) sum_i Q_c[i] T_i(y) with R(y) = sum_j r_j T_j(y), truncated at degree D.
// A block handles GCP = 32 consecutive cells of one instance with one warp per degree
// (lane = cell): the block's 32 + 2m - 1 grid values are loaded and scaled once into
// shared memory, each warp takes one arithmetic path and reads its tap coefficients as
// broadcasts; the fold runs with one warp per output degree on the [D][GCP] sums, and
// the outputs leave through shared memory as coalesced rows.
// ---------------------------------------------------------------------------------
constexpr int GCP = 32;

// block vb of D * GCP threads; smem4: the block's dynamic shared memory
template <int D>
__device__ __forceinline__ void gather_conv_df_block(const GridLaunch<float2> &L,
                                                     const float4 *__restrict__ buf_all,
                                                     float4 *__restrict__ Q_all, int vb,
                                                     float4 *smem4) {
    constexpr int B = D / 2;
    constexpr int NT = D * GCP;
    const int inst = block_instance(L.blk, L.ninst, vb);
    const GridInst<float2> G = L.inst[inst];
    const float4 *__restrict__ buf = buf_all + G.grid_base;
    float4 *__restrict__ Q4 = Q_all + (long long)G.cell_base * D;
    const float2 *__restrict__ rfit = L.fold ? G.rfit : nullptr;
    const int N2 = G.N2;
    const int m = L.m, ntap = 2 * L.m;
    const int nh = GCP + ntap - 1;
    float4 *hs = smem4;                                          // [nh] scaled grid values
    float4 *qs = hs + nh;                                        // [GCP][D] outputs
    float4 *qa = qs + GCP * D;                                   // [D][GCP] tap sums (fold only)
    float2 *coef = reinterpret_cast<float2 *>(qs + (L.fold ? 2 : 1) * GCP * D);   // [ntap][D]
    const int k = threadIdx.x & (GCP - 1), d = threadIdx.x / GCP;   // cell, degree
    const int ic0 = (vb - L.blk[inst]) * GCP;
    const int ncb = min(GCP, G.ncell - ic0);                     // cells of this block
    const long long pb = G.c_lo + ic0 - m + 1;                   // position of hs[0]
    for (int e = threadIdx.x; e < ntap * D; e += NT) coef[e] = G.coef[e];
    for (int e = threadIdx.x; e < ncb + ntap - 1; e += NT) {
        const long long p = pb + e;
        cdf h = ld(buf + wrap_index(p, N2));
        if (G.scale != nullptr) {
            const long long si = p + G.scale_off;
            const float2 sc = (si >= 0 && si < G.scale_len) ? G.scale[si] : make_float2(0.f, 0.f);
            h = cscale(h, mk(sc.x, sc.y));
        }
        st(hs + e, h);
    }
    __syncthreads();
    cdf q;
    if (d < B) {                                                 // warp-uniform branch
        df qr = mk(0.f), qi = mk(0.f);
        for (int t = 0; t < ntap; ++t) {
            const cdf h = ld(hs + k + t);
            const float2 c2 = coef[t * D + d];
            const df cd = mk(c2.x, c2.y);
            acc(qr, mul_u(cd, h.re));
            acc(qi, mul_u(cd, h.im));
        }
        q.re = norm(qr);
        q.im = norm(qi);
    } else {
        float fr = 0.f, fi = 0.f;
        for (int t = 0; t < ntap; ++t) {
            const float4 hv = hs[k + t];
            const float cc = coef[t * D + d].x;
            fr = fmaf(cc, hv.x, fr);
            fi = fmaf(cc, hv.z, fi);
        }
        q.re = mk(fr);
        q.im = mk(fi);
    }
    if (rfit == nullptr) {
        st(qs + k * D + d, q);
    } else {
        st(qa + d * GCP + k, q);
        __syncthreads();
        // coefficient n = d of R(y) S(y) = sum_{i,j} (r_j/2) Q_i (T_{i+j} + T_{|i-j|}):
        //   i = n - j (j <= n),  i = n + j,  and i = j - n (j >= n, n > 0)
        if (k < ncb) {
            const int n = d;
            df ar = mk(0.f), ai = mk(0.f);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const float2 rv = rfit[(long long)(ic0 + k) * NR + j];
                const df r = mk(rv.x, rv.y);
                if (j <= n) {
                    const cdf v = ld(qa + (n - j) * GCP + k);
                    acc(ar, mul_u(r, v.re));
                    acc(ai, mul_u(r, v.im));
                }
                if (n + j < D) {
                    const cdf v = ld(qa + (n + j) * GCP + k);
                    acc(ar, mul_u(r, v.re));
                    acc(ai, mul_u(r, v.im));
                }
                if (n > 0 && j >= n && j - n < D) {
                    const cdf v = ld(qa + (j - n) * GCP + k);
                    acc(ar, mul_u(r, v.re));
                    acc(ai, mul_u(r, v.im));
                }
            }
            cdf o;
            o.re = norm(ar);
            o.im = norm(ai);
            st(qs + k * D + n, o);
        }
    }
    __syncthreads();
    float4 *dst = Q4 + (long long)ic0 * D;
    for (int e = threadIdx.x; e < ncb * D; e += NT) dst[e] = qs[e];
}

template <int D>
__global__ void __launch_bounds__(512)
k_gather_conv_df(GridLaunch<float2> L, const float4 *__restrict__ buf_all,
                 float4 *__restrict__ Q_all) {
    extern __shared__ float4 smem4[];
    gather_conv_df_block<D>(L, buf_all, Q_all, blockIdx.x, smem4);
}

// Position-major form for launches with many blocks: one thread per cell with all D
// degrees in registers; the fold reads the thread's own row of sums from shared memory.
template <int D, bool FOLD>
__global__ void __launch_bounds__(GCP)
k_gather_conv_df_pos(GridLaunch<float2> L, const float4 *__restrict__ buf_all,
                     float4 *__restrict__ Q_all) {
    constexpr int B = D / 2;
    constexpr int F = D - B;
    extern __shared__ float4 smem4[];
    const int inst = block_instance(L.blk, L.ninst, blockIdx.x);
    const GridInst<float2> G = L.inst[inst];
    const float4 *__restrict__ buf = buf_all + G.grid_base;
    float4 *__restrict__ Q4 = Q_all + (long long)G.cell_base * D;
    const float2 *__restrict__ rfit = FOLD ? G.rfit : nullptr;
    const int N2 = G.N2;
    const int m = L.m, ntap = 2 * L.m;
    const int nh = GCP + ntap - 1;
    float4 *hs = smem4;                                          // [nh] scaled grid values
    float4 *qa = hs + nh;                                        // [GCP][D] tap sums
    float4 *qs = qa + GCP * D;                                   // [GCP][D] outputs (fold only)
    float2 *coef = reinterpret_cast<float2 *>(qa + (FOLD ? 2 : 1) * GCP * D);   // [ntap][D]
    const int k = threadIdx.x;
    const int ic0 = (blockIdx.x - L.blk[inst]) * GCP;
    const int ncb = min(GCP, G.ncell - ic0);
    const long long pb = G.c_lo + ic0 - m + 1;
    for (int e = k; e < ntap * D; e += GCP) coef[e] = G.coef[e];
    for (int e = k; e < ncb + ntap - 1; e += GCP) {
        const long long p = pb + e;
        cdf h = ld(buf + wrap_index(p, N2));
        if (G.scale != nullptr) {
            const long long si = p + G.scale_off;
            const float2 sc = (si >= 0 && si < G.scale_len) ? G.scale[si] : make_float2(0.f, 0.f);
            h = cscale(h, mk(sc.x, sc.y));
        }
        st(hs + e, h);
    }
    __syncthreads();
    if (k < ncb) {
        df qr[B], qi[B];
        float fr[F], fi[F];
#pragma unroll
        for (int d = 0; d < B; ++d) { qr[d] = mk(0.f); qi[d] = mk(0.f); }
#pragma unroll
        for (int d = 0; d < F; ++d) { fr[d] = 0.f; fi[d] = 0.f; }
        for (int t = 0; t < ntap; ++t) {
            const cdf h = ld(hs + k + t);
#pragma unroll
            for (int d = 0; d < B; ++d) {
                const float2 c2 = coef[t * D + d];
                const df cd = mk(c2.x, c2.y);
                acc(qr[d], mul_u(cd, h.re));
                acc(qi[d], mul_u(cd, h.im));
            }
#pragma unroll
            for (int d = 0; d < F; ++d) {
                const float cc = coef[t * D + B + d].x;
                fr[d] = fmaf(cc, h.re.h, fr[d]);
                fi[d] = fmaf(cc, h.im.h, fi[d]);
            }
        }
#pragma unroll
        for (int d = 0; d < B; ++d) {
            cdf q;
            q.re = norm(qr[d]);
            q.im = norm(qi[d]);
            st(qa + k * D + d, q);
        }
#pragma unroll
        for (int d = 0; d < F; ++d) {
            cdf q;
            q.re = mk(fr[d]);
            q.im = mk(fi[d]);
            st(qa + k * D + B + d, q);
        }
        if (FOLD && rfit != nullptr) {
            const float4 *qk = qa + k * D;
            df r[NR];
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const float2 rv = rfit[(long long)(ic0 + k) * NR + j];
                r[j] = mk(rv.x, rv.y);
            }
#pragma unroll 1
            for (int n = 0; n < D; ++n) {
                df ar = mk(0.f), ai = mk(0.f);
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    if (j <= n) {
                        const cdf v = ld(qk + n - j);
                        acc(ar, mul_u(r[j], v.re));
                        acc(ai, mul_u(r[j], v.im));
                    }
                    if (n + j < D) {
                        const cdf v = ld(qk + n + j);
                        acc(ar, mul_u(r[j], v.re));
                        acc(ai, mul_u(r[j], v.im));
                    }
                    if (n > 0 && j >= n && j - n < D) {
                        const cdf v = ld(qk + j - n);
                        acc(ar, mul_u(r[j], v.re));
                        acc(ai, mul_u(r[j], v.im));
                    }
                }
                cdf o;
                o.re = norm(ar);
                o.im = norm(ai);
                st(qs + k * D + n, o);
            }
        }
    }
    __syncthreads();
    const float4 *src = FOLD && rfit != nullptr ? qs : qa;
    float4 *dst = Q4 + (long long)ic0 * D;
    for (int e = k; e < ncb * D; e += GCP) dst[e] = src[e];
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------------
// The grid stage of one direction in one cooperative launch (GRID_FUSED_VARIANT): every
// block of D * 32 threads is resident; the blocks take the cell fold, the spread
// convolution, FFT pass 1, FFT pass 2 and the gather convolution in turn, each stage's
// blocks (the same block bodies as the stage-wide kernels above) spread round-robin over
// the launch, with a grid-wide barrier between two stages.  A barrier wait that gives up
// (gridsync.cuh) ends every block before its next stage; the plan reports NNFFT_ETIMEOUT.
// Two blocks per SM at most D * 32 threads each bound the registers; the launch takes half
// the resident blocks, so that the two directions' launches fit on the GPU together.
// ---------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(D * 32, 2) k_grid_stage_df(GridStageDf A) {
    extern __shared__ float4 smem4[];
    const unsigned nb = gridDim.x;
    const int ncell = A.fold_side.ncell;
    if (A.fold_tab.rfit != nullptr) {
        const int nv = (ncell + CFP - 1) / CFP;
        for (int vb = blockIdx.x; vb < nv; vb += gridDim.x) {
            cell_fold_df_fit_block<D>(A.fold_side, A.fold_tab, A.P4, A.Q4, vb);
            __syncthreads();
        }
    } else {
        const long long tot = (long long)ncell * D;
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += stride)
            cell_fold_df_elem<D>(A.fold_side, A.fold_tab, A.P4, A.Q4, idx);
    }
    if (!gsync::grid_barrier(A.bar, nb, A.limit, A.status)) return;
    for (int vb = blockIdx.x; vb < A.spread.nblocks; vb += gridDim.x) {
        spread_conv_df_block<D>(A.spread, A.Q4, A.bufA, vb, smem4, SpreadFoldDf{});
        __syncthreads();
    }
    if (!gsync::grid_barrier(A.bar, nb, A.limit, A.status)) return;
    for (int vb = blockIdx.x; vb < A.fft.nblk1; vb += gridDim.x) {
        fft_pass1_df_block(A.bufA, A.bufB, A.fft, A.sign, vb, smem4);
        __syncthreads();
    }
    if (!gsync::grid_barrier(A.bar, nb, A.limit, A.status)) return;
    for (int vb = blockIdx.x; vb < A.fft.nblk2; vb += gridDim.x) {
        fft_pass2_df_block(A.bufB, A.bufC, A.fft, A.sign, vb, smem4);
        __syncthreads();
    }
    if (!gsync::grid_barrier(A.bar, nb, A.limit, A.status)) return;
    for (int vb = blockIdx.x; vb < A.gather.nblocks; vb += gridDim.x) {
        gather_conv_df_block<D>(A.gather, A.bufC, A.Q4, vb, smem4);
        __syncthreads();
    }
}

}  // namespace

#define NNFFT_DISPATCH_DF2(D_, ...)                             \
    switch (D_) {                                               \
        case 8: { constexpr int DD = 8; __VA_ARGS__; } break;   \
        case 10: { constexpr int DD = 10; __VA_ARGS__; } break; \
        case 12: { constexpr int DD = 12; __VA_ARGS__; } break; \
        case 14: { constexpr int DD = 14; __VA_ARGS__; } break; \
        case 16: { constexpr int DD = 16; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                  \
    }

cudaError_t launch_cell_fold_df(const SideK<double> &S, const SideDf &T, const void *P4,
                                void *Pc4, cudaStream_t s) {
    if (S.ncell <= 0) return cudaSuccess;
    const float4 *in = static_cast<const float4 *>(P4);
    float4 *o = static_cast<float4 *>(Pc4);
    if (T.rfit != nullptr) {
        NNFFT_DISPATCH_DF2(S.D, (k_cell_fold_df_fit<DD><<<cdiv(S.ncell, CFP), DD * CFP, 0, s>>>(S, T, in, o)));
    } else {
        NNFFT_DISPATCH_DF2(S.D, (k_cell_fold_df<DD><<<cdiv((long long)S.ncell * S.D, 128), 128, 0, s>>>(S, T, in, o)));
    }
    count_launches(1);
    return cudaGetLastError();
}

int spread_blocks_df(int N2, int D) { return cdiv(N2, SCP); }
int gather_blocks_df(int ncell, int D) { return cdiv(ncell, GCP); }

bool spread_df_folds(const GridLaunch<float2> &L) {
    return L.nblocks > 0 && L.nblocks < POS_MAJOR_BLOCKS_PER_SM * device_sm_count();
}

cudaError_t launch_spread_conv_df(const GridLaunch<float2> &L, const void *Pc4, void *out,
                                  cudaStream_t s, const SpreadFoldDf &F) {
    if (L.nblocks <= 0) return cudaSuccess;
    const int ntap = 2 * L.m;
    const float4 *in = static_cast<const float4 *>(Pc4);
    float4 *o = static_cast<float4 *>(out);
    if (F.P4 != nullptr && !spread_df_folds(L)) return cudaErrorInvalidValue;
    if (L.nblocks >= POS_MAJOR_BLOCKS_PER_SM * device_sm_count()) {
        const size_t sm = sizeof(float4) * (size_t)L.D * (SCP + ntap - 1) +
                          sizeof(float2) * (size_t)ntap * L.D;
        NNFFT_DISPATCH_DF2(L.D, (k_spread_conv_df_pos<DD><<<L.nblocks, SCP, sm, s>>>(L, in, o)));
    } else {
        const size_t sm = sizeof(float4) * (size_t)L.D * (SCP + ntap - 1 + SCP) +
                          sizeof(float2) * (size_t)ntap * L.D +
                          (F.rfit != nullptr ? sizeof(float4) * (size_t)L.D * (SCP + ntap - 1) : 0);
        NNFFT_DISPATCH_DF2(L.D, (k_spread_conv_df<DD><<<L.nblocks, DD * SCP, sm, s>>>(L, in, o, F)));
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fft_df(const FftLaunch<FftDf> &F, const void *in, void *tmp, void *out,
                          int sign, cudaStream_t s) {
    if (F.nblk1 <= 0) return cudaSuccess;
    const size_t sm1 = sizeof(float4) * F.smem1;
    const size_t sm2 = sizeof(float4) * F.smem2;
    if (sm1 > 48 * 1024)
        cudaFuncSetAttribute(k_fft_pass1_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (sm2 > 48 * 1024)
        cudaFuncSetAttribute(k_fft_pass2_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    k_fft_pass1_df<<<F.nblk1, 128, sm1, s>>>(static_cast<const float4 *>(in),
                                              static_cast<float4 *>(tmp), F, sign);
    k_fft_pass2_df<<<F.nblk2, 128, sm2, s>>>(static_cast<const float4 *>(tmp),
                                              static_cast<float4 *>(out), F, sign);
    count_launches(2);
    return cudaGetLastError();
}

size_t fft_cluster_smem(int n1, int n2) {
    const int per1 = (n2 + FFT_CLUSTER - 1) / FFT_CLUSTER, per2 = (n1 + FFT_CLUSTER - 1) / FFT_CLUSTER;
    const size_t cap = (size_t)std::max(per1 * n1, per2 * n2);
    return sizeof(float4) * (3 * cap + (size_t)n1 + (size_t)n2);
}

cudaError_t prepare_fft_cluster_df() {
    // the kernel's limit is one value for every plan: the largest any plan may use
    return cudaFuncSetAttribute(k_fft_cluster_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FFT_CLUSTER_SMEM_MAX);
}

cudaError_t launch_fft_cluster_df(const FftLaunch<FftDf> &F, int n1, int n2, const void *in,
                                  void *out, int sign, cudaStream_t s) {
    const size_t sm = fft_cluster_smem(n1, n2);
    if (F.ninst != 1 || sm > FFT_CLUSTER_SMEM_MAX) return cudaErrorInvalidValue;
    k_fft_cluster_df<<<FFT_CLUSTER, FFT_CLUSTER_THREADS, sm, s>>>(
        static_cast<const float4 *>(in), static_cast<float4 *>(out), F, sign);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_conv_df(const GridLaunch<float2> &L, const void *buf, void *Q4,
                                  cudaStream_t s) {
    if (L.nblocks <= 0) return cudaSuccess;
    const int ntap = 2 * L.m;
    const size_t sm = sizeof(float4) * (size_t)(GCP + ntap - 1 + (L.fold ? 2 : 1) * GCP * L.D) +
                      sizeof(float2) * (size_t)ntap * L.D;
    const float4 *in = static_cast<const float4 *>(buf);
    float4 *o = static_cast<float4 *>(Q4);
    if (L.nblocks >= POS_MAJOR_BLOCKS_PER_SM * device_sm_count()) {
        if (L.fold) {
            NNFFT_DISPATCH_DF2(L.D, (k_gather_conv_df_pos<DD, true><<<L.nblocks, GCP, sm, s>>>(L, in, o)));
        } else {
            NNFFT_DISPATCH_DF2(L.D, (k_gather_conv_df_pos<DD, false><<<L.nblocks, GCP, sm, s>>>(L, in, o)));
        }
    } else {
        NNFFT_DISPATCH_DF2(L.D, (k_gather_conv_df<DD><<<L.nblocks, DD * GCP, sm, s>>>(L, in, o)));
    }
    count_launches(1);
    return cudaGetLastError();
}

size_t grid_stage_df_smem(int D, int m_spread, int m_gather, int smem1, int smem2) {
    const int ts = 2 * m_spread, tg = 2 * m_gather;
    const size_t spread = sizeof(float4) * (size_t)D * (SCP + ts - 1 + SCP) + sizeof(float2) * (size_t)ts * D;
    const size_t gather = sizeof(float4) * (size_t)(GCP + tg - 1 + 2 * GCP * D) + sizeof(float2) * (size_t)tg * D;
    const size_t fft = sizeof(float4) * (size_t)std::max(smem1, smem2);
    return std::max(std::max(spread, gather), fft);
}

namespace {
template <int D>
int prepare_grid_stage_d(size_t smem) {
    if (cudaFuncSetAttribute(k_grid_stage_df<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_grid_stage_df<D>, D * 32, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <int D>
cudaError_t launch_grid_stage_d(const GridStageDf &A, int blocks, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(D * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_grid_stage_df<D>, A);
}
}  // namespace

int prepare_grid_stage_df(int D, size_t smem) {
    switch (D) {
        case 8: return prepare_grid_stage_d<8>(smem);
        case 10: return prepare_grid_stage_d<10>(smem);
        case 12: return prepare_grid_stage_d<12>(smem);
        case 14: return prepare_grid_stage_d<14>(smem);
        case 16: return prepare_grid_stage_d<16>(smem);
        default: return 0;
    }
}

cudaError_t launch_grid_stage_df(const GridStageDf &A, int D, int blocks, size_t smem,
                                 cudaStream_t s) {
    if (blocks <= 0) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (D) {
        case 8: e = launch_grid_stage_d<8>(A, blocks, smem, s); break;
        case 10: e = launch_grid_stage_d<10>(A, blocks, smem, s); break;
        case 12: e = launch_grid_stage_d<12>(A, blocks, smem, s); break;
        case 14: e = launch_grid_stage_d<14>(A, blocks, smem, s); break;
        case 16: e = launch_grid_stage_d<16>(A, blocks, smem, s); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return e;
}

}  // namespace nnfft
