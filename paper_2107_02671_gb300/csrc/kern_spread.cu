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
#include "tma.cuh"

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

// points per lane of a work item (ITEM_CAP points, 32 lanes)
constexpr int PPL = ITEM_CAP / 32;
// points a small-item thread loads at a time
constexpr int SMALL_BATCH = 4;

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
// Warp reduce-scatter of 32 values per lane: after the five halving steps lane L
// holds the warp-wide sum of value L (31 adds per lane instead of 5 x 32).
// ---------------------------------------------------------------------------------
template <typename Real, int O>
__device__ __forceinline__ void rs_step(Real (&v)[32], int lane) {
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const Real send = up ? v[i] : v[O + i];
        const Real keep = up ? v[O + i] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

// ---------------------------------------------------------------------------------
// Cell moments (spread, step 1).  One warp per work item (<= ITEM_CAP sorted
// points of one cell): lanes stride over the points and accumulate
// sum_k val_k T_d(y_k) in registers; the warp then reduces the D complex sums.
// ---------------------------------------------------------------------------------
// Work item of warp w: w itself, or the w-th entry of the big-item list; -1 past the end.
template <typename Real>
__device__ __forceinline__ int warp_item(const SideK<Real> &S, int w) {
    if (S.list_big) return w < *S.n_big ? S.list_big[w] : -1;
    return w < *S.nitems ? w : -1;
}

template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_moments(SideK<Real> S, const C2<Real> *__restrict__ vals, C2<Real> *__restrict__ P) {
    const int item = warp_item(S, (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5));
    const int lane = threadIdx.x & 31;
    if (item < 0) return;
    const int pb = S.item_pb[item], pe = S.item_pe[item];
    Real ar[D], ai[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { ar[d] = Real(0); ai[d] = Real(0); }
    // issue every load of the item first (coordinates and indices, then the gathers)
    Real yv[PPL];
    int jv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int p = pb + lane + 32 * k;
        yv[k] = p < pe ? S.ys[p] : Real(0);
        jv[k] = p < pe ? S.perm[p] : -1;
    }
    C2<Real> fv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) fv[k] = jv[k] >= 0 ? vals[jv[k]] : mk2<Real>(Real(0), Real(0));
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        if (pb + 32 * k >= pe) break;                 // warp-uniform: no point in this round
        Real T[D];
        cheb<Real, D>(yv[k], T);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            ar[d] = fma(fv[k].x, T[d], ar[d]);
            ai[d] = fma(fv[k].y, T[d], ai[d]);
        }
    }
    if constexpr (2 * D <= 32) {
        Real vv[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) vv[i] = Real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            vv[d] = ar[d];
            vv[D + d] = ai[d];
        }
        rs_step<Real, 16>(vv, lane);
        rs_step<Real, 8>(vv, lane);
        rs_step<Real, 4>(vv, lane);
        rs_step<Real, 2>(vv, lane);
        rs_step<Real, 1>(vv, lane);
        Real *Pr = reinterpret_cast<Real *>(P + (long long)item * D);
        if (lane < D) Pr[2 * lane] = vv[0];
        else if (lane < 2 * D) Pr[2 * (lane - D) + 1] = vv[0];
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            ar[d] = warp_sum(ar[d]);
            ai[d] = warp_sum(ai[d]);
        }
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (lane == d) P[(long long)item * D + d] = mk2<Real>(ar[d], ai[d]);
    }
}

// ---------------------------------------------------------------------------------
// Cell moments of small work items (<= SMALL_ITEM points): one thread per item walks
// its points in order, no reduction.
// ---------------------------------------------------------------------------------
template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_moments_small(SideK<Real> S, const C2<Real> *__restrict__ vals, C2<Real> *__restrict__ P) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= *S.n_small) return;
    const int item = S.list_small[idx];
    const int pb = S.item_pb[item], pe = S.item_pe[item];
    Real ar[D], ai[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { ar[d] = Real(0); ai[d] = Real(0); }
    for (int p0 = pb; p0 < pe; p0 += SMALL_BATCH) {   // loads of SMALL_BATCH points first
        Real yv[SMALL_BATCH];
        int jv[SMALL_BATCH];
#pragma unroll
        for (int k = 0; k < SMALL_BATCH; ++k) {
            const int p = p0 + k;
            yv[k] = p < pe ? S.ys[p] : Real(0);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
        C2<Real> fv[SMALL_BATCH];
#pragma unroll
        for (int k = 0; k < SMALL_BATCH; ++k) fv[k] = jv[k] >= 0 ? vals[jv[k]] : mk2<Real>(Real(0), Real(0));
#pragma unroll
        for (int k = 0; k < SMALL_BATCH; ++k) {
            if (jv[k] < 0) break;
            Real T[D];
            cheb<Real, D>(yv[k], T);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                ar[d] = fma(fv[k].x, T[d], ar[d]);
                ai[d] = fma(fv[k].y, T[d], ai[d]);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) P[(long long)item * D + d] = mk2<Real>(ar[d], ai[d]);
}

// ---------------------------------------------------------------------------------
// Cell fold: one thread per cell sums its items' moments (fixed order) into
// Pc[cell][d].  With a 1/phihat1 fit r (adjoint, x side) it also applies the
// per-point factor R(y) = sum_j r_j T_j(y) exactly in the Chebyshev basis,
//   sum_k g_k R(y_k) T_d(y_k) = sum_j r_j (M_{d+j} + M_{|d-j|}) / 2,
// truncated at degree D (the dropped moments carry weight below 1e-16).
// ---------------------------------------------------------------------------------
template <typename Real, int D>
__global__ void __launch_bounds__(128)
k_cell_fold(SideK<Real> S, const C2<Real> *__restrict__ P, C2<Real> *__restrict__ Pc) {
    const int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic >= S.ncell) return;
    Real mr[D], mi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { mr[d] = Real(0); mi[d] = Real(0); }
    const int i0 = S.item_off[ic], i1 = S.item_off[ic + 1];
    for (int it = i0; it < i1; ++it) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const C2<Real> v = P[(long long)it * D + d];
            mr[d] += v.x;
            mi[d] += v.y;
        }
    }
    if (S.rfit != nullptr) {
        Real r[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) r[j] = Real(0.5) * S.rfit[(long long)ic * NR + j];
        Real orr[D], oi[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            Real a = Real(0), b = Real(0);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const int hi = d + j, lo = d > j ? d - j : j - d;
                if (hi < D) { a = fma(r[j], mr[hi], a); b = fma(r[j], mi[hi], b); }
                if (lo < D) { a = fma(r[j], mr[lo], a); b = fma(r[j], mi[lo], b); }
            }
            orr[d] = a;
            oi[d] = b;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) Pc[(long long)ic * D + d] = mk2<Real>(orr[d], oi[d]);
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) Pc[(long long)ic * D + d] = mk2<Real>(mr[d], mi[d]);
    }
}

// ---------------------------------------------------------------------------------
// Spread convolution.  Thread i handles grid position p = p_lo + i (centered
// coordinates; the taps of all cells cover [p_lo, p_hi], which is never wider
// than N2) and writes buffer index p mod N2:
//   g_p = scale(p) * sum_t sum_d coef[t][d] * Pc[p + m - 1 - t][d],
// and 0 for p > p_hi (the zero padding of step 3).  The block's cell range is
// staged in shared memory ([d][cell] layout), coef is broadcast from shared
// memory, and the D partial sums are independent accumulator chains.
// v side (forward): scale = 1/(N1 N2 phihat2(l)); x side (adjoint): scale = 1.
// ---------------------------------------------------------------------------------
constexpr int SC_THREADS = 32;
constexpr int GCN_THREADS = 32;

template <typename Real, int D>
__global__ void __launch_bounds__(SC_THREADS)
k_spread_conv(GridLaunch<Real> L, const C2<Real> *__restrict__ Pc_all,
              C2<Real> *__restrict__ out_all) {
    extern __shared__ unsigned char smem_raw[];
    const int inst = block_instance(L.blk, L.ninst, blockIdx.x);
    const GridInst<Real> G = L.inst[inst];
    const C2<Real> *__restrict__ Pc = Pc_all + (long long)G.cell_base * D;
    C2<Real> *__restrict__ out = out_all + G.grid_base;
    const Real *__restrict__ scale = G.scale;
    const long long scale_off = G.scale_off, scale_len = G.scale_len;
    const int N2 = G.N2;
    const int lb = blockIdx.x - L.blk[inst];
    const int m = L.m, ntap = 2 * L.m;
    const int ncl = SC_THREADS + ntap - 1;                    // staged cells
    Real *coef = reinterpret_cast<Real *>(smem_raw);
    C2<Real> *Ps = reinterpret_cast<C2<Real> *>(coef + ((ntap * D + 1) & ~1));   // [D][ncl]
    const long long p_lo = G.c_lo - m + 1, p_hi = G.c_lo + G.ncell - 1 + m;
    const long long p0 = p_lo + (long long)lb * SC_THREADS;
    const long long cbase = p0 - m;                           // cell of local index 0
    for (int i = threadIdx.x; i < ntap * D; i += SC_THREADS) coef[i] = G.coef[i];
    for (int i = threadIdx.x; i < ncl * D; i += SC_THREADS) {
        const int lc = i / D, d = i - lc * D;
        const long long ic = cbase + lc - G.c_lo;
        C2<Real> v = mk2<Real>(Real(0), Real(0));
        if (ic >= 0 && ic < G.ncell) v = Pc[ic * D + d];
        Ps[d * ncl + lc] = v;
    }
    __syncthreads();
    const long long i = (long long)lb * SC_THREADS + threadIdx.x;
    if (i >= N2) return;
    const long long p = p_lo + i;
    const int q = wrap_index(p, N2);
    if (p > p_hi) {
        out[q] = mk2<Real>(Real(0), Real(0));
        return;
    }
    Real ar[D], ai[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { ar[d] = Real(0); ai[d] = Real(0); }
    const int lbase = threadIdx.x + ntap - 1;                 // local cell of tap t = 0
    for (int t = 0; t < ntap; ++t) {
        const int lc = lbase - t;
        const Real *ct = coef + t * D;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const C2<Real> pv = Ps[d * ncl + lc];
            ar[d] = fma(ct[d], pv.x, ar[d]);
            ai[d] = fma(ct[d], pv.y, ai[d]);
        }
    }
    Real gr = Real(0), gi = Real(0);
#pragma unroll
    for (int d = 0; d < D; ++d) { gr += ar[d]; gi += ai[d]; }
    if (scale != nullptr) {
        const long long si = p + scale_off;
        const Real sc = (si >= 0 && si < scale_len) ? scale[si] : Real(0);
        gr *= sc;
        gi *= sc;
    }
    out[q] = mk2<Real>(gr, gi);
}

// ---------------------------------------------------------------------------------
// Gather convolution: one thread per cell c of the gathering side,
//   Q_c[d] = sum_t coef[t][d] * scale(p) * buf[p mod N2],  p = c - m + 1 + t.
// x side (forward): buf = h of step 3, scale = 1, and the output division by
// phihat1(N* x) is folded in per cell: with R(y) = sum_j r_j T_j(y),
//   R(y) sum_i Q_i T_i(y) = sum_n Q'_n T_n(y),  Q'_n = sum_{i,j} r_j Q_i [n = i+j or |i-j|] / 2,
// truncated at degree D.
// v side (adjoint): buf = the +sign FFT of the x-side spread, scale = 1/(N1 N2 phihat2(l)).
// ---------------------------------------------------------------------------------
template <typename Real, int D>
__global__ void __launch_bounds__(GCN_THREADS)
k_gather_conv(GridLaunch<Real> L, const C2<Real> *__restrict__ buf_all,
              C2<Real> *__restrict__ Q_all) {
    extern __shared__ unsigned char smem_raw[];
    const int inst = block_instance(L.blk, L.ninst, blockIdx.x);
    const GridInst<Real> G = L.inst[inst];
    const C2<Real> *__restrict__ buf = buf_all + G.grid_base;
    C2<Real> *__restrict__ Q = Q_all + (long long)G.cell_base * D;
    const Real *__restrict__ scale = G.scale;
    const Real *__restrict__ rfit = L.fold ? G.rfit : nullptr;
    const long long scale_off = G.scale_off, scale_len = G.scale_len;
    const int N2 = G.N2;
    Real *coef = reinterpret_cast<Real *>(smem_raw);
    const int m = L.m, ntap = 2 * L.m;
    for (int i = threadIdx.x; i < ntap * D; i += blockDim.x) coef[i] = G.coef[i];
    __syncthreads();
    const int ic = (blockIdx.x - L.blk[inst]) * GCN_THREADS + threadIdx.x;
    if (ic >= G.ncell) return;
    const long long c = G.c_lo + ic;
    Real qr[D], qi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { qr[d] = Real(0); qi[d] = Real(0); }
    int qidx = wrap_index(c - m + 1, N2);                     // buffer index of tap 0
    for (int t = 0; t < ntap; ++t, qidx = qidx + 1 == N2 ? 0 : qidx + 1) {
        const long long p = c - m + 1 + t;
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
    if (rfit != nullptr) {
        Real r[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) r[j] = Real(0.5) * rfit[(long long)ic * NR + j];
        Real orr[D], oi[D];
#pragma unroll
        for (int n = 0; n < D; ++n) { orr[n] = Real(0); oi[n] = Real(0); }
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const int hi = i + j, lo = i > j ? i - j : j - i;
                if (hi < D) { orr[hi] = fma(r[j], qr[i], orr[hi]); oi[hi] = fma(r[j], qi[i], oi[hi]); }
                if (lo < D) { orr[lo] = fma(r[j], qr[i], orr[lo]); oi[lo] = fma(r[j], qi[i], oi[lo]); }
            }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) { qr[d] = orr[d]; qi[d] = oi[d]; }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) Q[(long long)ic * D + d] = mk2<Real>(qr[d], qi[d]);
}

// ---------------------------------------------------------------------------------
// Point evaluation (gather, step 4 and the output division).  One warp per work
// item; the cell's D complex coefficients are loaded once (uniform loads) and
// every lane evaluates sum_d T_d(y) Q_c[d] for its points, scattered to the
// caller's order.
// ---------------------------------------------------------------------------------
template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_eval(SideK<Real> S, const C2<Real> *__restrict__ Q, C2<Real> *__restrict__ out) {
    const int item = warp_item(S, (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5));
    const int lane = threadIdx.x & 31;
    if (item < 0) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    Real qr[D], qi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const C2<Real> q = Q[(long long)c * D + d];
        qr[d] = q.x;
        qi[d] = q.y;
    }
    Real yv[PPL];
    int jv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int p = pb + lane + 32 * k;
        yv[k] = p < pe ? S.ys[p] : Real(0);
        jv[k] = p < pe ? S.perm[p] : -1;
    }
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        if (pb + 32 * k >= pe) break;
        Real T[D];
        cheb<Real, D>(yv[k], T);
        Real sr = Real(0), si = Real(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            sr = fma(qr[d], T[d], sr);
            si = fma(qi[d], T[d], si);
        }
        if (jv[k] >= 0) out[jv[k]] = mk2<Real>(sr, si);
    }
}

// ---------------------------------------------------------------------------------
// Team variants: TEAM = 8 lanes per work item, four items per warp.  For sparse cells
// (a few dozen points per item) a whole warp per item leaves most lanes idle and pays a
// 32-lane reduction per item; a team of 8 reduces in 3 exchange steps and every lane has
// points.  Moments: the 2D sums (padded to 32) are reduce-scattered over the team, after
// which lane s of the team holds sums 4s .. 4s+3 (real parts first, then imaginary).
// ---------------------------------------------------------------------------------
constexpr int TEAM = 8;

template <typename Real, int O, int LB>
__device__ __forceinline__ void rs_team(Real (&v)[32], int sub) {
    const bool up = (sub & LB) != 0;
#pragma unroll
    for (int i = 0; i < O; ++i) {
        const Real send = up ? v[i] : v[O + i];
        const Real keep = up ? v[O + i] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, LB);
    }
}

// Points per lane loaded at a time and blocks per SM for the team moments kernel: FP32
// at 4 points and 6 blocks for D <= 8 (40 registers without spills: 75 % occupancy for
// the latency of the value gathers), 4 blocks above; FP64 at the work item's 8 per lane.
template <typename Real, int D> struct TeamCfg {
    static constexpr bool f32 = std::is_same<Real, float>::value;
    static constexpr int CH = f32 ? 4 : PPL;
    static constexpr int MINB = f32 ? (D <= 8 ? 6 : 4) : 1;
};

template <typename Real, int D>
__global__ void __launch_bounds__(256, TeamCfg<Real, D>::MINB)
k_moments_team(SideK<Real> S, const C2<Real> *__restrict__ vals, C2<Real> *__restrict__ P) {
    constexpr int CH = TeamCfg<Real, D>::CH;
    static_assert(2 * D <= 32, "team moments hold at most 16 degrees");
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = threadIdx.x & (TEAM - 1);
    const int item = warp_item(S, gt / TEAM);
    int pb = 0, pe = 0;
    if (item >= 0) {                                 // every lane stays for the exchanges
        pb = S.item_pb[item];
        pe = S.item_pe[item];
    }
    Real ar[D], ai[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { ar[d] = Real(0); ai[d] = Real(0); }
    for (int c0 = pb; c0 < pe; c0 += TEAM * CH) {
        Real yv[CH];
        int jv[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int p = c0 + sub + TEAM * k;
            yv[k] = p < pe ? S.ys[p] : Real(0);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
        C2<Real> fv[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) fv[k] = jv[k] >= 0 ? vals[jv[k]] : mk2<Real>(Real(0), Real(0));
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if (jv[k] < 0) continue;
            Real T[D];
            cheb<Real, D>(yv[k], T);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                ar[d] = fma(fv[k].x, T[d], ar[d]);
                ai[d] = fma(fv[k].y, T[d], ai[d]);
            }
        }
    }
    Real vv[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) vv[i] = Real(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        vv[d] = ar[d];
        vv[D + d] = ai[d];
    }
    rs_team<Real, 16, 4>(vv, sub);
    rs_team<Real, 8, 2>(vv, sub);
    rs_team<Real, 4, 1>(vv, sub);
    if (item < 0) return;
    Real *Pr = reinterpret_cast<Real *>(P + (long long)item * D);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int idx = 4 * sub + t;
        if (idx < D) Pr[2 * idx] = vv[t];
        else if (idx < 2 * D) Pr[2 * (idx - D) + 1] = vv[t];
    }
}

template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_eval_team(SideK<Real> S, const C2<Real> *__restrict__ Q, C2<Real> *__restrict__ out) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = threadIdx.x & (TEAM - 1);
    const int item = warp_item(S, gt / TEAM);
    if (item < 0) return;
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    Real qr[D], qi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const C2<Real> q = Q[(long long)c * D + d];
        qr[d] = q.x;
        qi[d] = q.y;
    }
    for (int c0 = pb; c0 < pe; c0 += TEAM * PPL) {
        Real yv[PPL];
        int jv[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int p = c0 + sub + TEAM * k;
            yv[k] = p < pe ? S.ys[p] : Real(0);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            if (jv[k] < 0) continue;
            Real T[D];
            cheb<Real, D>(yv[k], T);
            Real sr = Real(0), si = Real(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                sr = fma(qr[d], T[d], sr);
                si = fma(qi[d], T[d], si);
            }
            out[jv[k]] = mk2<Real>(sr, si);
        }
    }
}

// Flat point evaluation: one thread per sorted point, its cell read from the sorted cell
// keys.  There is no work-item indirection, the point loads are coalesced, and threads of
// the same cell share the cell's coefficients through L1; for sparse cells this hides
// far more latency than item teams, at 4 extra bytes (the key) per point.
template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_eval_flat(SideK<Real> S, const C2<Real> *__restrict__ Q, C2<Real> *__restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.M) return;
    const int c = (int)S.keys[p];
    const Real y = S.ys[p];
    const int j = S.perm[p];
    const C2<Real> *q = Q + (long long)c * D;
    Real T[D];
    cheb<Real, D>(y, T);
    Real sr = Real(0), si = Real(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const C2<Real> qd = q[d];
        sr = fma(qd.x, T[d], sr);
        si = fma(qd.y, T[d], si);
    }
    out[j] = mk2<Real>(sr, si);
}

// The flat evaluation with the block's cells [c0, c1] staged in shared memory by one bulk
// (TMA) copy of Q[c0*D .. (c1+1)*D) (see k_eval_df_flat_tma); blocks spanning more than
// TMA_MAX_CELLS cells read Q from global memory.
template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_eval_flat_tma(SideK<Real> S, const C2<Real> *__restrict__ Q, C2<Real> *__restrict__ out) {
    __shared__ __align__(128) C2<Real> qs[TMA_MAX_CELLS * D];
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
            const unsigned bytes = (unsigned)nc * D * (unsigned)sizeof(C2<Real>);
            tma::bar_expect(&bar, bytes);
            tma::copy_g2s(qs, Q + (long long)c0 * D, bytes, &bar);
        }
        __syncthreads();
    }
    int c = 0, j = -1;
    Real y = Real(0);
    if (p < S.M) {
        c = (int)S.keys[p];
        y = S.ys[p];
        j = S.perm[p];
    }
    const C2<Real> *q = Q + (long long)c * D;
    if (staged) {
        if (!tma::bar_wait(&bar, 0, tma::WAIT_LIMIT_CYCLES)) {
            if (threadIdx.x == 0) atomicOr(S.status, STATUS_TIMEOUT);
            tma::bar_wait(&bar, 0, tma::WAIT_LIMIT_CYCLES);
            return;
        }
        q = qs + (c - c0) * D;
    }
    if (p >= S.M) return;
    Real T[D];
    cheb<Real, D>(y, T);
    Real sr = Real(0), si = Real(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const C2<Real> qd = q[d];
        sr = fma(qd.x, T[d], sr);
        si = fma(qd.y, T[d], si);
    }
    out[j] = mk2<Real>(sr, si);
}

// Point evaluation of small work items: one thread per item.
template <typename Real, int D>
__global__ void __launch_bounds__(256)
k_eval_small(SideK<Real> S, const C2<Real> *__restrict__ Q, C2<Real> *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= *S.n_small) return;
    const int item = S.list_small[idx];
    const int c = S.item_cell[item], pb = S.item_pb[item], pe = S.item_pe[item];
    Real qr[D], qi[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const C2<Real> q = Q[(long long)c * D + d];
        qr[d] = q.x;
        qi[d] = q.y;
    }
    for (int p0 = pb; p0 < pe; p0 += SMALL_BATCH) {
        Real yv[SMALL_BATCH];
        int jv[SMALL_BATCH];
#pragma unroll
        for (int k = 0; k < SMALL_BATCH; ++k) {
            const int p = p0 + k;
            yv[k] = p < pe ? S.ys[p] : Real(0);
            jv[k] = p < pe ? S.perm[p] : -1;
        }
#pragma unroll
        for (int k = 0; k < SMALL_BATCH; ++k) {
            if (jv[k] < 0) break;
            Real T[D];
            cheb<Real, D>(yv[k], T);
            Real sr = Real(0), si = Real(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                sr = fma(qr[d], T[d], sr);
                si = fma(qi[d], T[d], si);
            }
            out[jv[k]] = mk2<Real>(sr, si);
        }
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
cudaError_t launch_cell_fold(const SideK<Real> &S, const void *P, void *Pc, cudaStream_t s) {
    if (S.ncell > 0) {
        NNFFT_DISPATCH_D(S.D, (k_cell_fold<Real, DD><<<cdiv(S.ncell, 128), 128, 0, s>>>(
                                  S, static_cast<const C2<Real> *>(P), static_cast<C2<Real> *>(Pc))));
        count_launches(1);
    }
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_moments(const SideK<Real> &S, const void *vals, void *P, int lanes,
                           cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    const C2<Real> *v = static_cast<const C2<Real> *>(vals);
    C2<Real> *Pp = static_cast<C2<Real> *>(P);
    if (lanes == TEAM && S.D <= 16) {
        const int blocks = cdiv((long long)S.max_items * TEAM, 256);
        NNFFT_DISPATCH_D(S.D, (k_moments_team<Real, (DD <= 16 ? DD : 16)><<<blocks, 256, 0, s>>>(S, v, Pp)));
    } else {
        const int blocks = cdiv((long long)S.max_items * 32, 256);
        NNFFT_DISPATCH_D(S.D, (k_moments<Real, DD><<<blocks, 256, 0, s>>>(S, v, Pp)));
    }
    count_launches(1);
    if (S.list_small) {
        NNFFT_DISPATCH_D(S.D, (k_moments_small<Real, DD><<<cdiv(S.max_items, 256), 256, 0, s>>>(S, v, Pp)));
        count_launches(1);
    }
    return cudaGetLastError();
}

int spread_blocks_native(int N2, int D) { return cdiv(N2, SC_THREADS); }
int gather_blocks_native(int ncell, int D) { return cdiv(ncell, GCN_THREADS); }

template <typename Real>
cudaError_t launch_spread_conv(const GridLaunch<Real> &L, const void *Pc, void *out,
                               cudaStream_t s) {
    if (L.nblocks <= 0) return cudaSuccess;
    const int ntap = 2 * L.m;
    const size_t sm = sizeof(Real) * (size_t)((ntap * L.D + 1) & ~1) +
                      sizeof(C2<Real>) * (size_t)L.D * (SC_THREADS + ntap - 1);
    const C2<Real> *pc = static_cast<const C2<Real> *>(Pc);
    C2<Real> *o = static_cast<C2<Real> *>(out);
    NNFFT_DISPATCH_D(L.D, (k_spread_conv<Real, DD><<<L.nblocks, SC_THREADS, sm, s>>>(L, pc, o)));
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_gather_conv(const GridLaunch<Real> &L, const void *buf, void *Q,
                               cudaStream_t s) {
    if (L.nblocks <= 0) return cudaSuccess;
    const size_t sm = sizeof(Real) * 2 * L.m * L.D;
    const C2<Real> *b = static_cast<const C2<Real> *>(buf);
    C2<Real> *q = static_cast<C2<Real> *>(Q);
    NNFFT_DISPATCH_D(L.D, (k_gather_conv<Real, DD><<<L.nblocks, GCN_THREADS, sm, s>>>(L, b, q)));
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_eval(const SideK<Real> &S, const void *Q, void *out, int lanes,
                        cudaStream_t s) {
    if (S.max_items <= 0) return cudaSuccess;
    const C2<Real> *q = static_cast<const C2<Real> *>(Q);
    C2<Real> *o = static_cast<C2<Real> *>(out);
    if (lanes == EVAL_FLAT) {                       // covers every point: no small-item pass
        if (S.M <= 0) return cudaSuccess;
        NNFFT_DISPATCH_D(S.D, (k_eval_flat<Real, DD><<<cdiv(S.M, 256), 256, 0, s>>>(S, q, o)));
        count_launches(1);
        return cudaGetLastError();
    }
    if (lanes == EVAL_FLAT_TMA) {
        if (S.M <= 0) return cudaSuccess;
        NNFFT_DISPATCH_D(S.D, (k_eval_flat_tma<Real, DD><<<cdiv(S.M, 256), 256, 0, s>>>(S, q, o)));
        count_launches(1);
        return cudaGetLastError();
    }
    if (lanes == TEAM) {
        const int blocks = cdiv((long long)S.max_items * TEAM, 256);
        NNFFT_DISPATCH_D(S.D, (k_eval_team<Real, DD><<<blocks, 256, 0, s>>>(S, q, o)));
    } else {
        const int blocks = cdiv((long long)S.max_items * 32, 256);
        NNFFT_DISPATCH_D(S.D, (k_eval<Real, DD><<<blocks, 256, 0, s>>>(S, q, o)));
    }
    count_launches(1);
    if (S.list_small) {
        NNFFT_DISPATCH_D(S.D, (k_eval_small<Real, DD><<<cdiv(S.max_items, 256), 256, 0, s>>>(S, q, o)));
        count_launches(1);
    }
    return cudaGetLastError();
}

#define NNFFT_INST(R)                                                                      \
    template cudaError_t launch_moments<R>(const SideK<R> &, const void *, void *, int,    \
                                           cudaStream_t);                                  \
    template cudaError_t launch_spread_conv<R>(const GridLaunch<R> &, const void *, void *, \
                                               cudaStream_t);                              \
    template cudaError_t launch_gather_conv<R>(const GridLaunch<R> &, const void *, void *, \
                                               cudaStream_t);                              \
    template cudaError_t launch_cell_fold<R>(const SideK<R> &, const void *, void *,       \
                                             cudaStream_t);                                \
    template cudaError_t launch_eval<R>(const SideK<R> &, const void *, void *, int,       \
                                        cudaStream_t);

NNFFT_INST(double)
NNFFT_INST(float)

}  // namespace nnfft
