// kern_nodes.cu -- step 0 of Algorithm 2.2 for one node side: bin every node by
// the grid cell it falls in, sort the nodes by cell (stable LSD radix sort with
// digits of at most 8 bits), and build the per-cell offsets and the work items that the
// spread / gather kernels walk.  Deterministic: no order depends on timing.
#include <type_traits>

#include "internal.h"

namespace nnfft {

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Rank of this lane's key among the warp's 32 keys of one round, stably by bin d: every
// valid lane sets its bit in the warp's mask of bin d (one shared-memory atomicOr), and the
// mask read back is the set of lanes with the same bin; the lowest of them adds their
// number to the warp's bin counter and clears the mask for the next round.  rank = the
// counter before this round + the lanes of the same bin below this one (the same ranks
// as intersecting the ballots of the bits of d, in fewer issue slots).  mm: the warp's
// masks, zero on entry and on return; cnt: the warp's counters.
// The passes that move no carried 4-byte coordinates (the fp64 sorts) rank this way:
// measured at 2^20 keys per side, both sides' sorts 70 -> 66 us and the fp64 step 166 -> 162
// us; at 512 instances the fp64 node stage 3.56 -> 3.44 ms.  The passes that carry 4-byte
// coordinates (fp32) keep the ballots: ranked this way the 512-instance fp32 node stage took
// 3.41 ms against 3.14, and the single-instance sorts were no faster.
__device__ __forceinline__ int rank_or(unsigned *mm, int *cnt, unsigned d, bool valid,
                                       unsigned lt, int lane) {
    if (valid) atomicOr(&mm[d], 1u << lane);
    __syncwarp();
    unsigned peers = 0u;
    int before = 0;
    if (valid) {
        peers = mm[d];
        before = cnt[d];
    }
    __syncwarp();
    if (valid && (peers & lt) == 0) {
        cnt[d] = before + __popc(peers);
        mm[d] = 0u;
    }
    __syncwarp();
    return before + __popc(peers & lt);
}

// Cell and local coordinate of a node t in fixed point, with integer operations only.
// |t| is truncated to X = |t| 2^62 (exact for |t| >= 2^-10, absolute error < 2^-62), the
// scale is S = scale 2^FX_SB, so A = X S = |u| 2^(62 + FX_SB) exactly in 128 bits
// (|u| < 2^19).  Its integer part gives floor |u|, its top 63 fraction bits the local
// coordinate; for t < 0 the cell is -floor|u| - 1 (or -|u| when u is an integer).
// The error in u is below 2^-46 + 2^-62 |scale| (an FP64 product would round u to 2^-40).
// Returns false for |t| > 1/2 and NaN / Inf.  On success c = floor(u) and
// Y = (2 (u - c) - 1) 2^63 as a signed 64-bit integer.
constexpr int FX_SB = 44;   // matches the host's cell map
__device__ __forceinline__ bool node_fixed(double t, unsigned long long S, long long &c,
                                           long long &Y) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    const unsigned long long mant = (b & 0xfffffffffffffULL) | (e ? (1ULL << 52) : 0ULL);
    const bool ok = e < 1022u || (e == 1022u && mant == (1ULL << 52));
    unsigned long long X = 0;                              // |t| 2^62 = mant 2^(e - 1013)
    if (e >= 1013u && e <= 1022u) X = mant << (e - 1013u);
    else if (e > 949u && e < 1013u) X = mant >> (1013u - e);
    const unsigned long long lo = X * S, hi = __umul64hi(X, S);
    constexpr int SH = 62 + FX_SB - 64;                    // integer part = hi >> SH
    const unsigned long long ip = hi >> SH;
    const unsigned long long fm = hi & ((1ULL << SH) - 1);
    const unsigned long long f63 = (fm << (63 - SH)) | (lo >> (SH + 1));   // top 63 bits
    unsigned long long frac;
    if ((b >> 63) == 0) {
        c = (long long)ip;
        frac = f63;
    } else if ((fm | lo) == 0) {
        c = -(long long)ip;
        frac = 0;
    } else {
        c = -(long long)ip - 1;
        frac = (~f63) & 0x7fffffffffffffffULL;             // 1 - f, to 2^-63
    }
    Y = (long long)((frac << 1) ^ 0x8000000000000000ULL);  // 2 frac - 1, times 2^63
    return ok;
}

// The local coordinate y = Y 2^-63 (Y a signed 64-bit fixed-point value) as floats built
// from 32-bit conversions.  The node kernel is bound by the integer ALU pipe, and a 64-bit
// integer -> float conversion runs on the FP64 pipe (1/64 of the FP32 rate on GB300), so
// both formats start from the top word T = floor(Y / 2^32) (a signed 32-bit integer) and
// the low word L = Y - T 2^32 in [0, 2^32):
//   * fp32 plans: y ~ RN(T) 2^-31, |error| < 2^-31 + half an ulp;
//   * split plans, a float pair h + l: h = RN(T) 2^-31; the exact integer remainder
//     e = T - RN(T) (|e| <= 64) and L give l = RN(e 2^-31 + RN(L) 2^-63), so
//     |h + l - y| <= 2^-49 + 2^-56; then renormalised with Fast2Sum (|h| >= |l| or h = 0).
__device__ __forceinline__ float fixed63_to_float32(long long Y) {
    return __int2float_rn((int)(Y >> 32)) * 0x1p-31f;
}
__device__ __forceinline__ float2 fixed63_to_pair(long long Y) {
    const int top = (int)(Y >> 32);
    const unsigned low = (unsigned)(Y & 0xffffffffLL);
    const float hf = __int2float_rn(top);
    int e = top - __float2int_rn(hf);
    if (hf >= 0x1p31f) e -= 1;                    // the conversion saturates at 2^31 - 1
    const float h = hf * 0x1p-31f;
    const float l = fmaf(__int2float_rn(e), 0x1p-31f, __uint2float_rn(low) * 0x1p-63f);
    const float sh = h + l;                       // Fast2Sum
    return make_float2(sh, l - (sh - h));
}

// Store the local coordinate y = Y 2^-63 in the plan's format:
//   0: float (fp32 plans), 1: double (fp64 plans), 2: float pair hi + lo (split plans).
__device__ __forceinline__ void store_y(void *yout, int fmt, long long i, long long Y) {
    if (fmt == 0) {
        static_cast<float *>(yout)[i] = fixed63_to_float32(Y);
    } else if (fmt == 1) {
        static_cast<double *>(yout)[i] = __ll2double_rn(Y) * 0x1p-63;
    } else {
        static_cast<float2 *>(yout)[i] = fixed63_to_pair(Y);
    }
}

// Points of sort tile t and their instance: instance-aligned tiles of a batch, or tiles of
// SORT_TILE consecutive points of a single instance.
struct TileSpan {
    long long begin, end;
    int inst;
};
__device__ __forceinline__ TileSpan tile_span(const SortTiles &st, int t, int n) {
    TileSpan r;
    if (st.inst == nullptr) {
        r.inst = 0;
        r.begin = (long long)t * SORT_TILE;
        r.end = min(r.begin + SORT_TILE, (long long)n);
    } else {
        r.inst = st.inst[t];
        r.begin = st.start[t];
        r.end = min(r.begin + SORT_TILE, st.pt_off[r.inst + 1]);
    }
    return r;
}

// Step 0 for one node side in a single pass over the nodes: validate each node,
// compute its cell key (cell_base + c - c_lo) and local coordinate y = 2 (u - c) - 1
// (c = floor(u), u = node * scale, node_fixed), store y (caller order) in the plan's
// format, and count the digits of the first radix pass (of c - c_lo, the local cell: its
// low digit, or its high digit (c - c_lo) >> shift0 for the two-stage sort) for this
// block's tile (the tiles of the sort passes), into the per-tile counts and the digit
// totals of the tile's instance.
__global__ void __launch_bounds__(SORT_THREADS)
k_node_keys_y(const double *__restrict__ nodes, int n, NodeInst one, SortTiles st,
              uint32_t *__restrict__ keys, void *__restrict__ yout, int yfmt, int ntiles,
              int shift0, unsigned mask0, int *__restrict__ hist, int *__restrict__ tot,
              int *status) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    const TileSpan sp = tile_span(st, blockIdx.x, n);
    const NodeInst I = st.inst == nullptr ? one : st.tab[sp.inst];
    __syncthreads();
    constexpr int PER = SORT_TILE / SORT_THREADS;
    double xv[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {            // all loads of the thread first
        const long long i = sp.begin + threadIdx.x + (long long)r * SORT_THREADS;
        xv[r] = i < sp.end ? nodes[i] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const long long i = sp.begin + threadIdx.x + (long long)r * SORT_THREADS;
        if (i >= sp.end) break;
        long long c = 0, Y = -0x7fffffffffffffffLL - 1;
        long long ic = 0;
        if (!node_fixed(xv[r], I.S, c, Y)) {
            atomicOr(status, STATUS_RANGE);
            Y = -0x7fffffffffffffffLL - 1;
        } else {
            ic = c - I.c_lo;
            if (ic < 0 || ic >= I.ncell) {
                atomicOr(status, STATUS_INTERNAL);
                ic = ic < 0 ? 0 : I.ncell - 1;
            }
        }
        keys[i] = (uint32_t)(ic + I.cell_base);
        store_y(yout, yfmt, i, Y);
        atomicAdd(&h[(ic >> shift0) & mask0], 1);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
    if (h[threadIdx.x]) atomicAdd(&tot[sp.inst * 256 + threadIdx.x], h[threadIdx.x]);
}

// ---- radix sort ------------------------------------------------------------------
__global__ void __launch_bounds__(SORT_THREADS)
k_sort_upsweep(const uint32_t *__restrict__ keys, int n, int shift, unsigned mask, SortTiles st, int ntiles,
               int *__restrict__ hist, int *__restrict__ tot) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    const TileSpan sp = tile_span(st, blockIdx.x, n);
    const uint32_t cb = st.inst == nullptr ? 0u : (uint32_t)st.tab[sp.inst].cell_base;
    __syncthreads();
    for (long long i = sp.begin + threadIdx.x; i < sp.end; i += SORT_THREADS)
        atomicAdd(&h[((keys[i] - cb) >> shift) & mask], 1);
    __syncthreads();
    hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
    if (h[threadIdx.x]) atomicAdd(&tot[sp.inst * 256 + threadIdx.x], h[threadIdx.x]);   // order-free
}

// Exclusive scan of a batch's digit-major tile counts, one warp per (instance, digit):
// the digit's first position in the instance's sorted range (the instance's first point
// plus its keys with a smaller digit), then a scan over the instance's tiles.
__global__ void __launch_bounds__(256)
k_seg_scan(int *__restrict__ hist, int ntiles, const int *__restrict__ tot, SortTiles st) {
    const int g = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int inst = g >> 8, d = g & 255;
    if (inst >= st.ninst) return;
    const int *ti = tot + inst * 256;
    int part = 0;
    for (int j = lane; j < d; j += 32) part += ti[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    int carry = (int)st.pt_off[inst] + part;
    const int t0 = st.inst_tile0[inst], t1 = st.inst_tile0[inst + 1];
    int *row = hist + (long long)d * ntiles;
    for (int t = t0; t < t1; t += 32) {
        const int i = t + lane;
        const int v = i < t1 ? row[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (i < t1) row[i] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Exclusive scan of the digit-major histogram: block d scans row d (the counts of
// digit d in every tile) starting from the number of keys with a smaller digit,
// sum_{d' < d} digit_tot[d'].  Rows of up to 8 x 256 tiles (2^22 keys): thread t loads its
// contiguous share of at most 8 counts together with the digit totals (one round of
// loads), a block scan of the 256 thread sums gives each thread its start, and the thread
// writes its share.  Longer rows: warp w owns a contiguous eighth of the row, a first pass
// sums it, a block scan of the eight warp totals gives each warp its start, and a second
// pass scans the warp's segment in chunks of 32 with a running carry.
__global__ void __launch_bounds__(256)
k_sort_scan_rows(int *__restrict__ hist, int nblocks, const int *__restrict__ digit_tot) {
    __shared__ int wsum[8];
    __shared__ int dbase[8];
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int *row = hist + (long long)d * nblocks;
    const int per = (nblocks + 255) / 256;
    if (per <= 8) {
        const int a = tid * per;
        int v[8];
        int t = tid < d ? digit_tot[tid] : 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (q < per && a + q < nblocks) ? row[a + q] : 0;
        int s = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[w] = incl;
        if (lane == 0) dbase[w] = t;
        __syncthreads();
        int pre = incl - s;
#pragma unroll
        for (int k = 0; k < 8; ++k) pre += dbase[k] + (k < w ? wsum[k] : 0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q < per && a + q < nblocks) {
                row[a + q] = pre;
                pre += v[q];
            }
        }
        return;
    }
    int t = tid < d ? digit_tot[tid] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) dbase[w] = t;
    const int seg = (((nblocks + 7) / 8) + 31) & ~31;
    const int a = min(w * seg, nblocks), b = min(a + seg, nblocks);
    int s = 0;
#pragma unroll 4
    for (int i = a + lane; i < b; i += 32) s += row[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[w] = s;
    __syncthreads();
    int pre = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) pre += dbase[k] + (k < w ? wsum[k] : 0);
    for (int i0 = a; i0 < b; i0 += 32) {
        const int i = i0 + lane;
        const int v = i < b ? row[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (i < b) row[i] = pre + incl - v;
        pre += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Stable scatter.  Warp w of a block owns 32 * ROUNDS consecutive keys of the
// tile and visits them in ROUNDS rounds of 32 in index order; within a round lanes with the
// same digit are ranked by lane (ballots of the digit bits), across rounds by a per-warp
// digit counter, and across warps by an exclusive scan of those counters.  So keys
// with equal digits keep their input order.  The tile is first reordered by digit in
// shared memory and then written out in that order, so each digit's run of the tile
// leaves as consecutive addresses (coalesced) instead of one scattered store per key.
// FIRST: the values are the identity (vin unused).  Y: the local coordinates, or void.
// A 4-byte Y is carried through every pass with its key (yout[pos] = yin[input position],
// read coalesced); an 8-byte Y (float pairs) is gathered in the last pass only,
// yout[pos] = yin[value] (measured: carrying pays for 4 bytes and costs for 8, whose
// random reads fetch a larger share of each sector).  The digit, (key - cell_base of the
// tile's instance) >> shift & mask, is at most 8 bits wide (NARROW: mask < 255; else the
// literal 255, measured cheaper for the fp64 batch's scatters).  MATCH: the lanes with the
// same digit from one match instruction instead of nine ballots (measured: fewer issue
// slots, faster for large sorts; longer latency, slower for small ones).  Otherwise a pass
// without carried coordinates ranks by shared-memory masks (rank_or), one that carries them
// by the ballots.  The ballot-ranked
// passes that move 8-byte coordinates (the sorts below 8M keys) are bounded to four blocks
// per SM (64 registers, no spills; 73 unbounded, three blocks per SM, so that a 2^20-key
// sort's 512 tiles took two waves on 152 SMs: node stage 95 -> 93.6 us per side); the others
// keep the compiler's choice (minimum 0: unspecified; the bound measured 2 % slower on the
// match-ranked pass of the fp64 batch).
template <bool FIRST, typename Y, bool MATCH, bool NARROW>
__global__ void __launch_bounds__(SORT_THREADS,
                                  std::is_same<Y, unsigned long long>::value && !MATCH ? 4 : 0)
k_sort_scatter(const uint32_t *__restrict__ kin, const int *__restrict__ vin,
               uint32_t *__restrict__ kout, int *__restrict__ vout, int n, int shift,
               unsigned mask_arg, SortTiles st, int ntiles, const int *__restrict__ hist_scanned,
               const Y *__restrict__ yin, Y *__restrict__ yout) {
    const unsigned mask = NARROW ? mask_arg : 255u;
    constexpr int WARPS = SORT_THREADS / 32;
    constexpr int ROUNDS = SORT_TILE / SORT_THREADS;   // 8
    static_assert(SORT_THREADS == 256, "one thread per digit in the digit scans");
    __shared__ int cnt[WARPS][256];
    __shared__ int lstart[256];          // first tile-local slot of each digit
    __shared__ int delta[256];           // global position - tile-local slot, per digit
    __shared__ int wtot[WARPS];
    __shared__ uint32_t skey[SORT_TILE];
    __shared__ int sval[SORT_TILE];
    using YS = typename std::conditional<std::is_void<Y>::value, char, Y>::type;
    constexpr bool CARRY = !std::is_void<Y>::value && sizeof(YS) == 4;
    __shared__ YS sy[CARRY ? SORT_TILE : 1];
    constexpr bool OR = !MATCH && !CARRY;       // ranked by rank_or
    __shared__ unsigned mmask[OR ? WARPS : 1][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) {
        cnt[w][d] = 0;
        if constexpr (OR) mmask[w][d] = 0u;
    }
    __syncwarp();
    const TileSpan sp = tile_span(st, blockIdx.x, n);
    const uint32_t cb = st.inst == nullptr ? 0u : (uint32_t)st.tab[sp.inst].cell_base;
    const long long tile0 = sp.begin;
    const long long base = tile0 + (long long)w * (32 * ROUNDS);
    uint32_t key[ROUNDS];
    int val[ROUNDS], rank[ROUNDS];
    YS yv[CARRY ? ROUNDS : 1];
    const unsigned lt = lanemask_lt();
    // issue every load of the warp's keys (and values) before the ranking rounds
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const long long idx = base + r * 32 + lane;
        const bool valid = idx < sp.end;
        key[r] = valid ? kin[idx] : 0u;
        if (FIRST) val[r] = (int)idx;
        else val[r] = valid ? vin[idx] : 0;
        if constexpr (CARRY) yv[r] = valid ? yin[idx] : YS(0);
    }
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const long long idx = base + r * 32 + lane;
        const bool valid = idx < sp.end;
        const unsigned d = valid ? (((key[r] - cb) >> shift) & mask) : 256u;
        if constexpr (OR) {
            rank[r] = rank_or(mmask[w], cnt[w], d, valid, lt, lane);
            continue;
        }
        // lanes with the same 9-bit value d (256 marks an invalid lane)
        unsigned peers = 0xffffffffu;
        if constexpr (MATCH) {
            peers = __match_any_sync(0xffffffffu, d);
        } else {                                  // intersect the ballots of the bits of d
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const unsigned bit = (d >> b) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
        }
        const int before = valid ? cnt[w][d] : 0;
        __syncwarp();
        if (valid && (peers & lt) == 0) cnt[w][d] += __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {   // digit d = threadIdx.x: exclusive scan over warps, then over digits (tile-local)
        const int d = threadIdx.x;
        int run = 0;
#pragma unroll
        for (int ww = 0; ww < WARPS; ++ww) {
            const int t = cnt[ww][d];
            cnt[ww][d] = run;
            run += t;
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wtot[w] = incl;
        __syncthreads();
        int wpre = 0;
#pragma unroll
        for (int ww = 0; ww < WARPS; ++ww) wpre += ww < w ? wtot[ww] : 0;
        const int start = wpre + incl - run;
        lstart[d] = start;
        delta[d] = hist_scanned[(long long)d * ntiles + blockIdx.x] - start;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const long long idx = base + r * 32 + lane;
        if (idx < sp.end) {
            const unsigned d = ((key[r] - cb) >> shift) & mask;
            const int loc = lstart[d] + cnt[w][d] + rank[r];
            skey[loc] = key[r];
            sval[loc] = val[r];
            if constexpr (CARRY) sy[loc] = yv[r];
        }
    }
    __syncthreads();
    const int tn = (int)(sp.end - tile0);
    for (int i = threadIdx.x; i < tn; i += SORT_THREADS) {
        const uint32_t k = skey[i];
        const int v = sval[i];
        const int pos = delta[((k - cb) >> shift) & mask] + i;
        kout[pos] = k;
        vout[pos] = v;
        if constexpr (CARRY) yout[pos] = sy[i];
        else if constexpr (!std::is_void<Y>::value) yout[pos] = yin[v];
    }
}

// Second stage of the two-stage sort (see radix_sort_cells_local): the keys arrive
// stably partitioned by their high digit key >> lbits (bucket b is the position range
// [hist[b ntiles], hist[(b + 1) ntiles]) of the first pass's scanned digit-major counts),
// in input order within each bucket, and are sorted stably by the low lbits bits (the
// cell within the bucket, NB = 2^lbits bins).  A block takes one range of a bucket:
//   * a single instance splits every bucket into ranges of local_range keys (clustered
//     nodes make some buckets many times larger than others), each block finding its
//     bucket and range from the bucket sizes;
//   * a batch (st.inst != nullptr) takes one block per (instance, bucket), whole buckets.
// The block counts the bucket's keys per bin (their first positions are the cell offsets
// and, for dense plans (per_cell_first), one work item per cell; a cell above cap sets
// *overflow and the scan-based item builder runs next; the bucket's first block writes
// them) and the keys of its bucket before its range per bin (run[]).  Then its range in
// chunks: ranks within the chunk as in k_sort_scatter (per-warp counters; rank_or, or the
// ballots of the digit bits when 4-byte coordinates are carried), the chunk reordered by bin in shared memory and written out bin run by
// bin run (coalesced) after the same bin's earlier keys.  So the result is the stable
// sort by cell, the same order as the LSD passes.  The coordinates: 4-byte ones are
// carried (yin in first-pass order), 8-byte ones gathered from the caller-order array
// (yin[value]).
// Blocks of 256 threads (several per SM, so that one block's barrier waits overlap another's
// work): a batch takes one per (instance, bucket), a single instance one per range of
// local_range(256) = 2048 keys of a bucket.  Measured at 2^20 uniform keys: 1024-thread
// blocks over 8192-key ranges (one range per bucket, every key counted once instead of
// four times) took 28.3 us per launch against 23.5 us.  A chunk is 8 rounds of 256 keys
// (a whole 2048-key range at once): measured 1-3 % faster per step than 4 rounds; 4096-key
// ranges and a 5-blocks-per-SM register bound measured no better.
constexpr int LOCAL_ROUNDS = 8;
constexpr int LOCAL_SINGLE_THREADS = 256;
__host__ __device__ constexpr int local_range(int threads) { return threads * 8; }
__host__ __device__ constexpr int local_min_blocks(int threads) { return threads >= 1024 ? 1 : 4; }
// keys per thread loaded at a time by the counting pass over a bucket
constexpr int LOCAL_COUNT_UNROLL = 16;

__host__ __device__ constexpr size_t local_sort_smem(int threads, int lbits, int ybytes) {
    return sizeof(int) * ((size_t)(threads / 32) * (1u << lbits) * (ybytes == 4 ? 1u : 2u) +
                          5u * (1u << lbits) + 32u) +
           (size_t)threads * LOCAL_ROUNDS * (sizeof(uint32_t) + sizeof(int) + (ybytes == 4 ? 4u : 0u));
}

// A batch (st.inst != nullptr) sorts each instance by its local cell: block -> (instance
// i, bucket b) through blk_first, the bucket's range from the instance's first tile's
// scanned counts, bins of key - cell_base_i; ncell is then the side's total cell count.
template <int LOCAL_THREADS, typename Y, bool CARRY>
__device__ __forceinline__ void
sort_local_body(const uint32_t *__restrict__ kin, const int *__restrict__ vin,
                const Y *__restrict__ yin, uint32_t *__restrict__ kout, int *__restrict__ vout,
                Y *__restrict__ yout, int n, int lbits, int ncell, const int *__restrict__ hist,
                int ntiles, const SortTiles &st, const int *__restrict__ blk_first, int cap,
                int per_cell_first, int *__restrict__ off,
                int *__restrict__ item_off, int *__restrict__ item_cell, int *__restrict__ item_pb,
                int *__restrict__ item_pe, int *__restrict__ nitems, int *__restrict__ overflow) {
    constexpr int LOCAL_CHUNK = LOCAL_THREADS * LOCAL_ROUNDS;
    constexpr int LOCAL_WARPS = LOCAL_THREADS / 32;
    constexpr int RANGE = local_range(LOCAL_THREADS);
    constexpr bool RANK_OR = !CARRY;            // bins ranked by rank_or, else by ballots
    extern __shared__ __align__(16) int smem_i[];
    const int NB = 1 << lbits;
    const unsigned lmask = (unsigned)NB - 1u;
    int *cnt = smem_i;                           // [LOCAL_WARPS][NB] per-warp counts, then offsets
    int *btot = cnt + LOCAL_WARPS * NB;          // [NB] keys of each bin in the bucket
    int *bstart = btot + NB;                     // [NB] first bucket position of each bin
    int *run = bstart + NB;                      // [NB] keys of each bin in earlier chunks
    int *ctot = run + NB;                        // [NB] keys of each bin in this chunk
    int *cst = ctot + NB;                        // [NB] first chunk slot of each bin
    int *wtot = cst + NB;                        // [32]
    unsigned *mm = reinterpret_cast<unsigned *>(wtot + 32);   // [LOCAL_WARPS][NB] bin masks
    uint32_t *skey = reinterpret_cast<uint32_t *>(mm + (RANK_OR ? LOCAL_WARPS * NB : 0));
    int *sval = reinterpret_cast<int *>(skey + LOCAL_CHUNK);
    Y *sy = reinterpret_cast<Y *>(sval + LOCAL_CHUNK);   // CARRY only
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int b = blockIdx.x, t0 = 0, ncell_i = ncell, j = 0;
    unsigned cb = 0;
    int s0, s1, r0, r1;
    if (st.inst != nullptr) {
        const int inst = block_instance(blk_first, st.ninst, blockIdx.x);
        b = blockIdx.x - blk_first[inst];
        t0 = st.inst_tile0[inst];
        const NodeInst I = st.tab[inst];
        cb = (unsigned)I.cell_base;
        ncell_i = I.ncell;
        const int p_beg = (int)st.pt_off[inst], p_end = (int)st.pt_off[inst + 1];
        const int nb_i = ((ncell_i - 1) >> lbits) + 1;
        s0 = s1 = p_beg;                         // an instance without points: empty buckets
        if (p_end > p_beg) {
            s0 = hist[(long long)b * ntiles + t0];
            s1 = b + 1 < nb_i ? hist[(long long)(b + 1) * ntiles + t0] : p_end;
        }
        r0 = s0;
        r1 = s1;
    } else {
        // bucket i holds [start(i), start(i + 1)) and takes max(1, ceil(size / range)) blocks;
        // the sizes are the first pass's digit totals (one contiguous row, all loads first)
        __shared__ int bmap[257];
        __shared__ int bst[257];
        const int nbk = ((ncell - 1) >> lbits) + 1;   // <= 256
        if (w == 0) {
            const int *tot = hist + 256LL * ntiles;
            int sz[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = k * 32 + lane;
                sz[k] = i < nbk ? tot[i] : 0;
            }
            int carry = 0, carry_s = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int i = k * 32 + lane;
                const int v = i < nbk ? max(1, (sz[k] + RANGE - 1) / RANGE) : 0;
                int incl = v, incs = sz[k];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, incl, o);
                    const int us = __shfl_up_sync(0xffffffffu, incs, o);
                    if (lane >= o) {
                        incl += u;
                        incs += us;
                    }
                }
                if (i < nbk) {
                    bmap[i] = carry + incl - v;
                    bst[i] = carry_s + incs - sz[k];
                }
                carry += __shfl_sync(0xffffffffu, incl, 31);
                carry_s += __shfl_sync(0xffffffffu, incs, 31);
            }
            if (lane == 0) {
                bmap[nbk] = carry;
                bst[nbk] = carry_s;
            }
        }
        __syncthreads();
        if ((int)blockIdx.x >= bmap[nbk]) return;      // block-uniform: beyond the last range
        int lo = 0, hi = nbk;                           // largest i with bmap[i] <= block
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (bmap[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
        }
        b = lo;
        j = (int)blockIdx.x - bmap[b];
        s0 = bst[b];
        s1 = bst[b + 1];
        r0 = min(s0 + j * RANGE, s1);
        r1 = min(r0 + RANGE, s1);
    }
    for (int i = tid; i < NB; i += LOCAL_THREADS) {
        btot[i] = 0;
        run[i] = 0;
    }
    if constexpr (RANK_OR)
        for (int i = tid; i < LOCAL_WARPS * NB; i += LOCAL_THREADS) mm[i] = 0u;
    // the first chunk's keys, values (and carried coordinates) are loaded before the
    // counting pass, so that their latency overlaps it
    uint32_t key[LOCAL_ROUNDS];
    int val[LOCAL_ROUNDS], rank[LOCAL_ROUNDS];
    Y yv[CARRY ? LOCAL_ROUNDS : 1];
    auto load_chunk = [&](int c0, int cend) {
        const int base = c0 + w * (32 * LOCAL_ROUNDS);
#pragma unroll
        for (int r = 0; r < LOCAL_ROUNDS; ++r) {
            const int idx = base + r * 32 + lane;
            const bool valid = idx < cend;
            key[r] = valid ? kin[idx] : 0u;
            val[r] = valid ? vin[idx] : 0;
            if constexpr (CARRY) yv[r] = valid ? yin[idx] : Y(0);
        }
    };
    if (r0 < r1) load_chunk(r0, min(r0 + LOCAL_CHUNK, r1));
    __syncthreads();
    for (int i0 = s0; i0 < s1; i0 += LOCAL_COUNT_UNROLL * LOCAL_THREADS) {
        uint32_t kk[LOCAL_COUNT_UNROLL];
#pragma unroll
        for (int q = 0; q < LOCAL_COUNT_UNROLL; ++q) {   // the loads first
            const int i = i0 + q * LOCAL_THREADS + tid;
            kk[q] = i < s1 ? kin[i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < LOCAL_COUNT_UNROLL; ++q) {
            const int i = i0 + q * LOCAL_THREADS + tid;
            if (i >= s1) break;
            const unsigned d = (kk[q] - cb) & lmask;
            atomicAdd(&btot[d], 1);
            if (i < r0) atomicAdd(&run[d], 1);   // the bucket's keys before this range
        }
    }
    __syncthreads();
    if (w == 0) {                                // exclusive scan of the bin sizes
        int carry = 0;
        for (int i0 = 0; i0 < NB; i0 += 32) {
            const int i = i0 + lane;
            const int v = i < NB ? btot[i] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (i < NB) bstart[i] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int d = tid; d < NB && j == 0; d += LOCAL_THREADS) {   // cell offsets (and items)
        const int cl = (b << lbits) + d;
        if (cl >= ncell_i) continue;
        const int c = (int)cb + cl;
        const int pb = s0 + bstart[d];
        off[c] = pb;
        if (per_cell_first) {
            item_off[c] = c;
            item_cell[c] = c;
            item_pb[c] = pb;
            item_pe[c] = pb + btot[d];
            if (btot[d] > cap) *overflow = 1;
        }
    }
    const bool last = st.inst != nullptr ? blockIdx.x == gridDim.x - 1
                                         : (b == ((ncell - 1) >> lbits) && j == 0);
    if (last && tid == 0) {
        off[ncell] = n;
        if (per_cell_first) {
            item_off[ncell] = ncell;
            *nitems = ncell;
        }
    }
    const unsigned lt = lanemask_lt();
    for (int c0 = r0; c0 < r1; c0 += LOCAL_CHUNK) {
        const int cend = min(c0 + LOCAL_CHUNK, r1);
        for (int i = lane; i < NB; i += 32) cnt[w * NB + i] = 0;
        __syncwarp();
        const int base = c0 + w * (32 * LOCAL_ROUNDS);
        if (c0 != r0) load_chunk(c0, cend);
#pragma unroll
        for (int r = 0; r < LOCAL_ROUNDS; ++r) {
            const int idx = base + r * 32 + lane;
            const bool valid = idx < cend;
            const unsigned d = valid ? ((key[r] - cb) & lmask) : (unsigned)NB;   // NB: invalid
            if constexpr (RANK_OR) {
                rank[r] = rank_or(mm + w * NB, cnt + w * NB, d, valid, lt, lane);
                continue;
            }
            // a round without invalid lanes has d < NB in every lane: bit lbits is 0 for all
            // of them and its ballot would change nothing
            const int nbits = base + r * 32 + 31 < cend ? lbits : lbits + 1;
            unsigned peers = 0xffffffffu;
#pragma unroll
            for (int bt = 0; bt < 9; ++bt) {         // the ballots of the bits of d
                if (bt >= nbits) break;
                const unsigned bit = (d >> bt) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
            const int before = valid ? cnt[w * NB + d] : 0;
            __syncwarp();
            if (valid && (peers & lt) == 0) cnt[w * NB + d] += __popc(peers);
            __syncwarp();
            rank[r] = before + __popc(peers & lt);
        }
        __syncthreads();
        {   // one block-wide exclusive scan of the counters in (bin, warp) order: afterwards
            // cnt[w NB + d] is the chunk slot of warp w's first key of bin d
            const int total = NB * LOCAL_WARPS;
            const int per = (total + LOCAL_THREADS - 1) / LOCAL_THREADS;   // <= 8
            const int e0 = tid * per;
            int v[8];
            int sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q;                                      // e = d * WARPS + w
                v[q] = (q < per && e < total) ? cnt[(e % LOCAL_WARPS) * NB + e / LOCAL_WARPS] : 0;
                sum += v[q];
            }
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane == 31) wtot[w] = incl;
            __syncthreads();
            if (w == 0) {
                const int x = lane < LOCAL_WARPS ? wtot[lane] : 0;
                int xi = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, xi, o);
                    if (lane >= o) xi += u;
                }
                if (lane < LOCAL_WARPS) wtot[lane] = xi - x;
            }
            __syncthreads();
            int run_e = wtot[w] + incl - sum;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = e0 + q;
                if (q < per && e < total) {
                    cnt[(e % LOCAL_WARPS) * NB + e / LOCAL_WARPS] = run_e;
                    run_e += v[q];
                }
            }
        }
        __syncthreads();
        for (int d = tid; d < NB; d += LOCAL_THREADS) {   // chunk start and size of each bin
            const int a = cnt[d];                           // warp 0's slot = the bin's start
            cst[d] = a;
            ctot[d] = (d + 1 < NB ? cnt[d + 1] : (cend - c0)) - a;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < LOCAL_ROUNDS; ++r) {
            const int idx = base + r * 32 + lane;
            if (idx < cend) {
                const unsigned d = (key[r] - cb) & lmask;
                const int loc = cnt[w * NB + d] + rank[r];
                skey[loc] = key[r];
                sval[loc] = val[r];
                if constexpr (CARRY) sy[loc] = yv[r];
            }
        }
        __syncthreads();
        const int tn = cend - c0;
        for (int i = tid; i < tn; i += LOCAL_THREADS) {
            const uint32_t k = skey[i];
            const int v = sval[i];
            const unsigned d = (k - cb) & lmask;
            const int pos = s0 + bstart[d] + run[d] + (i - cst[d]);
            kout[pos] = k;
            vout[pos] = v;
            if constexpr (CARRY) yout[pos] = sy[i];
            else yout[pos] = yin[v];
        }
        __syncthreads();
        for (int d = tid; d < NB; d += LOCAL_THREADS) run[d] += ctot[d];
        __syncthreads();
    }
}

// Work items of every cell (as k_build_items) by one block of T threads, four cells per
// thread per tile: for the last block of the local pass when a cell exceeds the item cap.
// The cell offsets were written by the other blocks of the launch: read through L2.
template <int T>
__device__ __forceinline__ void build_items_block(const int *__restrict__ off, int ncell,
                                                  int *__restrict__ item_off,
                                                  int *__restrict__ item_cell,
                                                  int *__restrict__ item_pb,
                                                  int *__restrict__ item_pe,
                                                  int *__restrict__ nitems, int cap) {
    constexpr int PER = 4;
    constexpr int WARPS = T / 32;
    __shared__ int wsum[WARPS];
    __shared__ int carry_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += T * PER) {
        const int c0 = base + tid * PER;
        int p[PER + 1];
#pragma unroll
        for (int q = 0; q <= PER; ++q) p[q] = c0 + q <= ncell ? __ldcg(off + c0 + q) : 0;
        int v[PER];
        int sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            v[q] = c0 + q < ncell ? (p[q + 1] - p[q] + cap - 1) / cap : 0;
            sum += v[q];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int x = lane < WARPS ? wsum[lane] : 0;
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            if (lane < WARPS) wsum[lane] = xi - x;
        }
        __syncthreads();
        int first = carry_s + wsum[w] + incl - sum;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int c = c0 + q;
            if (c < ncell) {
                item_off[c] = first;
                for (int j = 0; j < v[q]; ++j) {
                    const int pb = p[q] + j * cap;
                    item_cell[first + j] = c;
                    item_pb[first + j] = pb;
                    item_pe[first + j] = pb + cap < p[q + 1] ? pb + cap : p[q + 1];
                }
            }
            first += v[q];
        }
        __syncthreads();
        if (tid == T - 1) carry_s = first;
        __syncthreads();
    }
    if (tid == 0) {
        item_off[ncell] = carry_s;
        *nitems = carry_s;
    }
}

// The local pass as a kernel.  ticket != nullptr (single instance, one work item per cell,
// ncell <= ITEMS_ONE_BLOCK_MAX; *ticket zero at launch): every block takes a ticket when it
// is done, and the last one, if some cell exceeded the item cap (*overflow), rebuilds the work
// items by the scan -- what k_build_items does in a launch of its own otherwise.  No block
// waits for another.
template <int LOCAL_THREADS, typename Y, bool CARRY>
__global__ void __launch_bounds__(LOCAL_THREADS, local_min_blocks(LOCAL_THREADS))
k_sort_local(const uint32_t *__restrict__ kin, const int *__restrict__ vin,
             const Y *__restrict__ yin, uint32_t *__restrict__ kout, int *__restrict__ vout,
             Y *__restrict__ yout, int n, int lbits, int ncell, const int *__restrict__ hist,
             int ntiles, SortTiles st, const int *__restrict__ blk_first, int cap,
             int per_cell_first, int *__restrict__ off,
             int *__restrict__ item_off, int *__restrict__ item_cell, int *__restrict__ item_pb,
             int *__restrict__ item_pe, int *__restrict__ nitems, int *__restrict__ overflow,
             int *__restrict__ ticket) {
    sort_local_body<LOCAL_THREADS, Y, CARRY>(kin, vin, yin, kout, vout, yout, n, lbits, ncell,
                                             hist, ntiles, st, blk_first, cap, per_cell_first,
                                             off, item_off, item_cell, item_pb, item_pe, nitems,
                                             overflow);
    if (ticket == nullptr) return;
    __shared__ int last_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_s = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    if (__ldcg(overflow) == 0) return;
    build_items_block<LOCAL_THREADS>(off, ncell, item_off, item_cell, item_pb, item_pe, nitems, cap);
}

// Single-block exclusive scan of n ints: out[i] = sum_{j<i} in[j], out[n] = total.
// Coalesced tiles of 1024 (one element per thread) with a running carry.
// in and out may alias.
__global__ void __launch_bounds__(1024) k_scan_exclusive(const int *in, int *out, int n,
                                                         const int *run_if = nullptr) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (run_if && *run_if == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < n; base += 1024) {
        const long long i = base + tid;
        const int v = i < n ? in[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int x = wsum[lane];
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            wsum[lane] = xi - x;           // exclusive prefix of the warp totals
        }
        __syncthreads();
        const int c0 = carry;
        if (i < n) out[i] = c0 + wsum[w] + incl - v;
        __syncthreads();
        if (tid == 1023) carry = c0 + wsum[31] + incl;   // last thread: tile total
        __syncthreads();
    }
    if (tid == 0) out[n] = carry;
}

// Cell offsets from the sorted keys and, in the same pass, one work item per cell (empty
// cells included: pb = pe) for the common case that no cell holds more than cap points.
// The first point i of a cell with more (keys[i + cap] still in the cell) sets *overflow;
// the scan-based builders launched next then rebuild the items (they return at once
// otherwise), so the decision stays on the device.
__global__ void __launch_bounds__(256)
k_cell_offsets_items(const uint32_t *__restrict__ keys, int n, int ncell, int cap,
                     int *__restrict__ off, int *__restrict__ item_off,
                     int *__restrict__ item_cell, int *__restrict__ item_pb,
                     int *__restrict__ item_pe, int *__restrict__ nitems,
                     int *__restrict__ overflow) {
    // four consecutive boundaries i = i0 .. i0 + 3 per thread (one 16-byte key load)
    const long long i0 = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 > n) return;
    int k[5];                                   // keys i0 - 1 .. i0 + 3 (ncell at n)
    k[0] = i0 == 0 ? -1 : (int)keys[i0 - 1];
    if (i0 + 3 < n) {
        const uint4 q = *reinterpret_cast<const uint4 *>(keys + i0);
        k[1] = (int)q.x;
        k[2] = (int)q.y;
        k[3] = (int)q.z;
        k[4] = (int)q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) k[1 + j] = i0 + j < n ? (int)keys[i0 + j] : ncell;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = (int)(i0 + j);
        if (i > n) break;
        const int prev = k[j], cur = k[j + 1];
        if (overflow == nullptr) {                        // offsets only
            for (int c = prev + 1; c <= cur; ++c) off[c] = i;
            continue;
        }
        if (cur > prev && i + cap < n && (int)keys[i + cap] == cur) *overflow = 1;
        for (int c = prev + 1; c <= cur; ++c) {
            off[c] = i;
            if (c < ncell) {
                item_off[c] = c;
                item_cell[c] = c;
                item_pb[c] = i;
            }
            if (c > 0) item_pe[c - 1] = i;
        }
        if (i == n) {
            item_off[ncell] = ncell;
            *nitems = ncell;
        }
    }
}

// Work items in one block: for every cell, ceil(count / cap) items of at most cap
// (<= ITEM_CAP) consecutive sorted points; item_off[c] = first item of cell c, nitems = total.
// Coalesced tiles of 1024 cells (one per thread), exclusive scan with a running carry;
// the next tile's offsets are loaded before the current tile is scanned.
__global__ void __launch_bounds__(1024)
k_build_items(const int *__restrict__ off, int ncell, int *__restrict__ item_off,
              int *__restrict__ item_cell, int *__restrict__ item_pb, int *__restrict__ item_pe,
              int *__restrict__ nitems, int cap, const int *__restrict__ run_if) {
    if (run_if && *run_if == 0) return;                 // items already one per cell
    __shared__ int wsum[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    int c = tid;
    int p0 = c < ncell ? off[c] : 0, p1 = c < ncell ? off[c + 1] : 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += 1024) {
        const int cn = c + 1024;
        const int q0 = cn < ncell ? off[cn] : 0, q1 = cn < ncell ? off[cn + 1] : 0;   // prefetch
        const int v = c < ncell ? (p1 - p0 + cap - 1) / cap : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int x = wsum[lane];
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            wsum[lane] = xi - x;
        }
        __syncthreads();
        const int first = carry + wsum[w] + incl - v;
        if (c < ncell) {
            item_off[c] = first;
            for (int j = 0; j < v; ++j) {
                const int pb = p0 + j * cap;
                item_cell[first + j] = c;
                item_pb[first + j] = pb;
                item_pe[first + j] = pb + cap < p1 ? pb + cap : p1;
            }
        }
        __syncthreads();
        if (tid == 1023) carry = first + v;
        __syncthreads();
        c = cn;
        p0 = q0;
        p1 = q1;
    }
    if (tid == 0) {
        item_off[ncell] = carry;
        *nitems = carry;
    }
}

// Work items for many cells (a batch), in three launches: per block of 1024 cells the
// number of items, a single-block scan of those block sums, then per block the local
// scan, the items and item_off.  Same items as k_build_items.
__device__ __forceinline__ int cell_items(const int *off, int c, int ncell, int cap) {
    return c < ncell ? (off[c + 1] - off[c] + cap - 1) / cap : 0;
}

__global__ void __launch_bounds__(1024)
k_item_block_sums(const int *__restrict__ off, int ncell, int *__restrict__ bsum, int cap,
                  const int *__restrict__ run_if) {
    __shared__ int wsum[32];
    if (run_if && *run_if == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int v = cell_items(off, blockIdx.x * 1024 + tid, ncell, cap);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int t = wsum[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024)
k_item_fill_blocks(const int *__restrict__ off, int ncell, const int *__restrict__ bbase,
                   int nblocks, int *__restrict__ item_off, int *__restrict__ item_cell,
                   int *__restrict__ item_pb, int *__restrict__ item_pe,
                   int *__restrict__ nitems, int cap, const int *__restrict__ run_if) {
    __shared__ int wsum[32];
    if (run_if && *run_if == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int c = blockIdx.x * 1024 + tid;
    const int v = cell_items(off, c, ncell, cap);
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = wsum[lane];
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += u;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    const int first = bbase[blockIdx.x] + wsum[w] + incl - v;
    if (c < ncell) {
        item_off[c] = first;
        const int p0 = off[c], p1 = off[c + 1];
        for (int j = 0; j < v; ++j) {
            const int pb = p0 + j * cap;
            item_cell[first + j] = c;
            item_pb[first + j] = pb;
            item_pe[first + j] = pb + cap < p1 ? pb + cap : p1;
        }
    }
    if (blockIdx.x == nblocks - 1 && tid == 0) {
        item_off[ncell] = bbase[nblocks];
        *nitems = bbase[nblocks];
    }
}

// Work items of at most SMALL_ITEM points to list_small, the rest to list_big; one
// warp-aggregated atomic per warp and list (the order within a list does not matter:
// every item is computed independently).
__global__ void k_split_items(const int *__restrict__ nitems, const int *__restrict__ item_pb,
                              const int *__restrict__ item_pe, int *__restrict__ list_small,
                              int *__restrict__ list_big, int *__restrict__ n2) {
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = it < *nitems;
    const bool small = valid && item_pe[it] - item_pb[it] <= SMALL_ITEM;
    const unsigned ms = __ballot_sync(0xffffffffu, small);
    const unsigned mb = __ballot_sync(0xffffffffu, valid && !small);
    int bs = 0, bb = 0;
    if (lane == 0) {
        if (ms) bs = atomicAdd(&n2[0], __popc(ms));
        if (mb) bb = atomicAdd(&n2[1], __popc(mb));
    }
    bs = __shfl_sync(0xffffffffu, bs, 0);
    bb = __shfl_sync(0xffffffffu, bb, 0);
    const unsigned lt = lanemask_lt();
    if (small) list_small[bs + __popc(ms & lt)] = it;
    else if (valid) list_big[bb + __popc(mb & lt)] = it;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

cudaError_t launch_split_items(const int *nitems, const int *item_pb, const int *item_pe,
                               int max_items, int *list_small, int *list_big, int *n2,
                               cudaStream_t s) {
    if (max_items <= 0) return cudaSuccess;
    k_split_items<<<cdiv(max_items, 256), 256, 0, s>>>(nitems, item_pb, item_pe, list_small,
                                                       list_big, n2);
    count_launches(1);
    return cudaGetLastError();
}

size_t radix_sort_hist_len(int ntiles, int ninst) {
    // per-tile digit counts (digit-major), then the digit totals of every instance
    return (size_t)256 * (size_t)(ntiles > 0 ? ntiles : 1) + (size_t)256 * (size_t)(ninst > 0 ? ninst : 1);
}

namespace {
SortTiles single_tiles() {
    SortTiles t;
    t.inst = nullptr;
    t.start = nullptr;
    t.inst_tile0 = nullptr;
    t.pt_off = nullptr;
    t.tab = nullptr;
    t.ntiles = 0;
    t.ninst = 1;
    return t;
}
}  // namespace

cudaError_t launch_node_keys_y(const double *nodes, int n, const NodeInst &one,
                               const SortTiles *tiles, int ntiles, uint32_t *keys, void *y_user,
                               int yfmt, int key_bits, int ybytes, int *hist, int *status,
                               cudaStream_t s, bool two_stage) {
    if (n <= 0) return cudaSuccess;
    const SortTiles st = tiles ? *tiles : single_tiles();
    if (!tiles) ntiles = cdiv(n, SORT_TILE);
    int *tot = hist + 256LL * ntiles;
    cudaError_t e = cudaMemsetAsync(tot, 0, 256 * sizeof(int) * (size_t)st.ninst, s);
    if (e != cudaSuccess) return e;
    const int shift0 = two_stage ? local_sort_low_bits(key_bits) : 0;
    const unsigned mask0 = two_stage ? 255u : radix_digit(key_bits, 0, radix_wide_first(ybytes)).mask;
    k_node_keys_y<<<ntiles, SORT_THREADS, 0, s>>>(nodes, n, one, st, keys, y_user, yfmt, ntiles,
                                                  shift0, mask0, hist, tot, status);
    count_launches(1);
    return cudaGetLastError();
}

namespace {
// keys from which the scatter passes after the first rank with match instructions.  The
// first pass ranks with ballots at every size: its digits are the keys' low bits, so a
// warp's 32 keys hold ~30 distinct digits, for which one match costs more than the nine
// ballots (measured at 512 instances: node stage 3.64 -> 3.49 ms fp32, 4.12 -> 4.01 ms
// fp64; the later passes' digits repeat more within a warp and keep match).
constexpr int SORT_MATCH_MIN = 1 << 23;

template <bool FIRST, typename Y, bool NARROW>
void scatter_launch_w(int ntiles, cudaStream_t s, const uint32_t *ka, const int *va, uint32_t *kb,
                      int *vb, int n, int shift, unsigned mask, const SortTiles &st, const int *hist,
                      const void *yin, void *yout) {
    if constexpr (!FIRST) {
        if (n >= SORT_MATCH_MIN) {
            k_sort_scatter<FIRST, Y, true, NARROW><<<ntiles, SORT_THREADS, 0, s>>>(
                ka, va, kb, vb, n, shift, mask, st, ntiles, hist, static_cast<const Y *>(yin),
                static_cast<Y *>(yout));
            return;
        }
    }
    k_sort_scatter<FIRST, Y, false, NARROW><<<ntiles, SORT_THREADS, 0, s>>>(
        ka, va, kb, vb, n, shift, mask, st, ntiles, hist, static_cast<const Y *>(yin),
        static_cast<Y *>(yout));
}
template <bool FIRST, typename Y>
void scatter_launch(int ntiles, cudaStream_t s, const uint32_t *ka, const int *va, uint32_t *kb,
                    int *vb, int n, int shift, unsigned mask, const SortTiles &st, const int *hist,
                    const void *yin, void *yout) {
    if (mask == 255u)
        scatter_launch_w<FIRST, Y, false>(ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist, yin, yout);
    else
        scatter_launch_w<FIRST, Y, true>(ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist, yin, yout);
}
template <bool FIRST>
void scatter_dispatch(int ybytes, int ntiles, cudaStream_t s, const uint32_t *ka, const int *va,
                      uint32_t *kb, int *vb, int n, int shift, unsigned mask, const SortTiles &st,
                      const int *hist, const void *yin, void *yout) {
    if (ybytes == 4)
        scatter_launch<FIRST, unsigned>(ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist, yin, yout);
    else if (ybytes == 8)
        scatter_launch<FIRST, unsigned long long>(ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist,
                                                  yin, yout);
    else
        scatter_launch<FIRST, void>(ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist, yin, yout);
}
}  // namespace

cudaError_t radix_sort_cells(uint32_t *keys, int *vals, uint32_t *keys_alt, int *vals_alt,
                             int *hist, const SortTiles *tiles, int ntiles, int n, int key_bits,
                             const void *y_user, void *ys, void *y_tmp, int ybytes, cudaStream_t s,
                             uint32_t **keys_sorted, int **vals_sorted) {
    uint32_t *ka = keys, *kb = keys_alt;
    int *va = vals, *vb = vals_alt;
    if (n <= 1) {
        if (n == 1) {
            cudaError_t e = cudaMemsetAsync(vals, 0, sizeof(int), s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ys, y_user, ybytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
        *keys_sorted = ka;
        *vals_sorted = va;
        return cudaSuccess;
    }
    const SortTiles st = tiles ? *tiles : single_tiles();
    if (!tiles) ntiles = cdiv(n, SORT_TILE);
    int *tot = hist + 256LL * ntiles;
    const int passes = radix_passes(key_bits);
    for (int pass = 0; pass < passes; ++pass) {
        const RadixDigit dg = radix_digit(key_bits, pass, radix_wide_first(ybytes));
        const int shift = dg.shift;
        // the key bits above the last digit are zero: its mask can be the full 8 bits
        const unsigned mask = pass == passes - 1 ? 255u : dg.mask;
        if (pass > 0) {
            cudaError_t e0 = cudaMemsetAsync(tot, 0, 256 * sizeof(int) * (size_t)st.ninst, s);
            if (e0 != cudaSuccess) return e0;
            k_sort_upsweep<<<ntiles, SORT_THREADS, 0, s>>>(ka, n, shift, mask, st, ntiles, hist, tot);
            count_launches(1);
        }   // pass 0: tile counts and digit totals come from k_node_keys_y
        if (tiles)
            k_seg_scan<<<cdiv((long long)st.ninst * 256, 8), 256, 0, s>>>(hist, ntiles, tot, st);
        else
            k_sort_scan_rows<<<256, 256, 0, s>>>(hist, ntiles, tot);
        // 4-byte coordinates move with their keys in every pass, alternating between y_tmp
        // and ys so that the last pass writes ys; 8-byte ones are gathered from y_user by
        // the last pass
        const bool carry = ybytes == 4;
        const void *yin = !carry ? y_user : pass == 0 ? y_user : ((passes - pass) % 2 == 0 ? ys : y_tmp);
        void *yout = !carry ? ys : (passes - 1 - pass) % 2 == 0 ? ys : y_tmp;
        const int yb = carry || pass == passes - 1 ? ybytes : 0;
        if (pass == 0)
            scatter_dispatch<true>(yb, ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist, yin, yout);
        else
            scatter_dispatch<false>(yb, ntiles, s, ka, va, kb, vb, n, shift, mask, st, hist, yin, yout);
        count_launches(2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint32_t *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    *keys_sorted = ka;
    *vals_sorted = va;
    return cudaSuccess;
}

namespace {
template <int T, typename Y, bool CARRY>
void local_attr(int ybytes) {
    cudaFuncSetAttribute(k_sort_local<T, Y, CARRY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)local_sort_smem(T, 8, ybytes));
}

template <int T>
void local_launch(int nblocks, size_t sm, cudaStream_t s, int ybytes, const uint32_t *kin,
                  const int *vin, const void *y_carried, const void *y_user, uint32_t *kout,
                  int *vout, void *ys, int n, int lbits, int ncell, const int *hist, int ntiles,
                  const SortTiles &st, const int *blk_first, int cap, int per_cell_first,
                  int *off, int *item_off, int *item_cell, int *item_pb, int *item_pe,
                  int *nitems, int *overflow, int *ticket) {
    if (ybytes == 4)
        k_sort_local<T, unsigned, true><<<nblocks, T, sm, s>>>(
            kin, vin, static_cast<const unsigned *>(y_carried), kout, vout,
            static_cast<unsigned *>(ys), n, lbits, ncell, hist, ntiles, st, blk_first, cap,
            per_cell_first, off, item_off, item_cell, item_pb, item_pe, nitems, overflow, ticket);
    else
        k_sort_local<T, unsigned long long, false><<<nblocks, T, sm, s>>>(
            kin, vin, static_cast<const unsigned long long *>(y_user), kout, vout,
            static_cast<unsigned long long *>(ys), n, lbits, ncell, hist, ntiles, st, blk_first,
            cap, per_cell_first, off, item_off, item_cell, item_pb, item_pe, nitems, overflow,
            ticket);
}
}  // namespace

cudaError_t prepare_local_sort() {
    local_attr<256, unsigned, true>(4);
    local_attr<256, unsigned long long, false>(8);
    return cudaGetLastError();
}

cudaError_t radix_sort_cells_local(uint32_t *keys, int *vals, uint32_t *keys_alt, int *vals_alt,
                                   int *hist, const SortTiles *tiles, int ntiles,
                                   const int *blk_first, int nblocks, int n, int ncell,
                                   int key_bits, const void *y_user,
                                   void *ys, void *y_tmp, int ybytes, int cap, bool per_cell_first,
                                   int *cell_off, int *item_off, int *item_cell, int *item_pb,
                                   int *item_pe, int *nitems, int *scratch, cudaStream_t s,
                                   uint32_t **keys_sorted, int **vals_sorted) {
    if (cap < ITEM_CAP_MIN || cap > ITEM_CAP || !local_sort_ok(key_bits) || n < 2 ||
        (ybytes != 4 && ybytes != 8) || (tiles && (per_cell_first || !blk_first || nblocks < 1)) ||
        (!tiles && ncell > (1 << key_bits)))
        return cudaErrorInvalidValue;
    const SortTiles st = tiles ? *tiles : single_tiles();
    const int lbits = local_sort_low_bits(key_bits);
    if (!tiles) {           // an upper bound of sum over buckets of max(1, ceil(size / range))
        ntiles = cdiv(n, SORT_TILE);
        nblocks = ((ncell - 1) >> lbits) + 1 + cdiv(n, local_range(LOCAL_SINGLE_THREADS));
    }
    int *tot = hist + 256LL * ntiles;
    // first stage: stable scatter by the high digit (counts from k_node_keys_y); 4-byte
    // coordinates move with their keys into y_tmp
    if (tiles)
        k_seg_scan<<<cdiv((long long)st.ninst * 256, 8), 256, 0, s>>>(hist, ntiles, tot, st);
    else
        k_sort_scan_rows<<<256, 256, 0, s>>>(hist, ntiles, tot);
    scatter_dispatch<true>(ybytes == 4 ? 4 : 0, ntiles, s, keys, vals, keys_alt, vals_alt, n,
                           lbits, 255u, st, hist, y_user, y_tmp);
    count_launches(2);
    int *overflow = nullptr, *ticket = nullptr;
    // one work item per cell from the local pass; its last block rebuilds the items when a
    // cell exceeds cap (up to ITEMS_ONE_BLOCK_MAX cells; more: the multi-block builder below)
    const bool items_in_pass = per_cell_first && ncell <= ITEMS_ONE_BLOCK_MAX;
    if (per_cell_first) {
        overflow = scratch + build_items_scratch_len(ncell) - 1;
        ticket = items_in_pass ? overflow - 1 : nullptr;
        cudaError_t e = cudaMemsetAsync(overflow - 1, 0, 2 * sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    // second stage: each bucket sorted by its low bits, cell offsets and items
    if (tiles)
        local_launch<256>(nblocks, local_sort_smem(256, lbits, ybytes), s, ybytes, keys_alt,
                          vals_alt, y_tmp, y_user, keys, vals, ys, n, lbits, ncell, hist, ntiles,
                          st, blk_first, cap, 0, cell_off, item_off, item_cell, item_pb, item_pe,
                          nitems, overflow, nullptr);
    else
        local_launch<LOCAL_SINGLE_THREADS>(nblocks, local_sort_smem(LOCAL_SINGLE_THREADS, lbits, ybytes),
                          s, ybytes, keys_alt,
                          vals_alt, y_tmp, y_user, keys, vals, ys, n, lbits, ncell, hist, ntiles,
                          st, blk_first, cap, per_cell_first ? 1 : 0, cell_off, item_off,
                          item_cell, item_pb, item_pe, nitems, overflow, ticket);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // cells above cap (or sparse plans): items by a scan of ceil(count / cap) over the cells
    if (items_in_pass) {
        // done by the local pass's last block
    } else if (ncell <= ITEMS_ONE_BLOCK_MAX) {
        k_build_items<<<1, 1024, 0, s>>>(cell_off, ncell, item_off, item_cell, item_pb, item_pe,
                                         nitems, cap, overflow);
        count_launches(1);
    } else {
        const int nb = cdiv(ncell, 1024);
        k_item_block_sums<<<nb, 1024, 0, s>>>(cell_off, ncell, scratch, cap, overflow);
        k_scan_exclusive<<<1, 1024, 0, s>>>(scratch, scratch, nb, overflow);
        k_item_fill_blocks<<<nb, 1024, 0, s>>>(cell_off, ncell, scratch, nb, item_off, item_cell,
                                               item_pb, item_pe, nitems, cap, overflow);
        count_launches(3);
    }
    *keys_sorted = keys;
    *vals_sorted = vals;
    return cudaGetLastError();
}

cudaError_t launch_cells_and_items(const uint32_t *keys_sorted, int n, int ncell, int cap,
                                   bool per_cell_first, int *cell_off, int *item_off,
                                   int *item_cell, int *item_pb, int *item_pe, int *nitems,
                                   int *scratch, cudaStream_t s) {
    if (cap < ITEM_CAP_MIN || cap > ITEM_CAP) return cudaErrorInvalidValue;
    const int nb = cdiv(ncell, 1024);
    int *overflow = nullptr;                              // nullptr: the scan always runs
    if (per_cell_first) {
        overflow = scratch + nb + 1;
        cudaError_t e = cudaMemsetAsync(overflow, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    k_cell_offsets_items<<<cdiv(((long long)n + 4) / 4, 256), 256, 0, s>>>(
        keys_sorted, n, ncell, cap, cell_off, item_off, item_cell, item_pb, item_pe, nitems, overflow);
    // cells above cap: items by a scan of ceil(count / cap) over the cells
    if (ncell <= ITEMS_ONE_BLOCK_MAX) {
        k_build_items<<<1, 1024, 0, s>>>(cell_off, ncell, item_off, item_cell, item_pb, item_pe,
                                         nitems, cap, overflow);
        count_launches(2);
        return cudaGetLastError();
    }
    k_item_block_sums<<<nb, 1024, 0, s>>>(cell_off, ncell, scratch, cap, overflow);
    k_scan_exclusive<<<1, 1024, 0, s>>>(scratch, scratch, nb, overflow);
    k_item_fill_blocks<<<nb, 1024, 0, s>>>(cell_off, ncell, scratch, nb, item_off, item_cell,
                                           item_pb, item_pe, nitems, cap, overflow);
    count_launches(4);
    return cudaGetLastError();
}

// block sums of the multi-block builder (cdiv(ncell, 1024) + 1), the local pass's ticket, and
// the overflow flag last
size_t build_items_scratch_len(int ncell) { return (size_t)cdiv(ncell, 1024) + 3; }

namespace {
// four floats per input: the node kernel's fp32 coordinate, its float pair (h, l), and
// CUDA's own rounding conversion of the same integer (the self-test checks the error bounds)
__global__ void k_selftest_fixed63(const long long *__restrict__ in, float *__restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long v = in[i];
    const float2 pr = fixed63_to_pair(v);
    out[4 * i + 0] = fixed63_to_float32(v);
    out[4 * i + 1] = pr.x;
    out[4 * i + 2] = pr.y;
    out[4 * i + 3] = __ll2float_rn(v) * 0x1p-63f;
}
}  // namespace

cudaError_t selftest_fixed63(const long long *in, float *out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_selftest_fixed63<<<cdiv(n, 256), 256, 0, s>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnfft
