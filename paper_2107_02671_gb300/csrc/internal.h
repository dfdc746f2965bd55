// internal.h -- declarations shared by the translation units of the NNFFT
// library (kernels + host orchestration).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>
#include <type_traits>

#include "nnfft.h"

namespace nnfft {

// Coefficients of the per-cell Chebyshev fit of 1/phihat1(N* x) on the x side.
constexpr int NR = 8;
// Radix sort: digits of at most 8 bits (256 counters), tiles of SORT_TILE keys per block
// (8 warps x 256).
constexpr int SORT_TILE = 2048;
constexpr int SORT_THREADS = 256;
// Largest supported FFT factor (one CTA transforms a column in shared memory).
constexpr int FFT_MAX_FACTOR = 1024;
constexpr int FFT_MAX_STAGES = 12;

// Kernel status bits (OR-ed into the plan's device status word).
constexpr int STATUS_RANGE = 1;      // node outside [-1/2, 1/2] or NaN
constexpr int STATUS_INTERNAL = 2;   // inconsistent cell assignment (should not happen)
constexpr int STATUS_TIMEOUT = 4;    // a bounded device-side wait gave up

// Kernels launched by this library (nnfft_launch_count); bumped by every launch wrapper.
void count_launches(int n);
long long launches_so_far();

}  // namespace nnfft

#include "side.h"

namespace nnfft {

// Double-float tables of one side for the split-precision grid kernels.
struct SideDf {
    const float2 *coef;   // [2m][D] (hi, lo) of the Chebyshev coefficients of the taps
    const float2 *rfit;   // [ncell][NR] (hi, lo) of r_j / 2 (x side) or nullptr
};

// One instance's FFT of length N2 = n1 * n2 (four-step, radix lists r1, r2), on the
// grid buffer elements [grid_base, grid_base + N2).
// A pass-1 block transforms cols1 columns (of length n1), a pass-2 block cols2 rows
// (of length n2), so short transforms share a block.
struct FftDf {
    int N2, n1, n2;
    int nr1, nr2;
    int r1[FFT_MAX_STAGES], r2[FFT_MAX_STAGES];
    const float4 *tw1, *tw2, *twN;   // exp(-2 pi i k / n) as (re.h, re.l, im.h, im.l)
    long long grid_base;
    int cols1, cols2;
};

struct FftPlanDev {
    int N2, n1, n2;
    int nr1, nr2;
    int r1[FFT_MAX_STAGES], r2[FFT_MAX_STAGES];
    const void *tw1, *tw2, *twN;   // C2<Real>: exp(-2 pi i k / n) for n = n1, n2, N2
    long long grid_base;
    int cols1, cols2;
};
// Elements per FFT block when short columns are packed together.
constexpr int FFT_TILE = 1024;

// ---- instances -----------------------------------------------------------------
// A plan holds one or more independent NNFFT instances (a batch).  On each node side
// their points and cells are concatenated: instance i owns points [pt_off[i],
// pt_off[i+1]) and cells [cell_base, cell_base + ncell); the point kernels, the sort
// and the cell fold see one side with all cells.  The grid stage runs per instance,
// one launch for all instances: block b belongs to the instance i with
// blk[i] <= b < blk[i+1] and works on that instance's grid of length N2 at
// grid_base in the concatenated grid buffers.

// Node binning of one instance: u = node * scale with the scale in fixed point,
// S = scale * 2^44 (see kern_nodes.cu); cell key cell_base + floor(u) - c_lo.
struct NodeInst {
    unsigned long long S;
    long long c_lo;
    int ncell, cell_base;
};

// Radix-sort tiles of a batch side, aligned to the instances: tile t holds the points
// [start[t], min(start[t] + SORT_TILE, pt_off[inst[t] + 1])) of instance inst[t], and
// inst_tile0[i] is the first tile of instance i.  A batch sorts each instance by its
// local cell (key - cell_base), so the passes cover the largest instance's cells, not
// all cells of the side.  inst == nullptr: one instance, tiles of SORT_TILE points.
struct SortTiles {
    const int *inst;
    const long long *start;
    const int *inst_tile0;
    const long long *pt_off;
    const NodeInst *tab;
    int ntiles, ninst;
};

// Grid-stage geometry of one instance on one side.  CoefT: Real, or float2 (hi, lo)
// pairs for split precision.
template <typename CoefT> struct GridInst {
    long long c_lo;                   // centered index of the instance's first cell
    long long grid_base;              // first element of its grid buffer
    long long scale_off, scale_len;   // scale index p + scale_off, valid below scale_len
    const CoefT *coef;                // [2m][D] tap coefficients
    const CoefT *scale;               // deconvolution factors (v side) or nullptr
    const CoefT *rfit;                // [ncell][NR] 1/phihat1 fits (x side) or nullptr
    int ncell, cell_base, N2, pad;
};

// One grid-stage launch over all instances.
template <typename CoefT> struct GridLaunch {
    const GridInst<CoefT> *inst;   // [ninst] device
    const int *blk;                // [ninst + 1] device: first block of each instance
    int ninst, nblocks, m, D;
    bool fold;                     // gather: apply the instance's rfit (1/phihat1)
};

template <typename F> struct FftLaunch {
    const F *inst;                 // [ninst] device
    const int *blk1, *blk2;        // [ninst + 1] device: first pass-1 / pass-2 block
    int ninst, nblk1, nblk2;
    int smem1, smem2;              // elements of shared memory per pass-1 / pass-2 block
};

// p mod n in [0, n) for a grid position p with |p| < 2^31 and 0 < n < 2^31 (one 32-bit
// remainder; the grids are far shorter than 2^31).
__device__ __forceinline__ int wrap_index(long long p, int n) {
    const int r = (int)p % n;
    return r < 0 ? r + n : r;
}

// Instance of block b: the largest i with blk[i] <= b (blk[0] = 0, increasing).
__device__ __forceinline__ int block_instance(const int *blk, int ninst, int b) {
    int lo = 0, hi = ninst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(blk + mid) <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// Self-test of the integer-built fixed-point conversions of the node kernel: per input
// four floats (truncated, rounded, and CUDA's conversions of the same value).
cudaError_t selftest_fixed63(const long long *in, float *out, int n, cudaStream_t s);

// ---- nnfft_host.cu (for the other translation units) -------------------------------
// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();
// Grid-stage kernels with two thread layouts (degree-major: one warp per degree, many
// warps for small grids; position-major: one thread per position, fewer instructions)
// take the position-major one from this many blocks per SM on.
constexpr int POS_MAJOR_BLOCKS_PER_SM = 16;
// Record a status code and message for nnfft_last_error; returns code.
int report_error(int code, const std::string &msg);
// The stream a plan was created with.
cudaStream_t plan_stream(nnfft_plan_t p);
// The device that was current when the plan was created (its buffers and streams live there).
int plan_device(nnfft_plan_t p);
// Device bytes a plan holds.
size_t plan_bytes(nnfft_plan_t p);
// Fast sinc transform through plans cached per (sizes rounded up to capacities, stream);
// *plan_bytes receives the device bytes of the plans used.
int sinc_exec_capacity(int64_t N, int64_t L1, int64_t L2, int64_t L1cap, int64_t L2cap, int m,
                       nnfft_dtype dtype, int rule, int64_t n, const double *a_dev,
                       const void *c_dev, const double *b_dev, void *h_dev, int is_complex,
                       cudaStream_t stream, size_t *plan_bytes);
size_t sinc_release_stream(cudaStream_t stream);

// ---- kern_nodes.cu ----------------------------------------------------------------
// Sort buffer (ints) for ntiles tiles and ninst instances: per-tile digit counts and
// per-instance digit totals.
size_t radix_sort_hist_len(int ntiles, int ninst);
// Fused step 0: keys (global cell), local coordinates (caller order, format yfmt: 0 float,
// 1 double, 2 float pair) and the first radix pass's per-tile digit counts and digit
// totals in hist (radix_sort_hist_len ints).  tiles: a batch's instance-aligned tiles
// (each point takes its instance's binning, keys offset by the instance's first cell), or
// nullptr for one instance with binning `one` and ntiles = ceil(n / SORT_TILE).
// two_stage: count the high digit (key >> local_sort_low_bits) for radix_sort_cells_local
// instead of the low digit of the LSD passes.
cudaError_t launch_node_keys_y(const double *nodes, int n, const NodeInst &one,
                               const SortTiles *tiles, int ntiles, uint32_t *keys, void *y_user,
                               int yfmt, int key_bits, int ybytes, int *hist, int *status,
                               cudaStream_t s, bool two_stage = false);
// Digits of the radix sort of key_bits-bit keys, ceil(key_bits / 8) passes.  A tile of
// SORT_TILE keys leaves each digit's keys as one run of consecutive addresses, so a narrower
// digit gives longer runs.  Where the coordinates travel with the keys in every pass
// (4-byte coordinates) the widths differ by at most one bit, the narrower ones first
// (14 bits: 7 + 7; 15: 7 + 8; measured at 512 instances, fp32: node stage 3.49 -> 3.43 ms
// against 8 + 6).  Where the last pass also gathers 8-byte coordinates (wide_first) the
// digits are 8 bits wide with the remainder last (14 bits: 8 + 6), which measured 6 %
// faster there than 7 + 7 (fp64 node stage 4.01 against 4.26 ms).
struct RadixDigit {
    int shift;
    unsigned mask;
};
inline int radix_passes(int key_bits) { return key_bits < 1 ? 1 : (key_bits + 7) / 8; }
inline RadixDigit radix_digit(int key_bits, int pass, bool wide_first) {
    const int np = radix_passes(key_bits), b = key_bits < 1 ? 1 : key_bits;
    const int lo = b / np, wide = b % np;   // balanced: the last `wide` passes take lo + 1 bits
    RadixDigit d{0, 0u};
    for (int q = 0; q <= pass; ++q) {
        const int w = wide_first ? (b - 8 * q < 8 ? b - 8 * q : 8) : lo + (q >= np - wide ? 1 : 0);
        if (q < pass) d.shift += w;
        else d.mask = (1u << w) - 1u;
    }
    return d;
}
// the digit order radix_sort_cells uses for ybytes-byte coordinates
inline bool radix_wide_first(int ybytes) { return ybytes == 8; }
// Stable LSD radix sort of the keys from launch_node_keys_y (values: the identity
// permutation, generated in pass 0) by the low key_bits bits of key - cell_base (the
// whole key for one instance; within each instance for a batch, whose points are
// grouped by instance in cell_base order, so the result is sorted by key).  The
// ybytes-byte coordinates end as ys[sorted position] = y_user[original index]: 4-byte ones
// move with their keys in every pass (y_tmp: scratch of the same size), 8-byte ones are
// gathered by the last pass.
cudaError_t radix_sort_cells(uint32_t *keys, int *vals, uint32_t *keys_alt, int *vals_alt,
                             int *hist, const SortTiles *tiles, int ntiles, int n, int key_bits,
                             const void *y_user, void *ys, void *y_tmp, int ybytes, cudaStream_t s,
                             uint32_t **keys_sorted, int **vals_sorted);
// Two-stage sort of 9- to 16-bit cell keys: one stable scatter pass by
// the high 8-bit digit (counts from launch_node_keys_y with two_stage), then one block per
// bucket of 2^(key_bits - 8) cells sorts its bucket by the low bits in shared memory and
// writes the cell offsets and work items of launch_cells_and_items (the scan-based item
// builder follows, returning at once when every cell fits one item).  The same order as
// radix_sort_cells; the sorted keys and values end in keys / vals, the coordinates in ys
// (4-byte ones through y_tmp, 8-byte ones gathered from y_user).  prepare_local_sort
// sets the kernels' shared-memory limits (once per device, outside stream capture).
inline bool local_sort_ok(int key_bits) { return key_bits >= 9 && key_bits <= 16; }
inline int local_sort_low_bits(int key_bits) { return key_bits - 8; }
cudaError_t prepare_local_sort();
// Batches (tiles != nullptr, their instance-aligned tiles): keys sorted within each
// instance by the local cell, blk_first[i] = first second-stage block of instance i
// (nblocks in all); per_cell_first must be false (the scan-based items follow).
cudaError_t radix_sort_cells_local(uint32_t *keys, int *vals, uint32_t *keys_alt, int *vals_alt,
                                   int *hist, const SortTiles *tiles, int ntiles,
                                   const int *blk_first, int nblocks, int n, int ncell,
                                   int key_bits, const void *y_user,
                                   void *ys, void *y_tmp, int ybytes, int cap, bool per_cell_first,
                                   int *cell_off, int *item_off, int *item_cell, int *item_pb,
                                   int *item_pe, int *nitems, int *scratch, cudaStream_t s,
                                   uint32_t **keys_sorted, int **vals_sorted);
// Cell offsets (cell_off[c] = first sorted point of cell c, cell_off[ncell] = n) and work
// items (at most cap sorted points of one cell each, ITEM_CAP_MIN <= cap <= ITEM_CAP;
// item_off[c] = first item of cell c, *nitems = total) from the sorted keys.  With
// per_cell_first (dense plans) the offsets pass also makes one item per cell (empty cells
// included) and the scan of ceil(count / cap) over the cells runs only if some cell holds
// more than cap points; otherwise the scan always runs (it skips empty cells).  The scan
// is one block up to ITEMS_ONE_BLOCK_MAX cells, else three launches.  scratch:
// build_items_scratch_len(ncell) ints.
constexpr int ITEMS_ONE_BLOCK_MAX = 65536;
cudaError_t launch_cells_and_items(const uint32_t *keys_sorted, int n, int ncell, int cap,
                                   bool per_cell_first, int *cell_off, int *item_off,
                                   int *item_cell, int *item_pb, int *item_pe, int *nitems,
                                   int *scratch, cudaStream_t s);
size_t build_items_scratch_len(int ncell);
// Split the work items into those of at most SMALL_ITEM points and the rest (lists of
// item ids in no particular order, counts in n2[0], n2[1]; n2 zeroed by the caller).
cudaError_t launch_split_items(const int *nitems, const int *item_pb, const int *item_pe,
                               int max_items, int *list_small, int *list_big, int *n2,
                               cudaStream_t s);

// ---- kern_spread.cu ---------------------------------------------------------------
// Cell moments of vals over the sorted points, one set per work item, into P; the
// per-cell fold (launch_cell_fold: item sum and, with S.rfit, the 1/phihat1 factor)
// follows as its own launch.
// lanes: 32 (one warp per work item) or 8 (four items per warp, D <= 16)
template <typename Real>
cudaError_t launch_moments(const SideK<Real> &S, const void *vals, void *P, int lanes,
                           cudaStream_t s);
// Spread convolution of every instance: cell sums Pc (all cells of the side) -> grid
// buffers out (concatenated).  Gather convolution: grid buffers buf -> per-cell window
// sums Q.  Block counts per instance: spread_blocks / gather_blocks.
template <typename Real>
cudaError_t launch_spread_conv(const GridLaunch<Real> &L, const void *Pc, void *out,
                               cudaStream_t s);
template <typename Real>
cudaError_t launch_cell_fold(const SideK<Real> &S, const void *P, void *Pc, cudaStream_t s);
template <typename Real>
cudaError_t launch_gather_conv(const GridLaunch<Real> &L, const void *buf, void *Q,
                               cudaStream_t s);
// blocks of one instance's spread / gather convolution (all-real and split kernels)
int spread_blocks_native(int N2, int D);
int gather_blocks_native(int ncell, int D);
int spread_blocks_df(int N2, int D);
int gather_blocks_df(int ncell, int D);
template <typename Real>
cudaError_t launch_eval(const SideK<Real> &S, const void *Q, void *out, int lanes,
                        cudaStream_t s);
bool supported_degree(int D);

// ---- kern_spread_df.cu / kern_grid_df.cu (fp64 plans, split precision) ------------
// S.ys holds float2 (hi, lo) coordinates; degrees < D/2 in double-float, the rest FP32;
// all intermediate complex arrays are float4 (re.h, re.l, im.h, im.l).
bool df_supported_degree(int D);
// lanes: 32 (one warp per work item), 16 (two items per warp) or 8 (four items per warp);
// the plan's autotuner picks.  Evaluation: 32 or 8.
cudaError_t launch_moments_df(const SideK<double> &S, const void *vals, void *P4, int lanes,
                              cudaStream_t s);
// The evaluation with the gather convolution done per work item (EVAL_GATHER): L is the
// gathering side's grid launch (one instance), grid the FFT output.  eval_gather_df_ok: L
// qualifies (one instance, 2m <= 32, D <= 16); the side must not split small items.
bool eval_gather_df_ok(const GridLaunch<float2> &L);
cudaError_t launch_eval_gather_df(const SideK<double> &S, const GridLaunch<float2> &L,
                                  const void *grid, void *out, cudaStream_t s);
cudaError_t launch_eval_df(const SideK<double> &S, const void *Q4, void *out, int lanes,
                           cudaStream_t s);
cudaError_t launch_cell_fold_df(const SideK<double> &S, const SideDf &T, const void *P4,
                                void *Pc4, cudaStream_t s);
// The cell fold done by the spread convolution: the side's work-item offsets per cell, the
// per-item moments, and the fit tables (x side, adjoint) or nullptr.  P4 == nullptr: the
// convolution reads the folded moments (Pc4) instead.
struct SpreadFoldDf {
    const int *item_off = nullptr;
    const float4 *P4 = nullptr;
    const float2 *rfit = nullptr;
};
// True when the spread convolution of L runs the degree-major blocks, which can fold.
bool spread_df_folds(const GridLaunch<float2> &L);
cudaError_t launch_spread_conv_df(const GridLaunch<float2> &L, const void *Pc4, void *out,
                                  cudaStream_t s, const SpreadFoldDf &F = SpreadFoldDf{});
cudaError_t launch_fft_df(const FftLaunch<FftDf> &F, const void *in, void *tmp, void *out,
                          int sign, cudaStream_t s);
cudaError_t launch_gather_conv_df(const GridLaunch<float2> &L, const void *buf, void *Q4,
                                  cudaStream_t s);
// The FFT of a single instance as one launch of a thread-block cluster (FFT_CLUSTER CTAs,
// the grid in distributed shared memory; out may equal in).  fft_cluster_smem: shared memory
// per CTA; usable while it is at most FFT_CLUSTER_SMEM_MAX.  prepare_fft_cluster_df sets the
// kernel's shared-memory limit to that maximum (once per device and process suffices).
constexpr int FFT_CLUSTER = 8;
constexpr int FFT_CLUSTER_VARIANT = 2;   // nnfft_tuning.fft_variant value selecting it
constexpr int FFT_CLUSTER_THREADS = 512;
constexpr size_t FFT_CLUSTER_SMEM_MAX = 200 * 1024;
size_t fft_cluster_smem(int n1, int n2);
cudaError_t prepare_fft_cluster_df();
cudaError_t launch_fft_cluster_df(const FftLaunch<FftDf> &F, int n1, int n2, const void *in,
                                  void *out, int sign, cudaStream_t s);

// The whole grid stage of one direction (cell fold, spread convolution with the step-2
// deconvolution, the two FFT passes of step 3, gather convolution) as one cooperative
// launch: persistent blocks of D * 32 threads take each stage's blocks in turn and meet at
// a grid-wide barrier with bounded waits (gridsync.cuh) between the stages.  Same
// arithmetic as the stage-wide launches, so the results are bitwise equal.
constexpr int GRID_FUSED_VARIANT = 3;   // nnfft_tuning.fft_variant value selecting it
// barrier wait limit: about one second at the GB300's 2.07 GHz SM clock
constexpr long long GRID_WAIT_LIMIT_CYCLES = 2000000000LL;
struct GridStageDf {
    SideK<double> fold_side;        // the spreading side's item lists (cell fold)
    SideDf fold_tab;                // its fit tables (rfit: x side, adjoint)
    const float4 *P4;               // per-item moments
    float4 *Q4;                     // per-cell moments, then per-cell window sums
    GridLaunch<float2> spread, gather;
    FftLaunch<FftDf> fft;           // the first column packing
    float4 *bufA, *bufB, *bufC;     // spread grid, FFT intermediate, FFT output
    int sign;
    unsigned long long *bar;        // barrier words (arrival counter, abort word)
    int *status;
    long long limit;                // barrier wait limit in SM clock cycles
};
// Dynamic shared memory of the fused kernel for degree D and window sizes m_spread,
// m_gather with FFT blocks of smem1 / smem2 float4 elements.
size_t grid_stage_df_smem(int D, int m_spread, int m_gather, int smem1, int smem2);
// Sets the kernel's shared-memory limit and returns the blocks per SM that can be resident
// (0: not launchable with this shared memory).
int prepare_grid_stage_df(int D, size_t smem);
cudaError_t launch_grid_stage_df(const GridStageDf &A, int D, int blocks, size_t smem,
                                 cudaStream_t s);
// Self-test of the grid barrier: a cooperative launch of `blocks` blocks passing two
// barriers that expect blocks + extra arrivals (extra > 0: nobody completes them, every
// wait gives up after `limit` cycles and sets STATUS_TIMEOUT in *status).  words: two
// zeroed 64-bit words.
cudaError_t selftest_grid_barrier(int blocks, int extra, long long limit,
                                  unsigned long long *words, int *status, cudaStream_t s);

// ---- kern_fft.cu ------------------------------------------------------------------
template <typename Real>
cudaError_t launch_fft(const FftLaunch<FftPlanDev> &F, const void *in, void *tmp, void *out,
                       int sign, cudaStream_t s);
// The cluster FFT of a single instance (see launch_fft_cluster_df) for complex64 / complex128
// grids.
template <typename Real> size_t fft_cluster_smem_real(int n1, int n2);
template <typename Real> cudaError_t prepare_fft_cluster();
template <typename Real>
cudaError_t launch_fft_cluster(const FftLaunch<FftPlanDev> &F, int n1, int n2, const void *in,
                               void *out, int sign, cudaStream_t s);

// ---- kern_misc.cu -----------------------------------------------------------------
template <typename Real>
cudaError_t launch_real_to_complex(const Real *in, int n, void *out, cudaStream_t s);
template <typename Real>
cudaError_t launch_scale_by_weights(void *vals, const double *w, int n, cudaStream_t s);
template <typename Real>
cudaError_t launch_complex_to_real(const void *in, int n, Real *out, cudaStream_t s);
// Clenshaw-Curtis weights (Algorithm 5.4): even extension of length 2n into x (double2),
// then, after a length-2n FFT of x into X, the weights w[0..n] and nodes +-cos(k pi/n)/2.
cudaError_t launch_cc_extend(long long n, void *x, cudaStream_t s);
cudaError_t launch_cc_finish(long long n, const void *X, double *w, double *half_z,
                             double *neg_half_z, cudaStream_t s);
// Self-test of the bulk (TMA) copy helpers (see nnfft_selftest_bulk_copy).
cudaError_t selftest_bulk_copy(const float *src, float *dst, int n, int arm_only,
                               long long limit, int *status, cudaStream_t s);
// Sharded transform: copy the n centered positions l in I_n of an N2 grid buffer (element
// format fmt: 0 float2, 1 double2, 2 double-float float4; p at p mod N2) to out[l + n/2]
// (complex64 for fmt 0, complex128 otherwise), or back (import writes every buffer
// element: the n positions and zeros).  n <= N2, both even.
cudaError_t launch_grid_export(int fmt, const void *buf, int N2, int n, void *out,
                               cudaStream_t s);
cudaError_t launch_grid_import(int fmt, const void *in, int N2, int n, void *buf,
                               cudaStream_t s);

}  // namespace nnfft
