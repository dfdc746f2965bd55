// side.h -- what the point kernels (cell moments and evaluation) know about one node
// side: the work-item limits and the SideK descriptor.  Kept apart from internal.h so
// that the point kernels' sources can be identified by hashing only the files they are
// built from.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace nnfft {

// A work item is a run of at most `cap` sorted points of one cell, ITEM_CAP_MIN <= cap <=
// ITEM_CAP (a plan setting; the point kernels are written for items of up to ITEM_CAP).
constexpr int ITEM_CAP = 256;
constexpr int ITEM_CAP_MIN = 32;
template <typename Real> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };
template <typename Real> using C2 = typename Cplx<Real>::T;

// Everything a spread / gather kernel needs to know about one node side.
//   v side: frequency nodes v_k, window phi1 (m1, beta1), grid I_{K1}
//   x side: spatial nodes x_j,   window phi2 (m2, beta2), grid I_{N2}
// A point with u = node * uscale lies in cell c = floor(u) (c_lo <= c < c_lo + ncell)
// and has local coordinate y = 2 (u - c) - 1 in [-1, 1).  Its 2m taps hit grid
// positions p = c - m + 1 + t, t = 0..2m-1, with weights
//   w_t(y) = omega((t - m + 1 - z)/m), z = (y + 1)/2,  ~  sum_d coef[t*D + d] T_d(y).
template <typename Real> struct SideK {
    int m, D, ncell;
    long long c_lo;
    const Real *coef;      // [2m][D] Chebyshev coefficients of the taps
    const Real *rfit;      // [ncell][NR] or nullptr (x side: 1/phihat1 per cell)
    const int *perm;       // [M] sorted position -> caller index
    const Real *ys;        // [M] sorted local coordinates
    const int *item_off;   // [ncell + 1] first work item of each cell
    const int *item_cell;  // [max_items]
    const int *item_pb;    // [max_items] first sorted point of the item
    const int *item_pe;    // [max_items] one past its last point
    const int *nitems;     // device scalar: number of items
    int max_items;
    // with small-item splitting: items of at most SMALL_ITEM points (list_small, count
    // *n_small) run one thread per item, the others (list_big, *n_big) one warp per item;
    // nullptr lists: every item runs one warp per item
    const int *list_small, *list_big, *n_small, *n_big;
    // sorted cell index of every point ([M], ascending) and the active point count, for
    // the flat (one thread per point) evaluation kernels
    const uint32_t *keys;
    int M;
    // the plan's device status word (kernels OR in STATUS_* bits)
    int *status;
};
// Moments lanes value that selects the split-precision 8-lane team kernel with two sets of
// accumulators (consecutive points of a lane accumulate independently).
constexpr int MOM_TEAM_PF = 4;
// Evaluation lanes value that selects the flat kernels: one thread per sorted point.
constexpr int EVAL_FLAT = 1;
// The flat kernels with each block's range of cell window sums staged in shared memory by
// one bulk (TMA) copy.
constexpr int EVAL_FLAT_TMA = 2;
// One warp per work item that computes its cell's window sums from the grid itself (the
// gather convolution inside the evaluation; split precision, single instances).
constexpr int EVAL_GATHER = 3;
// Cells a staged block holds at most (blocks spanning more read global memory directly).
constexpr int TMA_MAX_CELLS = 128;
// Largest work item handled by one thread (no reduction) when a plan splits items.
constexpr int SMALL_ITEM = 16;

}  // namespace nnfft
