/*
 * nnfft.h -- C ABI of the GB300 (sm_103a) NNFFT library.
 *
 * The library evaluates the NNFFT (nonuniform FFT with nonequispaced spatial
 * and frequency data, "type 3") of Kircheis, Potts and Tasche,
 *
 *     y_j = sum_{k < M1} f_k exp(-2 pi i N v_k x_j),   j < M2,      (eq. (1.2))
 *
 * for frequency nodes v_k and spatial nodes x_j in [-1/2, 1/2], by Algorithm 2.2
 * with two sinh-type windows (Example 2.1, Section 4), its adjoint
 *
 *     z_k = sum_{j < M2} g_j exp(+2 pi i N v_k x_j),   k < M1,
 *
 * and the fast sinc transform of Algorithm 6.1 (Section 6),
 *
 *     h_l = sum_{k < L1} c_k sinc(N pi (b_l - a_k)),   l < L2.      (eq. (6.2))
 *
 * Conventions shared by every entry point:
 *   - Index sets are 0-based arrays; outputs are in the caller's order.
 *   - Complex data is interleaved (re, im) in the plan's real type: float for
 *     NNFFT_C64, double for NNFFT_C128.  Nodes are always double.
 *   - Pointers named *_dev are device pointers; *_host are host pointers
 *     (pinned memory gives full copy bandwidth; pageable memory works).
 *   - The caller owns every buffer it passes.  A plan owns its tables, its
 *     sorted copies of the nodes and its work buffers, all in device memory.
 *   - Every call is asynchronous on the plan's stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream) except the *_host calls and
 *     nnfft_sync, which return after the stream has drained.
 *   - Errors detectable on the host are returned at once.  Errors found by a
 *     kernel (a node outside [-1/2, 1/2] or NaN) set a status word in the plan
 *     that the next nnfft_sync (or *_host call) returns.
 *   - There is no CPU fallback: without a usable CUDA device the calls fail
 *     with NNFFT_ECUDA.
 *   - A plan must not be used from two host threads at once.
 */
#ifndef NNFFT_GB300_H
#define NNFFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nnfft_plan_s *nnfft_plan_t;

/* coefficient / output type; nodes are always float64 */
typedef enum { NNFFT_C64 = 0, NNFFT_C128 = 1 } nnfft_dtype;

/* status codes */
enum {
    NNFFT_OK = 0,
    NNFFT_EINVAL = 1,   /* invalid argument or parameter combination              */
    NNFFT_ERANGE = 2,   /* a node outside [-1/2, 1/2] or NaN (reported by kernels) */
    NNFFT_ENOMEM = 3,   /* device or host allocation failed                      */
    NNFFT_ECUDA = 4,    /* CUDA runtime error (no device, launch failure, ...)   */
    NNFFT_ETIMEOUT = 5, /* a bounded device-side wait gave up                    */
    NNFFT_ESTATE = 6    /* call out of order (e.g. exec before set_nodes)        */
};

/* Parameters a plan derived from its arguments (Section 2 and Section 4). */
typedef struct {
    int64_t N, Nstar, N1, K1, N2;   /* N* = N + ceil(2 m1/sigma1); N1 = sigma1 N* rounded up to
                                       even; K1 = N1 + 2 m1 (= a N1, eq. (2.6)); N2 = sigma2 K1
                                       rounded up to an even 2^a 3^b 5^c                      */
    int64_t M1, M2;
    int m1, m2;
    double sigma1, sigma2;           /* effective oversampling N1/N*, N2/K1                   */
    double beta1, beta2;             /* 2 pi m_j (1 - 1/(2 sigma_j))                          */
    int dtype;                       /* nnfft_dtype                                           */
    int D1, D2;                      /* Chebyshev degrees + 1 of the piecewise window fits    */
    double fit_err1, fit_err2;       /* max abs error of those fits on [-1,1] (window max 1)  */
    int64_t ncell1, ncell2;          /* node cells (bins) of the v side and the x side        */
    int64_t fft_n1, fft_n2;          /* N2 = fft_n1 * fft_n2 (four-step split)                */
    int arith;                       /* NNFFT_ARITH_* used by the point kernels (nnfft_plan only) */
    int window;                      /* NNFFT_WINDOW_* of both steps                           */
} nnfft_info;

/*
 * Arithmetic of the point kernels (Algorithm 2.2 steps 1 and 4).
 *   NNFFT_ARITH_FP32:       complex64 plans.
 *   NNFFT_ARITH_FP64:       complex128 plans, every operation in FP64.
 *   NNFFT_ARITH_FP64_SPLIT: complex128 plans (default when available): Chebyshev degrees
 *       d < D/2 of the window series in double-float (pairs of floats, ~48 bits), higher
 *       degrees in FP32, sums assembled in FP64.  Available when the fitted window weights
 *       of the degrees >= D/2 are <= 2e-7, which bounds the extra error near 1e-13 of
 *       ||f||_1; coefficient magnitudes must lie in [2^-75, 2^127] for full accuracy.
 */
enum { NNFFT_ARITH_FP32 = 0, NNFFT_ARITH_FP64 = 1, NNFFT_ARITH_FP64_SPLIT = 2 };

/*
 * nnfft_params: derive the plan parameters without touching a GPU.
 * Same rules and validation as nnfft_plan (EINVAL on: N < 1, M1 < 0, M2 < 0,
 * sigma_j <= 1 or > 16, m_j < 2 or m_j > 16, M_j > 2^30, N2 > 2^20, or
 * 2 m2 > (1 - 1/sigma1) N2,
 * the condition of step 4 of Algorithm 2.2).  fit_err*, D* are filled too.
 */
int nnfft_params(int64_t N, int64_t M1, int64_t M2, double sigma1, double sigma2,
                 int m1, int m2, nnfft_dtype dtype, nnfft_info *out);

/*
 * nnfft_plan: create a plan for M1 frequency nodes, M2 spatial nodes,
 * bandwidth N (Algorithm 2.2, input line), oversampling sigma1, sigma2 > 1,
 * truncation m1, m2 in [2, 16] and dtype.  Allocates the plan's device
 * tables and work buffers (O(M1 + M2 + N2) bytes) and uploads the window
 * tables.  stream: cudaStream_t (or NULL) used by every later call.
 * On success *out receives the plan; on failure *out is set to NULL.
 */
int nnfft_plan(nnfft_plan_t *out, int64_t N, int64_t M1, int64_t M2,
               double sigma1, double sigma2, int m1, int m2, nnfft_dtype dtype,
               void *stream);

/*
 * nnfft_batch_plan: one plan holding `count` independent NNFFT instances (the paper has no
 * batched form; each instance is Algorithm 2.2 with its own N[i], M1[i], M2[i] and the
 * shared sigma1, sigma2, m1, m2, dtype).  Every later call (set_nodes, exec, adjoint, the
 * host-buffer forms, sync, timing) treats the instances' data as concatenated: v holds
 * the M1[0] nodes of instance 0, then the M1[1] nodes of instance 1, ...; likewise x
 * (M2), f and z (M1), y and g (M2).  Each call does all instances at once: one launch
 * per stage, the node sort of all instances in one pass.  The window series of a side
 * use one Chebyshev length for all instances (the largest any instance needs), so a
 * batch result can differ from the single-instance plan's in the last bits.
 * count >= 1; the totals sum(M1), sum(M2) must be <= 2^30.  Errors as nnfft_plan; an
 * invalid instance gives EINVAL with its index in the message.
 * nnfft_plan(N, M1, M2, ...) is nnfft_batch_plan with count = 1.
 */
int nnfft_batch_plan(nnfft_plan_t *out, int64_t count, const int64_t *N, const int64_t *M1,
                     const int64_t *M2, double sigma1, double sigma2, int m1, int m2,
                     nnfft_dtype dtype, void *stream);

/*
 * Window functions (Section 2): the set Omega of even windows supported on [-1, 1].
 *   NNFFT_WINDOW_SINH:           sinh(beta sqrt(1 - x^2)) / sinh(beta), beta = 2 pi m (1 - 1/(2 sigma))
 *                                (Example 2.1, Section 4; the default of nnfft_plan);
 *   NNFFT_WINDOW_KAISER_BESSEL:  I0(beta sqrt(1 - x^2)) / I0(beta), the same beta (the standard
 *                                window beside which the paper's Fig. 4.1(b) plots the sinh bound);
 *   NNFFT_WINDOW_BSPLINE:        B_{2m}(m x) / B_{2m}(0), the centered cardinal B-spline of order 2m
 *                                (Example 2.1; beta = 0 is reported);
 *   NNFFT_WINDOW_ALGEBRAIC:      (1 - x^2)^{beta - 1/2}, beta = 3 m (Example 2.1; sigma1, sigma2 must
 *                                exceed pi/3).
 * Every window enters the kernels through the same per-cell Chebyshev fits of its 2m taps and
 * the same deconvolution tables (built from its closed-form Fourier transform), so every other
 * call works unchanged.  Only the sinh-type window carries the bound of Theorem 4.1; the
 * B-spline and algebraic windows converge algebraically in m (errors about 3e-9 and 1e-8 at
 * m = 8, sigma = 2, N = 128 in the oracle's Algorithm 2.2), the Kaiser-Bessel window like the
 * sinh-type one.
 */
enum {
    NNFFT_WINDOW_SINH = 0,
    NNFFT_WINDOW_KAISER_BESSEL = 1,
    NNFFT_WINDOW_BSPLINE = 2,
    NNFFT_WINDOW_ALGEBRAIC = 3
};
/* nnfft_plan / nnfft_batch_plan / nnfft_params with a window; EINVAL for an unknown window or
 * the algebraic window with sigma_j <= pi/3. */
int nnfft_plan_window(nnfft_plan_t *out, int64_t N, int64_t M1, int64_t M2, double sigma1,
                      double sigma2, int m1, int m2, nnfft_dtype dtype, int window, void *stream);
int nnfft_batch_plan_window(nnfft_plan_t *out, int64_t count, const int64_t *N, const int64_t *M1,
                            const int64_t *M2, double sigma1, double sigma2, int m1, int m2,
                            nnfft_dtype dtype, int window, void *stream);
int nnfft_params_window(int64_t N, int64_t M1, int64_t M2, double sigma1, double sigma2, int m1,
                        int m2, int dtype, int window, nnfft_info *out);
/* Host-only: the window's value omega(x) and Fourier transform omegahat(v) (2 int_0^1 omega(x)
 * cos(2 pi v x) dx, closed forms) for truncation m and oversampling sigma. */
int nnfft_window(int window, int m, double sigma, double x, double v, double *omega_x,
                 double *omega_hat_v);

/*
 * nnfft_set_sizes: use a single-instance plan for M1 <= (M1 at creation) frequency nodes
 * and M2 <= (M2 at creation) spatial nodes from now on (a plan made for the largest size
 * serves smaller requests; the results are those of a plan made for the exact sizes).
 * Discards the node preprocessing: call nnfft_set_nodes next.  EINVAL for batches or
 * sizes above the capacity.  Host-side only; work already queued is unaffected.
 */
int nnfft_set_sizes(nnfft_plan_t p, int64_t M1, int64_t M2);

/*
 * nnfft_set_bandwidth: use a single-instance plan made for bandwidth N' for the
 * transform with bandwidth N <= N' (exp(-2 pi i N v x)): the frequency nodes are binned
 * with u = v N1 N / N* instead of v N1 N' / N*, which is the plan's transform at the
 * nodes v N / N' (in [-1/2, 1/2]).  The window parameters stay those of N' (oversampling
 * relative to N grows).  Discards the node preprocessing of the v side.  EINVAL for
 * batches or N outside [1, N'].
 */
int nnfft_set_bandwidth(nnfft_plan_t p, int64_t N);

/*
 * nnfft_set_stream: issue the plan's later work on `stream` (cudaStream_t or NULL).
 * The caller orders it after the plan's earlier work (e.g. by waiting for it).
 */
int nnfft_set_stream(nnfft_plan_t p, void *stream);

/* nnfft_batch_count: number of instances in the plan (1 for nnfft_plan). */
int nnfft_batch_count(nnfft_plan_t p, int64_t *count);

/* nnfft_batch_info: derived parameters of instance i (0 <= i < count; EINVAL otherwise). */
int nnfft_batch_info(nnfft_plan_t p, int64_t i, nnfft_info *out);

/*
 * nnfft_plan_info: copy the derived parameters of a plan.  For a batch: M1, M2, K1, N1,
 * N2, ncell1, ncell2 are sums over the instances (N2: total grid length), N, Nstar,
 * fit_err1/2 and fft_n1/n2 maxima, D1/D2 the common degrees, the other fields those of
 * instance 0.
 */
int nnfft_plan_info(nnfft_plan_t p, nnfft_info *out);

/*
 * Autotuning (the paper has no counterpart).  nnfft_autotune times the plan's kernel
 * variants with the caller's buffers and keeps the fastest: threads per work item of the
 * moments kernel (32: one warp per item; 16: two items per warp, split-precision kernel
 * only; 8: four items per warp; the same for both sides), the evaluation kernel (32 or 8
 * per item, or 1: one thread per sorted point with no work items), the FFT's packing of
 * short columns into blocks (variant 0 by the plan-size rule, variant 1 the other
 * extreme) and, when the nodes are given, the largest work item (item_cap: 256, 128, 64
 * or 32 points; smaller items give dense cells more parallel work) and whether work items
 * of at most 16 points run one thread per item (item_split; only tried where some
 * instance has few points per cell).  With v and x (device) every run is a full
 * nnfft_transform; with v = x = NULL it is nnfft_exec_adjoint on the current nodes.  The
 * settings are searched one at a time from the defaults with the others at their current
 * best (two sweeps); each value is timed in three interleaved rounds of `reps` runs (best
 * kept) and the current value stays unless another is more than 3 % faster.  flags:
 * NNFFT_TUNE_FLUSH_L2 writes a 192 MB buffer before every timed run (cold L2, as in a
 * stream of new problems).  y and z receive the transforms.  Synchronous.  Other variants
 * sum in another order, so later results may change in the last bits.
 */
enum { NNFFT_TUNE_FLUSH_L2 = 1 };
typedef struct {
    int moments_lanes_v, moments_lanes_x;   /* 32, 16 or 8 lanes per work item; 4: the 8-lane
                                               split-precision kernel with two accumulator sets
                                               per lane */
    int fft_variant;                        /* 0 or 1 (two-pass FFT), 2 (cluster FFT), 3 (the
                                               split-precision grid stage as one cooperative
                                               launch) */
    int tuned;                              /* 1 after nnfft_autotune */
    double default_ms, best_ms;             /* per run: default and chosen config */
    int item_split;                         /* 1: small work items one thread each (default 0) */
    int timed_transform;                    /* 1: runs were full transforms */
    int eval_lanes_v, eval_lanes_x;         /* evaluation lanes per item: 32 or 8; 1 = flat
                                               (thread per point); 2 = flat with each block's
                                               cell window sums staged by a TMA bulk copy;
                                               3 = 32 lanes that also compute their cell's
                                               window sums from the grid (the gather
                                               convolution inside the evaluation; split
                                               precision, single plans, else as 32) */
    int item_cap;                           /* points per work item at most: 256, 128, 64, 32 */
    int sort_lsd;                           /* node sort of 9- to 16-bit cell keys: 0 two-stage
                                               (high-digit scatter, then a shared-memory sort per
                                               bucket; default for single instances), 1 LSD radix
                                               passes (default for batches) */
} nnfft_tuning;
int nnfft_autotune(nnfft_plan_t p, const double *v_dev, const double *x_dev, const void *f_dev,
                   void *y_dev, const void *g_dev, void *z_dev, int reps, int flags);
int nnfft_get_tuning(nnfft_plan_t p, nnfft_tuning *out);
/* nnfft_set_tuning: apply a configuration (e.g. one kept from an earlier nnfft_autotune):
 * moments_lanes_v / _x in {4, 8, 16, 32}, eval_lanes_v / _x in {1, 2, 3, 8, 32} (0: 32), fft_variant in
 * {0, 1} (two-pass FFT, two column packings) or 2 (single-instance plans whose grid fits, N2 up
 * to about 32K: the FFT as one launch of an 8-CTA thread-block cluster holding the grid in
 * distributed shared memory; bitwise the same result) or 3 (complex128 plans in split precision
 * with D1 = D2: cell fold, spread convolution, both FFT passes and gather convolution of a
 * direction in one cooperative launch whose persistent blocks meet at grid-wide barriers with
 * bounded waits -- a wait that gives up makes the plan report NNFFT_ETIMEOUT; bitwise the same
 * result; exec/adjoint and transforms only, the split entry points nnfft_spread_grid ... keep
 * the separate launches), item_split in {0, 1}, item_cap in {32, 64, 128, 256} (0: 256), sort_lsd in {0, 1}
 * (both sorts give the same order: the same results bitwise); the other fields are
 * ignored (a lane count a kernel does not have runs as one warp per item).  EINVAL otherwise.
 * Takes effect for the work queued next; a changed item_split, item_cap or sort_lsd needs
 * nnfft_set_nodes again. */
int nnfft_set_tuning(nnfft_plan_t p, const nnfft_tuning *t);

/*
 * nnfft_set_arith: choose NNFFT_ARITH_FP64 or NNFFT_ARITH_FP64_SPLIT for a complex128 plan
 * (EINVAL if unavailable).  Changing the mode discards the plan's node preprocessing:
 * call nnfft_set_nodes again before the next exec/adjoint.
 */
int nnfft_set_arith(nnfft_plan_t p, int arith);

/*
 * nnfft_set_nodes: step 0 of Algorithm 2.2 for a new node set.
 * v_dev: M1 doubles, x_dev: M2 doubles, both device pointers, values in
 * [-1/2, 1/2].  Either may be NULL to keep that side's previous nodes.
 * The nodes are rescaled (v* = N v / N*, after eq. (2.7)), binned by grid
 * cell and sorted (stable), and the plan keeps the sorted local coordinates
 * and the permutation; the caller's arrays are not referenced afterwards.
 * Out-of-range or NaN nodes set NNFFT_ERANGE in the status word.
 */
int nnfft_set_nodes(nnfft_plan_t p, const double *v_dev, const double *x_dev);

/*
 * nnfft_exec: the NNFFT, y_j ~ sum_k f_k exp(-2 pi i N v_k x_j)
 * (Algorithm 2.2 steps 1-4 and the output division).
 * f_dev: M1 complex values, y_dev: M2 complex values (device, plan dtype).
 */
int nnfft_exec(nnfft_plan_t p, const void *f_dev, void *y_dev);

/*
 * nnfft_adjoint: z_k ~ sum_j g_j exp(+2 pi i N v_k x_j), computed as the exact
 * transpose of the fast forward map (every step of Algorithm 2.2 reversed).
 * g_dev: M2 complex values, z_dev: M1 complex values (device, plan dtype).
 */
int nnfft_adjoint(nnfft_plan_t p, const void *g_dev, void *z_dev);

/*
 * Sharded transform: Algorithm 2.2 split at its grid, for node sets divided among P
 * processes (one GPU each).  Step 1 (eq. (2.12)) is a sum over the frequency nodes k and
 * step 4 is independent per spatial node j, so each process holds a plan with the same
 * N, sigma1, sigma2, m1, m2 and dtype for its own share of the v nodes (M1_r of them)
 * and of the x nodes (M2_r), and a direction becomes
 *     forward: nnfft_spread_grid (steps 1-2 for its v share) -> sum of the P grids
 *              (an all-reduce, done by the caller) -> nnfft_exec_grid (steps 3-4 and the
 *              output division for its x share);
 *     adjoint: nnfft_adjoint_spread_grid (the transposed steps 4 for its x share) -> sum
 *              -> nnfft_adjoint_grid (the transposed steps 3-1 for its v share).
 * The results equal those of one plan over all nodes up to the rounding of the sum.
 * Grids are device arrays of complex values of the plan's type, centered index l stored
 * at l + n/2, n even:
 *     forward: n = K1 = N1 + 2 m1 values ghat_l / N2 = g_l / (N2 phihat2(l)), l in I_K1
 *              (steps 1-2: the deconvolved grid with the 1/N2 of step 3);
 *     adjoint: n = N2 values u_s = sum_j g_j phi2(x_j/sigma1 - s/N2) / phihat1(N* x_j),
 *              s in I_N2 (the window sums taken N2-periodically, N* the rescaled bandwidth of
 *              eq. (2.7)), the transpose of step 4.
 * K1 and N2 are in nnfft_plan_info.  Single-instance plans only (NNFFT_EINVAL for a
 * batch); nnfft_set_nodes first (NNFFT_ESTATE).  Asynchronous on the plan stream like
 * nnfft_exec; the grid is read or written in stream order.  A share may be empty: its
 * grid is then zero (spread) or the call does nothing (exec/adjoint from a grid).
 */
int nnfft_spread_grid(nnfft_plan_t p, const void *f_dev, void *grid_dev);
int nnfft_exec_grid(nnfft_plan_t p, const void *grid_dev, void *y_dev);
int nnfft_adjoint_spread_grid(nnfft_plan_t p, const void *g_dev, void *grid_dev);
int nnfft_adjoint_grid(nnfft_plan_t p, const void *grid_dev, void *z_dev);

/*
 * nnfft_exec_adjoint: y = A f and z = A^H g for the same nodes in one call, the two
 * directions running concurrently (the adjoint on the plan's second stream with its own
 * work buffers, allocated on the first call).  Same results, arguments and errors as
 * nnfft_exec followed by nnfft_adjoint; ordered on the plan stream like them.
 */
int nnfft_exec_adjoint(nnfft_plan_t p, const void *f_dev, void *y_dev, const void *g_dev,
                       void *z_dev);

/*
 * Host-buffer variants of set_nodes / exec / adjoint.  Same arguments as above
 * but host pointers: the call copies the inputs into plan-owned device
 * staging buffers, runs the transform, copies the result back and waits for
 * the stream.  Returns any pending kernel status like nnfft_sync.
 */
int nnfft_set_nodes_host(nnfft_plan_t p, const double *v_host, const double *x_host);
int nnfft_exec_host(nnfft_plan_t p, const void *f_host, void *y_host);
int nnfft_adjoint_host(nnfft_plan_t p, const void *g_host, void *z_host);

/*
 * nnfft_exec_host_noalloc: nnfft_exec_host without any device allocation.
 * The paper has no counterpart of this call; it exists for callers that cannot
 * allocate device memory when they call the library -- code whose GPU memory is
 * owned by another allocator (a framework's caching allocator that has reserved
 * nearly all of the device, where a cudaMalloc would fail or fragment it) and
 * latency-bound serving loops that must not stall on an allocation.
 * nnfft_exec_host allocates its device staging on first use; this call stages
 * f and y in one static 4 MiB device array of the library instead (held on every
 * GPU that loads the library until exit), so M1 and M2 complex values of the
 * plan's type must fit in 4 MiB (f's part rounded up to 256 bytes): about
 * 262,000 points in total for complex128.  Larger plans get NNFFT_EINVAL.
 * Same arguments and result as nnfft_exec_host (host pointers; returns after the
 * stream has drained, with any pending kernel status).  All calls on a device
 * share the array; calls whose GPU work overlaps race on it, so serialise them.
 * The call works on the plan's device (the one current at nnfft_plan), switching
 * to it for the call if another device is current and back before returning.
 * The first call on each device looks up the array's address (with that device
 * current); make that first call before any stream capture.
 */
int nnfft_exec_host_noalloc(nnfft_plan_t p, const void *f_host, void *y_host);

/*
 * nnfft_transform: new nodes and both directions in one call, device buffers:
 * y = A f and z = A^H g for the nodes v, x (sizes as nnfft_set_nodes / nnfft_exec).  The
 * two node sides are sorted concurrently; the forward starts as soon as v is sorted and
 * waits for x only before its gather half, the adjoint the other way round, so the
 * directions overlap each other and the sort.  f = y = NULL or g = z = NULL skips a
 * direction.  Asynchronous on the plan stream; results equal nnfft_set_nodes +
 * nnfft_exec + nnfft_adjoint.
 */
int nnfft_transform(nnfft_plan_t p, const double *v_dev, const double *x_dev, const void *f_dev,
                    void *y_dev, const void *g_dev, void *z_dev);

/*
 * CUDA graph of one nnfft_transform over fixed device buffers.  nnfft_transform_graph
 * records the whole call (both node sorts, forward and adjoint, both streams) into a
 * graph; each nnfft_graph_launch replays it on the plan stream with the buffers' contents
 * at that time (write new nodes or values into the same buffers between launches), with
 * one launch instead of a few dozen.  The kernel variants (nnfft_set_tuning /
 * nnfft_autotune) and sizes are those at capture time: capture again after changing
 * them.  The capture queues no work, but the plan then holds the captured nodes as its
 * node set: launch the graph before nnfft_exec / nnfft_adjoint on them.  The graph must
 * not outlive the plan or the buffers.
 * nnfft_graph_kernels: library kernels one replay runs (counted by nnfft_launch_count at
 * every launch).  Errors: EINVAL (null argument), ENOMEM, ECUDA.
 */
typedef struct nnfft_graph_s *nnfft_graph_t;
int nnfft_transform_graph(nnfft_plan_t p, const double *v_dev, const double *x_dev,
                          const void *f_dev, void *y_dev, const void *g_dev, void *z_dev,
                          nnfft_graph_t *out);
int nnfft_graph_launch(nnfft_graph_t g);
int64_t nnfft_graph_kernels(nnfft_graph_t g);
int nnfft_graph_destroy(nnfft_graph_t g);
/*
 * nnfft_transform_host_graph: the same for nnfft_transform_host (below) over fixed
 * page-locked host buffers (cudaHostAlloc / cudaHostRegister / pinned tensors): one replay
 * uploads the buffers' current contents, runs the transform and writes y and z back to the
 * host buffers.  nnfft_graph_launch only queues the work: nnfft_sync(p) waits for it and
 * returns the node status (ERANGE) that nnfft_transform_host returns directly.  EINVAL if
 * a given host buffer is not page-locked (a pageable copy cannot be captured).
 */
int nnfft_transform_host_graph(nnfft_plan_t p, const double *v_host, const double *x_host,
                               const void *f_host, void *y_host, const void *g_host,
                               void *z_host, nnfft_graph_t *out);

/*
 * nnfft_transform_host: new nodes and both directions from host memory in one call:
 * y = A f and z = A^H g for the nodes v, x (all host arrays of the plan's sizes; pinned
 * memory copies asynchronously).  The nodes are uploaded first and sorted (one side per
 * stream) while f and g go up on a third stream; the forward and the adjoint then run
 * concurrently and their results come back on their own streams.  Pass f = y = NULL or
 * g = z = NULL to skip a direction.  Synchronous; returns any kernel status (ERANGE for a
 * node outside [-1/2, 1/2]).  Results equal nnfft_set_nodes_host + nnfft_exec_host +
 * nnfft_adjoint_host.
 */
int nnfft_transform_host(nnfft_plan_t p, const double *v_host, const double *x_host,
                         const void *f_host, void *y_host, const void *g_host, void *z_host);

/* nnfft_sync: wait for the plan's stream; return and clear the kernel status. */
int nnfft_sync(nnfft_plan_t p);

/*
 * nnfft_node_order: the order step 0 of Algorithm 2.2 put one side's nodes in (the
 * binning by grid cell and the stable sort by cell of nnfft_set_nodes), copied to host
 * memory, for callers that keep their own data in the plan's cell order and for checks.
 * side 0: the frequency nodes v (M1 points, cells of the window phi1's grid), side 1: the
 * spatial nodes x (M2 points, cells of the N2-grid).  Cells are consecutive intervals of the
 * node axis, in increasing order of the node.
 * perm_host: NULL or M int32 (caller-owned host memory): perm[i] = caller index of sorted
 *   position i; within a cell the caller indices increase (the sort is stable).
 * off_host: NULL or ncell + 1 int32: the points of cell c are the sorted positions
 *   off[c] .. off[c + 1] - 1 (off[0] = 0, off[ncell] = M).
 * ncell_out: NULL or the number of cells of the side.
 * Waits for the plan's stream (without reading or clearing the kernel status: nnfft_sync
 * still reports it).  Single-instance plans only: EINVAL for a batch plan or a side other
 * than 0 or 1; ESTATE when perm_host or off_host is given and the side's nodes were never set.
 */
int nnfft_node_order(nnfft_plan_t p, int side, int32_t *perm_host, int32_t *off_host,
                     int64_t *ncell_out);

/* nnfft_destroy: free the plan (waits for its stream first).  NULL is a no-op. */
int nnfft_destroy(nnfft_plan_t p);

/*
 * sinc_exec: fast sinc transform, Algorithm 6.1 with an n = 2N node
 * Gauss-Legendre rule on [-1/2, 1/2] in place of Clenshaw-Curtis:
 *   g_j     = sum_k c_k exp(+2 pi i N tau_j a_k)        (NNFFT #1, nodes a -> -tau)
 *   alpha_j = w_j g_j                                    (step 2)
 *   h_l     = sum_j alpha_j exp(-2 pi i N tau_j b_l)    (NNFFT #2, nodes tau -> b)
 * which approximates h_l = sum_k c_k sinc(N pi (b_l - a_k)).
 * Both NNFFTs use sigma1 = sigma2 = 2 and m1 = m2 = m.
 * a_dev: L1 doubles, b_dev: L2 doubles in [-1/2, 1/2] (device).
 * c_dev / h_dev: L1 / L2 values in the dtype's real type when is_complex = 0
 * (h is then the real part; it is real up to rounding for real c because the
 * rule is symmetric), or interleaved complex when is_complex = 1.
 * The call keeps an internal plan cache keyed by (N, L1, L2, m, dtype, stream);
 * stream as in nnfft_plan.  Asynchronous like nnfft_exec; call sinc_sync to wait
 * and to collect a kernel status.
 */
int sinc_exec(int64_t N, int64_t L1, int64_t L2, int m, nnfft_dtype dtype,
              const double *a_dev, const void *c_dev, const double *b_dev, void *h_dev,
              int is_complex, void *stream);

/*
 * Quadrature rules for sinc(N pi x) = int_{-1/2}^{1/2} exp(-2 pi i N t x) dt
 * (Section 5; equivalently (1/2) int_{-1}^{1} exp(-pi i N z x) dz with z = 2t):
 *   SINC_RULE_GL  n-point Gauss-Legendre rule on [-1/2, 1/2] (n = 0 selects 2N);
 *   SINC_RULE_CC  Clenshaw-Curtis: nodes t_j = cos(j pi / n) / 2, j = 0..n, and the
 *                 weights of eq. (5.4) computed on the GPU by Algorithm 5.4 (a DCT-I,
 *                 done as one FFT of length 2n).  n = 0 selects 4N (Algorithm 6.1:
 *                 n >= 4N); n is rounded up to the next 5-smooth integer (the paper's
 *                 n = 2^t is one) and 2n may not exceed 2^20.  Theorem 5.3 bounds the
 *                 quadrature error by 36(1 + e^{-2CN})/(35(e^2 - 1)) e^{-N(n/N - C)},
 *                 C = pi (e^2 - 1)/(2e) ~ 3.69.
 */
enum { SINC_RULE_GL = 0, SINC_RULE_CC = 1 };

/*
 * sinc_exec_rule: Algorithm 6.1 with the given rule (t_j, w_j):
 *   step 1  g_j     = sum_k c_k exp(-2 pi i N a_k x1_j)   (NNFFT #1, nodes a -> x1)
 *   step 2  alpha_j = w_j g_j
 *   step 3  h_l     = sum_j alpha_j exp(-2 pi i N v2_j b_l) (NNFFT #2, nodes v2 -> b)
 * with x1 = t, v2 = -t for CC (the signs of Algorithm 6.1) and x1 = -t, v2 = t for GL
 * (the same sums, since the GL rule is symmetric).  Arguments, caching, streams and
 * errors as in sinc_exec; the cache key includes rule and n.  EINVAL for an unknown
 * rule or n < 0.
 */
int sinc_exec_rule(int64_t N, int64_t L1, int64_t L2, int m, nnfft_dtype dtype, int rule,
                   int64_t n, const double *a_dev, const void *c_dev, const double *b_dev,
                   void *h_dev, int is_complex, void *stream);

/*
 * sinc_quadrature: the rule sinc_exec_rule uses for (rule, N, n): *nodes_out = its
 * number of nodes (n for GL, n + 1 for CC after rounding); if t_host and w_host are
 * non-null they receive the nodes t_j (in [-1/2, 1/2]) and weights w_j (host arrays
 * of *nodes_out doubles).  GL needs no GPU; CC weights come from the device
 * (NNFFT_ECUDA without one).  Synchronous.
 */
int sinc_quadrature(int rule, int64_t N, int64_t n, double *t_host, double *w_host,
                    int64_t *nodes_out);

/* sinc_sync: wait for `stream` and return/clear the status of the cached sinc plans on it. */
int sinc_sync(void *stream);

/* sinc_release: free every cached sinc plan (all streams). */
int sinc_release(void);

/*
 * nnfft_gauss_legendre: the library's n-point Gauss-Legendre rule on [-1/2, 1/2]
 * (increasing nodes tau, weights w summing to 1), as used by sinc_exec.  Host
 * arrays of length n.  No GPU needed.
 */
int nnfft_gauss_legendre(int64_t n, double *tau_host, double *w_host);

/*
 * Per-stage device timing (tracing).  When enabled, every stage of set_nodes /
 * exec / adjoint is bracketed by CUDA events recorded on the plan stream; the
 * elapsed times accumulate until nnfft_timing_read (which waits for the stream).
 * Stage ids (index into ms[] / count[]):
 *   0 v-side node binning + sort     1 x-side node binning + sort
 *   2 forward cell moments (v)       3 forward spread convolution
 *   4 forward FFT (both passes)      5 forward gather convolution
 *   6 forward point evaluation (x)   7 adjoint cell moments (x)
 *   8 adjoint spread convolution     9 adjoint FFT
 *  10 adjoint gather convolution    11 adjoint point evaluation (v)
 *  12 forward per-cell fold (v)      13 adjoint per-cell fold (x, with 1/phihat1)
 */
#define NNFFT_NSTAGES 14
typedef struct {
    double ms[16];      /* accumulated milliseconds per stage */
    int64_t count[16];  /* number of timed executions per stage */
} nnfft_timing;
int nnfft_timing_enable(nnfft_plan_t p, int enable);
int nnfft_timing_read(nnfft_plan_t p, nnfft_timing *out, int reset);

/*
 * nnfft_selftest_fixed63: check of the node kernel's conversion of a signed 64-bit
 * fixed-point coordinate Y (value y = Y 2^-63) to floats.  For each of the n device inputs,
 * out_dev[4i .. 4i+3] = (the fp32 plans' float, the split plans' float pair h and l, CUDA's
 * own rounding conversion of Y); the caller checks |float - y| < 2^-31 + half an ulp and
 * |h + l - y| <= 2^-49 + 2^-56 with |l| <= ulp(h) / 2.  Synchronous on the legacy default
 * stream.  EINVAL for n < 0, n > 2^28 or null pointers with n > 0.
 */
int nnfft_selftest_fixed63(const int64_t *in_dev, float *out_dev, int64_t n);

/*
 * nnfft_selftest_bulk_copy: check of the bounded waits around the library's bulk (TMA)
 * copies into shared memory.  One block arms a shared-memory barrier for n floats
 * (0 < n <= 4096, n a multiple of 4), copies src_dev into shared memory with one bulk copy
 * and writes it to dst_dev.  With arm_only the copy is not issued, so the wait on the
 * barrier gives up after limit_cycles SM clock cycles: the block ORs the timeout bit (4)
 * into *status_dev (a device int) and returns without writing dst_dev, as the evaluation
 * kernels do, which turn that bit into NNFFT_ETIMEOUT.  Synchronous on the legacy default
 * stream.  EINVAL for invalid arguments.
 */
int nnfft_selftest_bulk_copy(const float *src_dev, float *dst_dev, int n, int arm_only,
                             int64_t limit_cycles, int *status_dev);

/*
 * nnfft_selftest_grid_barrier: check of the bounded grid-wide barrier of the fused grid
 * stage (nnfft_tuning.fft_variant 3).  A cooperative launch of `blocks` blocks (1 ..
 * the device's SM count) passes two barriers that each expect blocks + extra arrivals.
 * words_dev: two 64-bit device words, zero before the first call (an arrival counter that
 * only grows, and an abort word).  extra = 0: both barriers complete and the counter grows
 * by 2 * blocks.  extra > 0: nobody completes the first barrier, so every block's wait
 * gives up after limit_cycles SM clock cycles (or on seeing another block give up): the
 * timeout bit (4) is ORed into *status_dev, the abort word is set and the blocks return,
 * as the fused grid stage does, whose plan then reports NNFFT_ETIMEOUT.  Synchronous on the
 * legacy default stream.  EINVAL for invalid arguments, ECUDA if the launch fails.
 */
int nnfft_selftest_grid_barrier(int blocks, int extra, int64_t limit_cycles,
                                uint64_t *words_dev, int *status_dev);

/* nnfft_launch_count: number of kernels this library has launched in the process. */
int64_t nnfft_launch_count(void);

/*
 * Request loop (serving).  The paper has no counterpart: this serves many NNFFT and fast
 * sinc transform requests of different N, M1, M2 and tolerances on one GPU.
 *
 * nnfft_tolerance_params: the arithmetic a tolerance (max error / sum |f|) is served
 * with: *dtype = NNFFT_C64 for tol >= 1e-6, else NNFFT_C128; *m = the smallest window
 * half-width in [2, 12] with (24 m^{3/2} + 10) exp(-2 pi m sqrt(1/2)) <= tol (the first
 * term of Theorem 4.1 at sigma = 2).  Host only.
 */
int nnfft_tolerance_params(double tol, int *dtype, int *m);

enum { NNFFT_REQ_NNFFT = 0, NNFFT_REQ_SINC = 1 };

/*
 * One request.  NNFFT: y_j = sum_k f_k exp(-2 pi i N v_k x_j), M1 nodes v and values f,
 * M2 nodes x and outputs y.  Sinc (Algorithm 6.1): h_l = sum_k c_k sinc(N pi (b_l - a_k)),
 * with v = a and f = c (M1 = L1 of them), x = b and y = h (M2 = L2), `rule` a
 * SINC_RULE_* (2N Gauss-Legendre or 4N Clenshaw-Curtis for the request's bandwidth
 * bucket), `is_complex` selecting complex c / h (else real).  All pointers are HOST
 * memory (pinned memory gives asynchronous copies), owned by the caller and kept alive
 * until nnfft_server_wait returns for the request.  Values are in the tolerance's type
 * (nnfft_tolerance_params): complex64 / float for NNFFT_C64, complex128 / double else.
 */
typedef struct {
    int kind;              /* NNFFT_REQ_NNFFT or NNFFT_REQ_SINC */
    int rule;              /* sinc only */
    int is_complex;        /* sinc only */
    int reserved;
    int64_t N, M1, M2;     /* 1 <= N <= 65536 (sinc: <= 16384); M1, M2 <= max_points */
    double tol;            /* > 0 */
    const double *v, *x;
    const void *f;
    void *y;
} nnfft_request;

typedef struct {
    int64_t completed, failed, pending, in_flight;
    double p50_ms, p99_ms, mean_ms, max_ms;   /* latency submit -> completion */
    double points;                            /* sum of M1 + M2 of completed requests */
    double seconds;                           /* first submit -> last completion */
    int64_t plans_cached, plans_made, plans_evicted, device_bytes;
} nnfft_server_report;

/*
 * nnfft_server_create: start a request loop on the current device with `slots` request
 * slots (streams; 1..64), device buffers for requests of up to max_points nodes per side,
 * and a device-memory budget (bytes) for buffers plus cached plans.  Requests queue in
 * arrival order; a request starts when a slot is free and its plans fit in the budget
 * (idle cached plans are evicted least recently used first).  Plans are cached per
 * (bandwidth rounded up to a power of two >= 64, tolerance class) with capacities
 * rounded up to powers of two; a result equals that of the library's own plan for the
 * bucket's parameters (the same result alone and in any mix of requests).
 */
typedef struct nnfft_server_s *nnfft_server_t;
int nnfft_server_create(nnfft_server_t *out, int64_t mem_budget_bytes, int slots,
                        int64_t max_points);
/* Queue a request (copied); *id identifies it.  EINVAL for sizes outside the limits. */
int nnfft_server_submit(nnfft_server_t s, const nnfft_request *r, int64_t *id);
/* Block until request id is done; returns its status (the id is then released). */
int nnfft_server_wait(nnfft_server_t s, int64_t id, double *latency_ms);
/* nnfft_server_wait that also returns where the request's work ran on the device: four
 * times in ms since the server was created, from CUDA events on its slot stream, before its
 * uploads, before its first kernel, after its last kernel and after its download (device_ms
 * may be NULL; -1 for a failed request).  Requests whose [first, last] intervals intersect
 * had work on the device at the same time (copies of one beside kernels of the other, or
 * kernels of both). */
int nnfft_server_wait_device(nnfft_server_t s, int64_t id, double *latency_ms, double *device_ms);
/* Latency percentiles and throughput of the requests completed so far (reset: restart). */
int nnfft_server_stats(nnfft_server_t s, nnfft_server_report *out, int reset);
/* Finish the queued requests, stop the loop and free everything. */
int nnfft_server_destroy(nnfft_server_t s);

/* nnfft_last_error: thread-local message describing the last non-OK status. */
const char *nnfft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NNFFT_GB300_H */
