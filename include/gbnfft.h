/*
 * gbnfft: the gridding NFFT of the HP-NFFT paper on one GB300 GPU.
 *
 * C ABI.  All functions return an nfft_status (0 = success, < 0 = error)
 * unless stated otherwise; none throws.  Pointers named *_dev are device
 * pointers the caller owns (for example PyTorch tensors); the library never
 * frees them and never copies them to the host.  Work is queued on the plan's
 * CUDA stream and is asynchronous: argument errors are returned at once,
 * errors found on the device (non-finite points) are returned by nfft_sync.
 * A plan is not thread-safe; distinct plans may be used from distinct threads.
 *
 * Notation (paper, Section 1):
 *   I_N = { k in Z^d : -N_t/2 <= k_t < N_t/2 },  N_t even, d in {1, 2, 3}
 *   Eq. 5 (adjoint):  fhat(k) = sum_{j<M} f(x_j) exp(-2 pi i k.x_j),  k in I_N
 *   Eq. 6 (forward):  f(x_j)  = sum_{k in I_N} fhat(k) exp(+2 pi i k.x_j)
 * Eq. 6 is the transpose A^H of Eq. 5's matrix A, which the paper calls the
 * "inverse NDFT"; this library calls it the forward transform.
 *
 * Both transforms are computed by the gridding method of Section 2 on the
 * oversampled grid I_n, n_t = sigma N_t rounded up to an even 2,3,5,7-smooth
 * integer: spreading with a window phi, FFT, scaling by c_k(phi~) (Fig. 1,
 * Algorithm 2) and subdividing, inverse FFT, interpolating (Fig. 2,
 * Algorithm 5).  Each point reaches 2m + 2 cells per dimension (the
 * Kaiser-Bessel window is zero on two of them, which the kernels skip).
 *
 * Layouts
 *   x      M x d doubles, point-major: x[j*d + t] is coordinate t of point j,
 *          paired with N_t.  Any finite value (Eq. 5 is 1-periodic in x).
 *   f      R x M complex, right-hand side r at f + r*M.
 *   fhat   R x |I_N| complex, each in C order over (k_0, ..., k_{d-1}) with
 *          every k_t ascending from -N_t/2 (the last index varies fastest).
 *   complex = interleaved (re, im): double for NFFT_FP64, float for
 *          NFFT_FP32_MIXED.
 */
#ifndef GBNFFT_H
#define GBNFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nfft_plan nfft_plan;

/* Window functions named in Section 4 (Fig. 12), in the cell variable
 * u = n x of each dimension (formulas: the standard NFFT windows).
 * Gaussian: 2m + 2 taps; the others 2m taps (their weight vanishes at the
 * two outer cells).  B-spline and sinc-power evaluate slower and serve
 * precision studies; the picker chooses between Gaussian and Kaiser-Bessel. */
typedef enum {
  NFFT_GAUSSIAN = 0,      /* exp(-u^2 / b), b = 2 sigma m / ((2 sigma - 1) pi) */
  NFFT_KAISER_BESSEL = 1, /* sinh(b sqrt(m^2 - u^2)) / sqrt(m^2 - u^2), |u| < m, b = pi (2 - 1/sigma) */
  NFFT_B_SPLINE = 2,      /* M_2m(u), the centred cardinal B-spline of order 2m */
  NFFT_SINC_POWER = 3     /* sinc(pi u (2 sigma - 1) / (2 m sigma))^(2m), |u| < m (sinc t = sin t / t) */
} nfft_window;

/* NFFT_FP64: FP64 points, weights, grid and FFT (the plain form).
 * NFFT_FP32_MIXED: FP64 argument reduction of n x_j and FP64 scaling factors,
 * FP32 window weights, FP32 spreading / interpolation with FP32 accumulation,
 * FP32 FFT. */
typedef enum {
  NFFT_FP64 = 0,
  NFFT_FP32_MIXED = 1
} nfft_precision;

typedef enum {
  NFFT_OK = 0,
  NFFT_ERR_INVALID_ARG = -1,  /* bad size, null pointer, odd N, sigma < 1, ... */
  NFFT_ERR_DOMAIN = -2,       /* a point coordinate was NaN or infinite */
  NFFT_ERR_OOM = -3,          /* device allocation failed */
  NFFT_ERR_CUDA = -4,         /* a CUDA runtime call failed */
  NFFT_ERR_CUFFT = -5,        /* a cuFFT call failed */
  NFFT_ERR_NOT_READY = -6,    /* transform requested before nfft_set_points */
  NFFT_ERR_TIMEOUT = -7,      /* a bounded device wait gave up */
  NFFT_ERR_UNSUPPORTED = -8   /* valid request outside what this build supports */
} nfft_status;

/* Spreading / interpolation kernels. */
typedef enum {
  NFFT_METHOD_AUTO = 0,   /* warp if available, else tiled if the tile fits, else global */
  NFFT_METHOD_TILED = 1,  /* bin-sorted points, per-subproblem shared-memory tile */
  NFFT_METHOD_GLOBAL = 2, /* one thread per point, atomics straight into the grid
                             (the paper's spread kernel, Section 3) */
  NFFT_METHOD_WARP = 3,   /* d = 2 (up to 16 taps): one warp per point, lanes on
                             distinct cells, warp-private shared-memory tiles;
                             d = 3 (up to 26 taps): one shared tile per block,
                             spreading by plane-owner warps without atomics */
  NFFT_METHOD_GRID_WARP = 4 /* one warp per point straight on the grid (vector
                             atomics / gathers, no tile), every subproblem */
} nfft_method;

/* Options for nfft_set_option. */
typedef enum {
  NFFT_OPT_METHOD = 0,          /* nfft_method */
  NFFT_OPT_BIN_0 = 1,           /* bin edge in cells along dimension 0 (0 = default) */
  NFFT_OPT_BIN_1 = 2,
  NFFT_OPT_BIN_2 = 3,
  NFFT_OPT_MAX_SUBPROBLEM = 4,  /* points per subproblem (0 = default) */
  NFFT_OPT_RHS_CAPACITY = 5,    /* grids kept for right-hand sides processed together */
  NFFT_OPT_PROFILE = 6,         /* 1: record CUDA events around every stage */
  NFFT_OPT_THREADS = 7,         /* threads per block of the point kernels (0 = default) */
  NFFT_OPT_SPREAD_THREADS = 8,  /* threads per block of spreading only (overrides 7) */
  NFFT_OPT_INTERP_THREADS = 9,  /* threads per block of interpolation only (overrides 7) */
  NFFT_OPT_SPARSE_POINTS = 10,  /* with NFFT_METHOD_AUTO: spreading subproblems of
                                   fewer points than this run on the
                                   NFFT_METHOD_GRID_WARP kernel, the rest on the
                                   tiled one (0 = automatic: one point per
                                   W^d / 2 tile cells, -1 = never) */
  NFFT_OPT_SPARSE_POINTS_INTERP = 11, /* the same for interpolation (0 = automatic:
                                   one point per W^d / 5 tile cells; gathers
                                   need no atomics, so the split sits higher) */
  NFFT_OPT_OWNER_SPREAD = 12,   /* d = 3: 1 spreads the sparse bins by their
                                   cells' owners (a warp per bin, no atomics,
                                   every cell written once) where the grid
                                   allows (n_t >= bin_t + W - 1); 0 (default)
                                   uses the grid-warp atomics, which measure
                                   faster (an owner pass repeats each point's
                                   weights for every owner it touches) */
  NFFT_OPT_TENSOR_SPREAD = 13,  /* d = 3, NFFT_FP32_MIXED, windows of 4, 6 or 8
                                   taps, NFFT_METHOD_AUTO or _WARP: 1 spreads
                                   the dense bins on the tensor cores (tcgen05
                                   MMAs of TF32 operands split in two, so the
                                   products keep FP32 accuracy; the tile is the
                                   MMA accumulator in tensor memory).  Default
                                   bins become (12 - W, 12 - W, 16), so that the
                                   tile's (z, y) rows fit the MMA's 128; explicit
                                   bins must satisfy (b0 + W - 1)(b1 + W - 1) <= 128
                                   and 2 (b2 + W - 1) <= 112, else nfft_set_option
                                   returns NFFT_ERR_UNSUPPORTED.  Interpolation
                                   keeps the plane kernels unless
                                   NFFT_OPT_TENSOR_INTERP is set.  0 (default): the
                                   plane-owner shared-memory kernel */
  NFFT_OPT_TENSOR_INTERP = 14,  /* the same conditions: 1 interpolates the dense
                                   bins on the tensor cores (the chunk's points
                                   as the MMA's rows, the tile's (z, y) rows as
                                   its K; each point then sums its own x
                                   columns).  Takes the same bins as
                                   NFFT_OPT_TENSOR_SPREAD; either option alone
                                   or both.  0 (default): the plane kernels */
  NFFT_OPT_PRUNED_FFT = 15      /* d = 3 plans of one item with N_0 < n_0: 1
                                   splits the FFT of Section 2 into the
                                   1-D transforms along dimension 0 over the
                                   whole grid and the 2-D transforms of
                                   dimensions 1, 2 over the N_0 planes that hold
                                   I_N (the adjoint transforms along 0 first and
                                   then only the planes its crop reads; the
                                   forward transforms the planes its padding
                                   fills, the others being zero, then along 0):
                                   1 + 2 N_0 / n_0 passes over the grid instead of
                                   3.  0: one 3-D cuFFT over the whole grid.
                                   -1 (default): automatic, the split form for
                                   grids of at least 128 MiB (beyond the L2
                                   cache; a smaller grid's 3-D cuFFT runs from
                                   L2), and nfft_autotune times both forms and
                                   keeps the faster (the option then reads 0
                                   or 1 in effect) */
} nfft_option;

/* Stages timed when NFFT_OPT_PROFILE is on (index into nfft_stage_times). */
typedef enum {
  NFFT_STAGE_SORT = 0,      /* nfft_set_points: wrap, cell, bin-sort, subproblems */
  NFFT_STAGE_SPREAD = 1,    /* adjoint step 1 */
  NFFT_STAGE_FFT = 2,       /* adjoint step 2 (forward cuFFT) */
  NFFT_STAGE_DECONV = 3,    /* adjoint step 3 (scale + crop) */
  NFFT_STAGE_PAD = 4,       /* forward step 1 (subdivide: scale + zero pad) */
  NFFT_STAGE_IFFT = 5,      /* forward step 2 (inverse cuFFT) */
  NFFT_STAGE_INTERP = 6,    /* forward step 3 */
  NFFT_STAGE_COUNT = 7
} nfft_stage;

typedef struct {
  int d;
  int64_t N[3];
  int64_t n[3];              /* oversampled grid */
  int64_t M;
  int m;                     /* cut-off parameter */
  int taps;                  /* nonzero window taps per dimension the kernels visit */
  int window;
  int precision;
  int method;                /* the method in use (never AUTO) */
  int bin[3];                /* bin edges in cells */
  int64_t n_bins;
  int rhs_capacity;
  int threads;               /* threads per block of the point kernels */
  int64_t device_bytes;      /* device memory held by the plan (grids, sort buffers, tables) */
  double sigma[3];           /* actual n_t / N_t */
  int max_subproblem;        /* points per subproblem in use */
  int spread_threads;        /* NFFT_OPT_SPREAD_THREADS (0 = chosen per launch) */
  int interp_threads;        /* NFFT_OPT_INTERP_THREADS (0 = chosen per launch) */
  int sparse_points;         /* spreading subproblems below this many points use the grid-warp kernel */
  int sparse_points_interp;  /* the same for interpolation */
  int owner_spread;          /* 1: sparse bins are spread by the owner kernel */
  int64_t kernel_launches;   /* this library's kernels launched by the plan so far
                                (cuFFT's own kernels and memsets not included) */
  int spread_block_threads;  /* threads per block of the last launch of the tiled spreading
                                kernel (3-D plane kernels: 32 x warps; 0 = none yet) */
  int interp_block_threads;  /* the same for interpolation */
  int tensor_spread;         /* 1: dense bins are spread on the tensor cores (NFFT_OPT_TENSOR_SPREAD) */
  int tensor_interp;         /* 1: dense bins are interpolated on the tensor cores (NFFT_OPT_TENSOR_INTERP) */
  int pruned_fft;            /* 1: the FFT runs as the pruned passes of NFFT_OPT_PRUNED_FFT */
} nfft_plan_info;

/* Create a plan (Section 2 parameters: bandwidth N, M points, oversampling
 * sigma >= 1, cut-off m >= 1, window, precision).  N points to d int64 values,
 * each even and >= 2.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  Allocates all device memory the transforms need; no later call
 * allocates unless NFFT_OPT_RHS_CAPACITY, a bin size or the method changes.
 * On error *out is NULL. */
int nfft_plan_create(nfft_plan** out, int d, const int64_t* N, int64_t M, double sigma, int m,
                     int window, int precision, void* cuda_stream);

/* Free the plan and everything it holds (waits for its stream first). NULL is ignored. */
int nfft_plan_destroy(nfft_plan* plan);

/* Set the M points (x_dev: M*d doubles on the device, layout above).  Wraps
 * each coordinate into [-1/2, 1/2) (exact: Eq. 5 is 1-periodic), reduces
 * u = n_t x_t to a cell index and an in-cell offset in FP64, and bin-sorts the
 * points by spatial tile (the on-device form of the paper's subcells,
 * Eqs. 7-8).  x_dev is read during the call's kernels only and may be freed or
 * reused once the stream passes them.  A NaN/Inf coordinate sets the plan's
 * device error flag (reported by nfft_sync as NFFT_ERR_DOMAIN); such a point
 * is treated as x = 0. */
int nfft_set_points(nfft_plan* plan, const double* x_dev);

/* Eq. 5 for R right-hand sides (Fig. 1, Algorithm 2): fhat_dev[r] = A f_dev[r].
 * f_dev: R x M complex, fhat_dev: R x |I_N| complex (precision's type). */
int nfft_adjoint(nfft_plan* plan, const void* f_dev, void* fhat_dev, int R);

/* Eq. 6 for R right-hand sides (Fig. 2, Algorithm 5): f_dev[r] = A^H fhat_dev[r]. */
int nfft_forward(nfft_plan* plan, const void* fhat_dev, void* f_dev, int R);

/* Reciprocal-space Ewald energy of Section 5, Eq. 12, for charges q_j at the
 * points set by nfft_set_points (x_j = r_j / L in box units):
 *   U^K = 1/(2 pi L) sum_{n in I_N, n != 0} exp(-pi^2 |n|^2 / (alpha L)^2) / |n|^2 |S(n)|^2
 *         - alpha / sqrt(pi) sum_j q_j^2,
 *   S(n) = sum_j q_j exp(-2 pi i n.x_j)   (the adjoint, Eq. 5).
 * q_dev: M complex values of the plan's precision (real charges: imaginary
 * part 0).  Runs spreading and the FFT, then reduces the scaled spectrum in
 * FP64 without writing fhat.  out (host, 3 doubles): out[0] = U^K,
 * out[1] = the n-sum term, out[2] = the self term.  Waits for the stream.
 * The sum runs over I_N only: it is converged only if the Gaussian factor is
 * negligible outside I_N. */
int nfft_ewald_reciprocal(nfft_plan* plan, const void* q_dev, double L, double alpha, double* out);

/* The n-sum term of Eq. 12, 1/(2 pi L) sum_{n != 0} exp(-pi^2 |n|^2/(alpha L)^2) / |n|^2 |S(n)|^2,
 * from a structure factor S_dev given on the plan's I_N (|I_N| complex of the
 * plan's precision, layout of fhat).  Writes one double to sum_dev (device),
 * asynchronously on the plan's stream, with a deterministic FP64 reduction
 * (fixed tiles of 8192 elements, fixed summation tree). */
int nfft_ewald_reciprocal_sum(nfft_plan* plan, const void* S_dev, double L, double alpha, double* sum_dev);

/* Reciprocal-space Ewald forces on the points set (d = 3 only, else
 * NFFT_ERR_UNSUPPORTED): the negative gradient of Eq. 12 (Section 5; the
 * paper names molecular dynamics as the use of the method but prints no
 * force formula, so this is the derivative written out).  With x_i = r_i / L
 * (up to an integer shift, e.g. x = r / L - 1/2) and S(n) = sum_j q_j
 * exp(-2 pi i n.x_j),
 *   F_i = (2 q_i / L^2) sum_{n in I_N, n != 0} exp(-pi^2 |n|^2 / (alpha L)^2) / |n|^2
 *         n Im(S(n) exp(2 pi i n.x_i)):
 * an adjoint NFFT of the charges (Eq. 5), the weights w(n) n_t on I_N, and a
 * forward NFFT (Eq. 6) of three right-hand sides.  q_dev: M complex of the
 * plan's precision (real part = charge); F_dev: device, M x 3 doubles,
 * point-major, written asynchronously on the plan's stream.  The first call
 * allocates 3 |I_N| + 3 M complex values of scratch kept by the plan. */
int nfft_ewald_reciprocal_forces(nfft_plan* plan, const void* q_dev, double L, double alpha, double* F_dev);

/* Largest |I_N| nfft_ewald_reciprocal_sum_noalloc accepts (4096 tiles of 8192). */
#define NFFT_NOALLOC_MAX_MODES 33554432

/* The same n-sum as nfft_ewald_reciprocal_sum, for callers that cannot
 * allocate device memory when they need it: code inside a framework whose
 * caching allocator owns the GPU memory (a direct cudaMalloc there can fail
 * or synchronise the device), steady-state loops that forbid allocation, or
 * callers with no plan.  The paper has no counterpart; it is a library
 * convenience.  No plan is needed and nothing is allocated: the caller passes
 * S_dev (|I_N| complex of `precision`'s type, layout of fhat, with I_N given
 * by d and N) and sum_dev (one device double, written asynchronously on
 * cuda_stream, NULL = legacy default stream).  Scratch is a static 32 KiB
 * device array of the library, held on every GPU that loads it until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current); make that first
 * call outside any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys and
 * recreates the device's primary context) the array may move and this entry
 * point must not be called again in that process.  All calls share the array: calls whose
 * work overlaps on the GPU (different streams, different host threads) race
 * and must be serialised by the caller.  Returns NFFT_ERR_UNSUPPORTED without
 * touching the GPU when |I_N| > NFFT_NOALLOC_MAX_MODES, NFFT_ERR_INVALID_ARG
 * for bad arguments, NFFT_ERR_CUDA if the launch fails. */
int nfft_ewald_reciprocal_sum_noalloc(int d, const int64_t* N, int precision, const void* S_dev, double L,
                                      double alpha, double* sum_dev, void* cuda_stream);

/* Real-space Ewald energy, Eq. 11 (Section 5): 1/2 sum over pairs (i, j)
 * and periodic images n, omitting n = 0 for i = j, of q_i q_j erfc(alpha d)/d
 * with d = |r_i - r_j + n L| < rcut.  r_dev: n x 3 positions (device, FP64,
 * row-major, any finite values: reduced mod L per coordinate); q_dev: n
 * charges (device, FP64).  Requires 0 < rcut < L.  When L / rcut >= 3 the
 * ions are sorted into a cell list of edge >= rcut / 2 and each ion visits
 * the 5^3 cells around its own (only the minimum image of a pair is within
 * rcut) and the pair terms are FP32 from offsets to
 * the cells' centres, with FP64 sums per ion; otherwise every pair and its
 * 27 nearest images are summed in FP64 (n <= 65536, else
 * NFFT_ERR_UNSUPPORTED).  The total is a fixed-order FP64 reduction.
 * Allocates scratch, runs on cuda_stream (NULL = legacy default stream) and
 * waits for it; *energy gets U^R (host double).  The paper computes this term
 * on the CPU side of its method; the library adds it so that the whole
 * Madelung check (Eq. 10) runs on the GPU. */
int nfft_ewald_real_space(int64_t n, const double* r_dev, const double* q_dev, double L, double alpha, double rcut,
                          double* energy, void* cuda_stream);

/* Real-space Ewald forces, the negative gradient of Eq. 11 (Section 5; no
 * formula in the paper, the derivative written out):
 *   F_i = q_i sum_j q_j (erfc(alpha d)/d + 2 alpha/sqrt(pi) exp(-alpha^2 d^2)) (r_i - r_j + n L) / d^2
 * over the pairs and images with d = |r_i - r_j + n L| < rcut, by the same
 * two forms as nfft_ewald_real_space (cell list with FP32 pair terms and FP64
 * sums per ion, or all pairs in FP64).  F_dev: device, n x 3 doubles in the
 * input order; *energy gets U^R as nfft_ewald_real_space would.  Allocates
 * scratch, runs on cuda_stream and waits for it. */
int nfft_ewald_real_space_forces(int64_t n, const double* r_dev, const double* q_dev, double L, double alpha,
                                 double rcut, double* F_dev, double* energy, void* cuda_stream);

/* Wait for the plan's stream, then report (and clear) the device error flag. */
int nfft_sync(nfft_plan* plan);

/* Change the stream later calls queue on (NULL = legacy default stream). */
int nfft_set_stream(nfft_plan* plan, void* cuda_stream);

/* Set a tuning option (nfft_option).  Bins, method and subproblem size take
 * effect at the next nfft_set_points, which must follow. */
int nfft_set_option(nfft_plan* plan, int option, int64_t value);

int nfft_get_info(const nfft_plan* plan, nfft_plan_info* info);

/* With NFFT_OPT_PROFILE on: waits for the stream, then writes into
 * ms[NFFT_STAGE_COUNT] the milliseconds and into launches[NFFT_STAGE_COUNT]
 * (may be NULL) the number of timed calls accumulated per stage since the
 * last reset; reset != 0 clears the totals afterwards. */
int nfft_stage_times(nfft_plan* plan, double* ms, int64_t* launches, int reset);

/* Autotuner: with the points set, time adjoint + forward for candidate
 * layouts -- bin edges, points per subproblem, then the threads per block of
 * spreading and of interpolation, then (with NFFT_METHOD_AUTO) the sparse /
 * dense split of each (NFFT_OPT_SPARSE_POINTS and _INTERP: never, automatic,
 * or 32, 128, 512 or all points per bin) -- on synthetic values (median of
 * `reps` runs each, CUDA events) and keep the fastest.  The chosen values
 * replace the corresponding options.  Sets the points again for the winner;
 * allocates temporary buffers during the call.  *best_ms (may be NULL) gets
 * the winner's adjoint + forward milliseconds. */
int nfft_autotune(nfft_plan* plan, int reps, double* best_ms);

/* Host-only parameter rule (no device needed): the oversampled size n_t for
 * each of the d bandwidths and the number of window taps per dimension. */
int nfft_plan_params(int d, const int64_t* N, double sigma, int m, int window, int64_t* n_out, int* taps_out);

/* Host-only: how much the scaling step (Section 2, 1/c_k) amplifies
 * rounding on the oversampled grid.  With a_t(k) = c_t(0) / c_t(k_t) per
 * dimension, *rms (may be NULL) = prod_t sqrt(mean over I_N of a_t^2) and
 * *peak (may be NULL) = prod_t max a_t (at the edge of I_N).  Frequencies are
 * subsampled to at most 4097 per dimension.  FP32 errors scale with *rms. */
int nfft_deconv_amplification(int d, const int64_t* N, double sigma, int m, int window, double* rms, double* peak);

/* ---- batches ------------------------------------------------------------
 * Many independent transforms of uneven sizes (and items with several
 * right-hand sides sharing one point set), set up once and run together:
 * one sort pass over all items' points, one persistent spreading /
 * interpolation launch per group of items with the same d, taps and bin
 * shape, one cuFFT plan-many per oversampled grid size and one scaling
 * launch for all items, captured in a CUDA graph that each call replays.
 * Items keep their own parameters (Section 2); the precision is common. */
typedef struct nfft_batch nfft_batch;

typedef struct {
  int d;              /* 1, 2 or 3 */
  int64_t N[3];       /* bandwidths (first d used), even */
  int64_t M;          /* points */
  double sigma;       /* oversampling >= 1 */
  int m;              /* cut-off */
  int window;         /* nfft_window */
  int nrhs;           /* right-hand sides transformed per call (>= 1) */
} nfft_batch_item;

/* Create a batch of `count` items (allocates everything, including one grid
 * per right-hand side of every item and the cuFFT plans).  Returns
 * NFFT_ERR_UNSUPPORTED, before any device work, when the items' M add up to
 * more than INT32_MAX (the bin sort indexes all points of a batch with 32-bit
 * integers). */
int nfft_batch_create(nfft_batch** out, int count, const nfft_batch_item* items, int precision, void* cuda_stream);

int nfft_batch_destroy(nfft_batch* batch);

/* Set every item's points: x_dev is a host array of `count` device pointers
 * (item i: M_i x d_i doubles, layout of nfft_set_points).  Sorts all points in
 * one pass and waits for the stream (the pointer table is copied). */
int nfft_batch_set_points(nfft_batch* batch, const double* const* x_dev);

/* Eq. 5 for every item: f_dev and fhat_dev are host arrays of `count` device
 * pointers (item i: nrhs_i x M_i and nrhs_i x |I_N_i| complex).  One CUDA
 * graph launch: the pointer table upload, zeroing of the grids, one
 * spreading launch per item group, the batched FFTs and one scaling launch.
 * Asynchronous; the pointer arrays may be reused when the call returns. */
int nfft_batch_adjoint(nfft_batch* batch, const void* const* f_dev, void* const* fhat_dev);

/* Eq. 6 for every item (one graph launch: table upload, scaling + padding,
 * batched inverse FFTs, interpolation). */
int nfft_batch_forward(nfft_batch* batch, const void* const* fhat_dev, void* const* f_dev);

int nfft_batch_sync(nfft_batch* batch);

/* nfft_set_option for all items of the batch (NFFT_OPT_RHS_CAPACITY is not
 * available: a batch fixes each item's right-hand sides).  Layout options
 * require nfft_batch_set_points again. */
int nfft_batch_set_option(nfft_batch* batch, int option, int64_t value);

/* The autotuner of nfft_autotune for a batch (whole-batch graph timings). */
int nfft_batch_autotune(nfft_batch* batch, int reps, double* best_ms);

/* Stage times with NFFT_OPT_PROFILE on: a whole adjoint graph is booked as
 * NFFT_STAGE_SPREAD, a whole forward graph as NFFT_STAGE_INTERP. */
int nfft_batch_stage_times(nfft_batch* batch, double* ms, int64_t* launches, int reset);
/* This library's kernels launched by the batch so far, graph replays
 * included (cuFFT's own kernels and memsets not included). */
int nfft_batch_kernel_launches(const nfft_batch* batch, int64_t* count);

/* ---- learned parameter picker ---------------------------------------------
 * A small MLP, n_in -> n_hidden -> n_hidden -> n_out with ReLU, trained and
 * run by the library's own kernels: FP16 weights (used by forward and
 * backward), FP32 master weights (updated by Adam), FP32 accumulation.
 * Loss: masked mean squared error sum mask (y - t)^2 / (2 sum mask).
 * Parameters are flattened as W1 (n_hidden x n_in, row-major), b1, W2, b2,
 * W3 (n_out x n_hidden), b3.  The paper has no such component: it is the
 * parameter choice (sigma, m, window; Sections 2 and 4) made by a model. */
typedef struct nfft_mlp nfft_mlp;

#define NFFT_PICKER_FEATURES 8

int nfft_mlp_create(nfft_mlp** out, int n_in, int n_hidden, int n_out, uint64_t seed, void* cuda_stream);
int nfft_mlp_destroy(nfft_mlp* mlp);
int nfft_mlp_num_params(const nfft_mlp* mlp, int64_t* n);
/* Host FP32 parameters in / out (set_params also refreshes the FP16 copy and
 * resets the Adam state; get_params with fp16_copy != 0 returns the FP16
 * weights the kernels use, widened to float). */
int nfft_mlp_set_params(nfft_mlp* mlp, const float* host);
int nfft_mlp_get_params(nfft_mlp* mlp, float* host, int fp16_copy);
/* y_dev (B x n_out) = network(x_dev (B x n_in)), device float arrays. */
int nfft_mlp_forward(nfft_mlp* mlp, const float* x_dev, float* y_dev, int B);
/* Gradient of the masked loss with respect to all parameters (FP32, device,
 * n_params) and the loss (host float, may be NULL); no update. */
int nfft_mlp_gradients(nfft_mlp* mlp, const float* x_dev, const float* t_dev, const float* mask_dev, int B,
                       float* grad_dev, float* loss_host);
/* One Adam step (beta 0.9 / 0.999) on a minibatch; loss_dev (device float,
 * may be NULL) gets the minibatch loss before the step. */
int nfft_mlp_train_step(nfft_mlp* mlp, const float* x_dev, const float* t_dev, const float* mask_dev, int B, float lr,
                        float* loss_dev);

/* Picker features of a problem: d, log2 N_0, log2 N_1, log2 N_2 (0 if
 * unused), log10 M, cluster std (0 = uniform), log10 eps, log10(M / |I_N|). */
int nfft_picker_features(int d, const int64_t* N, int64_t M, double cluster_std, double eps, double* features8);
/* Attach the candidate table and the normalisation the network was trained
 * with: n_out = 2 n_candidates; output c is the normalised predicted
 * log10(error / eps) of candidate c, output n_candidates + c its normalised
 * log10(cost); denormalised output = y * out_std + out_mean, normalised
 * feature = (f - feat_mean) / feat_std.  A candidate qualifies when its
 * predicted error is at most eps * err_margin (0 < err_margin <= 1).  The
 * network predicts the window's error (FP64 runs); for the FP32 form a
 * candidate must also have fp32_floor * (nfft_deconv_amplification rms) at
 * most eps * err_margin: the rounding of the FP32 grid stage, amplified by
 * the scaling step. */
int nfft_picker_configure(nfft_mlp* mlp, int n_candidates, const double* cand_sigma, const int* cand_m,
                          const int* cand_window, const double* feat_mean, const double* feat_std,
                          const double* out_mean, const double* out_std, double err_margin, double fp32_floor);
/* The plain rule: Kaiser-Bessel, sigma = 2, m = ceil(ln(1/eps) / (2 pi sqrt(1 - 1/sigma))) in [2, 12]. */
int nfft_rule_of_thumb(double eps, double* sigma, int* m, int* window);
/* Choose (sigma, m, window) for a problem solved in `precision`
 * (nfft_precision): the candidate with the lowest predicted cost among those
 * valid for N and predicted to reach eps (see nfft_picker_configure); the
 * rule of thumb (used_fallback = 1) when none qualifies or mlp is NULL or not
 * configured.  Runs one forward pass on the device and waits. */
int nfft_pick_params(nfft_mlp* mlp, int d, const int64_t* N, int64_t M, double cluster_std, double eps,
                     int precision, double* sigma, int* m, int* window, int* used_fallback);

/* Human-readable name of a status code (static string). */
const char* nfft_status_string(int status);

/* Library version, major * 10000 + minor * 100 + patch. */
int nfft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBNFFT_H */
