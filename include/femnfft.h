/*
 * femnfft.h - C ABI of the GB300 (sm_103a) FEM-NFFT fast summation.
 *
 * The library evaluates, for N targets x_i and M sources y_j with charges q_j,
 *
 *     phi(x_i) = sum_{j : y_j != x_i} q_j G(x_i - y_j),   G(d) = -(1/2 pi) log|d|,
 *     H(x_i)   = -grad phi(x_i),
 *
 * the discretised Green convolution of Eq. (2) of Kritsikis, Toussaint and
 * Fruchart, "Fast computation of magnetostatic fields by Non-uniform Fast
 * Fourier Transforms" (Eq. (1) with G the 2D Green function), by the NFFT
 * fast summation the paper describes after Eq. (2): the charges are spread
 * onto an oversampled regular grid with a smooth localised window, the grid
 * is Fourier transformed, divided by the window's Fourier coefficients and
 * multiplied by the coefficients b_l of the log kernel smoothed near the
 * origin, transformed back and interpolated at the targets, and a near-field
 * correction is added for pairs inside the smoothing radius eps_I.
 *
 * Conventions shared by every entry point:
 *  - Pointers marked [device] are CUDA device pointers on the device that is
 *    current when the plan is created; [host] pointers are host memory.
 *  - Point arrays are interleaved (x, y) pairs, row-major: point k at [2k, 2k+1].
 *  - The caller owns every buffer it passes; the plan owns its workspace
 *    (grids, sorted copies, coefficient tables) until fs_plan_destroy.
 *  - Compute calls are enqueued on the plan's stream (fs_opts.stream) and
 *    return before the work finishes, unless stated otherwise.  FP32 plans
 *    (2D and 3D) also own a second, non-blocking stream: the near field of
 *    fs_eval_field / fs_eval_potential / fs3_eval_field and of fs_adjoint runs
 *    there beside the spreading and the transform, forked from and joined back
 *    into the plan's stream with events, so every call still completes, as
 *    seen from the plan's stream, in the order it was made (FS_FLAG_SERIAL
 *    turns this off for 2D plans).
 *  - No call exits or aborts the process.  On failure a call returns a
 *    non-zero fs_status and fs_last_error() describes it; the plan stays
 *    valid for fs_plan_destroy.  Errors raised by kernels (points outside
 *    the admissible radius) are reported by fs_sync_status.
 *  - Radii eps_I and eps_B are in torus units: the plan scales all points by
 *    s = (1/4 - eps_B/2) / R_max (R_max = largest |point|, points centred at
 *    the origin) onto the torus [-1/2, 1/2)^2; results are returned in the
 *    caller's (physical) units.
 */
#ifndef FEMNFFT_H
#define FEMNFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fs_plan fs_plan;

typedef enum {
    FS_OK = 0,
    FS_EINVAL = 1,        /* invalid argument (null pointer, size, parameter range) */
    FS_EDOMAIN = 2,       /* a point fell outside the admissible region */
    FS_ENOMEM = 3,        /* device or host allocation failed */
    FS_ECUDA = 4,         /* a CUDA runtime call failed */
    FS_ETIMEOUT = 5,      /* a bounded device wait gave up */
    FS_EUNSUPPORTED = 6   /* valid request this build does not implement */
} fs_status;

typedef enum { FS_F32 = 32, FS_F64 = 64 } fs_dtype;

/* Option flags (fs_opts.flags). */
#define FS_FLAG_NO_KAHAN 1u   /* FP32 path: plain (uncompensated) grid accumulation */
#define FS_FLAG_TIMING 2u     /* record per-stage CUDA events (see fs_stage_times) */
#define FS_FLAG_AUTOTUNE 4u   /* fs_batch_create: choose cell and tile_cells per instance class
                                 by timing candidate plans */
#define FS_FLAG_SERIAL 8u     /* FP32 plans: run the near field on the plan's stream after the
                                 interpolation instead of on a second stream beside spreading
                                 and the transform (slower; stage times then do not overlap) */
#define FS_FLAG_SPREAD_DIRECT 16u  /* 2D plans: spread every tap straight into the grid with global
                                      atomics (FP32: with a compensation plane) instead of through
                                      shared-memory tiles */
#define FS_FLAG_SPREAD_TILES 32u   /* 2D plans: use the shared-memory tiles (the default: on
                                      GB300 they were faster at every density measured, 1.4 to
                                      over 700 sources per occupied tile; fs_info.spread_direct
                                      reports the mode a plan uses) */

/* Plan options.  A zeroed struct (or NULL) selects every default. */
typedef struct {
    int precision;    /* 32 (default) or 64: arithmetic of spread, FFT, multiply,
                         interpolation and near field.  Coefficients b_l are always
                         computed in FP64. */
    int p;            /* smoothness degree of the regularised kernel;
                         0 -> max(2, round(n_grid * eps_I)) */
    double eps_B;     /* width of the torus-boundary smoothing zone; 0 -> eps_I */
    int cell;         /* near-field cell edge in oversampled-grid cells;
                         0 -> ceil(eps_I * n_os) (cells never narrower than eps_I) */
    int tile_cells;   /* spreading tile edge in near-field cells; 0 -> about 16 grid cells */
    unsigned flags;   /* FS_FLAG_* */
    void *stream;     /* cudaStream_t for every enqueued call; NULL = default stream */
} fs_opts;

/* Read-only plan facts (fs_plan_info). */
typedef struct {
    int64_t n_src, n_tgt;     /* M, N */
    int n_grid, n_os, m, p;   /* n, sigma*n, window half-width, smoothness degree */
    int precision;            /* 32 or 64 */
    double eps_I, eps_B;      /* torus units */
    double scale;             /* s: torus coordinate = s * physical coordinate */
    int window_lo, window_n;  /* active oversampled window [lo, lo+window_n)^2 */
    int cell, cells_per_dim;  /* near-field cells */
    int tile_cells, spread_items;
    int64_t near_pairs;       /* candidate-filtered pairs with r < eps_I (counted at plan time) */
    int64_t near_pairs_fp64;  /* of those, pairs with r < eps_I/8 (FP32 path: difference refined
                                 from the hi and lo parts of the positions) */
    int64_t workspace_bytes;
    int is_fem;               /* plan built by fs_plan_create_fem */
    int64_t n_nodes, n_tris, n_bedges;
    int spread_direct;        /* 1: the plan spreads with global atomics (FS_FLAG_SPREAD_DIRECT or
                                 too few sources per tile), 0: shared-memory tiles */
} fs_info;

/*
 * Create a plan for the fast summation from M sources to N targets.
 *
 * Method: NFFT fast summation (paper, paragraph after Eq. (2)): frequencies
 * l in I_n = {-n/2..n/2-1}^2, oversampled grid n_os = sigma_os * n_grid per
 * dimension, Kaiser-Bessel window of half-width m_window grid cells (support
 * |x| < m_window), near-field radius eps_I.  Binning (cell sort of sources and
 * targets), the FP64 coefficients b_l of the regularised kernel and the
 * deconvolution table are computed here, on the device.
 *
 *  src_xy  [device] (M, 2) float64 source positions
 *  tgt_xy  [device] (N, 2) float64 target positions (may equal src_xy)
 *  n_grid  even power of two, 8..2048
 *  sigma_os oversampling; n_os = sigma_os * n_grid must be a power of two, > n_grid, <= 4096
 *  m_window 2..8, and m_window < n_os / 4
 *  eps_I   0 < eps_I < 1/4, torus units
 *  opts    NULL for defaults
 *  out     receives the plan
 * Returns FS_EINVAL on a bad argument, FS_ENOMEM, FS_ECUDA.  Synchronises the
 * plan's stream (it reads the binning counts back to the host).
 */
fs_status fs_plan_create(const double *src_xy, int64_t M, const double *tgt_xy, int64_t N,
                         int n_grid, double sigma_os, int m_window, double eps_I,
                         const fs_opts *opts, fs_plan **out);

/*
 * Create a plan for a P1 triangle mesh (paper, Eq. (2) with the quadrature of
 * Eq. (1)): targets are the Nv mesh nodes; sources are the quadrature points,
 * in this order: 3 points per triangle at barycentric (2/3,1/6,1/6) and its
 * permutations (triangle-major), then 2 Gauss-Legendre points
 * t = 1/2 -+ 1/(2 sqrt 3) per boundary edge (edges used by one triangle only,
 * sorted by (lower node index, higher node index), the first point nearer the
 * lower index).
 *
 *  nodes [device] (Nv, 2) float64;  tris [device] (Nt, 3) int32 node indices
 *  Other arguments as fs_plan_create.
 */
fs_status fs_plan_create_fem(const double *nodes, int64_t Nv, const int32_t *tris, int64_t Nt,
                             int n_grid, double sigma_os, int m_window, double eps_I,
                             const fs_opts *opts, fs_plan **out);

/*
 * Set nrhs charge vectors q [device] (nrhs, M) of dtype FS_F32 or FS_F64
 * (converted to the plan's precision and permuted into cell order).
 * The values are copied; q may be reused once the stream reaches this call.
 */
fs_status fs_set_charges(fs_plan *plan, const void *q, fs_dtype dtype, int nrhs);

/*
 * FEM plans only: charges from nodal magnetisation (kernel (a), Eq. (2)):
 * rho_T = -div M constant per P1 triangle, q = rho_T |T| / 3 per triangle
 * point; sigma = M(t).n_e along boundary edges (outward unit normal, M linear
 * along the edge), q = sigma |e| / 2 per edge point.  The charges are computed
 * (in FP64) straight into the plan's cell order in one kernel, so a time loop
 * (one plan, a new M every step) costs one pass over the sources per step.
 * The first call (or one with more vectors than before) allocates the plan's
 * charge storage.
 *  mag [device] (nrhs, Nv, 2) float64, 16-byte aligned.
 */
fs_status fs_set_magnetization(fs_plan *plan, const double *mag, int nrhs);

/*
 * FEM plans only: the same as fs_set_magnetization, but the call allocates no
 * memory at all.  The paper has no counterpart; this exists for callers that
 * must not call cudaMalloc: code that runs while a CUDA stream capture is
 * active (allocation is not permitted there), code that works inside a fixed
 * memory budget or an external arena, and time-stepping loops that must not
 * stall on the allocator every step.
 *
 * It passes through intermediate charges in source order (nrhs x M doubles, as
 * fs_fem_charges writes them); these live in one static device array of 2^19
 * doubles (4 MiB) inside the library.  Every GPU that loads the library
 * holds that array until the process exits.
 *  - nrhs * M above 524288 is rejected with FS_EINVAL.
 *  - The plan's charge storage must already hold nrhs vectors, reserved by an
 *    earlier fs_set_charges or fs_set_magnetization call with at least nrhs
 *    vectors; otherwise FS_EINVAL (this call will not allocate it).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is cached per device and per CUDA context: after
 *    cudaDeviceReset (or under another context) the next call looks it up
 *    again, so that call too should come before any stream capture.
 *  - All calls share the one array and each call overwrites every element it
 *    reads, so nothing needs clearing; but calls that overlap on the GPU (on
 *    other streams, or for other plans on the same device) race on it, so the
 *    caller must serialise them.
 *  mag [device] (nrhs, Nv, 2) float64, 16-byte aligned.
 */
fs_status fs_set_magnetization_static(fs_plan *plan, const double *mag, int nrhs);

/* FEM plans only: kernel (a) alone, charges written in source order.
 *  mag [device] (nrhs, Nv, 2) float64;  q_out [device] (nrhs, M) float64. */
fs_status fs_fem_charges(fs_plan *plan, const double *mag, double *q_out, int nrhs);

/* FEM plans only: the quadrature points [device] (M, 2) float64, in source order. */
fs_status fs_fem_sources(fs_plan *plan, double *src_out);

/*
 * Evaluate phi at the targets for every charge vector set last.
 *  phi [device] (nrhs, N) of dtype FS_F32 or FS_F64.
 */
fs_status fs_eval_potential(fs_plan *plan, void *phi, fs_dtype dtype);

/*
 * Evaluate H = -grad phi (and phi, unless phi is NULL) in one pass.
 *  phi [device] (nrhs, N) or NULL;  H [device] (nrhs, N, 2); dtype FS_F32|FS_F64.
 */
fs_status fs_eval_field(fs_plan *plan, void *phi, void *H, fs_dtype dtype);

/*
 * End-to-end solve from host memory: copies q [host] (nrhs, M) to the device,
 * sets the charges, evaluates phi and H and copies them back to phi [host]
 * (nrhs, N) (may be NULL) and H [host] (nrhs, N, 2).  Blocking: returns after
 * the results are in host memory.  Page-locked host buffers make the copies
 * asynchronous DMA transfers.
 */
fs_status fs_solve_host(fs_plan *plan, const void *q, fs_dtype q_dtype, int nrhs,
                        void *phi, void *H, fs_dtype out_dtype);

/*
 * Adjoint: gradients of a loss L(phi, H) through the fast summation, for every charge
 * vector set last (the paper has no adjoint; it is the transpose of the steps above).
 * With gphi = dL/dphi and gH = dL/dH and
 *     A(y) = sum_i gphi_i G(x_i - y) - sum_i gH_i . grad G(x_i - y),
 *   dq   = dL/dq_j   = A(y_j)                          (the transposed fast summation:
 *                                                       spread gphi, gH at the targets with the
 *                                                       window and its slope, same spectral
 *                                                       multiply, interpolate at the sources)
 *   dsrc = dL/dy_j   = q_j grad A(y_j)
 *   dtgt = dL/dx_i   = -gphi_i H(x_i) - Hess phi(x_i) gH_i   (the forward grid is recomputed and
 *                                                       interpolated with the window's curvature)
 * The torus scale s is held fixed (gradients through R_max are not taken).
 *  g_phi [device] (nrhs, N) or NULL (zero);  g_H [device] (nrhs, N, 2) or NULL (zero);
 *  in_dtype FS_F32|FS_F64 for both; dq (nrhs, M), dsrc (nrhs, M, 2), dtgt (nrhs, N, 2) [device]
 *  of out_dtype, each may be NULL (not computed).  The first call allocates the adjoint
 *  workspace.
 */
fs_status fs_adjoint(fs_plan *plan, const void *g_phi, const void *g_H, fs_dtype in_dtype, void *dq,
                     void *dsrc, void *dtgt, fs_dtype out_dtype);

/* Wait for the plan's stream and report device-side errors (FS_EDOMAIN, FS_ETIMEOUT). */
fs_status fs_sync_status(fs_plan *plan);

/* Copy the plan's facts into *info (host). */
fs_status fs_plan_info(const fs_plan *plan, fs_info *info);

/*
 * With FS_FLAG_TIMING: milliseconds of each stage of the last evaluation,
 * measured with CUDA events on the plan's stream.  Stage order: 0 charges,
 * 1 spread, 2 fft rows fwd, 3 fft cols + multiply, 4 fft rows inv,
 * 5 interpolate, 6 near field, 7 unpermute.  FP32 plans without FS_FLAG_SERIAL
 * run the near field on a second stream beside stages 1-4 (stage 6 is its own
 * duration there) and write the output in the interpolation kernel (stage 5
 * includes it; stage 7 is empty).  Synchronises the stream.
 * count = number of doubles available in ms (8 or more).
 */
fs_status fs_stage_times(fs_plan *plan, double *ms, int count);

/* Release the plan and its workspace (synchronises its stream first). */
fs_status fs_plan_destroy(fs_plan *plan);

/*
 * Batched solves.  The paper has no counterpart: it solves one problem at a time.
 * A batch holds `count` independent instances (own points, grid size n_grid and
 * radius eps_I; shared sigma_os, m_window, precision and smoothness degree p) and
 * nrhs charge vectors per instance, and evaluates all of them with one launch per
 * stage (charges, spreading, FFT + multiply, interpolation, near field, output)
 * over all (instance, right-hand side, work unit) items, replayed as one CUDA
 * graph.  The FFT stage is one persistent launch whose blocks wait on each other
 * through counters; those waits are bounded and a wait that gives up sets an
 * error word reported by fs_batch_sync_status as FS_ETIMEOUT.
 */
typedef struct fs_batch fs_batch;

typedef struct {
    const double *src_xy;   /* [device] (M, 2) float64 */
    int64_t M;
    const double *tgt_xy;   /* [device] (N, 2) float64, may equal src_xy */
    int64_t N;
    int n_grid;             /* as fs_plan_create */
    double eps_I;           /* as fs_plan_create */
} fs_instance;

typedef struct {
    int count, nrhs, precision;
    int64_t total_src, total_tgt;
    int spread_items;       /* spreading work items over all instances (x nrhs per launch) */
    int fft_units;          /* row pairs + columns + inverse row pairs, all instances and rhs */
    int fft_blocks;         /* persistent blocks of the FFT launch */
    int64_t near_items;     /* FP32 near-field warp items over all instances */
    int64_t workspace_bytes;
} fs_batch_facts;

/*
 * Create a batch.  Every instance is planned as by fs_plan_create (its plan is
 * reachable through fs_batch_plan); opts applies to all (opts.cell and
 * opts.tile_cells, if set, to every instance).  With FS_FLAG_AUTOTUNE (and cell,
 * tile_cells left 0) each class of instances - same n_grid, m, sigma, p,
 * precision and rounded log2 of N and of M - gets the near-field cell (1, 1.5 or
 * 2 times the narrowest) and spreading tile (about 16, 32 or 64 grid lines, if its
 * shared-memory tile stays within 56 KB so that four spreading CTAs fit per SM)
 * that evaluated fastest on the class's first instance; choices are cached for
 * the process.
 *  inst   [host] count descriptors; the point arrays are read during the call only
 *  nrhs   1..4 charge vectors per instance
 * Returns FS_EINVAL (bad argument; instances with different p), FS_ENOMEM, FS_ECUDA.
 * With opts.stream NULL the batch creates its own blocking stream (the legacy
 * default stream cannot be captured into a graph).  Synchronising.
 */
fs_status fs_batch_create(const fs_instance *inst, int count, double sigma_os, int m_window, int nrhs,
                          const fs_opts *opts, fs_batch **out);

/*
 * Evaluate phi and H of every instance and charge vector.
 *  q   [host] array of count [device] pointers, instance i: (nrhs, M_i) of q_dtype
 *  phi [host] array of count [device] pointers (nrhs, N_i), or NULL (no potential);
 *      individual entries may be NULL
 *  H   [host] array of count [device] pointers (nrhs, N_i, 2), or NULL; entries may be NULL
 * The pointer arrays are read during the call; the first evaluation with a given
 * (q_dtype, out_dtype) captures and instantiates the graph, later ones replay it.
 * Enqueued on the batch's stream; device-side failures are reported by
 * fs_batch_sync_status.
 */
fs_status fs_batch_eval(fs_batch *batch, const void *const *q, fs_dtype q_dtype, void *const *phi,
                        void *const *H, fs_dtype out_dtype);

/* Wait for the batch's stream; FS_ETIMEOUT if a bounded device wait gave up since the last call. */
fs_status fs_batch_sync_status(fs_batch *batch);

/* Batch facts (host). */
fs_status fs_batch_info(const fs_batch *batch, fs_batch_facts *info);

/*
 * The plan of instance i (owned by the batch; valid until fs_batch_destroy).  It
 * accepts every fs_* plan call (fs_plan_info shows the chosen cell and tile;
 * fs_set_charges + fs_eval_field solve the instance on its own) on the batch's
 * stream; do not destroy it.
 */
fs_status fs_batch_plan(fs_batch *batch, int i, fs_plan **out);

/* Release the batch, its plans and graphs (synchronises its stream first). */
fs_status fs_batch_destroy(fs_batch *batch);

/*
 * Runs one bounded device wait (the wait of the batched FFT) on a counter that
 * nothing increments, giving up after `spins` polls of about 0.1 us.  Returns
 * FS_ETIMEOUT when the wait gave up and recorded it - the expected outcome - and
 * leaves the CUDA context usable.  The paper has no counterpart; it exists to
 * check the timeout path without a fault.
 */
fs_status fs_wait_selftest(int spins);

/*
 * Arithmetic throughput of the current device, measured: the denominators of the roofline
 * fractions of this library's ALU-bound kernels (near field, spreading, interpolation).
 * The paper has no counterpart.  A grid of 4 blocks x 256 threads per SM runs `iters`
 * steps of 8 independent chains per thread of one operation:
 *   FS_PROBE_FFMA   scalar FP32 fma, counted as 2 flop per lane
 *   FS_PROBE_FFMA2  packed two-wide FP32 fma, counted as 4 flop per lane
 *   FS_PROBE_MUFU   MUFU reciprocal and base-2 logarithm (rcp.approx, lg2.approx on alternate
 *                   chains, each followed by an add), counted as 1 op per lane
 * One warm-up launch, then `reps` launches timed with CUDA events on a private stream.
 *  ops_per_s      [host] out: flop/s (or MUFU op/s) over the timed launches
 *  ms_per_launch  [host] out: mean launch duration
 * Allocates and frees a small scratch buffer; synchronising.  FS_EINVAL for an unknown
 * mode or iters, reps < 1.
 */
#define FS_PROBE_FFMA 0
#define FS_PROBE_FFMA2 1
#define FS_PROBE_MUFU 2
fs_status fs_probe_throughput(int mode, int iters, int reps, double *ops_per_s, double *ms_per_launch);

/*
 * The 3D kernel G(r) = 1/(4 pi r): the paper names it (with tetrahedral P1 elements) as
 * the next step, with the same pipeline in three dimensions.  A 3D plan evaluates
 *
 *     phi(x_i) = sum_{j : y_j != x_i} q_j / (4 pi |x_i - y_j|),   H = -grad phi,
 *
 * for points in R^3: frequencies l in I_n^3, an oversampled n_os^3 grid (only the
 * active window cube around the scaled points is stored), the Kaiser-Bessel window in
 * each coordinate, 1/r smoothed inside eps_I by the even polynomial T_I and flattened
 * near |x| = 1/2 of the torus cube, and the near-field correction for pairs closer than
 * eps_I (cells at least eps_I wide, the 27 around a target's).  The points are scaled by
 * s = (1/4 - eps_B/2) / R_max; results are returned in physical units (phi = s phi~,
 * H = -s^2 grad~ phi~).  Conventions as for the 2D plan; points are (x, y, z) triples.
 */
typedef struct fs3_plan fs3_plan;

/*
 *  src_xyz [device] (M, 3) float64;  tgt_xyz [device] (N, 3) float64 (may equal src_xyz)
 *  n_grid  power of two in [4, 256];  sigma_os: n_os = sigma_os * n_grid a power of two in
 *          (n_grid, 512];  m_window in [2, 5], below n_os / 4;  eps_I in (0, 1/4) torus units
 *  opts    precision (32 | 64), p, eps_B, stream as for fs_plan_create; other fields ignored
 * Returns FS_EINVAL, FS_EDOMAIN (a point beyond the admissible radius), FS_ENOMEM,
 * FS_ECUDA.  Synchronising.
 */
fs_status fs3_plan_create(const double *src_xyz, int64_t M, const double *tgt_xyz, int64_t N, int n_grid,
                          double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs3_plan **out);

/*
 * Create a plan for a P1 tetrahedral mesh: the charge quadrature of Eq. (2) with d = 3
 * (the paper's next step; the 3D rule is this library's reading).  Targets are the Nv
 * nodes; sources are the quadrature points, in this order: 4 points per tetrahedron at
 * barycentric (a, b, b, b) and its permutations, a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20
 * (tetrahedron-major, the weight a on its node 0, 1, 2, 3 in turn), then 3 points per
 * boundary face at barycentric (2/3, 1/6, 1/6) and permutations (faces used by one
 * tetrahedron only, sorted by their ascending node triple i0 < i1 < i2, the weight 2/3 on
 * i0, i1, i2 in turn).  Tetrahedra of either orientation are accepted.
 *
 *  nodes [device] (Nv, 3) float64, kept by reference: it must outlive the plan
 *  tets  [device] (Nt, 4) int32 node indices (copied)
 *  Other arguments as fs3_plan_create.  FS_EINVAL for an index out of range, a repeated
 *  node, a face shared by more than two tetrahedra, or more than 2^31 - 1 sources.
 */
fs_status fs3_plan_create_fem(const double *nodes, int64_t Nv, const int32_t *tets, int64_t Nt, int n_grid,
                              double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs3_plan **out);

/*
 * Tetrahedral plans only: charges from the nodal magnetisation, computed in FP64 straight
 * into the plan's cell order: rho_T = -div M constant per P1 tetrahedron, q = rho_T |T| / 4
 * per tetrahedron point; sigma = M.n_F on boundary faces (outward unit normal, M linear on
 * the face), q = sigma |F| / 3 per face point.
 *  mag [device] (nrhs, Nv, 3) float64.
 */
fs_status fs3_set_magnetization(fs3_plan *plan, const double *mag, int nrhs);

/* Tetrahedral plans only: the assembly alone, in source order.
 *  mag [device] (nrhs, Nv, 3) float64;  q_out [device] (nrhs, M) float64. */
fs_status fs3_fem_charges(fs3_plan *plan, const double *mag, double *q_out, int nrhs);

/* Tetrahedral plans only: the quadrature points [device] (M, 3) float64, in source order. */
fs_status fs3_fem_sources(fs3_plan *plan, double *src_out);

/* nrhs charge vectors q [device] (nrhs, M) of dtype FS_F32 or FS_F64 (copied). */
fs_status fs3_set_charges(fs3_plan *plan, const void *q, fs_dtype dtype, int nrhs);

/* phi [device] (nrhs, N) or NULL;  H [device] (nrhs, N, 3) or NULL (not both);  FS_F32|FS_F64. */
fs_status fs3_eval_field(fs3_plan *plan, void *phi, void *H, fs_dtype dtype);

/* Wait for the plan's stream. */
fs_status fs3_sync_status(fs3_plan *plan);

/* The plan's facts (fields of the 2D plan that have no 3D meaning are zero; for a
 * tetrahedral plan n_nodes, n_tris and n_bedges count nodes, tetrahedra and boundary
 * faces).  spread_items counts the FP32 spreading's shared-memory tile items: 0 when the
 * plan spreads straight into the grid with atomics (its occupied cells hold fewer than
 * about 300 sources on average, or the tiles do not fit in shared memory). */
fs_status fs3_plan_info(const fs3_plan *plan, fs_info *info);

/* Release the plan (synchronises its stream first). */
fs_status fs3_plan_destroy(fs3_plan *plan);

/* Message for the last failing call on this host thread ("" if none). */
const char *fs_last_error(void);

/* Library version string. */
const char *fs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FEMNFFT_H */
