// Launch wrappers of the FEM-NFFT kernels; each is defined in the .cu file that holds its kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace fs {

// Warps per spreading CTA; each holds a private padded tile in shared memory.
constexpr int kSpreadWarps = 4;

// Shared memory of the spreading kernels: the warp tiles (PLANES planes of P rows at pitch Q),
// padded to 16 bytes, then each warp's window weights (a group's row weights vector-aligned,
// then the column weights), then the FP32 window polynomials.
template <typename real> __host__ __device__ constexpr int spread_weight_stride(int M2)
{
    const int G = spread_groups(M2), RPL = M2 / G, VW = 16 / (int)sizeof(real);
    return G * ((RPL + VW - 1) / VW * VW) + (M2 + VW - 1) / VW * VW;
}

template <typename real> __host__ __device__ inline size_t spread_tiles_bytes(int P, int Q, int planes)
{
    return ((size_t)kSpreadWarps * P * Q * planes * sizeof(real) + 15) / 16 * 16;
}

template <typename real> inline size_t spread_smem_bytes(int P, int M2, bool comp)   // k_spread, k_batch_spread
{
    return spread_tiles_bytes<real>(P, spread_group_pitch(P, M2), comp ? 2 : 1) +
           (size_t)kSpreadWarps * spread_weight_stride<real>(M2) * sizeof(real) + sizeof(float) * M2 * (kPolyD + 1);
}

// One spreading work unit: sources [start, start+count) of tile `tile` (cell-sorted order).
struct SpreadItem {
    int tile;
    int start;
    int count;
    int pad;
};

// Regularised-kernel description for the b_l samples and the near field (FP64, host-filled).
struct KernelParams {
    double eps_I;
    double eps_B;
    int p;
    int dim;               // 3: k(r) = 1/(4 pi r); otherwise k(r) = -(1/2 pi) log r
    double beta[kMaxP];    // T_I(r) = sum_k beta_k (r/eps_I)^(2k)
    double tb_f0[kMaxP];   // eps_B^j k^(j)(1/2 - eps_B) / j!   (two-point Taylor data at the left end)
    double tb_binom[kMaxP];// C(p-1+i, i)
    double k_half;         // k(1/2)
};

// Near-field constants in the arithmetic precision.
template <typename real> struct NearParams {
    real eps2;             // eps_I^2
    real inv_eps2;
    real close2;           // (eps_I/8)^2: closer pairs refine their coordinate difference
    real hcell;            // cell width in torus units (FP32 positions are relative to cell corners)
    real beta[kMaxP];      // T_I coefficients in w = (r/eps_I)^2
    real dbeta[kMaxP];     // coefficients of T_I'(r)/r in w: 2k beta_k / eps_I^2 (index k-1)
    real pbeta[kMaxP];     // P(w) = T_I - k(eps_I): beta with beta_0 - k(eps_I), so P(1) = 0
    real nptilde[kMaxP];   // -Ptilde(w) with P(w) = (w - 1) Ptilde(w): degree p - 2 (index < p - 1)
    real rcoef;            // (-1)^p / (2 pi eps_I^2): (k' - T_I')(r)/r = rcoef (w - 1)^(p-1) / w
    int p;
};

// ---- 3D kernel 1/(4 pi r) (kernels3d.cu; transform and coefficients in kernels_fft.cu)

// Near-field cells of the 3D path: n_c^3 cubes of `cell` grid lines, cell key
// (c1 n_c + c2) n_c + c3.  Points are sorted by cell and, inside a cell, by sub-cell (sub^3
// cubes, Morton order): sort key = cell key x sub^3 + Morton index, so the points of cell K
// occupy the sorted range [start[K sub^3], start[(K + 1) sub^3]).
struct CellGrid3 {
    int cell;
    int n_c;
    int sub;   // sub-cells per cell edge: 1, 2 or 4
    __host__ __device__ int key(int c1, int c2, int c3) const { return (c1 * n_c + c2) * n_c + c3; }
    __host__ __device__ int n_cells() const { return n_c * n_c * n_c; }
    __host__ __device__ int sub3() const { return sub * sub * sub; }
    __host__ __device__ int n_keys() const { return n_cells() * sub3(); }
};

// FP32 3D near field (distances in units of eps_I, w = |d|^2 / eps_I^2):
//   f(w)       = c1 w^(-1/2) - P(w),             c1 = 1 / (4 pi eps_I), P(w) = T_I = sum beta_k w^k
//   grad_x f   = -(1/eps_I) (c1 w^(-3/2) + 2 P'(w)) d,   d in units of eps_I
struct Near3Params {
    float H;               // cell edge / eps_I (>= 1)
    float reach2;          // squared culling radius, 1 plus a rounding margin
    float close_reach2;    // squared radius of the close list, 1/8 plus a rounding margin
    double inv_eps_d;      // 1 / eps_I, for the FP64 differences of close pairs
    float c1;              // 1 / (4 pi eps_I)
    float inv_eps;         // 1 / eps_I
    float beta0;           // T_I(0), removed for coincident pairs (G(0) := 0)
    float nbeta[kMaxP];    // -beta_k
    float dbeta2[kMaxP];   // 2 P'(w) = sum dbeta2_k w^k, dbeta2_k = 2 (k + 1) beta_{k+1}
    int p;
};

cudaError_t launch_rmax3(const double *xyz, int64_t n, unsigned long long *out, cudaStream_t st);
cudaError_t launch_point_keys3(const double *xyz, int64_t n, double s, int n_os, int window_lo, int n_a, int m,
                               CellGrid3 cg, int *key, int *count, int *status, cudaStream_t st);
// pos: torus coordinates (n x 3, FP64); frac (n x 3); base: window grid lines packed 10 bits each;
// pos32 (FP32 path, else null): offsets from the point's cell corner in units of eps_I (times inv_eps)
template <typename real>
cudaError_t launch_gather_points3(const double *xyz, const int *perm, int64_t n, double s, int n_os, int window_lo,
                                  int n_a, int m, int cell, double inv_eps, double *pos, real *frac, int *base,
                                  float4 *pos32, int *status, cudaStream_t st);
template <typename real>
cudaError_t launch_spread3(int64_t M, int m, const int *base, const real *frac, const real *q, Window<real> w,
                           const WindowPoly &wp, real *grid, int n_a, cudaStream_t st);
// FP32 spreading through warp-private shared tiles with compensation; items {first source,
// count <= kSpread3ItemMax} of one cell each.  spread3_tile_smem is 0 when the tiles do not fit.
constexpr int kSpread3ItemMax = 1024;
// A tile costs its zeroing and its flush (2 (cell + 2m - 1)^3 words) per item, against one
// global atomic per tap for direct spreading; FP32 plans take the tiles only where the cells
// that hold sources hold at least this many on average (measured on GB300: direct spreading
// wins up to ~190 sources per cell on tetrahedral meshes, tiles from ~440).
constexpr int kSpread3TileMinPerCell = 300;
size_t spread3_tile_smem(int cell, int m);
cudaError_t launch_spread3_tile(const int2 *items, int n_items, int m, int cell, const int *base, const float *frac,
                                const float *q, const WindowPoly &wp, float *grid, int n_a, cudaStream_t st);
// acc: add to phi_s / grad_s (the near field stored there first) instead of writing them
template <typename real>
cudaError_t launch_interp3(int64_t N, int m, const int *base, const real *frac, Window<real> w, const WindowPoly &wp,
                           const real *grid, int n_a, real n_os, real *phi_s, real *grad_s, bool acc,
                           cudaStream_t st);
// FP64 near field, thread per target over the 27 cells around its own
cudaError_t launch_near3_f64(int64_t N, const int *tgt_base, const double *tgt_pos, const double *src_pos,
                             const int *src_start, CellGrid3 cg, const double *q, NearParams<double> np,
                             double *phi_s, double *grad_s, cudaStream_t st);
// FP32 near field over warp items {first target, count <= 64} of one cell each (sorted order);
// coincident pairs (equal positions) are listed per target in coinc_start / coinc_src
// (pairs closer than eps_I / 8 refine their difference from the FP64 positions tgt_pos, src_pos)
// (assign: store phi_s / grad_s instead of adding, for the near field run beside the far field)
cudaError_t launch_near3_warp(const int2 *items, int n_items, const int *tgt_base, const float4 *tgt_p32,
                              const float4 *src_p32, const double *tgt_pos, const double *src_pos, const float *q,
                              const int *src_start, CellGrid3 cg, const Near3Params &np, const int *coinc_start,
                              const int *coinc_src, float *phi_s, float *grad_s, bool assign, cudaStream_t st);
// Source-major FP32 near field (many more sources than targets): items of at most 64 sources of
// one cell; phi and grad phi are added to the targets with atomics, then the coincident pairs'
// -q T_I(0) when any_coincident
cudaError_t launch_near3_src(const int2 *items, int n_items, const int *src_base, const float4 *src_p32,
                             const float4 *tgt_p32, const double *tgt_pos, const double *src_pos, const float *q,
                             const int *tgt_start, CellGrid3 cg, const Near3Params &np, int64_t N,
                             const int *coinc_start, const int *coinc_src, bool any_coincident, float *phi_s,
                             float *grad_s, cudaStream_t st);
// per target: count of sources at the same FP64 position (same cell) when coinc_src is null, or
// their sorted indices from coinc_start (coinc_src given)
cudaError_t launch_coincident3(int64_t N, const int *tgt_base, const double *tgt_pos, const double *src_pos,
                               const int *src_start, CellGrid3 cg, int *count, const int *coinc_start, int *coinc_src,
                               cudaStream_t st);
template <typename real>
cudaError_t launch_unpermute3(int64_t N, const real *phi_s, const real *grad_s, const int *perm, double s,
                              void *phi_out, void *H_out, int out_f64, cudaStream_t st);
// five-pass transform with the multiply on the n_a^3 window (spec1: n_a x (n/2+1) x n_a,
// spec2: n_a x (n/2+1) x (n+1) complex)
template <typename real>
cudaError_t launch_fft3(real *grid, int n_a, int L, int n, typename Cplx<real>::type *spec1,
                        typename Cplx<real>::type *spec2, const real *mul3, const typename Cplx<real>::type *tw,
                        cudaStream_t st);
// FP64 samples of K_R on the n^3 frequency grid, their 3D FFT (samp, tmp: n^3 each) and the
// multiplier (n/2+1) x (n+1) x (n+1) in the plan's precision
cudaError_t launch_coeffs3(double2 *samp, double2 *tmp, int n, KernelParams kp, const double2 *tw64,
                           const double *c_tab, void *mul3, int real_is_f64, cudaStream_t st);

// ---- batched solves: one launch per stage over all instances and right-hand sides

// One instance of a batch as its kernels see it (device memory, filled when the batch is
// created).  Point data, tables and twiddles belong to the instance's plan; the buffers per
// right-hand side belong to the batch (right-hand side r at offset r * stride).
template <typename real> struct BatchInst {
    int n, L, n_a, pitch, ld;
    CellGrid cg;
    int64_t M, N;
    const int *src_base, *tgt_base;
    const void *src_frac, *tgt_frac;
    const double2 *src_pos, *tgt_pos;               // FP64 positions (FP64 near field)
    const float2 *src_hi, *src_lo, *tgt_hi, *tgt_lo; // FP32 cell-relative positions
    const int *src_start, *src_perm, *tgt_perm;
    const real *mul;
    const typename Cplx<real>::type *tw;
    real *q;                                         // sorted charges, stride M
    real *grid;                                      // active window, stride grid_stride
    typename Cplx<real>::type *spec;                 // half spectrum, stride spec_stride
    real *phi_s, *grad_s, *coinc;                    // strides N, 2N, N
    double *q_sum;                                   // one per right-hand side
    int64_t grid_stride, spec_stride;
    double s, shift;
    NearParams<real> np;
};

// Caller buffers of one instance for one batched evaluation (device pointers).
struct BatchIO {
    const void *q;   // (nrhs, M)
    void *phi;       // (nrhs, N) or null
    void *H;         // (nrhs, N, 2) or null
};

// Block -> instance map of a per-point batched launch: block b belongs to instance inst[b]
// and is block b - first[inst[b]] of that instance.
struct BlockMap {
    const int *inst;
    const int *first;
};

// Work unit of the batched persistent FFT.  kind 0: forward row pair, 1: column (forward
// FFT, multiply, inverse FFT), 2: inverse row pair; index = row pair or column l1.
struct FftUnit {
    int inst, rhs, kind, index;
};

// Device-side wait budget of the persistent FFT (spins of ~0.1 us each before the wait
// gives up and records a timeout).
constexpr int kWaitSpins = 1 << 23;

template <typename real>
cudaError_t launch_batch_gather_charges(const BatchInst<real> *inst, const BatchIO *io, BlockMap bm, int blocks,
                                        int nrhs, int q_is_f64, cudaStream_t st);
template <typename real>
cudaError_t launch_batch_spread(const SpreadItem *items, int n_items, int nrhs, const BatchInst<real> *inst, int m,
                                int max_tile, Window<real> w, const WindowPoly &wp, bool kahan, cudaStream_t st);
template <typename real>
cudaError_t prepare_batch_spread(int m, int max_tile, bool kahan);
template <typename real>
cudaError_t launch_batch_interp(const BatchInst<real> *inst, BlockMap bm, int blocks, int nrhs, int m,
                                Window<real> w, const WindowPoly &wp, cudaStream_t st);
// FP32 batches: interpolation and output in one pass, after the near field stored its sums
template <typename real>
cudaError_t launch_batch_interp_out(const BatchInst<real> *inst, const BatchIO *io, BlockMap bm, int blocks, int nrhs,
                                    int m, Window<real> w, const WindowPoly &wp, int out_is_f64, cudaStream_t st);
// counters: 2 * n_inst * nrhs ints (rows done, columns done) plus the queue head, zeroed
// before each launch; err: set to 1 when a wait ran out of spins
template <typename real>
cudaError_t launch_batch_fft(const BatchInst<real> *inst, const FftUnit *units, int n_units, int n_inst, int nrhs,
                             int L_max, int grid_blocks, int *counters, int *err, int spins, cudaStream_t st);
template <typename real> cudaError_t batch_fft_blocks(int L_max, int *blocks);
// one bounded wait on a counter that nothing increments (the timeout path, for tests)
cudaError_t launch_wait_selftest(int *counter, int *err, int spins, cudaStream_t st);
// items: (first target, count <= 64, instance, 0) per warp
cudaError_t launch_batch_near32(int64_t n_items, const int4 *items, const BatchInst<float> *inst, int p, int nrhs,
                                bool assign, cudaStream_t st);
cudaError_t launch_batch_near64(const BatchInst<double> *inst, BlockMap bm, int blocks, int nrhs, cudaStream_t st);
template <typename real>
cudaError_t launch_batch_unpermute(const BatchInst<real> *inst, const BatchIO *io, BlockMap bm, int blocks, int nrhs,
                                   int out_is_f64, cudaStream_t st);

// ---- binning (kernels_bin.cu)
cudaError_t launch_rmax(const double *xy, int64_t n, unsigned long long *out, cudaStream_t st);
cudaError_t launch_point_keys(const double *xy, int64_t n, double s, int n_os, int window_lo, int n_a,
                              int m, CellGrid cg, int *key, int *count, int *status, cudaStream_t st);
cudaError_t launch_exclusive_scan(const int *count, int *start, int n, int *block_tmp, cudaStream_t st);
cudaError_t launch_scatter(const int *key, int64_t n, int *fill, int *perm, cudaStream_t st);
template <typename real>
cudaError_t launch_gather_points(const double *xy, const int *perm, int64_t n, double s, int n_os,
                                 int window_lo, int n_a, int m, int cell, double2 *pos, void *frac, int *base,
                                 float2 *pos32, float2 *pos32_lo, cudaStream_t st);
template <typename real>
cudaError_t launch_gather_charges(const void *q, int q_is_f64, const int *perm, int64_t M, int nrhs,
                                  real *q_sorted, double *q_sum, cudaStream_t st);
cudaError_t launch_near_count(const double2 *tgt_pos, const int *tgt_base, int64_t N,
                              const double2 *src_pos, const int *src_start, CellGrid cg, double eps2,
                              double close2, unsigned long long *counts, cudaStream_t st);

// ---- spreading / interpolation (kernels_spread.cu)
template <typename real>
cudaError_t launch_spread(const SpreadItem *items, int n_items, CellGrid cg, int m, const int *base,
                          const void *frac, const real *q, Window<real> w, const WindowPoly &wp, real *grid,
                          int pitch, int n_a, bool kahan, cudaStream_t st);
// direct spreading (global atomics, no tiles); comp: compensation plane of the grid's size
// (FP32 with compensation; folded into the grid at the end), may be null otherwise
template <typename real>
cudaError_t launch_spread_direct(int64_t M, int m, const int *base, const void *frac, const real *q, Window<real> w,
                                 const WindowPoly &wp, real *grid, real *comp, int pitch, int n_a, bool kahan,
                                 cudaStream_t st);
template <typename real>
// acc: add to phi_s / grad_s (the near field already stored there) instead of writing them
cudaError_t launch_interp(int64_t N, int m, const int *base, const void *frac, Window<real> w,
                          const WindowPoly &wp, const real *grid, int pitch, real n_os, real *phi_s, real *grad_s,
                          bool acc, cudaStream_t st);

// Interpolation and output in one pass (plans whose near field stored phi_s / grad_s / coinc
// first): the caller's phi and H at perm[k], as launch_interp with acc followed by launch_unpermute.
template <typename real>
cudaError_t launch_interp_out(int64_t N, int m, const int *base, const void *frac, Window<real> w,
                              const WindowPoly &wp, const real *grid, int pitch, real n_os, const real *phi_s,
                              const real *grad_s, const real *coinc, const int *perm, double shift,
                              const double *q_sum, double s, void *phi_out, void *H_out, int out_is_f64,
                              cudaStream_t st);

template <typename real>
cudaError_t launch_spread_dip(const SpreadItem *items, int n_items, CellGrid cg, int m, const int *base,
                              const void *frac, const real *cq, const void *dq, Window<real> w, const WindowPoly &wp,
                              real *grid, int pitch, int n_a, bool kahan, cudaStream_t st);
template <typename real>
// (acc: add to grad_s / hess_s, where the near part was stored first)
cudaError_t launch_interp_hess(int64_t N, int m, const int *base, const void *frac, Window<real> w,
                               const WindowPoly &wp, const real *grid, int pitch, real n_os, real *grad_s,
                               real *hess_s, bool acc, cudaStream_t st);

// ---- FFT and spectral multiply (kernels_fft.cu)
// Radix of the Stockham pass that follows the first L / rest points: 8 while 8 divides the
// rest, then one pass of 4 or 2.
__host__ __device__ constexpr int fft_pass_radix(int rest) { return rest % 8 == 0 ? 8 : (rest == 4 ? 4 : 2); }
// Twiddles of a length-L transform (L a power of two, 2 L values re, im): for each pass
// (Ns points already combined, radix R) the entries Ns - 1 + (r - 1) Ns + k, r = 1..R-1,
// k = 0..Ns-1, hold exp(-2 pi i r k / (Ns R)); entry L - 1 is 1.  Computed in FP64.
template <typename real> void fft_twiddle_table(int L, real *re_im);
template <typename real>
cudaError_t launch_fft_rows_fwd(const real *grid, int pitch, int n_a, int L, int n_half,
                                typename Cplx<real>::type *spec, int ld, const typename Cplx<real>::type *tw,
                                cudaStream_t st);
template <typename real>
cudaError_t launch_fft_cols(typename Cplx<real>::type *spec, int ld, int n_a, int L, int n,
                            const real *mul, const typename Cplx<real>::type *tw, cudaStream_t st);
template <typename real>
cudaError_t launch_fft_rows_inv(const typename Cplx<real>::type *spec, int ld, int n_a, int L, int n_half,
                                real *grid, int pitch, const typename Cplx<real>::type *tw, cudaStream_t st);
cudaError_t launch_kernel_samples(double2 *samp, int n, KernelParams kp, cudaStream_t st);
cudaError_t launch_fft_lines_c64(double2 *data, int lines, int L, const double2 *tw, cudaStream_t st);
cudaError_t launch_transpose_c64(const double2 *in, double2 *out, int n, cudaStream_t st);
template <typename real>
cudaError_t launch_build_mul(const double2 *bhat, int n, const double *c_tab, real *mul, cudaStream_t st);

// ---- near field and output (kernels_near.cu)
cudaError_t launch_near64(int64_t N, const int *tgt_base, const double2 *tgt_pos, const double2 *src_pos,
                          const int *src_start, CellGrid cg, const double *q, NearParams<double> np, double *phi_s,
                          double *grad_s, double *coinc, cudaStream_t st);
// items: (first target, count <= 64) per warp, never spanning two cells
// (assign: store phi_s and grad_s instead of adding to them, for the near field that runs on a
// second stream beside spreading and the transform)
cudaError_t launch_near32(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                          const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start,
                          CellGrid cg, const float *q, NearParams<float> np, float *phi_s, float *grad_s, float *coinc,
                          bool assign, cudaStream_t st);
// source-major variant for plans with many more sources than targets: items (first source,
// count <= 64) per warp; phi_s, grad_s and coinc (zeroed by the caller) receive atomic adds
cudaError_t launch_near_src32(int64_t n_items, const int2 *items, const int *src_base, const float2 *src_hi,
                              const float2 *src_lo, const float2 *tgt_hi, const float2 *tgt_lo, const int *tgt_start,
                              CellGrid cg, const float *q, NearParams<float> np, float *phi_s, float *grad_s,
                              float *coinc, cudaStream_t st);
// plan-time pair statistics over the FP32 near-field items: counts[2 s] (r < eps_I) and
// counts[2 s + 1] (r < eps_I / 8) for s < kNearCountSlots, to be summed
constexpr int kNearCountSlots = 64;
cudaError_t launch_near_count32(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                                const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start,
                                CellGrid cg, NearParams<float> np, unsigned long long *counts, cudaStream_t st);
template <typename real>
cudaError_t launch_unpermute(int64_t N, const real *phi_s, const real *grad_s, const real *coinc,
                             const int *perm, double shift, const double *q_sum, double s, void *phi_out,
                             void *H_out, int out_is_f64, cudaStream_t st);

// ---- adjoint (kernels_adjoint.cu)
template <typename real>
cudaError_t launch_gather_adj(int64_t N, const int *perm, const void *gphi, const void *gH, int in_f64, double s,
                              double n_os, real *c, void *dn, void *df, double *gsum, cudaStream_t st);
// FP64: one thread per point over the 3 x 3 cells
cudaError_t launch_near_adj64(int64_t M, const int *src_base, const double2 *src_pos, const double2 *tgt_pos,
                              const int *tgt_start, CellGrid cg, const double *c, const void *dn,
                              NearParams<double> np, double *a_s, double *ga_s, double *cg_s, cudaStream_t st);
cudaError_t launch_near_hess64(int64_t N, const int *tgt_base, const double2 *tgt_pos, const double2 *src_pos,
                               const int *src_start, CellGrid cg, const double *q, NearParams<double> np,
                               double *grad_s, double *hess_s, cudaStream_t st);
// FP32: warp items over the sources (adjoint potential) or the targets (Hessian)
cudaError_t launch_near_adj32(int64_t n_items, const int2 *items, const int *src_base, const float2 *src_hi,
                              const float2 *src_lo, const float2 *tgt_hi, const float2 *tgt_lo, const int *tgt_start,
                              CellGrid cg, const float *c, const void *dn, NearParams<float> np, float *a_s,
                              float *ga_s, float *cg_s, bool assign, cudaStream_t st);
// (assign: store instead of adding, for the near parts run beside the spreading and transform)
cudaError_t launch_near_hess32(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                               const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start,
                               CellGrid cg, const float *q, NearParams<float> np, float *grad_s, float *hess_s,
                               bool assign, cudaStream_t st);
template <typename real>
cudaError_t launch_adj_finish_src(int64_t M, const int *perm, const real *a_s, const real *ga_s, const real *cg_s,
                                  const real *q, double shift, const double *gsum, double s, void *dq, void *dy,
                                  int out_f64, cudaStream_t st);
template <typename real>
cudaError_t launch_adj_finish_tgt(int64_t N, const int *perm, const real *grad_s, const real *hess_s, const real *c,
                                  const void *dn, double s, void *dx, int out_f64, cudaStream_t st);

// ---- FEM charge assembly (kernels_fem.cu)
cudaError_t launch_fem_sources(const double2 *nodes, const int *tris, int64_t Nt, const int *bedges,
                               int64_t Ne, double2 *src, cudaStream_t st);
cudaError_t launch_fem_charges(const double2 *nodes, const int *tris, int64_t Nt, const int *bedges,
                               int64_t Ne, const double2 *mag, int64_t Nv, int nrhs, double *q,
                               int64_t M, cudaStream_t st);
// charges straight into cell order (q_sorted, stride M per rhs; inv_perm: source -> sorted index)
// and their sums (q_sum, zeroed), one thread per triangle or boundary edge
template <typename real>
cudaError_t launch_fem_charges_scatter(const double2 *nodes, const int *tris, int64_t Nt, const double2 *tri_coef,
                                       const int *bedges, int64_t Ne, const double2 *mag, int64_t Nv, int nrhs,
                                       const int *inv_perm, int64_t M, real *q_sorted, double *q_sum, cudaStream_t st);
// per triangle, the coefficients c_k of its charge sum_k M_k . c_k (3 per triangle)
cudaError_t launch_fem_tri_coef(const double2 *nodes, const int *tris, int64_t Nt, double2 *coef, cudaStream_t st);
// inv[perm[k]] = k
cudaError_t launch_invert_perm(const int *perm, int64_t n, int *inv, cudaStream_t st);
// tetrahedra: nodes (Nv, 3), tets (Nt, 4), faces (Nf, 4) = (i0 < i1 < i2, fourth node), mag (nrhs, Nv, 3)
cudaError_t launch_fem3_sources(const double *nodes, const int *tets, int64_t Nt, const int *faces, int64_t Nf,
                                double *src, cudaStream_t st);
cudaError_t launch_fem3_charges(const double *nodes, const int *tets, int64_t Nt, const int *faces,
                                const double *mag, int64_t Nv, int nrhs, double *q, int64_t M, cudaStream_t st);
template <typename real>
cudaError_t launch_fem3_charges_scatter(const double *nodes, const int *tets, int64_t Nt, const double *tet_coef,
                                        const int *faces, int64_t Nf, const double *mag, int64_t Nv, int nrhs,
                                        const int *inv_perm, int64_t M, real *q_sorted, double *q_sum,
                                        cudaStream_t st);
// per tetrahedron, the 9 coefficients g_1..g_3 of its charge sum_k (M_k - M_0) . g_k
cudaError_t launch_fem3_tet_coef(const double *nodes, const int *tets, int64_t Nt, double *coef, cudaStream_t st);

}  // namespace fs
