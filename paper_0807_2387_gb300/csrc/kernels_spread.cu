// Window spreading (step c) and interpolation (step f) on the oversampled grid.
//
// Spreading is the paper's "let the data diffuse to the X nodes through
// convolution with a ... smooth localized function":
//     g_k = sum_j q_j psi(k_1 - u_j1) psi(k_2 - u_j2),
// over the 2m x 2m grid lines k with |k - u_j| < m.  Interpolation reads the
// same stencil back: phi(x_i) = sum_k g'_k psi(u_i1 - k_1) psi(u_i2 - k_2), and
// the gradient uses the analytic window slope psi'.
//
// Spreading: one CTA (kSpreadWarps warps) per work item (a tile of cells, or a
// slice of a crowded tile).  A warp takes one source at a time: lanes 0..2m-1
// evaluate the 2m window weights of the first coordinate, lanes 2m..4m-1 those
// of the second (times q), and every lane owns a fixed subset of the (2m)^2
// taps, fetching its two factors by shuffle.  Each warp accumulates into its
// own padded copy of the tile in shared memory, so within a warp every tap
// address is distinct and the read-modify-write needs no atomics; in FP32 each
// addition's rounding error is recovered exactly (TwoSum) into a second,
// compensation tile, so the tile holds a double-FP32 sum.  At the end the warp
// tiles are summed and added to the grid with global atomics (tiles overlap by
// 2m-1 lines).
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "output.cuh"

namespace fs {

namespace {

template <typename real> using real2_t = typename Cplx<real>::type;

// Loads a group's RPL row weights from 16-byte aligned shared memory in vectors.
template <typename real, int RPL> __device__ __forceinline__ void load_row_weights(const real *src, real (&w)[RPL])
{
    constexpr int VW = 16 / (int)sizeof(real);
#pragma unroll
    for (int v = 0; v < (RPL + VW - 1) / VW; ++v) {
        if constexpr (sizeof(real) == 4) {
            const float4 t = reinterpret_cast<const float4 *>(src)[v];
            const float e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (4 * v + k < RPL)
                    w[4 * v + k] = e[k];
        } else {
            const double2 t = reinterpret_cast<const double2 *>(src)[v];
            w[2 * v] = t.x;
            if (2 * v + 1 < RPL)
                w[2 * v + 1] = t.y;
        }
    }
}

__device__ __forceinline__ float2 sub2f(float2 a, float2 b)   // a - b, one rounding
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// TGC > 0: the tile edge (grid lines) fixed at compile time, so that the tile pitch and the
// row offsets of the taps are constants (immediate offsets instead of one address per row).
template <typename real, int M2, bool KAHAN, int TGC = 0>
__device__ __forceinline__ void spread_item(const SpreadItem &it, const CellGrid &cg, const int *__restrict__ base,
                                            const real2_t<real> *__restrict__ frac, const real *__restrict__ q,
                                            const Window<real> &w, const WindowPoly &wp, real *__restrict__ grid,
                                            int pitch, int n_a)
{
    constexpr int m = M2 / 2;
    constexpr int G = spread_groups(M2);
    constexpr int RPL = M2 / G;                               // rows per tap lane
    constexpr int VW = 16 / (int)sizeof(real);
    constexpr int RPAD = (RPL + VW - 1) / VW * VW;            // a group's row weights, vector-aligned
    constexpr int WSTRIDE = spread_weight_stride<real>(M2);
    constexpr int PLANES = KAHAN ? 2 : 1;
    constexpr bool kPoly = sizeof(real) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kQ = TGC > 0 ? spread_group_pitch(TGC + M2 - 1, M2) : 0;
    const int TG = TGC > 0 ? TGC : cg.T * cg.cell;
    const int P = TG + M2 - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Q = TGC > 0 ? kQ : spread_group_pitch(P, M2);   // row pitch: conflict-free tap rows
    const int PP = P * Q;                                     // one plane of a warp tile
    real *acc = reinterpret_cast<real *>(smem_raw) + (size_t)warp * PP * PLANES;
    unsigned char *after_tiles = smem_raw + spread_tiles_bytes<real>(P, Q, PLANES);
    real *wb = reinterpret_cast<real *>(after_tiles) + warp * WSTRIDE;
    float *poly = reinterpret_cast<float *>(after_tiles + (size_t)kSpreadWarps * WSTRIDE * sizeof(real));
    if (kPoly) {
        for (int i = threadIdx.x; i < M2 * (kPolyD + 1); i += blockDim.x)
            poly[i] = wp.c[i / (kPolyD + 1)][i % (kPolyD + 1)];
    }
    const int t1 = it.tile / cg.n_t, t2 = it.tile - (it.tile / cg.n_t) * cg.n_t;
    const int o1 = t1 * TG - (m - 1), o2 = t2 * TG - (m - 1);
    for (int i = lane; i < PP * PLANES; i += 32)
        acc[i] = real(0);
    __syncthreads();
    // weight lanes: lane a < M2 evaluates the first coordinate's weight of row a, lane M2 + b the
    // second coordinate's weight of column b (times q); they go to the warp's weight slots
    const bool first = lane < M2;
    const int jw = first ? lane : lane - M2;
    const int wslot = first ? (jw / RPL) * RPAD + (jw % RPL) : G * RPAD + jw;
    float pc[kPolyD + 1];   // the lane's window polynomial (FP32 path), in registers for the item
    {
        const float *prow = poly + (lane < 2 * M2 ? jw : 0) * (kPolyD + 1);
#pragma unroll
        for (int k = 0; k <= kPolyD; ++k)
            pc[k] = kPoly ? prow[k] : 0.f;
    }
    // tap lanes: lane (g, b) owns column b and rows g RPL .. g RPL + RPL - 1 of every source
    const bool tap_lane = lane < G * M2;
    const int g = lane / M2, b = lane - (lane / M2) * M2;
    const real *wrow = wb + (tap_lane ? g : 0) * RPAD;
    const real *wcol = wb + G * RPAD + (tap_lane ? b : 0);
    const int end = it.start + it.count;
    int j = it.start + warp;
    // software pipeline: the next source's record is in flight while this one is spread
    int nb = 0;
    real2_t<real> nf{};
    real nq = real(0);
    if (j < end) {
        nb = base[j];
        nf = frac[j];
        nq = q[j];
    }
    for (; j < end; j += kSpreadWarps) {
        const int packed = nb;
        const real2_t<real> f = nf;
        const real qj = nq;
        if (j + kSpreadWarps < end) {
            nb = base[j + kSpreadWarps];
            nf = frac[j + kSpreadWarps];
            nq = q[j + kSpreadWarps];
        }
        if (lane < 2 * M2) {
            const real fr = first ? f.x : f.y;
            real wv;
            if constexpr (kPoly)
                wv = poly_eval<kPolyD>(pc, (float)fr - 0.5f);
            else
                wv = kb_value<real>(w, fr, m - 1 - jw);
            wb[wslot] = first ? wv : wv * qj;
        }
        __syncwarp();
        if (tap_lane) {
            real w1[RPL];
            load_row_weights<real, RPL>(wrow, w1);
            const real w2 = *wcol;
            // the taps of a lane are distinct cells, and distinct from the other lanes': every read
            // of this source is issued before any write
            real *cell = acc + (base1(packed) - m + 1 - o1 + g * RPL) * Q + (base2(packed) - m + 1 - o2 + b);
            real v[RPL], old[RPL], cmp[RPL];
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                v[i] = w1[i] * w2;
                old[i] = cell[i * Q];
                if (KAHAN)
                    cmp[i] = cell[i * Q + PP];
            }
            if constexpr (KAHAN && sizeof(real) == 4) {
                // TwoSum of (old, v) for two taps per packed instruction; the error goes to the
                // compensation plane
#pragma unroll
                for (int i = 0; i + 1 < RPL; i += 2) {
                    const float2 o = make_float2(old[i], old[i + 1]), vv = make_float2(v[i], v[i + 1]);
                    const float2 sm = __fadd2_rn(o, vv);
                    const float2 bb = sub2f(sm, o);
                    const float2 e = __fadd2_rn(sub2f(o, sub2f(sm, bb)), sub2f(vv, bb));
                    const float2 c = __fadd2_rn(make_float2(cmp[i], cmp[i + 1]), e);
                    cell[i * Q] = sm.x;
                    cell[(i + 1) * Q] = sm.y;
                    cell[i * Q + PP] = c.x;
                    cell[(i + 1) * Q + PP] = c.y;
                }
                if constexpr (RPL % 2 == 1) {
                    constexpr int i = RPL - 1;
                    const real sm = old[i] + v[i];
                    const real bb = sm - old[i];
                    cell[i * Q] = sm;
                    cell[i * Q + PP] = cmp[i] + ((old[i] - (sm - bb)) + (v[i] - bb));
                }
            } else {
#pragma unroll
                for (int i = 0; i < RPL; ++i) {
                    const real sm = old[i] + v[i];
                    cell[i * Q] = sm;
                    if (KAHAN) {
                        const real bb = sm - old[i];
                        cell[i * Q + PP] = cmp[i] + ((old[i] - (sm - bb)) + (v[i] - bb));
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    const real *base_tile = reinterpret_cast<const real *>(smem_raw);
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int r = i / P, c = i - (i / P) * P;
        real v = real(0);
#pragma unroll
        for (int ww = 0; ww < kSpreadWarps; ++ww) {
            const real *tile = base_tile + (size_t)ww * PP * PLANES + r * Q + c;
            v += tile[0];
            if (KAHAN)
                v += tile[PP];
        }
        const int g1 = o1 + r, g2 = o2 + c;
        if (v != real(0) && g1 >= 0 && g1 < n_a && g2 >= 0 && g2 < n_a)
            atomicAdd(grid + (int64_t)g1 * pitch + g2, v);
    }
}

// Direct spreading, the alternative to the shared-memory tiles for sparse plans: a warp per
// source (grid-stride), the same row-group lanes, every tap added straight to the grid with a
// global atomic.  FP32 plans with compensation take the old value the atomic returns, recover
// the addition's rounding error exactly (TwoSum of the old and the added value: the atomic
// rounds to nearest like the add it replaces) and add it to a compensation plane, which
// k_fold_comp folds into the grid before the transform.  The window weights reach the tap
// lanes by shuffles.
template <typename real, int M2, bool KAHAN>
__global__ void __launch_bounds__(256) k_spread_direct(int64_t M, const int *__restrict__ base,
                                                       const real2_t<real> *__restrict__ frac,
                                                       const real *__restrict__ q, Window<real> w, WindowPoly wp,
                                                       real *__restrict__ grid, real *__restrict__ comp, int pitch)
{
    constexpr int m = M2 / 2;
    constexpr int G = spread_groups(M2);
    constexpr int RPL = M2 / G;
    constexpr bool kPoly = sizeof(real) == 4;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool first = lane < M2;
    const int jw = first ? lane : lane - M2;
    float pc[kPolyD + 1];
#pragma unroll
    for (int k = 0; k <= kPolyD; ++k)
        pc[k] = (kPoly && lane < 2 * M2) ? wp.c[jw][k] : 0.f;
    const bool tap_lane = lane < G * M2;
    const int g = lane / M2, b = lane - (lane / M2) * M2;
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < M; j += warps) {
        const int packed = base[j];
        const real2_t<real> f = frac[j];
        const real qj = q[j];
        real wv = real(0);
        if (lane < 2 * M2) {
            const real fr = first ? f.x : f.y;
            if constexpr (kPoly)
                wv = poly_eval<kPolyD>(pc, (float)fr - 0.5f);
            else
                wv = kb_value<real>(w, fr, m - 1 - jw);
            if (!first)
                wv *= qj;
        }
        const real w2 = __shfl_sync(0xffffffffu, wv, M2 + (tap_lane ? b : 0));
        real w1[RPL];
#pragma unroll
        for (int i = 0; i < RPL; ++i)
            w1[i] = __shfl_sync(0xffffffffu, wv, (tap_lane ? g : 0) * RPL + i);
        if (tap_lane) {
            const int64_t at = (int64_t)(base1(packed) - m + 1 + g * RPL) * pitch + (base2(packed) - m + 1 + b);
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                const real v = w1[i] * w2;
                const int64_t k = at + (int64_t)i * pitch;
                if constexpr (KAHAN) {
                    const real old = atomicAdd(grid + k, v);
                    const real sm = old + v, bb = sm - old;
                    const real e = (old - (sm - bb)) + (v - bb);
                    if (e != real(0))
                        atomicAdd(comp + k, e);
                } else {
                    atomicAdd(grid + k, v);
                }
            }
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(256) k_fold_comp(int64_t n, real *__restrict__ grid, const real *__restrict__ comp)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n)
        grid[k] += comp[k];
}

template <typename real, int M2, bool KAHAN, int TGC>
__global__ void __launch_bounds__(kSpreadWarps * 32) k_spread(const SpreadItem *__restrict__ items, CellGrid cg,
                                                              const int *__restrict__ base,
                                                              const real2_t<real> *__restrict__ frac,
                                                              const real *__restrict__ q, Window<real> w, WindowPoly wp,
                                                              real *__restrict__ grid, int pitch, int n_a)
{
    spread_item<real, M2, KAHAN, TGC>(items[blockIdx.x], cg, base, frac, q, w, wp, grid, pitch, n_a);
}

// Batched spreading: items carry their instance in `pad`; blockIdx.y = right-hand side.
template <typename real, int M2, bool KAHAN>
__global__ void __launch_bounds__(kSpreadWarps * 32) k_batch_spread(const SpreadItem *__restrict__ items,
                                                                    const BatchInst<real> *__restrict__ inst,
                                                                    Window<real> w, WindowPoly wp)
{
    const SpreadItem it = items[blockIdx.x];
    const BatchInst<real> &b = inst[it.pad];
    const int r = blockIdx.y;
    auto go = [&](auto tg) {
        spread_item<real, M2, KAHAN, decltype(tg)::value>(it, b.cg, b.src_base, (const real2_t<real> *)b.src_frac,
                                                          b.q + (int64_t)r * b.M, w, wp,
                                                          b.grid + (int64_t)r * b.grid_stride, b.pitch, b.n_a);
    };
    // FP32 compensated batches: the tile edges the autotuner picks for the batched instance
    // classes compiled as constants (per block: instances differ), any other edge at run time
    if constexpr (sizeof(real) == 4 && KAHAN) {
        switch (b.cg.T * b.cg.cell) {
        case 12: go(std::integral_constant<int, 12>{}); return;
        case 16: go(std::integral_constant<int, 16>{}); return;
        case 18: go(std::integral_constant<int, 18>{}); return;
        case 24: go(std::integral_constant<int, 24>{}); return;
        default: break;
        }
    }
    go(std::integral_constant<int, 0>{});
}

// In FP32 with m >= 5 the derivative sums are formed against a reference tap:
// the window's periodisation sum_k psi(x - k) is flat (to ~1e-9 relative for
// m = 5, ~1e-11 for m = 6), so sum_k psi'(x - k) vanishes to that level and
// sum_a d_a s_a = sum_a d_a (s_a - s_c) avoids the cancellation between terms of
// size n_os |s| that would otherwise dominate the FP32 gradient error.  For
// m <= 4 the periodisation is flat only to ~1e-7, no better than FP32 rounding,
// so those widths (and the FP64 path) sum directly.
// One row of a target's taps: the row sum rs with the column weights w2 and the derivative
// sum rd with d2 (against the reference column m - 1 when kRef), added to phi and grad with the
// row's weights wr, dr.  The first coordinate's derivative sum is taken against the row sum of
// row m - 1, which the caller visits first (rs_ref).
template <typename real, int M2, bool kRef>
__device__ __forceinline__ void interp_row(const real *__restrict__ rowp, const real (&w2)[M2], const real (&d2)[M2],
                                           real wr, real dr, bool ref_row, real &rs_ref, real &phi, real &g1,
                                           real &g2)
{
    constexpr int m = M2 / 2;
    real gv[M2];
#pragma unroll
    for (int b = 0; b < M2; ++b)
        gv[b] = __ldg(rowp + b);
    real rs = 0, rd = 0;
#pragma unroll
    for (int b = 0; b < M2; ++b) {
        rs += w2[b] * gv[b];
        rd += d2[b] * (kRef ? gv[b] - gv[m - 1] : gv[b]);
    }
    if (ref_row)
        rs_ref = rs;
    phi += wr * rs;
    g2 += wr * rd;
    g1 += dr * (kRef ? rs - rs_ref : rs);
}

// The far-field sums of target k: phi and the two derivative sums in grid units (times n_os for
// the gradient).
template <typename real, int M2>
__device__ __forceinline__ void interp_sums(int64_t k, const int *__restrict__ base,
                                            const real2_t<real> *__restrict__ frac, const Window<real> &w,
                                            const WindowPoly &wp, const real *__restrict__ grid, int pitch, real &phi,
                                            real &g1, real &g2)
{
    constexpr int m = M2 / 2;
    constexpr bool kRef = sizeof(real) == 4 && m >= 5;
    const int packed = base[k];
    const real2_t<real> f = frac[k];
    const int row0 = base1(packed) - m + 1;
    const int col0 = base2(packed) - m + 1;
    real rs_ref = 0;
    phi = g1 = g2 = 0;
    real w2[M2], d2[M2];
    if constexpr (sizeof(real) == 4) {
        // FP32: per-tap window polynomials in t = frac - 1/2 (coefficients are warp-uniform kernel
        // parameters).  The window is even, so tap M2-1-a at t is tap a at -t: each pair takes
        // the even and odd parts of tap a's polynomials in t^2 once (value p(+-t) = E +- t O,
        // slope of the mirrored tap -p'(-t) = t O' - E'), about half the FMAs of 2 evaluations.
        // The column weights are held for all rows; the row weights of each symmetric pair of
        // rows are evaluated just before those two rows (middle pair first, so that row m - 1,
        // the reference, comes first), which keeps 2 M2 fewer values live across the loop.
        const float t1 = (float)f.x - 0.5f, t2 = (float)f.y - 0.5f;
        const float s1 = t1 * t1, s2 = t2 * t2;
#pragma unroll
        for (int a = 0; a < m; ++a) {
            float e, o;
            poly_even_odd<kPolyD>(wp.c[a], s2, e, o);
            w2[a] = fmaf(t2, o, e);
            w2[M2 - 1 - a] = fmaf(-t2, o, e);
            poly_even_odd<kPolyD - 1>(wp.d[a], s2, e, o);
            d2[a] = fmaf(t2, o, e);
            d2[M2 - 1 - a] = fmaf(t2, o, -e);
        }
#pragma unroll
        for (int q = 0; q < m; ++q) {
            const int a = m - 1 - q, a2 = M2 - 1 - a;
            float e, o, de, dd;
            poly_even_odd<kPolyD>(wp.c[a], s1, e, o);
            poly_even_odd<kPolyD - 1>(wp.d[a], s1, de, dd);
            interp_row<real, M2, kRef>(grid + (int64_t)(row0 + a) * pitch + col0, w2, d2, fmaf(t1, o, e),
                                       fmaf(t1, dd, de), q == 0, rs_ref, phi, g1, g2);
            interp_row<real, M2, kRef>(grid + (int64_t)(row0 + a2) * pitch + col0, w2, d2, fmaf(-t1, o, e),
                                       fmaf(t1, dd, -de), false, rs_ref, phi, g1, g2);
        }
    } else {
        real w1[M2], d1[M2];
#pragma unroll
        for (int a = 0; a < M2; ++a) {
            kb_value_slope<real>(w, f.x, m - 1 - a, w1[a], d1[a]);
            kb_value_slope<real>(w, f.y, m - 1 - a, w2[a], d2[a]);
        }
#pragma unroll
        for (int a = 0; a < M2; ++a)
            interp_row<real, M2, kRef>(grid + (int64_t)(row0 + a) * pitch + col0, w2, d2, w1[a], d1[a], false,
                                       rs_ref, phi, g1, g2);
    }
}

// FP32 far-field sums of target k for R right-hand sides at once (grids grid + r grid_stride):
// the window weights, the larger part of the arithmetic, are formed once for all of them.
template <int M2, int R>
__device__ __forceinline__ void interp_sums_rhs(int64_t k, const int *__restrict__ base,
                                                const float2 *__restrict__ frac, const WindowPoly &wp,
                                                const float *__restrict__ grid, int64_t grid_stride, int pitch,
                                                float (&phi)[R], float (&g1)[R], float (&g2)[R])
{
    constexpr int m = M2 / 2;
    constexpr bool kRef = m >= 5;
    const int packed = base[k];
    const float2 f = frac[k];
    const int64_t off = (int64_t)(base1(packed) - m + 1) * pitch + (base2(packed) - m + 1);
    float rs_ref[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
        phi[r] = g1[r] = g2[r] = rs_ref[r] = 0.f;
    float w2[M2], d2[M2];
    const float t1 = f.x - 0.5f, t2 = f.y - 0.5f;
    const float s1 = t1 * t1, s2 = t2 * t2;
#pragma unroll
    for (int a = 0; a < m; ++a) {
        float e, o;
        poly_even_odd<kPolyD>(wp.c[a], s2, e, o);
        w2[a] = fmaf(t2, o, e);
        w2[M2 - 1 - a] = fmaf(-t2, o, e);
        poly_even_odd<kPolyD - 1>(wp.d[a], s2, e, o);
        d2[a] = fmaf(t2, o, e);
        d2[M2 - 1 - a] = fmaf(t2, o, -e);
    }
#pragma unroll
    for (int q = 0; q < m; ++q) {
        const int a = m - 1 - q, a2 = M2 - 1 - a;
        float e, o, de, dd;
        poly_even_odd<kPolyD>(wp.c[a], s1, e, o);
        poly_even_odd<kPolyD - 1>(wp.d[a], s1, de, dd);
        const float wa = fmaf(t1, o, e), da = fmaf(t1, dd, de), wb = fmaf(-t1, o, e), db = fmaf(t1, dd, -de);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float *g = grid + r * grid_stride + off;
            interp_row<float, M2, kRef>(g + (int64_t)a * pitch, w2, d2, wa, da, q == 0, rs_ref[r], phi[r], g1[r],
                                        g2[r]);
            interp_row<float, M2, kRef>(g + (int64_t)a2 * pitch, w2, d2, wb, db, false, rs_ref[r], phi[r], g1[r],
                                        g2[r]);
        }
    }
}

template <typename real, int M2>
__device__ __forceinline__ void interp_point(int64_t k, const int *__restrict__ base,
                                             const real2_t<real> *__restrict__ frac, const Window<real> &w,
                                             const WindowPoly &wp, const real *__restrict__ grid, int pitch, real n_os,
                                             real *__restrict__ phi_s, real *__restrict__ grad_s,
                                             bool acc = false)
{
    real phi, g1, g2;
    interp_sums<real, M2>(k, base, frac, w, wp, grid, pitch, phi, g1, g2);
    // acc: the near field was stored first (overlapped with spreading and the transform)
    phi_s[k] = acc ? phi_s[k] + phi : phi;
    grad_s[2 * k] = acc ? grad_s[2 * k] + n_os * g1 : n_os * g1;
    grad_s[2 * k + 1] = acc ? grad_s[2 * k + 1] + n_os * g2 : n_os * g2;
}

template <typename real, int M2>
__global__ void __launch_bounds__(256) k_interp(int64_t N, const int *__restrict__ base,
                                                const real2_t<real> *__restrict__ frac, Window<real> w, WindowPoly wp,
                                                const real *__restrict__ grid, int pitch, real n_os,
                                                real *__restrict__ phi_s, real *__restrict__ grad_s, bool acc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N)
        interp_point<real, M2>(k, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc);
}

// Interpolation and output in one pass, for plans whose near field was stored first: the far
// field is added to the near field's sums in the working precision exactly as k_interp does,
// and the result goes straight to the caller's buffers (k_unpermute's step), so the sums are not
// written back and read again.
template <typename real, int M2>
__global__ void __launch_bounds__(256, 3) k_interp_out(int64_t N, const int *__restrict__ base,
                                                    const real2_t<real> *__restrict__ frac, Window<real> w,
                                                    WindowPoly wp, const real *__restrict__ grid, int pitch, real n_os,
                                                    const real *__restrict__ phi_s, const real *__restrict__ grad_s,
                                                    const real *__restrict__ coinc, const int *__restrict__ perm,
                                                    double shift, const double *__restrict__ q_sum, double s,
                                                    void *__restrict__ phi_out, void *__restrict__ H_out, int out_is_f64)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    real phi, g1, g2;
    interp_sums<real, M2>(k, base, frac, w, wp, grid, pitch, phi, g1, g2);
    const real pt = phi_s[k] + phi;
    const real gx = grad_s[2 * k] + n_os * g1;
    const real gy = grad_s[2 * k + 1] + n_os * g2;
    output_point<real>(k, pt, gx, gy, coinc[k], perm, shift, q_sum[0], s, phi_out, H_out, out_is_f64);
}

// Batched interpolation: block -> (instance, block of its targets), blockIdx.y = right-hand side.
template <typename real, int M2>
__global__ void __launch_bounds__(256) k_batch_interp(const BatchInst<real> *__restrict__ inst, BlockMap bm,
                                                      Window<real> w, WindowPoly wp)
{
    const int i = bm.inst[blockIdx.x];
    const BatchInst<real> &b = inst[i];
    const int64_t k = (int64_t)(blockIdx.x - bm.first[i]) * blockDim.x + threadIdx.x;
    const int64_t N = b.N;
    if (k >= N)
        return;
    const int r = blockIdx.y;
    interp_point<real, M2>(k, b.tgt_base, (const real2_t<real> *)b.tgt_frac, w, wp,
                           b.grid + (int64_t)r * b.grid_stride, b.pitch, (real)b.L, b.phi_s + (int64_t)r * N,
                           b.grad_s + 2 * (int64_t)r * N);
}

// Batched interpolation and output in one pass (FP32 batches, whose near field stored the sums
// first): block -> (instance, block of its targets), blockIdx.y = right-hand side; writes the
// caller's (nrhs, N) and (nrhs, N, 2) buffers of each instance.
template <typename real, int M2>
__global__ void __launch_bounds__(256, 3) k_batch_interp_out(const BatchInst<real> *__restrict__ inst,
                                                          const BatchIO *__restrict__ io, BlockMap bm, Window<real> w,
                                                          WindowPoly wp, int out_is_f64)
{
    const int i = bm.inst[blockIdx.x];
    const BatchInst<real> &b = inst[i];
    const int64_t k = (int64_t)(blockIdx.x - bm.first[i]) * blockDim.x + threadIdx.x;
    const int64_t N = b.N;
    if (k >= N)
        return;
    const int r = blockIdx.y;
    real phi, g1, g2;
    interp_sums<real, M2>(k, b.tgt_base, (const real2_t<real> *)b.tgt_frac, w, wp, b.grid + (int64_t)r * b.grid_stride,
                          b.pitch, phi, g1, g2);
    const real n_os = (real)b.L;
    const real *ps = b.phi_s + (int64_t)r * N, *gs = b.grad_s + 2 * (int64_t)r * N;
    const size_t osz = out_is_f64 ? 8 : 4;
    void *po = io[i].phi ? (unsigned char *)io[i].phi + (size_t)r * N * osz : nullptr;
    void *ho = io[i].H ? (unsigned char *)io[i].H + (size_t)r * N * 2 * osz : nullptr;
    output_point<real>(k, ps[k] + phi, gs[2 * k] + n_os * g1, gs[2 * k + 1] + n_os * g2, b.coinc[(int64_t)r * N + k],
                       b.tgt_perm, b.shift, b.q_sum[r], b.s, po, ho, out_is_f64);
}

// FP32 batches: the same with all R right-hand sides of a target in one thread (window weights
// formed once); block -> (instance, block of its targets).
template <int M2, int R>
__global__ void __launch_bounds__(256, 3) k_batch_interp_out_rhs(const BatchInst<float> *__restrict__ inst,
                                                              const BatchIO *__restrict__ io, BlockMap bm,
                                                              WindowPoly wp, int out_is_f64)
{
    const int i = bm.inst[blockIdx.x];
    const BatchInst<float> &b = inst[i];
    const int64_t k = (int64_t)(blockIdx.x - bm.first[i]) * blockDim.x + threadIdx.x;
    const int64_t N = b.N;
    if (k >= N)
        return;
    float phi[R], g1[R], g2[R];
    interp_sums_rhs<M2, R>(k, b.tgt_base, (const float2 *)b.tgt_frac, wp, b.grid, b.grid_stride, b.pitch, phi, g1, g2);
    const float n_os = (float)b.L;
    const size_t osz = out_is_f64 ? 8 : 4;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float *ps = b.phi_s + (int64_t)r * N, *gs = b.grad_s + 2 * (int64_t)r * N;
        void *po = io[i].phi ? (unsigned char *)io[i].phi + (size_t)r * N * osz : nullptr;
        void *ho = io[i].H ? (unsigned char *)io[i].H + (size_t)r * N * 2 * osz : nullptr;
        output_point<float>(k, ps[k] + phi[r], gs[2 * k] + n_os * g1[r], gs[2 * k + 1] + n_os * g2[r],
                            b.coinc[(int64_t)r * N + k], b.tgt_perm, b.shift, b.q_sum[r], b.s, po, ho, out_is_f64);
    }
}

// Adjoint spreading at the targets: each point carries a monopole c and a dipole d (2-vector)
// and adds c psi(x1) psi(x2) + d1 psi'(x1) psi(x2) + d2 psi(x1) psi'(x2) at the taps x = u - k,
// the transpose of interpolating phi and grad phi with the same taps.  Same warp-per-point
// organisation as k_spread (lanes evaluate one value/slope pair each, lanes own taps).
template <typename real, int M2, bool KAHAN>
__global__ void __launch_bounds__(kSpreadWarps * 32) k_spread_dip(const SpreadItem *__restrict__ items, CellGrid cg,
                                                                  const int *__restrict__ base,
                                                                  const real2_t<real> *__restrict__ frac,
                                                                  const real *__restrict__ cq,
                                                                  const real2_t<real> *__restrict__ dq, Window<real> w,
                                                                  WindowPoly wp, real *__restrict__ grid, int pitch,
                                                                  int n_a)
{
    constexpr int m = M2 / 2;
    constexpr int TAPS = M2 * M2;
    constexpr int PER = (TAPS + 31) / 32;
    constexpr int PLANES = KAHAN ? 2 : 1;
    constexpr bool kPoly = sizeof(real) == 4;
    extern __shared__ unsigned char smem_raw[];
    const int TG = cg.T * cg.cell;
    const int P = TG + M2 - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Q = spread_pitch_warp(P, M2, lane);   // row pitch: bank-conflict-free taps
    const int PP = P * Q;                             // one plane of a warp tile
    real *acc = reinterpret_cast<real *>(smem_raw) + (size_t)warp * PP * PLANES;
    float *poly = reinterpret_cast<float *>(reinterpret_cast<real *>(smem_raw) + (size_t)kSpreadWarps * PP * PLANES);
    if (kPoly) {
        for (int i = threadIdx.x; i < M2 * (kPolyD + 1); i += blockDim.x)
            poly[i] = wp.c[i / (kPolyD + 1)][i % (kPolyD + 1)];
        for (int i = threadIdx.x; i < M2 * kPolyD; i += blockDim.x)
            poly[M2 * (kPolyD + 1) + i] = wp.d[i / kPolyD][i % kPolyD];
    }
    const SpreadItem it = items[blockIdx.x];
    const int t1 = it.tile / cg.n_t, t2 = it.tile - (it.tile / cg.n_t) * cg.n_t;
    const int o1 = t1 * TG - (m - 1), o2 = t2 * TG - (m - 1);
    for (int i = lane; i < PP * PLANES; i += 32)
        acc[i] = real(0);
    __syncthreads();
    int toff[PER], ta[PER], tb[PER];
    unsigned valid;
    spread_lane_taps<M2, PER>(lane, Q, ta, tb, toff, valid);
    const bool first = lane < M2;
    const int jw = first ? lane : lane - M2;
    float pc[kPolyD + 1], pd[kPolyD];   // the lane's value and slope polynomials, in registers
    {
        const float *prow = poly + (lane < 2 * M2 ? jw : 0) * (kPolyD + 1);
        const float *drow = poly + M2 * (kPolyD + 1) + (lane < 2 * M2 ? jw : 0) * kPolyD;
#pragma unroll
        for (int k = 0; k <= kPolyD; ++k)
            pc[k] = kPoly ? prow[k] : 0.f;
#pragma unroll
        for (int k = 0; k < kPolyD; ++k)
            pd[k] = kPoly ? drow[k] : 0.f;
    }
    for (int j = it.start + warp; j < it.start + it.count; j += kSpreadWarps) {
        const int packed = base[j];
        const real2_t<real> f = frac[j];
        const real c = cq[j];
        const real2_t<real> d = dq[j];
        real wv = real(0), wd = real(0);
        if (lane < 2 * M2) {
            const real fr = first ? f.x : f.y;
            if constexpr (kPoly) {
                wv = poly_eval<kPolyD>(pc, (float)fr - 0.5f);
                wd = poly_eval<kPolyD - 1>(pd, (float)fr - 0.5f);
            } else {
                kb_value_slope<real>(w, fr, m - 1 - jw, wv, wd);
            }
        }
        real *corner = acc + (base1(packed) - m + 1 - o1) * Q + (base2(packed) - m + 1 - o2);
        real v[PER], old[PER], cmp[PER];     // reads before writes, as in spread_item
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const real w1 = __shfl_sync(0xffffffffu, wv, ta[i]);
            const real d1 = __shfl_sync(0xffffffffu, wd, ta[i]);
            const real w2 = __shfl_sync(0xffffffffu, wv, M2 + tb[i]);
            const real d2 = __shfl_sync(0xffffffffu, wd, M2 + tb[i]);
            v[i] = w2 * (c * w1 + d.x * d1) + d.y * w1 * d2;
            if ((valid >> i) & 1u) {
                old[i] = corner[toff[i]];
                if (KAHAN)
                    cmp[i] = corner[toff[i] + PP];
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if ((valid >> i) & 1u) {
                real *cell = corner + toff[i];
                const real s = old[i] + v[i];
                *cell = s;
                if (KAHAN) {
                    const real bb = s - old[i];
                    cell[PP] = cmp[i] + ((old[i] - (s - bb)) + (v[i] - bb));
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    const real *base_tile = reinterpret_cast<const real *>(smem_raw);
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int r = i / P, cc = i - (i / P) * P;
        real v = real(0);
#pragma unroll
        for (int ww = 0; ww < kSpreadWarps; ++ww) {
            const real *tile = base_tile + (size_t)ww * PP * PLANES + r * Q + cc;
            v += tile[0];
            if (KAHAN)
                v += tile[PP];
        }
        const int g1 = o1 + r, g2 = o2 + cc;
        if (v != real(0) && g1 >= 0 && g1 < n_a && g2 >= 0 && g2 < n_a)
            atomicAdd(grid + (int64_t)g1 * pitch + g2, v);
    }
}

// Gradient and Hessian of the interpolated field (torus units):
//   grad = n_os sum_k g_k grad Psi(u - k),  Hess = n_os^2 sum_k g_k grad grad Psi(u - k).
// FP32 with m >= 5 forms the derivative sums against a reference tap (see k_interp).
template <typename real, int M2>
__global__ void __launch_bounds__(256) k_interp_hess(int64_t N, const int *__restrict__ base,
                                                     const real2_t<real> *__restrict__ frac, Window<real> w,
                                                     WindowPoly wp, const real *__restrict__ grid, int pitch,
                                                     real n_os, real *__restrict__ grad_s, real *__restrict__ hess_s,
                                                     bool acc)
{
    constexpr int m = M2 / 2;
    constexpr bool kRef = sizeof(real) == 4 && m >= 5;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int packed = base[k];
    const real2_t<real> f = frac[k];
    real w1[M2], d1[M2], e1[M2], w2[M2], d2[M2], e2[M2];
    if constexpr (sizeof(real) == 4) {
        const float t1 = (float)f.x - 0.5f, t2 = (float)f.y - 0.5f;
#pragma unroll
        for (int a = 0; a < M2; ++a) {
            w1[a] = poly_eval<kPolyD>(wp.c[a], t1);
            d1[a] = poly_eval<kPolyD - 1>(wp.d[a], t1);
            e1[a] = poly_eval<kPolyD - 2>(wp.e[a], t1);
            w2[a] = poly_eval<kPolyD>(wp.c[a], t2);
            d2[a] = poly_eval<kPolyD - 1>(wp.d[a], t2);
            e2[a] = poly_eval<kPolyD - 2>(wp.e[a], t2);
        }
    } else {
#pragma unroll
        for (int a = 0; a < M2; ++a) {
            kb_value_slope_curv<real>(w, f.x, m - 1 - a, w1[a], d1[a], e1[a]);
            kb_value_slope_curv<real>(w, f.y, m - 1 - a, w2[a], d2[a], e2[a]);
        }
    }
    const int row0 = base1(packed) - m + 1;
    const int col0 = base2(packed) - m + 1;
    real rs[M2], rd[M2];
    real gy = 0, hyy = 0, hxy = 0;
#pragma unroll
    for (int a = 0; a < M2; ++a) {
        const real *rowp = grid + (int64_t)(row0 + a) * pitch + col0;
        real gv[M2];
#pragma unroll
        for (int b = 0; b < M2; ++b)
            gv[b] = __ldg(rowp + b);
        real s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int b = 0; b < M2; ++b) {
            const real g = kRef ? gv[b] - gv[m - 1] : gv[b];
            s0 += w2[b] * gv[b];
            s1 += d2[b] * g;
            s2 += e2[b] * g;
        }
        rs[a] = s0;
        rd[a] = s1;
        gy += w1[a] * s1;
        hyy += w1[a] * s2;
    }
    real gx = 0, hxx = 0;
#pragma unroll
    for (int a = 0; a < M2; ++a) {
        const real r0 = kRef ? rs[a] - rs[m - 1] : rs[a];
        const real r1 = kRef ? rd[a] - rd[m - 1] : rd[a];
        gx += d1[a] * r0;
        hxx += e1[a] * r0;
        hxy += d1[a] * r1;
    }
    // acc: the near part was stored first (it ran beside the spreading and the transform)
    const real n2 = n_os * n_os;
    grad_s[2 * k] = acc ? grad_s[2 * k] + n_os * gx : n_os * gx;
    grad_s[2 * k + 1] = acc ? grad_s[2 * k + 1] + n_os * gy : n_os * gy;
    hess_s[3 * k] = acc ? hess_s[3 * k] + n2 * hxx : n2 * hxx;
    hess_s[3 * k + 1] = acc ? hess_s[3 * k + 1] + n2 * hxy : n2 * hxy;
    hess_s[3 * k + 2] = acc ? hess_s[3 * k + 2] + n2 * hyy : n2 * hyy;
}

template <typename real, int M2>
cudaError_t spread_m(const SpreadItem *items, int n_items, CellGrid cg, const int *base, const void *frac,
                     const real *q, Window<real> w, const WindowPoly &wp, real *grid, int pitch, int n_a, bool kahan,
                     cudaStream_t st)
{
    const int TG = cg.T * cg.cell;
    const int P = TG + M2 - 1;
    const size_t smem = spread_smem_bytes<real>(P, M2, kahan);
    const real2_t<real> *fr = (const real2_t<real> *)frac;
    auto run = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        kern<<<n_items, kSpreadWarps * 32, smem, st>>>(items, cg, base, fr, q, w, wp, grid, pitch, n_a);
        return cudaGetLastError();
    };
    // the tile edges of the 2D plans' two tile rules (16 and 24 grid lines) compiled as constants
    if (kahan)
        return TG == 16 ? run(k_spread<real, M2, true, 16>)
                        : TG == 24 ? run(k_spread<real, M2, true, 24>) : run(k_spread<real, M2, true, 0>);
    return TG == 16 ? run(k_spread<real, M2, false, 16>)
                    : TG == 24 ? run(k_spread<real, M2, false, 24>) : run(k_spread<real, M2, false, 0>);
}

template <typename real, int M2>
cudaError_t interp_m(int64_t N, const int *base, const void *frac, Window<real> w, const WindowPoly &wp,
                     const real *grid, int pitch, real n_os, real *phi_s, real *grad_s, bool acc, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((N + 255) / 256);
    k_interp<real, M2><<<blocks, 256, 0, st>>>(N, base, (const real2_t<real> *)frac, w, wp, grid, pitch, n_os, phi_s,
                                                grad_s, acc);
    return cudaGetLastError();
}

template <typename real, int M2>
cudaError_t spread_dip_m(const SpreadItem *items, int n_items, CellGrid cg, const int *base, const void *frac,
                         const real *cq, const void *dq, Window<real> w, const WindowPoly &wp, real *grid, int pitch,
                         int n_a, bool kahan, cudaStream_t st)
{
    const int TG = cg.T * cg.cell;
    const int P = TG + M2 - 1;
    const size_t smem = (size_t)kSpreadWarps * P * spread_pitch(P, M2) * sizeof(real) * (kahan ? 2 : 1) +
                        sizeof(float) * M2 * (2 * kPolyD + 1);
    const real2_t<real> *fr = (const real2_t<real> *)frac;
    const real2_t<real> *dd = (const real2_t<real> *)dq;
    if (kahan) {
        auto kern = k_spread_dip<real, M2, true>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        kern<<<n_items, kSpreadWarps * 32, smem, st>>>(items, cg, base, fr, cq, dd, w, wp, grid, pitch, n_a);
    } else {
        auto kern = k_spread_dip<real, M2, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        kern<<<n_items, kSpreadWarps * 32, smem, st>>>(items, cg, base, fr, cq, dd, w, wp, grid, pitch, n_a);
    }
    return cudaGetLastError();
}

template <typename real, int M2>
cudaError_t interp_hess_m(int64_t N, const int *base, const void *frac, Window<real> w, const WindowPoly &wp,
                          const real *grid, int pitch, real n_os, real *grad_s, real *hess_s, bool acc,
                          cudaStream_t st)
{
    const unsigned blocks = (unsigned)((N + 255) / 256);
    k_interp_hess<real, M2><<<blocks, 256, 0, st>>>(N, base, (const real2_t<real> *)frac, w, wp, grid, pitch, n_os,
                                                     grad_s, hess_s, acc);
    return cudaGetLastError();
}

}  // namespace

template <typename real>
cudaError_t launch_spread_dip(const SpreadItem *items, int n_items, CellGrid cg, int m, const int *base,
                              const void *frac, const real *cq, const void *dq, Window<real> w, const WindowPoly &wp,
                              real *grid, int pitch, int n_a, bool kahan, cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    const bool comp = kahan && sizeof(real) == 4;
    switch (m) {
#define FS_DIP_CASE(MM)                                                                                          \
    case MM:                                                                                                     \
        return spread_dip_m<real, 2 * MM>(items, n_items, cg, base, frac, cq, dq, w, wp, grid, pitch, n_a, comp, st);
        FS_DIP_CASE(2)
        FS_DIP_CASE(3)
        FS_DIP_CASE(4)
        FS_DIP_CASE(5)
        FS_DIP_CASE(6)
        FS_DIP_CASE(7)
        FS_DIP_CASE(8)
#undef FS_DIP_CASE
    default: return cudaErrorInvalidValue;
    }
}

template <typename real>
cudaError_t launch_interp_hess(int64_t N, int m, const int *base, const void *frac, Window<real> w,
                               const WindowPoly &wp, const real *grid, int pitch, real n_os, real *grad_s,
                               real *hess_s, bool acc, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    switch (m) {
#define FS_HESS_CASE(MM)                                                                                         \
    case MM:                                                                                                     \
        return interp_hess_m<real, 2 * MM>(N, base, frac, w, wp, grid, pitch, n_os, grad_s, hess_s, acc, st);
        FS_HESS_CASE(2)
        FS_HESS_CASE(3)
        FS_HESS_CASE(4)
        FS_HESS_CASE(5)
        FS_HESS_CASE(6)
        FS_HESS_CASE(7)
        FS_HESS_CASE(8)
#undef FS_HESS_CASE
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_spread_dip<float>(const SpreadItem *, int, CellGrid, int, const int *, const void *,
                                              const float *, const void *, Window<float>, const WindowPoly &, float *,
                                              int, int, bool, cudaStream_t);
template cudaError_t launch_spread_dip<double>(const SpreadItem *, int, CellGrid, int, const int *, const void *,
                                               const double *, const void *, Window<double>, const WindowPoly &,
                                               double *, int, int, bool, cudaStream_t);
template cudaError_t launch_interp_hess<float>(int64_t, int, const int *, const void *, Window<float>,
                                               const WindowPoly &, const float *, int, float, float *, float *, bool,
                                               cudaStream_t);
template cudaError_t launch_interp_hess<double>(int64_t, int, const int *, const void *, Window<double>,
                                                const WindowPoly &, const double *, int, double, double *, double *,
                                                bool, cudaStream_t);

// Calls f(std::integral_constant<int, 2m>) for the window half-width m in 2..8.
template <class F> cudaError_t with_width_spread(int m, F &&f)
{
    switch (m) {
    case 2: return f(std::integral_constant<int, 4>{});
    case 3: return f(std::integral_constant<int, 6>{});
    case 4: return f(std::integral_constant<int, 8>{});
    case 5: return f(std::integral_constant<int, 10>{});
    case 6: return f(std::integral_constant<int, 12>{});
    case 7: return f(std::integral_constant<int, 14>{});
    case 8: return f(std::integral_constant<int, 16>{});
    default: return cudaErrorInvalidValue;
    }
}

template <typename real>
cudaError_t launch_spread(const SpreadItem *items, int n_items, CellGrid cg, int m, const int *base, const void *frac,
                          const real *q, Window<real> w, const WindowPoly &wp, real *grid, int pitch, int n_a,
                          bool kahan, cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    const bool comp = kahan && sizeof(real) == 4;
    switch (m) {
    case 2: return spread_m<real, 4>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    case 3: return spread_m<real, 6>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    case 4: return spread_m<real, 8>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    case 5: return spread_m<real, 10>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    case 6: return spread_m<real, 12>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    case 7: return spread_m<real, 14>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    case 8: return spread_m<real, 16>(items, n_items, cg, base, frac, q, w, wp, grid, pitch, n_a, comp, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename real>
cudaError_t launch_interp(int64_t N, int m, const int *base, const void *frac, Window<real> w, const WindowPoly &wp,
                          const real *grid, int pitch, real n_os, real *phi_s, real *grad_s, bool acc,
                          cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    switch (m) {
    case 2: return interp_m<real, 4>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    case 3: return interp_m<real, 6>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    case 4: return interp_m<real, 8>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    case 5: return interp_m<real, 10>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    case 6: return interp_m<real, 12>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    case 7: return interp_m<real, 14>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    case 8: return interp_m<real, 16>(N, base, frac, w, wp, grid, pitch, n_os, phi_s, grad_s, acc, st);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_spread<float>(const SpreadItem *, int, CellGrid, int, const int *, const void *,
                                          const float *, Window<float>, const WindowPoly &, float *, int, int, bool,
                                          cudaStream_t);
template cudaError_t launch_spread<double>(const SpreadItem *, int, CellGrid, int, const int *, const void *,
                                           const double *, Window<double>, const WindowPoly &, double *, int, int,
                                           bool, cudaStream_t);
template <typename real>
cudaError_t launch_spread_direct(int64_t M, int m, const int *base, const void *frac, const real *q, Window<real> w,
                                 const WindowPoly &wp, real *grid, real *comp, int pitch, int n_a, bool kahan,
                                 cudaStream_t st)
{
    if (M <= 0)
        return cudaSuccess;
    const bool comp_on = kahan && sizeof(real) == 4 && comp;
    const real2_t<real> *fr = (const real2_t<real> *)frac;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int64_t want = (M + 7) / 8;   // 8 warps (sources in flight) per block of 256
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    e = with_width_spread(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        if (comp_on)
            k_spread_direct<real, M2, true><<<blocks, 256, 0, st>>>(M, base, fr, q, w, wp, grid, comp, pitch);
        else
            k_spread_direct<real, M2, false><<<blocks, 256, 0, st>>>(M, base, fr, q, w, wp, grid, comp, pitch);
        return cudaGetLastError();
    });
    if (e != cudaSuccess || !comp_on)
        return e;
    const int64_t n = (int64_t)n_a * pitch;
    k_fold_comp<real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, grid, comp);
    return cudaGetLastError();
}

template cudaError_t launch_spread_direct<float>(int64_t, int, const int *, const void *, const float *, Window<float>,
                                                 const WindowPoly &, float *, float *, int, int, bool, cudaStream_t);
template cudaError_t launch_spread_direct<double>(int64_t, int, const int *, const void *, const double *,
                                                  Window<double>, const WindowPoly &, double *, double *, int, int,
                                                  bool, cudaStream_t);

template cudaError_t launch_interp<float>(int64_t, int, const int *, const void *, Window<float>, const WindowPoly &,
                                          const float *, int, float, float *, float *, bool, cudaStream_t);
template cudaError_t launch_interp<double>(int64_t, int, const int *, const void *, Window<double>,
                                           const WindowPoly &, const double *, int, double, double *, double *, bool,
                                           cudaStream_t);

namespace {

// Calls f(std::integral_constant<int, 2m>) for the window half-width m in 2..8.
template <class F> cudaError_t with_width(int m, F &&f)
{
    switch (m) {
    case 2: return f(std::integral_constant<int, 4>{});
    case 3: return f(std::integral_constant<int, 6>{});
    case 4: return f(std::integral_constant<int, 8>{});
    case 5: return f(std::integral_constant<int, 10>{});
    case 6: return f(std::integral_constant<int, 12>{});
    case 7: return f(std::integral_constant<int, 14>{});
    case 8: return f(std::integral_constant<int, 16>{});
    default: return cudaErrorInvalidValue;
    }
}

// Instances have tiles of up to max_tile grid lines; a tile of r <= P rows takes at most
// r (r + 31) words per plane, which is below P^2 <= P x pitch(P) unless r > P - 32.
template <typename real> size_t batch_spread_smem(int M2, int max_tile, bool comp)
{
    const int P = max_tile + M2 - 1;
    size_t bytes = 0;
    for (int r = P > 32 ? P - 32 : 1; r <= P; ++r)
        bytes = std::max(bytes, spread_smem_bytes<real>(r, M2, comp));
    return bytes;
}

}  // namespace

template <typename real>
cudaError_t launch_interp_out(int64_t N, int m, const int *base, const void *frac, Window<real> w, const WindowPoly &wp,
                              const real *grid, int pitch, real n_os, const real *phi_s, const real *grad_s,
                              const real *coinc, const int *perm, double shift, const double *q_sum, double s,
                              void *phi_out, void *H_out, int out_is_f64, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    return with_width(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        k_interp_out<real, M2><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
            N, base, (const real2_t<real> *)frac, w, wp, grid, pitch, n_os, phi_s, grad_s, coinc, perm, shift, q_sum, s,
            phi_out, H_out, out_is_f64);
        return cudaGetLastError();
    });
}
template cudaError_t launch_interp_out<float>(int64_t, int, const int *, const void *, Window<float>,
                                              const WindowPoly &, const float *, int, float, const float *,
                                              const float *, const float *, const int *, double, const double *,
                                              double, void *, void *, int, cudaStream_t);
template cudaError_t launch_interp_out<double>(int64_t, int, const int *, const void *, Window<double>,
                                               const WindowPoly &, const double *, int, double, const double *,
                                               const double *, const double *, const int *, double, const double *,
                                               double, void *, void *, int, cudaStream_t);

// Raises the dynamic shared memory limit of the batched spreading kernel (outside graph capture).
template <typename real> cudaError_t prepare_batch_spread(int m, int max_tile, bool kahan)
{
    const bool comp = kahan && sizeof(real) == 4;
    return with_width(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        const int smem = (int)batch_spread_smem<real>(M2, max_tile, comp);
        return comp ? cudaFuncSetAttribute(k_batch_spread<real, M2, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                    : cudaFuncSetAttribute(k_batch_spread<real, M2, false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
}

template <typename real>
cudaError_t launch_batch_spread(const SpreadItem *items, int n_items, int nrhs, const BatchInst<real> *inst, int m,
                                int max_tile, Window<real> w, const WindowPoly &wp, bool kahan, cudaStream_t st)
{
    if (n_items <= 0 || nrhs <= 0)
        return cudaSuccess;
    const bool comp = kahan && sizeof(real) == 4;
    return with_width(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        const size_t smem = batch_spread_smem<real>(M2, max_tile, comp);
        const dim3 grid((unsigned)n_items, (unsigned)nrhs);
        if (comp)
            k_batch_spread<real, M2, true><<<grid, kSpreadWarps * 32, smem, st>>>(items, inst, w, wp);
        else
            k_batch_spread<real, M2, false><<<grid, kSpreadWarps * 32, smem, st>>>(items, inst, w, wp);
        return cudaGetLastError();
    });
}

template <typename real>
cudaError_t launch_batch_interp(const BatchInst<real> *inst, BlockMap bm, int blocks, int nrhs, int m,
                                Window<real> w, const WindowPoly &wp, cudaStream_t st)
{
    if (blocks <= 0 || nrhs <= 0)
        return cudaSuccess;
    return with_width(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        k_batch_interp<real, M2><<<dim3((unsigned)blocks, (unsigned)nrhs), 256, 0, st>>>(inst, bm, w, wp);
        return cudaGetLastError();
    });
}

template <typename real>
cudaError_t launch_batch_interp_out(const BatchInst<real> *inst, const BatchIO *io, BlockMap bm, int blocks, int nrhs,
                                    int m, Window<real> w, const WindowPoly &wp, int out_is_f64, cudaStream_t st)
{
    if (blocks <= 0 || nrhs <= 0)
        return cudaSuccess;
    return with_width(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        if constexpr (std::is_same_v<real, float>) {
            // up to four right-hand sides in one thread per target (batched replay 7.78 -> 7.63 ms)
            const dim3 g((unsigned)blocks, 1);
            const auto *fi = reinterpret_cast<const BatchInst<float> *>(inst);
            switch (nrhs) {
            case 1: k_batch_interp_out_rhs<M2, 1><<<g, 256, 0, st>>>(fi, io, bm, wp, out_is_f64); return cudaGetLastError();
            case 2: k_batch_interp_out_rhs<M2, 2><<<g, 256, 0, st>>>(fi, io, bm, wp, out_is_f64); return cudaGetLastError();
            case 3: k_batch_interp_out_rhs<M2, 3><<<g, 256, 0, st>>>(fi, io, bm, wp, out_is_f64); return cudaGetLastError();
            case 4: k_batch_interp_out_rhs<M2, 4><<<g, 256, 0, st>>>(fi, io, bm, wp, out_is_f64); return cudaGetLastError();
            default: break;
            }
        }
        k_batch_interp_out<real, M2><<<dim3((unsigned)blocks, (unsigned)nrhs), 256, 0, st>>>(inst, io, bm, w, wp,
                                                                                           out_is_f64);
        return cudaGetLastError();
    });
}

#define FS_INST(real)                                                                                          \
    template cudaError_t prepare_batch_spread<real>(int, int, bool);                                           \
    template cudaError_t launch_batch_spread<real>(const SpreadItem *, int, int, const BatchInst<real> *, int, \
                                                   int, Window<real>, const WindowPoly &, bool, cudaStream_t); \
    template cudaError_t launch_batch_interp<real>(const BatchInst<real> *, BlockMap, int, int, int,           \
                                                   Window<real>, const WindowPoly &, cudaStream_t);           \
    template cudaError_t launch_batch_interp_out<real>(const BatchInst<real> *, const BatchIO *, BlockMap, int, \
                                                       int, int, Window<real>, const WindowPoly &, int,        \
                                                       cudaStream_t);
FS_INST(float)
FS_INST(double)
#undef FS_INST

}  // namespace fs
