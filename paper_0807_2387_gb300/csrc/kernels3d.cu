// The fast summation for the 3D kernel G(r) = 1/(4 pi r): binning, spreading, interpolation,
// near field and output (the transform is in kernels_fft.cu).
//
// The paper names the 3D Green function as the next step with the same pipeline; each
// kernel here is the 2D one with a third coordinate:
//   spreading    g_k = sum_j q_j psi(k1 - u_j1) psi(k2 - u_j2) psi(k3 - u_j3) over the
//                (2m)^3 grid lines around each source; one warp per source, lanes 0..6m-1
//                hold the window values of the three coordinates and every lane owns
//                (2m)^3 / 32 taps.  FP32: warp-private shared tiles of the source cell with a
//                TwoSum compensation plane, flushed once per item (k_spread3_tile); FP64 (or
//                tiles too large for shared memory): global atomics (k_spread3);
//   interpolation phi and grad phi from the same taps, the window and its slope;
//   near field   q (1/(4 pi r) - T_I(r)) and its gradient for 0 < r < eps_I over the 27
//                cells around, -q T_I(0) for coincident points.  FP32: warp items over the
//                targets with candidate lists (k_near3_warp) or, when sources outnumber
//                targets three to one, over the sources (k_near3_src); pairs closer than
//                eps_I / 8 take their difference from the FP64 positions.  FP64: thread per
//                target (k_near3_f64);
//   output       phi = s phi~, H = -s^2 grad~ phi~ (1/r is homogeneous of degree -1).
// Grid layout: g[z][y][x], x fastest, edge n_a (the active window); a point's base grid
// line per coordinate is packed into 10 bits each.
#include "near_warp.cuh"

namespace fs {

namespace {

template <typename real> using real2_t = typename Cplx<real>::type;

__device__ __forceinline__ int b3x(int p) { return p & 1023; }
__device__ __forceinline__ int b3y(int p) { return (p >> 10) & 1023; }
__device__ __forceinline__ int b3z(int p) { return (p >> 20) & 1023; }

__global__ void k_rmax3(const double *__restrict__ xyz, int64_t n, unsigned long long *out)
{
    double best = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
        best = fmax(best, x * x + y * y + z * z);
    }
    for (int o = 16; o > 0; o >>= 1)
        best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, (unsigned long long)__double_as_longlong(best));   // non-negative: bit order = value order
}

// Window grid line of torus coordinate s x: floor(n_os s x) + n_os/2 - window_lo, and the
// fraction n_os s x - floor(n_os s x); status 1 when the taps leave the active window (the
// point lies beyond the admissible radius).
__device__ __forceinline__ int grid_line3(double x, double s, int n_os, int window_lo, int m, int n_a, double &frac,
                                          int *status)
{
    const double v = (double)n_os * (s * x);
    const double fl = floor(v);
    frac = v - fl;
    int b = (int)fl + n_os / 2 - window_lo;
    if (b - m + 1 < 0 || b + m > n_a - 1) {
        atomicExch(status, 1);
        b = b - m + 1 < 0 ? m - 1 : n_a - 1 - m;
        frac = 0.0;
    }
    return b;
}

__global__ void k_point_keys3(const double *__restrict__ xyz, int64_t n, double s, int n_os, int window_lo, int n_a,
                              int m, CellGrid3 cg, int *__restrict__ key, int *__restrict__ count, int *status)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    int b[3], sc[3];
    for (int d = 0; d < 3; ++d) {
        double f;
        b[d] = grid_line3(xyz[3 * k + d], s, n_os, window_lo, m, n_a, f, status);
        // sub-cell from the offset inside the cell, (b mod cell + frac) / cell in [0, 1)
        const int sidx = (int)(((double)(b[d] % cg.cell) + f) * cg.sub / cg.cell);
        sc[d] = sidx < cg.sub ? sidx : cg.sub - 1;
    }
    int morton = 0;
    for (int bit = 0; bit < 2; ++bit)
        morton |= (((sc[2] >> bit) & 1) << (3 * bit)) | (((sc[1] >> bit) & 1) << (3 * bit + 1)) |
                  (((sc[0] >> bit) & 1) << (3 * bit + 2));
    const int kk = cg.key(b[0] / cg.cell, b[1] / cg.cell, b[2] / cg.cell) * cg.sub3() + morton;
    key[k] = kk;
    atomicAdd(&count[kk], 1);
}

template <typename real>
__global__ void k_gather_points3(const double *__restrict__ xyz, const int *__restrict__ perm, int64_t n, double s,
                                 int n_os, int window_lo, int n_a, int m, int cell, double inv_eps,
                                 double *__restrict__ pos, real *__restrict__ frac, int *__restrict__ base,
                                 float4 *__restrict__ pos32, int *status)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    const int64_t i = perm[k];
    int b[3];
    double fr[3];
    for (int d = 0; d < 3; ++d) {
        b[d] = grid_line3(xyz[3 * i + d], s, n_os, window_lo, m, n_a, fr[d], status);
        pos[3 * k + d] = s * xyz[3 * i + d];
        frac[3 * k + d] = (real)fr[d];
    }
    base[k] = b[0] | (b[1] << 10) | (b[2] << 20);
    if (pos32) {
        // offset from the lower corner of the point's cell, in units of eps_I
        float o[3];
        for (int d = 0; d < 3; ++d) {
            const double corner = (double)((b[d] / cell) * cell + window_lo) / n_os - 0.5;
            o[d] = (float)((s * xyz[3 * i + d] - corner) * inv_eps);
        }
        pos32[k] = make_float4(o[0], o[1], o[2], 0.f);
    }
}

// One warp per source: lanes 0..M2-1, M2..2M2-1, 2M2..3M2-1 evaluate the x, y, z window values
// (x times q), every lane adds its taps (t = lane + 32 i: x fastest) to the grid.
template <typename real, int M2>
__global__ void __launch_bounds__(256) k_spread3(int64_t M, const int *__restrict__ base, const real *__restrict__ frac,
                                                 const real *__restrict__ q, Window<real> w, WindowPoly wp,
                                                 real *__restrict__ grid, int n_a)
{
    constexpr int m = M2 / 2;
    constexpr int TAPS = M2 * M2 * M2;
    constexpr int PER = (TAPS + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int dim = lane / M2, jw = lane - (lane / M2) * M2;
    // software pipeline: the next source's record is in flight while this one is spread
    int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int nb = 0;
    real nf = real(0), nq = real(0);
    if (j < M) {
        nb = base[j];
        nf = lane < 3 * M2 ? frac[3 * j + dim] : real(0);
        nq = q[j];
    }
    for (; j < M; j += warps) {
        const int packed = nb;
        const real fr = nf, qj = nq;
        if (j + warps < M) {
            nb = base[j + warps];
            nf = lane < 3 * M2 ? frac[3 * (j + warps) + dim] : real(0);
            nq = q[j + warps];
        }
        real wv = real(0);
        if (lane < 3 * M2) {
            if constexpr (sizeof(real) == 4)
                wv = poly_eval<kPolyD>(wp.c[jw], (float)fr - 0.5f);
            else
                wv = kb_value<real>(w, fr, m - 1 - jw);
            if (dim == 0)
                wv *= qj;
        }
        const int x0 = b3x(packed) - m + 1, y0 = b3y(packed) - m + 1, z0 = b3z(packed) - m + 1;
        if constexpr (M2 == 8) {
            // t = lane + 32 i: tx = lane % 8 for every i, ty takes two values (i even / odd) and
            // tz = i / 2, so 11 shuffles serve the 16 taps of a lane
            const real vx = __shfl_sync(0xffffffffu, wv, lane & 7);
            const real vxy0 = vx * __shfl_sync(0xffffffffu, wv, 8 + (lane >> 3));
            const real vxy1 = vx * __shfl_sync(0xffffffffu, wv, 12 + (lane >> 3));
            real* row = grid + ((int64_t)z0 * n_a + (y0 + (lane >> 3))) * n_a + (x0 + (lane & 7));
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const real vz = __shfl_sync(0xffffffffu, wv, 16 + (i >> 1));
                atomicAdd(row + ((int64_t)(i >> 1) * n_a + 4 * (i & 1)) * n_a, ((i & 1) ? vxy1 : vxy0) * vz);
            }
        } else {
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int t = lane + 32 * i;
                const int tx = t % M2, ty = (t / M2) % M2, tz = t / (M2 * M2);
                const real vx = __shfl_sync(0xffffffffu, wv, tx);
                const real vy = __shfl_sync(0xffffffffu, wv, M2 + ty);
                const real vz = __shfl_sync(0xffffffffu, wv, 2 * M2 + (tz < M2 ? tz : 0));
                if (t < TAPS)
                    atomicAdd(grid + ((int64_t)(z0 + tz) * n_a + (y0 + ty)) * n_a + (x0 + tx), vx * vy * vz);
            }
        }
    }
}

// FP32 spreading through warp-private tiles in shared memory (items of at most
// kSpread3ItemMax sources of one cell).  Each warp owns a tile covering the cell's taps, edge
// P = cell + 2m - 1 grid lines, plus a compensation plane: a warp handles one source at a time
// and every tap of a source is a distinct cell, so the read-modify-write needs no atomics, and
// the rounding error of each addition is recovered exactly (TwoSum) into the compensation
// plane.  The warps' tiles are summed and added to the grid once per item with global atomics.
// This replaces 512 global atomics per source (at m = 4) by 2 shared reads and 2 writes per tap.
constexpr int kSpread3Warps = 4;

template <int M2>
__global__ void __launch_bounds__(kSpread3Warps * 32) k_spread3_tile(const int2 *__restrict__ items,
                                                                     const int *__restrict__ base,
                                                                     const float *__restrict__ frac,
                                                                     const float *__restrict__ q, WindowPoly wp,
                                                                     int cell, float *__restrict__ grid, int n_a)
{
    constexpr int m = M2 / 2;
    constexpr int TAPS = M2 * M2 * M2;
    constexpr int PER = (TAPS + 31) / 32;
    extern __shared__ float tiles[];
    const int P = cell + M2 - 1, P3 = P * P * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *acc = tiles + (size_t)warp * 2 * P3;   // value plane, then compensation plane
    const int2 it = items[blockIdx.x];
    for (int i = lane; i < 2 * P3; i += 32)
        acc[i] = 0.f;
    const int pk = base[it.x];
    const int ox = (b3x(pk) / cell) * cell - (m - 1), oy = (b3y(pk) / cell) * cell - (m - 1),
              oz = (b3z(pk) / cell) * cell - (m - 1);
    const int dim = lane / M2, jw = lane - (lane / M2) * M2;
    float pc[kPolyD + 1];   // this lane's window polynomial
#pragma unroll
    for (int k = 0; k <= kPolyD; ++k)
        pc[k] = wp.c[lane < 3 * M2 ? jw : 0][k];
    __syncwarp();
    // software pipeline: the next source's record is in flight while this one is spread
    const int end = it.x + it.y;
    int j = it.x + warp;
    int nb = 0;
    float nf = 0.f, nq = 0.f;
    if (j < end) {
        nb = base[j];
        nf = lane < 3 * M2 ? frac[3 * j + dim] : 0.f;
        nq = q[j];
    }
    for (; j < end; j += kSpread3Warps) {
        const int packed = nb;
        const float fr = nf, qj = nq;
        if (j + kSpread3Warps < end) {
            nb = base[j + kSpread3Warps];
            nf = lane < 3 * M2 ? frac[3 * (j + kSpread3Warps) + dim] : 0.f;
            nq = q[j + kSpread3Warps];
        }
        float wv = 0.f;
        if (lane < 3 * M2) {
            wv = poly_eval<kPolyD>(pc, fr - 0.5f);
            if (dim == 0)
                wv *= qj;
        }
        const int lx = b3x(packed) - m + 1 - ox, ly = b3y(packed) - m + 1 - oy, lz = b3z(packed) - m + 1 - oz;
        float v[PER];
        int idx[PER];
        bool on[PER];
        if constexpr (M2 == 8) {
            const float vx = __shfl_sync(0xffffffffu, wv, lane & 7);
            const float vxy0 = vx * __shfl_sync(0xffffffffu, wv, 8 + (lane >> 3));
            const float vxy1 = vx * __shfl_sync(0xffffffffu, wv, 12 + (lane >> 3));
            const int row = (lz * P + ly + (lane >> 3)) * P + lx + (lane & 7);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = ((i & 1) ? vxy1 : vxy0) * __shfl_sync(0xffffffffu, wv, 16 + (i >> 1));
                idx[i] = row + ((i >> 1) * P + 4 * (i & 1)) * P;
                on[i] = true;
            }
        } else {
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int t = lane + 32 * i;
                const int tx = t % M2, ty = (t / M2) % M2, tz = t / (M2 * M2);
                const float vx = __shfl_sync(0xffffffffu, wv, tx);
                const float vy = __shfl_sync(0xffffffffu, wv, M2 + ty);
                const float vz = __shfl_sync(0xffffffffu, wv, 2 * M2 + (tz < M2 ? tz : 0));
                v[i] = vx * vy * vz;
                idx[i] = ((lz + tz) * P + (ly + ty)) * P + (lx + tx);
                on[i] = t < TAPS;
            }
        }
        // a source's taps are distinct cells: all reads before the writes
        float old[PER], cmp[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (on[i]) {
                old[i] = acc[idx[i]];
                cmp[i] = acc[P3 + idx[i]];
            }
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (on[i]) {
                const float s = old[i] + v[i];
                const float bb = s - old[i];
                acc[idx[i]] = s;
                acc[P3 + idx[i]] = cmp[i] + ((old[i] - (s - bb)) + (v[i] - bb));
            }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P3; i += blockDim.x) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kSpread3Warps; ++w)
            v += tiles[(size_t)w * 2 * P3 + i] + tiles[(size_t)w * 2 * P3 + P3 + i];
        const int x = i % P, y = (i / P) % P, z = i / (P * P);
        const int gx = ox + x, gy = oy + y, gz = oz + z;
        if (v != 0.f && gx >= 0 && gx < n_a && gy >= 0 && gy < n_a && gz >= 0 && gz < n_a)
            atomicAdd(grid + ((int64_t)gz * n_a + gy) * n_a + gx, v);
    }
}

// phi~ and grad~ phi~ at the targets from the filtered grid (thread per target).
template <typename real, int M2>
__global__ void __launch_bounds__(256) k_interp3(int64_t N, const int *__restrict__ base, const real *__restrict__ frac,
                                                 Window<real> w, WindowPoly wp, const real *__restrict__ grid, int n_a,
                                                 real n_os, real *__restrict__ phi_s, real *__restrict__ grad_s,
                                                 bool acc)
{
    constexpr int m = M2 / 2;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    real wt[3][M2], dt[3][M2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const real fr = frac[3 * k + d];
#pragma unroll
        for (int a = 0; a < M2; ++a) {
            if constexpr (sizeof(real) == 4) {
                wt[d][a] = poly_eval<kPolyD>(wp.c[a], (float)fr - 0.5f);
                dt[d][a] = poly_eval<kPolyD - 1>(wp.d[a], (float)fr - 0.5f);
            } else {
                kb_value_slope<real>(w, fr, m - 1 - a, wt[d][a], dt[d][a]);
            }
        }
    }
    const int packed = base[k];
    const int x0 = b3x(packed) - m + 1, y0 = b3y(packed) - m + 1, z0 = b3z(packed) - m + 1;
    real phi = 0, gx = 0, gy = 0, gz = 0;
    for (int c = 0; c < M2; ++c) {
        real t = 0, tx = 0, ty = 0;
        for (int b = 0; b < M2; ++b) {
            const real *row = grid + ((int64_t)(z0 + c) * n_a + (y0 + b)) * n_a + x0;
            real s = 0, sx = 0;
#pragma unroll
            for (int a = 0; a < M2; ++a) {
                const real g = __ldg(row + a);
                s += wt[0][a] * g;
                sx += dt[0][a] * g;
            }
            t += wt[1][b] * s;
            tx += wt[1][b] * sx;
            ty += dt[1][b] * s;
        }
        phi += wt[2][c] * t;
        gx += wt[2][c] * tx;
        gy += wt[2][c] * ty;
        gz += dt[2][c] * t;
    }
    // acc: the near field was stored first (it ran beside spreading and the transform)
    phi_s[k] = acc ? phi_s[k] + phi : phi;
    grad_s[3 * k] = acc ? grad_s[3 * k] + n_os * gx : n_os * gx;
    grad_s[3 * k + 1] = acc ? grad_s[3 * k + 1] + n_os * gy : n_os * gy;
    grad_s[3 * k + 2] = acc ? grad_s[3 * k + 2] + n_os * gz : n_os * gz;
}

// FP64 near-field correction at target k (thread per target) over the 27 cells around its cell.
__global__ void __launch_bounds__(256) k_near3_f64(int64_t N, const int *__restrict__ tgt_base,
                                                   const double *__restrict__ tgt_pos,
                                                   const double *__restrict__ src_pos,
                                                   const int *__restrict__ src_start, CellGrid3 cg,
                                                   const double *__restrict__ q, NearParams<double> np,
                                                   double *__restrict__ phi_s, double *__restrict__ grad_s)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int packed = tgt_base[k];
    const int c1 = b3x(packed) / cg.cell, c2 = b3y(packed) / cg.cell, c3 = b3z(packed) / cg.cell;
    const double xt0 = tgt_pos[3 * k], xt1 = tgt_pos[3 * k + 1], xt2 = tgt_pos[3 * k + 2];
    const double inv4pi = 1.0 / (4.0 * kPi);
    const int S3 = cg.sub3();
    double phi = 0, g0 = 0, g1 = 0, g2 = 0;
    for (int e1 = max(c1 - 1, 0); e1 <= min(c1 + 1, cg.n_c - 1); ++e1)
        for (int e2 = max(c2 - 1, 0); e2 <= min(c2 + 1, cg.n_c - 1); ++e2)
            for (int e3 = max(c3 - 1, 0); e3 <= min(c3 + 1, cg.n_c - 1); ++e3) {
                const int key = cg.key(e1, e2, e3);
                const int end = src_start[(key + 1) * S3];
                for (int j = src_start[key * S3]; j < end; ++j) {
                    const double dx = xt0 - src_pos[3 * j];
                    const double dy = xt1 - src_pos[3 * j + 1];
                    const double dz = xt2 - src_pos[3 * j + 2];
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 < np.eps2))
                        continue;
                    const double qj = q[j];
                    if (r2 == 0.0) {
                        phi -= qj * np.beta[0];
                        continue;
                    }
                    const double u2 = r2 * np.inv_eps2;
                    double t = np.beta[np.p - 1];
                    for (int i = np.p - 2; i >= 0; --i)
                        t = t * u2 + np.beta[i];
                    double tp = 0.0;
                    if (np.p > 1) {
                        tp = np.dbeta[np.p - 2];
                        for (int i = np.p - 3; i >= 0; --i)
                            tp = tp * u2 + np.dbeta[i];
                    }
                    const double inv_r = 1.0 / sqrt(r2);
                    const double val = inv4pi * inv_r - t;
                    const double coef = -inv4pi * inv_r * inv_r * inv_r - tp;
                    phi += qj * val;
                    g0 += qj * coef * dx;
                    g1 += qj * coef * dy;
                    g2 += qj * coef * dz;
                }
            }
    phi_s[k] += phi;
    grad_s[3 * k] += g0;
    grad_s[3 * k + 1] += g1;
    grad_s[3 * k + 2] += g2;
}

// ---- FP32 near field: warp items, candidate lists, packed pairs
//
// A warp takes one item, at most 64 consecutive targets of one cell (two per lane; Morton
// sub-cell order keeps them compact) and forms their bounding box.  Coordinates are offsets
// from the target cell's corner in units of eps_I.  For each of the 27 cells around (skipping
// cells beyond the culling radius of the box), the lanes read 32 sources at a time, keep those
// within the culling radius of the box (ballot) and append them to the warp's candidate list
// in shared memory, pre-broadcast as (x, x, y, y), (z, z, q, q).  The list is evaluated by
// all lanes against both of their targets as packed FP32 pairs: no branch, pairs outside
// 0 < w < 1 get charge 0 (an integer compare of the bits of w: 0 < w < 1 iff
// bits(w) - 1 < bits(1) - 1 as unsigned), and coincident pairs (w = 0) are accounted from the
// per-target lists built with the plan.  Sources within eps_I / 8 of the box go to a second
// list, whose pairs closer than eps_I / 8 take their difference from the FP64 positions.
constexpr int kNear3Warps = 4;
constexpr int kNear3Cap = 256;        // far candidate entries per warp (32 B each)
constexpr int kNear3CloseCap = 64;    // close candidate entries per warp (32 B + index)
constexpr int kNear3Unroll = 2;

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// q if 0 < w < 1, else 0
__device__ __forceinline__ float in_range(float w, float q)
{
    return (__float_as_uint(w) - 1u) < 0x3f7fffffu ? q : 0.f;
}

// The packed pair arithmetic for one candidate at (w, dx, dy, dz) (units of eps_I).
template <int P>
__device__ __forceinline__ void near3_pair(const Near3Params &np, float2 w, float2 dx, float2 dy, float2 dz,
                                           float2 qq, float2 &phi, float2 &gx, float2 &gy, float2 &gz)
{
    const float2 c1 = make_float2(np.c1, np.c1);
    const float2 qe = make_float2(in_range(w.x, qq.x), in_range(w.y, qq.y));
    // w = 0 only for coincident pairs (charge 0 here): floor w so that w^-3/2 stays finite
    // (distinct points give w >= ~1e-14, far above the floor)
    const float2 rs = make_float2(rsqrt_approx(fmaxf(w.x, 1e-20f)), rsqrt_approx(fmaxf(w.y, 1e-20f)));
    float2 t = make_float2(np.nbeta[P - 1], np.nbeta[P - 1]);
#pragma unroll
    for (int i = P - 2; i >= 0; --i)
        t = __ffma2_rn(t, w, make_float2(np.nbeta[i], np.nbeta[i]));
    float2 u = make_float2(0.f, 0.f);
    if constexpr (P >= 2) {
        u = make_float2(np.dbeta2[P - 2], np.dbeta2[P - 2]);
#pragma unroll
        for (int i = P - 3; i >= 0; --i)
            u = __ffma2_rn(u, w, make_float2(np.dbeta2[i], np.dbeta2[i]));
    }
    const float2 val = __ffma2_rn(c1, rs, t);                                  // c1 w^-1/2 - P(w)
    const float2 gc = __ffma2_rn(c1, __fmul2_rn(__fmul2_rn(rs, rs), rs), u);   // c1 w^-3/2 + 2 P'(w)
    phi = __ffma2_rn(qe, val, phi);
    const float2 qc = __fmul2_rn(qe, gc);
    gx = __ffma2_rn(qc, dx, gx);
    gy = __ffma2_rn(qc, dy, gy);
    gz = __ffma2_rn(qc, dz, gz);
}

// Far candidates: no pair can be closer than eps_I / 8.
template <int P>
__device__ __forceinline__ void near3_eval(const float4 (*list)[2], int n, float2 X, float2 Y, float2 Z,
                                           const Near3Params &np, float2 &phi, float2 &gx, float2 &gy, float2 &gz)
{
#pragma unroll kNear3Unroll
    for (int e = 0; e < n; ++e) {
        const float4 A = list[e][0], B = list[e][1];
        const float2 dx = __fadd2_rn(X, make_float2(-A.x, -A.y));
        const float2 dy = __fadd2_rn(Y, make_float2(-A.z, -A.w));
        const float2 dz = __fadd2_rn(Z, make_float2(-B.x, -B.y));
        const float2 w = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        near3_pair<P>(np, w, dx, dy, dz, make_float2(B.z, B.w), phi, gx, gy, gz);
    }
}

// Close candidates (within eps_I / 8 of the box): pairs closer than eps_I / 8 take their
// difference from the FP64 positions (the FP32 cell offsets lose relative precision as r
// shrinks, and such pairs dominate H), then the same arithmetic.
template <int P>
__device__ __forceinline__ void near3_eval_close(const float4 (*list)[2], const int *jlist, int n, float2 X,
                                                 float2 Y, float2 Z, const int (&kt)[2],
                                                 const double *__restrict__ tgt_pos,
                                                 const double *__restrict__ src_pos, const Near3Params &np,
                                                 float2 &phi, float2 &gx, float2 &gy, float2 &gz)
{
    for (int e = 0; e < n; ++e) {
        const float4 A = list[e][0], B = list[e][1];
        float2 dx = __fadd2_rn(X, make_float2(-A.x, -A.y));
        float2 dy = __fadd2_rn(Y, make_float2(-A.z, -A.w));
        float2 dz = __fadd2_rn(Z, make_float2(-B.x, -B.y));
        float2 w = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const bool c0 = w.x < 1.f / 64.f, c1 = w.y < 1.f / 64.f;
        if (__any_sync(0xffffffffu, c0 || c1)) {
            const int j = jlist[e];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (t == 0 ? c0 : c1) {
                    const int64_t k = kt[t];
                    const float ex = (float)((tgt_pos[3 * k] - src_pos[3 * (int64_t)j]) * np.inv_eps_d);
                    const float ey = (float)((tgt_pos[3 * k + 1] - src_pos[3 * (int64_t)j + 1]) * np.inv_eps_d);
                    const float ez = (float)((tgt_pos[3 * k + 2] - src_pos[3 * (int64_t)j + 2]) * np.inv_eps_d);
                    const float e2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                    if (t == 0) {
                        dx.x = ex;
                        dy.x = ey;
                        dz.x = ez;
                        w.x = e2;
                    } else {
                        dx.y = ex;
                        dy.y = ey;
                        dz.y = ez;
                        w.y = e2;
                    }
                }
            }
        }
        near3_pair<P>(np, w, dx, dy, dz, make_float2(B.z, B.w), phi, gx, gy, gz);
    }
}

template <int P>
__global__ void __launch_bounds__(kNear3Warps * 32) k_near3_warp(const int2 *__restrict__ items, int n_items,
                                                                 const int *__restrict__ tgt_base,
                                                                 const float4 *__restrict__ tgt_p32,
                                                                 const float4 *__restrict__ src_p32,
                                                                 const double *__restrict__ tgt_pos,
                                                                 const double *__restrict__ src_pos,
                                                                 const float *__restrict__ q,
                                                                 const int *__restrict__ src_start, CellGrid3 cg,
                                                                 Near3Params np, const int *__restrict__ coinc_start,
                                                                 const int *__restrict__ coinc_src,
                                                                 float *__restrict__ phi_s, float *__restrict__ grad_s,
                                                                 bool assign)
{
    __shared__ float4 lists[kNear3Warps][kNear3Cap][2];
    __shared__ float4 clists[kNear3Warps][kNear3CloseCap][2];
    __shared__ int cjs[kNear3Warps][kNear3CloseCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = blockIdx.x * kNear3Warps + warp;
    if (item >= n_items)
        return;   // whole warp; the kernel has no block-wide barrier
    float4(*list)[2] = lists[warp];
    float4(*clist)[2] = clists[warp];
    int *cj = cjs[warp];
    const int2 it = items[item];
    const int first = it.x, count = it.y;
    const bool va = lane < count, vb = lane + 32 < count;
    const int ka = va ? first + lane : first, kb = vb ? first + 32 + lane : ka;
    const float4 pa = tgt_p32[ka], pb = tgt_p32[kb];
    const float2 X = make_float2(pa.x, pb.x), Y = make_float2(pa.y, pb.y), Z = make_float2(pa.z, pb.z);
    const int kt[2] = {ka, kb};
    const float lox = warp_min(fminf(pa.x, pb.x)), hix = warp_max(fmaxf(pa.x, pb.x));
    const float loy = warp_min(fminf(pa.y, pb.y)), hiy = warp_max(fmaxf(pa.y, pb.y));
    const float loz = warp_min(fminf(pa.z, pb.z)), hiz = warp_max(fmaxf(pa.z, pb.z));
    const int packed = tgt_base[first];
    const int c1 = b3x(packed) / cg.cell, c2 = b3y(packed) / cg.cell, c3 = b3z(packed) / cg.cell;
    const int S3 = cg.sub3();
    float2 phi = make_float2(0.f, 0.f), gx = phi, gy = phi, gz = phi;
    int n = 0, nc = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int e1 = max(c1 - 1, 0); e1 <= min(c1 + 1, cg.n_c - 1); ++e1) {
        const float o1 = (float)(e1 - c1) * np.H;
        const float bx = fmaxf(0.f, fmaxf(o1 - hix, lox - (o1 + np.H)));
        for (int e2 = max(c2 - 1, 0); e2 <= min(c2 + 1, cg.n_c - 1); ++e2) {
            const float o2 = (float)(e2 - c2) * np.H;
            const float by = fmaxf(0.f, fmaxf(o2 - hiy, loy - (o2 + np.H)));
            for (int e3 = max(c3 - 1, 0); e3 <= min(c3 + 1, cg.n_c - 1); ++e3) {
                const float o3 = (float)(e3 - c3) * np.H;
                const float bz = fmaxf(0.f, fmaxf(o3 - hiz, loz - (o3 + np.H)));
                if (bx * bx + by * by + bz * bz >= np.reach2)
                    continue;   // the whole cell is beyond reach of the box (warp-uniform)
                const int key = cg.key(e1, e2, e3);
                const int end = src_start[(key + 1) * S3];
                for (int j0 = src_start[key * S3]; j0 < end; j0 += 32) {
                    const int j = j0 + lane;
                    bool keep = false, close = false;
                    float sx = 0.f, sy = 0.f, sz = 0.f, qj = 0.f;
                    if (j < end) {
                        const float4 sp = src_p32[j];
                        qj = q[j];
                        sx = sp.x + o1;
                        sy = sp.y + o2;
                        sz = sp.z + o3;
                        const float dx = fmaxf(0.f, fmaxf(sx - hix, lox - sx));
                        const float dy = fmaxf(0.f, fmaxf(sy - hiy, loy - sy));
                        const float dz = fmaxf(0.f, fmaxf(sz - hiz, loz - sz));
                        const float g2 = dx * dx + dy * dy + dz * dz;
                        keep = g2 < np.reach2;
                        close = g2 < np.close_reach2;
                    }
                    const unsigned mf = __ballot_sync(0xffffffffu, keep && !close);
                    const unsigned mc = __ballot_sync(0xffffffffu, close);
                    if (keep && !close) {
                        const int at = n + __popc(mf & below);
                        list[at][0] = make_float4(sx, sx, sy, sy);
                        list[at][1] = make_float4(sz, sz, qj, qj);
                    }
                    if (close) {
                        const int at = nc + __popc(mc & below);
                        clist[at][0] = make_float4(sx, sx, sy, sy);
                        clist[at][1] = make_float4(sz, sz, qj, qj);
                        cj[at] = j;
                    }
                    n += __popc(mf);
                    nc += __popc(mc);
                    if (n > kNear3Cap - 32) {
                        __syncwarp();
                        near3_eval<P>(list, n, X, Y, Z, np, phi, gx, gy, gz);
                        n = 0;
                        __syncwarp();
                    }
                    if (nc > kNear3CloseCap - 32) {
                        __syncwarp();
                        near3_eval_close<P>(clist, cj, nc, X, Y, Z, kt, tgt_pos, src_pos, np, phi, gx, gy, gz);
                        nc = 0;
                        __syncwarp();
                    }
                }
            }
        }
    }
    __syncwarp();
    near3_eval<P>(list, n, X, Y, Z, np, phi, gx, gy, gz);
    near3_eval_close<P>(clist, cj, nc, X, Y, Z, kt, tgt_pos, src_pos, np, phi, gx, gy, gz);
    // coincident pairs: G(0) := 0, so only -q T_I(0) remains of the far field's self term
    const bool vt[2] = {va, vb};
    const float ph[2] = {phi.x, phi.y}, ggx[2] = {gx.x, gx.y}, ggy[2] = {gy.x, gy.y}, ggz[2] = {gz.x, gz.y};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (!vt[t])
            continue;
        const int k = kt[t];
        float self = 0.f;
        for (int c = coinc_start[k]; c < coinc_start[k + 1]; ++c)
            self += q[coinc_src[c]];
        const float p0 = assign ? 0.f : phi_s[k];
        phi_s[k] = p0 + (ph[t] - np.beta0 * self);
        grad_s[3 * k] = (assign ? 0.f : grad_s[3 * k]) - np.inv_eps * ggx[t];
        grad_s[3 * k + 1] = (assign ? 0.f : grad_s[3 * k + 1]) - np.inv_eps * ggy[t];
        grad_s[3 * k + 2] = (assign ? 0.f : grad_s[3 * k + 2]) - np.inv_eps * ggz[t];
    }
}

// ---- FP32 near field, source-major (plans with many more sources than targets: FEM meshes,
// where every node meets the quadrature points of several elements)
//
// Target items hold only the few targets of a cell, so their box is the whole cell and most
// candidates lie beyond eps_I of most targets.  Here a warp takes an item of at most 64 sources
// of one cell (compact: Morton sub-cell order) and keeps them in shared memory as packed pairs;
// it reads the targets of the 27 cells around 32 at a time, keeps those within eps_I of the
// sources' box (ballot) in a list (those within eps_I / 8 of the box in a second one), and
// each lane then takes one listed target and sums the item's sources on it, two per packed
// operation, adding phi and grad phi to the target with atomics.  Pairs closer than eps_I / 8
// take their difference from the FP64 positions, as in k_near3_warp; coincident pairs are
// removed by k_coincident3_apply.
constexpr int kSrcListCap = 128;

template <int P, bool CLOSE>
__device__ __forceinline__ void near3_src_eval(const float4 (*spairs)[2], const float4 *tlist, int n, int first,
                                               int count, float dummy, const double *__restrict__ tgt_pos,
                                               const double *__restrict__ src_pos, const Near3Params &np,
                                               float *__restrict__ phi_s, float *__restrict__ grad_s, int lane)
{
    for (int base = 0; base < n; base += 32) {
        const int e = base + lane;
        const bool valid = e < n;
        const float4 T = valid ? tlist[e] : make_float4(dummy, dummy, dummy, 0.f);
        const int k = __float_as_int(T.w);
        const float2 X = make_float2(T.x, T.x), Y = make_float2(T.y, T.y), Z = make_float2(T.z, T.z);
        float2 phi = make_float2(0.f, 0.f), gx = phi, gy = phi, gz = phi;
#pragma unroll 2
        for (int i = 0; i < 32; ++i) {
            const float4 A = spairs[i][0], B = spairs[i][1];   // (xa, xb, ya, yb), (za, zb, qa, qb)
            float2 dx = __fadd2_rn(X, make_float2(-A.x, -A.y));
            float2 dy = __fadd2_rn(Y, make_float2(-A.z, -A.w));
            float2 dz = __fadd2_rn(Z, make_float2(-B.x, -B.y));
            float2 w = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            if constexpr (CLOSE) {
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    // (idle source slots, i + 32 t >= count, carry charge 0 and are not refined)
                    if (valid && i + 32 * t < count && (t == 0 ? w.x : w.y) < 1.f / 64.f) {
                        const int64_t j = first + i + 32 * t;
                        const float ex = (float)((tgt_pos[3 * (int64_t)k] - src_pos[3 * j]) * np.inv_eps_d);
                        const float ey = (float)((tgt_pos[3 * (int64_t)k + 1] - src_pos[3 * j + 1]) * np.inv_eps_d);
                        const float ez = (float)((tgt_pos[3 * (int64_t)k + 2] - src_pos[3 * j + 2]) * np.inv_eps_d);
                        const float e2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                        if (t == 0) {
                            dx.x = ex;
                            dy.x = ey;
                            dz.x = ez;
                            w.x = e2;
                        } else {
                            dx.y = ex;
                            dy.y = ey;
                            dz.y = ez;
                            w.y = e2;
                        }
                    }
                }
            }
            near3_pair<P>(np, w, dx, dy, dz, make_float2(B.z, B.w), phi, gx, gy, gz);
        }
        if (valid) {
            atomicAdd(phi_s + k, phi.x + phi.y);
            atomicAdd(grad_s + 3 * (int64_t)k, -np.inv_eps * (gx.x + gx.y));
            atomicAdd(grad_s + 3 * (int64_t)k + 1, -np.inv_eps * (gy.x + gy.y));
            atomicAdd(grad_s + 3 * (int64_t)k + 2, -np.inv_eps * (gz.x + gz.y));
        }
    }
}

template <int P>
__global__ void __launch_bounds__(kNear3Warps * 32) k_near3_src(const int2 *__restrict__ items, int n_items,
                                                                const int *__restrict__ src_base,
                                                                const float4 *__restrict__ src_p32,
                                                                const float4 *__restrict__ tgt_p32,
                                                                const double *__restrict__ tgt_pos,
                                                                const double *__restrict__ src_pos,
                                                                const float *__restrict__ q,
                                                                const int *__restrict__ tgt_start, CellGrid3 cg,
                                                                Near3Params np, float *__restrict__ phi_s,
                                                                float *__restrict__ grad_s)
{
    __shared__ float4 spairs_all[kNear3Warps][32][2];
    __shared__ float4 flist_all[kNear3Warps][kSrcListCap];
    __shared__ float4 clist_all[kNear3Warps][kSrcListCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = blockIdx.x * kNear3Warps + warp;
    if (item >= n_items)
        return;   // whole warp; the kernel has no block-wide barrier
    float4(*spairs)[2] = spairs_all[warp];
    float4 *flist = flist_all[warp], *clist = clist_all[warp];
    const int2 it = items[item];
    const int first = it.x, count = it.y;
    const bool va = lane < count, vb = lane + 32 < count;
    const float4 pa = src_p32[va ? first + lane : first], pb = src_p32[vb ? first + 32 + lane : first];
    spairs[lane][0] = make_float4(pa.x, pb.x, pa.y, pb.y);
    spairs[lane][1] = make_float4(pa.z, pb.z, va ? q[first + lane] : 0.f, vb ? q[first + 32 + lane] : 0.f);
    const float lox = warp_min(fminf(pa.x, pb.x)), hix = warp_max(fmaxf(pa.x, pb.x));
    const float loy = warp_min(fminf(pa.y, pb.y)), hiy = warp_max(fmaxf(pa.y, pb.y));
    const float loz = warp_min(fminf(pa.z, pb.z)), hiz = warp_max(fmaxf(pa.z, pb.z));
    const float dummy = fminf(lox, fminf(loy, loz)) - 3.f;   // idle lanes: every pair beyond eps_I
    __syncwarp();
    const int packed = src_base[first];
    const int c1 = b3x(packed) / cg.cell, c2 = b3y(packed) / cg.cell, c3 = b3z(packed) / cg.cell;
    const int S3 = cg.sub3();
    const unsigned below = (1u << lane) - 1u;
    int nf = 0, nc = 0;
    for (int e1 = max(c1 - 1, 0); e1 <= min(c1 + 1, cg.n_c - 1); ++e1) {
        const float o1 = (float)(e1 - c1) * np.H;
        const float bx = fmaxf(0.f, fmaxf(o1 - hix, lox - (o1 + np.H)));
        for (int e2 = max(c2 - 1, 0); e2 <= min(c2 + 1, cg.n_c - 1); ++e2) {
            const float o2 = (float)(e2 - c2) * np.H;
            const float by = fmaxf(0.f, fmaxf(o2 - hiy, loy - (o2 + np.H)));
            for (int e3 = max(c3 - 1, 0); e3 <= min(c3 + 1, cg.n_c - 1); ++e3) {
                const float o3 = (float)(e3 - c3) * np.H;
                const float bz = fmaxf(0.f, fmaxf(o3 - hiz, loz - (o3 + np.H)));
                if (bx * bx + by * by + bz * bz >= np.reach2)
                    continue;
                const int key = cg.key(e1, e2, e3);
                const int end = tgt_start[(key + 1) * S3];
                for (int j0 = tgt_start[key * S3]; j0 < end; j0 += 32) {
                    const int j = j0 + lane;
                    bool keep = false, close = false;
                    float tx = 0.f, ty = 0.f, tz = 0.f;
                    if (j < end) {
                        const float4 tp = tgt_p32[j];
                        tx = tp.x + o1;
                        ty = tp.y + o2;
                        tz = tp.z + o3;
                        const float dx = fmaxf(0.f, fmaxf(tx - hix, lox - tx));
                        const float dy = fmaxf(0.f, fmaxf(ty - hiy, loy - ty));
                        const float dz = fmaxf(0.f, fmaxf(tz - hiz, loz - tz));
                        const float g2 = dx * dx + dy * dy + dz * dz;
                        keep = g2 < np.reach2;
                        close = g2 < np.close_reach2;
                    }
                    const unsigned mf = __ballot_sync(0xffffffffu, keep && !close);
                    const unsigned mc = __ballot_sync(0xffffffffu, close);
                    if (keep && !close)
                        flist[nf + __popc(mf & below)] = make_float4(tx, ty, tz, __int_as_float(j));
                    if (close)
                        clist[nc + __popc(mc & below)] = make_float4(tx, ty, tz, __int_as_float(j));
                    nf += __popc(mf);
                    nc += __popc(mc);
                    if (nf > kSrcListCap - 32) {
                        __syncwarp();
                        near3_src_eval<P, false>(spairs, flist, nf, first, count, dummy, tgt_pos, src_pos, np, phi_s, grad_s,
                                                 lane);
                        nf = 0;
                        __syncwarp();
                    }
                    if (nc > kSrcListCap - 32) {
                        __syncwarp();
                        near3_src_eval<P, true>(spairs, clist, nc, first, count, dummy, tgt_pos, src_pos, np, phi_s, grad_s,
                                                lane);
                        nc = 0;
                        __syncwarp();
                    }
                }
            }
        }
    }
    __syncwarp();
    near3_src_eval<P, false>(spairs, flist, nf, first, count, dummy, tgt_pos, src_pos, np, phi_s, grad_s, lane);
    near3_src_eval<P, true>(spairs, clist, nc, first, count, dummy, tgt_pos, src_pos, np, phi_s, grad_s, lane);
}

// Coincident pairs for the source-major kernel: phi -= T_I(0) (sum of the coincident charges).
__global__ void k_coincident3_apply(int64_t N, const int *__restrict__ coinc_start, const int *__restrict__ coinc_src,
                                    const float *__restrict__ q, float beta0, float *__restrict__ phi_s)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    float self = 0.f;
    for (int c = coinc_start[k]; c < coinc_start[k + 1]; ++c)
        self += q[coinc_src[c]];
    if (self != 0.f)
        phi_s[k] -= beta0 * self;
}

// Coincident pairs: sources of the target's own cell at the same (FP64) position.
__global__ void k_coincident3(int64_t N, const int *__restrict__ tgt_base, const double *__restrict__ tgt_pos,
                              const double *__restrict__ src_pos, const int *__restrict__ src_start, CellGrid3 cg,
                              int *__restrict__ count, const int *__restrict__ coinc_start, int *__restrict__ coinc_src)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int packed = tgt_base[k];
    const int key = cg.key(b3x(packed) / cg.cell, b3y(packed) / cg.cell, b3z(packed) / cg.cell);
    const double tx = tgt_pos[3 * k], ty = tgt_pos[3 * k + 1], tz = tgt_pos[3 * k + 2];
    const int S3 = cg.sub3();
    int c = 0, at = coinc_src ? coinc_start[k] : 0;
    for (int j = src_start[key * S3]; j < src_start[(key + 1) * S3]; ++j) {
        if (src_pos[3 * (int64_t)j] == tx && src_pos[3 * (int64_t)j + 1] == ty && src_pos[3 * (int64_t)j + 2] == tz) {
            if (coinc_src)
                coinc_src[at++] = j;
            ++c;
        }
    }
    if (!coinc_src)
        count[k] = c;
}

template <typename real>
__global__ void k_unpermute3(int64_t N, const real *__restrict__ phi_s, const real *__restrict__ grad_s,
                             const int *__restrict__ perm, double s, void *__restrict__ phi_out,
                             void *__restrict__ H_out, int out_f64)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int64_t i = perm[k];
    const double phi = s * (double)phi_s[k];
    const double s2 = -s * s;
    if (out_f64) {
        if (phi_out)
            ((double *)phi_out)[i] = phi;
        if (H_out)
            for (int d = 0; d < 3; ++d)
                ((double *)H_out)[3 * i + d] = s2 * (double)grad_s[3 * k + d];
    } else {
        if (phi_out)
            ((float *)phi_out)[i] = (float)phi;
        if (H_out)
            for (int d = 0; d < 3; ++d)
                ((float *)H_out)[3 * i + d] = (float)(s2 * (double)grad_s[3 * k + d]);
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class F> cudaError_t with_width3(int m, F &&f)
{
    switch (m) {
    case 2: return f(std::integral_constant<int, 4>{});
    case 3: return f(std::integral_constant<int, 6>{});
    case 4: return f(std::integral_constant<int, 8>{});
    case 5: return f(std::integral_constant<int, 10>{});
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_rmax3(const double *xyz, int64_t n, unsigned long long *out, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    unsigned b = nblk(n, 256);
    if (b > 1024)
        b = 1024;
    k_rmax3<<<b, 256, 0, st>>>(xyz, n, out);
    return cudaGetLastError();
}

cudaError_t launch_point_keys3(const double *xyz, int64_t n, double s, int n_os, int window_lo, int n_a, int m,
                               CellGrid3 cg, int *key, int *count, int *status, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_point_keys3<<<nblk(n, 256), 256, 0, st>>>(xyz, n, s, n_os, window_lo, n_a, m, cg, key, count, status);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gather_points3(const double *xyz, const int *perm, int64_t n, double s, int n_os, int window_lo,
                                  int n_a, int m, int cell, double inv_eps, double *pos, real *frac, int *base,
                                  float4 *pos32, int *status, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_gather_points3<real><<<nblk(n, 256), 256, 0, st>>>(xyz, perm, n, s, n_os, window_lo, n_a, m, cell, inv_eps, pos,
                                                        frac, base, pos32, status);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_spread3(int64_t M, int m, const int *base, const real *frac, const real *q, Window<real> w,
                           const WindowPoly &wp, real *grid, int n_a, cudaStream_t st)
{
    if (M <= 0)
        return cudaSuccess;
    return with_width3(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        int64_t blocks = (M + 7) / 8;   // eight warps (sources) per block, then grid-stride
        if (blocks > 152 * 16)
            blocks = 152 * 16;
        k_spread3<real, M2><<<(unsigned)blocks, 256, 0, st>>>(M, base, frac, q, w, wp, grid, n_a);
        return cudaGetLastError();
    });
}

// Shared memory of the tiled FP32 spreading (0 when the tiles do not fit: use k_spread3).
size_t spread3_tile_smem(int cell, int m)
{
    const size_t P = (size_t)cell + 2 * m - 1;
    const size_t bytes = (size_t)kSpread3Warps * 2 * P * P * P * sizeof(float);
    return bytes <= 112 * 1024 ? bytes : 0;
}

cudaError_t launch_spread3_tile(const int2 *items, int n_items, int m, int cell, const int *base, const float *frac,
                                const float *q, const WindowPoly &wp, float *grid, int n_a, cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    const size_t smem = spread3_tile_smem(cell, m);
    if (smem == 0)
        return cudaErrorInvalidValue;
    return with_width3(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        cudaError_t e = cudaFuncSetAttribute(k_spread3_tile<M2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        k_spread3_tile<M2><<<(unsigned)n_items, kSpread3Warps * 32, smem, st>>>(items, base, frac, q, wp, cell, grid,
                                                                                n_a);
        return cudaGetLastError();
    });
}

template <typename real>
cudaError_t launch_interp3(int64_t N, int m, const int *base, const real *frac, Window<real> w, const WindowPoly &wp,
                           const real *grid, int n_a, real n_os, real *phi_s, real *grad_s, bool acc,
                           cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    return with_width3(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        k_interp3<real, M2><<<nblk(N, 256), 256, 0, st>>>(N, base, frac, w, wp, grid, n_a, n_os, phi_s, grad_s, acc);
        return cudaGetLastError();
    });
}

cudaError_t launch_near3_f64(int64_t N, const int *tgt_base, const double *tgt_pos, const double *src_pos,
                             const int *src_start, CellGrid3 cg, const double *q, NearParams<double> np,
                             double *phi_s, double *grad_s, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near3_f64<<<nblk(N, 256), 256, 0, st>>>(N, tgt_base, tgt_pos, src_pos, src_start, cg, q, np, phi_s, grad_s);
    return cudaGetLastError();
}

cudaError_t launch_near3_warp(const int2 *items, int n_items, const int *tgt_base, const float4 *tgt_p32,
                              const float4 *src_p32, const double *tgt_pos, const double *src_pos, const float *q,
                              const int *src_start, CellGrid3 cg, const Near3Params &np, const int *coinc_start,
                              const int *coinc_src, float *phi_s, float *grad_s, bool assign, cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    const unsigned blocks = (unsigned)((n_items + kNear3Warps - 1) / kNear3Warps);
    return with_degree(np.p, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        k_near3_warp<P><<<blocks, kNear3Warps * 32, 0, st>>>(items, n_items, tgt_base, tgt_p32, src_p32, tgt_pos,
                                                              src_pos, q, src_start, cg, np, coinc_start, coinc_src,
                                                              phi_s, grad_s, assign);
        return cudaGetLastError();
    });
}

cudaError_t launch_near3_src(const int2 *items, int n_items, const int *src_base, const float4 *src_p32,
                             const float4 *tgt_p32, const double *tgt_pos, const double *src_pos, const float *q,
                             const int *tgt_start, CellGrid3 cg, const Near3Params &np, int64_t N,
                             const int *coinc_start, const int *coinc_src, bool any_coincident, float *phi_s,
                             float *grad_s, cudaStream_t st)
{
    if (n_items > 0) {
        const unsigned blocks = (unsigned)((n_items + kNear3Warps - 1) / kNear3Warps);
        cudaError_t e = with_degree(np.p, [&](auto pc) {
            constexpr int P = decltype(pc)::value;
            k_near3_src<P><<<blocks, kNear3Warps * 32, 0, st>>>(items, n_items, src_base, src_p32, tgt_p32, tgt_pos,
                                                                 src_pos, q, tgt_start, cg, np, phi_s, grad_s);
            return cudaGetLastError();
        });
        if (e != cudaSuccess)
            return e;
    }
    if (any_coincident && N > 0) {
        k_coincident3_apply<<<nblk(N, 256), 256, 0, st>>>(N, coinc_start, coinc_src, q, np.beta0, phi_s);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_coincident3(int64_t N, const int *tgt_base, const double *tgt_pos, const double *src_pos,
                               const int *src_start, CellGrid3 cg, int *count, const int *coinc_start, int *coinc_src,
                               cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_coincident3<<<nblk(N, 256), 256, 0, st>>>(N, tgt_base, tgt_pos, src_pos, src_start, cg, count, coinc_start,
                                                coinc_src);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpermute3(int64_t N, const real *phi_s, const real *grad_s, const int *perm, double s,
                              void *phi_out, void *H_out, int out_f64, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_unpermute3<real><<<nblk(N, 256), 256, 0, st>>>(N, phi_s, grad_s, perm, s, phi_out, H_out, out_f64);
    return cudaGetLastError();
}

#define FS_INST3(real)                                                                                            \
    template cudaError_t launch_gather_points3<real>(const double *, const int *, int64_t, double, int, int, int, \
                                                     int, int, double, double *, real *, int *, float4 *, int *,  \
                                                     cudaStream_t);                                               \
    template cudaError_t launch_spread3<real>(int64_t, int, const int *, const real *, const real *, Window<real>, \
                                              const WindowPoly &, real *, int, cudaStream_t);                     \
    template cudaError_t launch_interp3<real>(int64_t, int, const int *, const real *, Window<real>,               \
                                              const WindowPoly &, const real *, int, real, real *, real *, bool,  \
                                              cudaStream_t);                                                      \
    template cudaError_t launch_unpermute3<real>(int64_t, const real *, const real *, const int *, double, void *, \
                                                 void *, int, cudaStream_t);
FS_INST3(float)
FS_INST3(double)
#undef FS_INST3

}  // namespace fs
