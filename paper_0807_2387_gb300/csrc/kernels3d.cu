// The fast summation for the 3D kernel G(r) = 1/(4 pi r): binning, spreading, interpolation,
// near field and output (the transform is in kernels_fft.cu).
//
// The paper names the 3D Green function as the next step with the same pipeline; each
// kernel here is the 2D one with a third coordinate:
//   spreading    g_k = sum_j q_j psi(k1 - u_j1) psi(k2 - u_j2) psi(k3 - u_j3) over the
//                (2m)^3 grid lines around each source; one warp per source, lanes 0..6m-1
//                hold the window values of the three coordinates, every lane owns
//                (2m)^3 / 32 taps and adds them to the grid with atomics (the grid of the
//                active window stays in L2 for the sizes this path serves);
//   interpolation phi and grad phi from the same taps, the window and its slope;
//   near field   q (1/(4 pi r) - T_I(r)) and its gradient for 0 < r < eps_I over the 27
//                cells around the target's (cells at least eps_I wide), -q T_I(0) for
//                coincident points;
//   output       phi = s phi~, H = -s^2 grad~ phi~ (1/r is homogeneous of degree -1).
// Grid layout: g[z][y][x], x fastest, edge n_a (the active window); a point's base grid
// line per coordinate is packed into 10 bits each.
#include "internal.h"

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
    double f;
    const int b1 = grid_line3(xyz[3 * k], s, n_os, window_lo, m, n_a, f, status);
    const int b2 = grid_line3(xyz[3 * k + 1], s, n_os, window_lo, m, n_a, f, status);
    const int b3 = grid_line3(xyz[3 * k + 2], s, n_os, window_lo, m, n_a, f, status);
    const int kk = cg.key(b1 / cg.cell, b2 / cg.cell, b3 / cg.cell);
    key[k] = kk;
    atomicAdd(&count[kk], 1);
}

template <typename real>
__global__ void k_gather_points3(const double *__restrict__ xyz, const int *__restrict__ perm, int64_t n, double s,
                                 int n_os, int window_lo, int n_a, int m, int cell, double *__restrict__ pos,
                                 real *__restrict__ frac, int *__restrict__ base, float4 *__restrict__ pos32,
                                 int *status)
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
        // offset from the lower corner of the point's cell, torus units
        float o[3];
        for (int d = 0; d < 3; ++d) {
            const double corner = (double)((b[d] / cell) * cell + window_lo) / n_os - 0.5;
            o[d] = (float)(s * xyz[3 * i + d] - corner);
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
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < M; j += warps) {
        const int packed = base[j];
        real wv = real(0);
        if (lane < 3 * M2) {
            const real fr = frac[3 * j + dim];
            if constexpr (sizeof(real) == 4)
                wv = poly_eval<kPolyD>(wp.c[jw], (float)fr - 0.5f);
            else
                wv = kb_value<real>(w, fr, m - 1 - jw);
            if (dim == 0)
                wv *= q[j];
        }
        const int x0 = b3x(packed) - m + 1, y0 = b3y(packed) - m + 1, z0 = b3z(packed) - m + 1;
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

// phi~ and grad~ phi~ at the targets from the filtered grid (thread per target).
template <typename real, int M2>
__global__ void __launch_bounds__(256) k_interp3(int64_t N, const int *__restrict__ base, const real *__restrict__ frac,
                                                 Window<real> w, WindowPoly wp, const real *__restrict__ grid, int n_a,
                                                 real n_os, real *__restrict__ phi_s, real *__restrict__ grad_s)
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
    phi_s[k] = phi;
    grad_s[3 * k] = n_os * gx;
    grad_s[3 * k + 1] = n_os * gy;
    grad_s[3 * k + 2] = n_os * gz;
}

// Near-field correction at target k (thread per target) over the 27 cells around its cell.
template <typename real>
__global__ void __launch_bounds__(256) k_near3(int64_t N, const int *__restrict__ tgt_base,
                                               const double *__restrict__ tgt_pos, const float4 *__restrict__ tgt_p32,
                                               const double *__restrict__ src_pos, const float4 *__restrict__ src_p32,
                                               const int *__restrict__ src_start, CellGrid3 cg,
                                               const real *__restrict__ q, NearParams<real> np,
                                               real *__restrict__ phi_s, real *__restrict__ grad_s)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int packed = tgt_base[k];
    const int c1 = b3x(packed) / cg.cell, c2 = b3y(packed) / cg.cell, c3 = b3z(packed) / cg.cell;
    real xt[3];
    if constexpr (sizeof(real) == 4) {
        const float4 p = tgt_p32[k];
        xt[0] = p.x;
        xt[1] = p.y;
        xt[2] = p.z;
    } else {
        for (int d = 0; d < 3; ++d)
            xt[d] = tgt_pos[3 * k + d];
    }
    const real inv4pi = real(1.0 / (4.0 * kPi));
    real phi = 0, g0 = 0, g1 = 0, g2 = 0;
    for (int e1 = max(c1 - 1, 0); e1 <= min(c1 + 1, cg.n_c - 1); ++e1)
        for (int e2 = max(c2 - 1, 0); e2 <= min(c2 + 1, cg.n_c - 1); ++e2)
            for (int e3 = max(c3 - 1, 0); e3 <= min(c3 + 1, cg.n_c - 1); ++e3) {
                const int key = cg.key(e1, e2, e3);
                // FP32 offsets are relative to the cell corners: add the cell step
                const real o1 = sizeof(real) == 4 ? (real)(c1 - e1) * np.hcell : real(0);
                const real o2 = sizeof(real) == 4 ? (real)(c2 - e2) * np.hcell : real(0);
                const real o3 = sizeof(real) == 4 ? (real)(c3 - e3) * np.hcell : real(0);
                const int end = src_start[key + 1];
                for (int j = src_start[key]; j < end; ++j) {
                    real dx, dy, dz;
                    if constexpr (sizeof(real) == 4) {
                        const float4 p = __ldg(src_p32 + j);
                        dx = (xt[0] - p.x) + o1;
                        dy = (xt[1] - p.y) + o2;
                        dz = (xt[2] - p.z) + o3;
                    } else {
                        dx = xt[0] - src_pos[3 * j];
                        dy = xt[1] - src_pos[3 * j + 1];
                        dz = xt[2] - src_pos[3 * j + 2];
                    }
                    const real r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 < np.eps2))
                        continue;
                    const real qj = q[j];
                    if (r2 == real(0)) {
                        phi -= qj * np.beta[0];
                        continue;
                    }
                    const real u2 = r2 * np.inv_eps2;
                    real t = np.beta[np.p - 1];
                    for (int i = np.p - 2; i >= 0; --i)
                        t = t * u2 + np.beta[i];
                    real tp = real(0);
                    if (np.p > 1) {
                        tp = np.dbeta[np.p - 2];
                        for (int i = np.p - 3; i >= 0; --i)
                            tp = tp * u2 + np.dbeta[i];
                    }
                    const real inv_r = real(1) / sqrt(r2);
                    const real val = inv4pi * inv_r - t;
                    const real coef = -inv4pi * inv_r * inv_r * inv_r - tp;
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
                                  int n_a, int m, int cell, double *pos, real *frac, int *base, float4 *pos32,
                                  int *status, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_gather_points3<real><<<nblk(n, 256), 256, 0, st>>>(xyz, perm, n, s, n_os, window_lo, n_a, m, cell, pos, frac,
                                                        base, pos32, status);
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

template <typename real>
cudaError_t launch_interp3(int64_t N, int m, const int *base, const real *frac, Window<real> w, const WindowPoly &wp,
                           const real *grid, int n_a, real n_os, real *phi_s, real *grad_s, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    return with_width3(m, [&](auto mc) {
        constexpr int M2 = decltype(mc)::value;
        k_interp3<real, M2><<<nblk(N, 256), 256, 0, st>>>(N, base, frac, w, wp, grid, n_a, n_os, phi_s, grad_s);
        return cudaGetLastError();
    });
}

template <typename real>
cudaError_t launch_near3(int64_t N, const int *tgt_base, const double *tgt_pos, const float4 *tgt_p32,
                         const double *src_pos, const float4 *src_p32, const int *src_start, CellGrid3 cg,
                         const real *q, NearParams<real> np, real *phi_s, real *grad_s, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near3<real><<<nblk(N, 256), 256, 0, st>>>(N, tgt_base, tgt_pos, tgt_p32, src_pos, src_p32, src_start, cg, q, np,
                                               phi_s, grad_s);
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
                                                     int, int, double *, real *, int *, float4 *, int *,          \
                                                     cudaStream_t);                                               \
    template cudaError_t launch_spread3<real>(int64_t, int, const int *, const real *, const real *, Window<real>, \
                                              const WindowPoly &, real *, int, cudaStream_t);                     \
    template cudaError_t launch_interp3<real>(int64_t, int, const int *, const real *, Window<real>,               \
                                              const WindowPoly &, const real *, int, real, real *, real *,        \
                                              cudaStream_t);                                                      \
    template cudaError_t launch_near3<real>(int64_t, const int *, const double *, const float4 *, const double *,  \
                                            const float4 *, const int *, CellGrid3, const real *, NearParams<real>, \
                                            real *, real *, cudaStream_t);                                        \
    template cudaError_t launch_unpermute3<real>(int64_t, const real *, const real *, const int *, double, void *, \
                                                 void *, int, cudaStream_t);
FS_INST3(float)
FS_INST3(double)
#undef FS_INST3

}  // namespace fs
