// Adjoint of the fast summation (gradients of a loss L(phi, H)) and the Hessian of phi.
//
// The forward map is linear in q: phi = A q, H = B q, and the far field is
// interp o (symmetric spectral multiply) o spread, so its transpose is the same
// pipeline read backwards: the loss gradients gphi = dL/dphi and gH = dL/dH are
// spread at the targets as monopoles and dipoles (kernels_spread.cu), multiplied
// by the same table, and interpolated at the sources (value and gradient).  With
//   A(y) = sum_i gphi_i G(x_i - y) - sum_i gH_i . grad G(x_i - y)
// the gradients are dL/dq_j = A(y_j), dL/dy_j = q_j grad A(y_j) and
// dL/dx_i = -gphi_i H(x_i) - Hess phi(x_i) gH_i.  This file holds the near-field
// parts (the kernel difference f = G - T_I inside eps_I, its gradient c(w) d and
// Hessian c(w) I + (2 c'(w) / eps_I^2) d d^T, w = r^2 / eps_I^2), the gathers and
// the final assembly in physical units.
#include "internal.h"

namespace fs {

namespace {

template <typename real> using real2_t = typename Cplx<real>::type;

// f(w) = G - T_I, c(w) = (G' - T_I')(r) / r and c'(w) = dc/dw at w = r^2 / eps_I^2.
template <typename real>
__device__ __forceinline__ void near_fcd(const NearParams<real> &np, real r2, real &f, real &c, real &cp)
{
    const real w = r2 * np.inv_eps2;
    const int p = np.p;
    if (sizeof(real) == 4) {
        // P(w) = T_I - k(eps_I) with P(1) = 0; c = rc (w-1)^(p-1) / w; c' = rc (w-1)^(p-2) ((p-2) w + 1) / w^2
        real t = np.pbeta[p - 1];
        for (int i = p - 2; i >= 0; --i)
            t = t * w + np.pbeta[i];
        f = real(-1.0 / (4.0 * kPi)) * flog<real>(w) - t;
        const real om = w - real(1);
        real pw2 = real(1);   // (w-1)^(p-2)
        for (int i = 0; i < p - 2; ++i)
            pw2 *= om;
        if (p >= 2) {
            c = np.rcoef * pw2 * om / w;
            cp = np.rcoef * pw2 * (real(p - 2) * w + real(1)) / (w * w);
        } else {
            c = np.rcoef / w;
            cp = -np.rcoef / (w * w);
        }
    } else {
        real t = np.beta[p - 1];
        for (int i = p - 2; i >= 0; --i)
            t = t * w + np.beta[i];
        f = real(-1.0 / (4.0 * kPi)) * flog<real>(r2) - t;
        real tp = real(0), tpp = real(0);
        for (int k = p - 1; k >= 1; --k)
            tp = tp * w + real(2 * k) * np.beta[k];
        for (int k = p - 1; k >= 2; --k)
            tpp = tpp * w + real(2 * k * (k - 1)) * np.beta[k];
        const real inv2pi = real(1.0 / (2.0 * kPi));
        c = (-inv2pi / w - tp) * np.inv_eps2;
        cp = (inv2pi / (w * w) - tpp) * np.inv_eps2;
    }
}

// Loss gradients into sorted target order: c = gphi, dn = -s gH (near field, torus units),
// df = n_os dn (far-field dipole weight), and sum of gphi.
template <typename real>
__global__ void k_gather_adj(int64_t N, const int *__restrict__ perm, const void *__restrict__ gphi,
                             const void *__restrict__ gH, int in_f64, double s, double n_os, real *__restrict__ c,
                             real2_t<real> *__restrict__ dn, real2_t<real> *__restrict__ df, double *__restrict__ gsum)
{
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        double g = 0.0, hx = 0.0, hy = 0.0;
        if (gphi)
            g = in_f64 ? ((const double *)gphi)[i] : (double)((const float *)gphi)[i];
        if (gH) {
            hx = in_f64 ? ((const double *)gH)[2 * i] : (double)((const float *)gH)[2 * i];
            hy = in_f64 ? ((const double *)gH)[2 * i + 1] : (double)((const float *)gH)[2 * i + 1];
        }
        c[k] = (real)g;
        real2_t<real> a, b;
        a.x = (real)(-s * hx);
        a.y = (real)(-s * hy);
        b.x = (real)(-s * n_os * hx);
        b.y = (real)(-s * n_os * hy);
        dn[k] = a;
        df[k] = b;
        acc += g;
    }
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0)
            atomicAdd(gsum, acc);
    }
}

// Near part of the adjoint potential at the sources (sorted source order): value, gradient
// with respect to the source position, and the coincident gphi.
template <typename real>
__global__ void __launch_bounds__(256) k_near_adj(int64_t M, const int *__restrict__ src_base,
                                                  const double2 *__restrict__ src_pos,
                                                  const double2 *__restrict__ tgt_pos, const int *__restrict__ tgt_start,
                                                  CellGrid cg, const real *__restrict__ c,
                                                  const real2_t<real> *__restrict__ dn, NearParams<real> np,
                                                  real *__restrict__ a_s, real *__restrict__ ga_s,
                                                  real *__restrict__ cg_s)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= M)
        return;
    const double2 Y = src_pos[j];
    const int packed = src_base[j];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const real two_over_eps2 = real(2) * np.inv_eps2;
    real A = 0, gx = 0, gy = 0, gco = 0;
    for (int d1 = -1; d1 <= 1; ++d1) {
        const int e1 = c1 + d1;
        if (e1 < 0 || e1 >= cg.n_c)
            continue;
        for (int d2 = -1; d2 <= 1; ++d2) {
            const int e2 = c2 + d2;
            if (e2 < 0 || e2 >= cg.n_c)
                continue;
            const int key = cg.key(e1, e2);
            const int end = tgt_start[(key + 1) * kSub];
            for (int i = tgt_start[key * kSub]; i < end; ++i) {
                const double2 X = tgt_pos[i];
                const real Dx = (real)(X.x - Y.x), Dy = (real)(X.y - Y.y);
                const double rr2 = (X.x - Y.x) * (X.x - Y.x) + (X.y - Y.y) * (X.y - Y.y);
                if (!(rr2 < (double)np.eps2))
                    continue;
                const real gp = c[i];
                if (rr2 == 0.0) {
                    A -= gp * np.beta[0];
                    gco += gp;
                    continue;
                }
                real f, cc, cp;
                near_fcd<real>(np, (real)rr2, f, cc, cp);
                const real2_t<real> dd = dn[i];
                const real dD = dd.x * Dx + dd.y * Dy;
                A += gp * f + dD * cc;
                const real k2 = two_over_eps2 * cp * dD;
                gx -= gp * cc * Dx + cc * dd.x + k2 * Dx;
                gy -= gp * cc * Dy + cc * dd.y + k2 * Dy;
            }
        }
    }
    a_s[j] += A;
    ga_s[2 * j] += gx;
    ga_s[2 * j + 1] += gy;
    cg_s[j] = gco;
}

// Near part of grad phi and Hess phi at the targets (sorted target order), torus units.
template <typename real>
__global__ void __launch_bounds__(256) k_near_hess(int64_t N, const int *__restrict__ tgt_base,
                                                   const double2 *__restrict__ tgt_pos,
                                                   const double2 *__restrict__ src_pos, const int *__restrict__ src_start,
                                                   CellGrid cg, const real *__restrict__ q, NearParams<real> np,
                                                   real *__restrict__ grad_s, real *__restrict__ hess_s)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const double2 X = tgt_pos[k];
    const int packed = tgt_base[k];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const real two_over_eps2 = real(2) * np.inv_eps2;
    real gx = 0, gy = 0, hxx = 0, hxy = 0, hyy = 0;
    for (int d1 = -1; d1 <= 1; ++d1) {
        const int e1 = c1 + d1;
        if (e1 < 0 || e1 >= cg.n_c)
            continue;
        for (int d2 = -1; d2 <= 1; ++d2) {
            const int e2 = c2 + d2;
            if (e2 < 0 || e2 >= cg.n_c)
                continue;
            const int key = cg.key(e1, e2);
            const int end = src_start[(key + 1) * kSub];
            for (int j = src_start[key * kSub]; j < end; ++j) {
                const double2 Y = src_pos[j];
                const double rr2 = (X.x - Y.x) * (X.x - Y.x) + (X.y - Y.y) * (X.y - Y.y);
                if (!(rr2 < (double)np.eps2) || rr2 == 0.0)
                    continue;
                const real Dx = (real)(X.x - Y.x), Dy = (real)(X.y - Y.y);
                real f, cc, cp;
                near_fcd<real>(np, (real)rr2, f, cc, cp);
                const real qj = q[j];
                gx += qj * cc * Dx;
                gy += qj * cc * Dy;
                const real k2 = qj * two_over_eps2 * cp;
                hxx += qj * cc + k2 * Dx * Dx;
                hxy += k2 * Dx * Dy;
                hyy += qj * cc + k2 * Dy * Dy;
            }
        }
    }
    grad_s[2 * k] += gx;
    grad_s[2 * k + 1] += gy;
    hess_s[3 * k] += hxx;
    hess_s[3 * k + 1] += hxy;
    hess_s[3 * k + 2] += hyy;
}

// dL/dq_j = A(y_j) + (log s / 2pi)(sum gphi - coincident gphi);  dL/dy_j = q_j s grad~ A(y_j).
template <typename real>
__global__ void k_adj_finish_src(int64_t M, const int *__restrict__ perm, const real *__restrict__ a_s,
                                 const real *__restrict__ ga_s, const real *__restrict__ cg_s,
                                 const real *__restrict__ q, double shift, const double *__restrict__ gsum, double s,
                                 void *__restrict__ dq, void *__restrict__ dy, int out_f64)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= M)
        return;
    const int64_t j = perm[k];
    const double v = (double)a_s[k] + shift * (gsum[0] - (double)cg_s[k]);
    const double gx = s * (double)q[k] * (double)ga_s[2 * k];
    const double gy = s * (double)q[k] * (double)ga_s[2 * k + 1];
    if (out_f64) {
        if (dq)
            ((double *)dq)[j] = v;
        if (dy) {
            ((double *)dy)[2 * j] = gx;
            ((double *)dy)[2 * j + 1] = gy;
        }
    } else {
        if (dq)
            ((float *)dq)[j] = (float)v;
        if (dy) {
            ((float *)dy)[2 * j] = (float)gx;
            ((float *)dy)[2 * j + 1] = (float)gy;
        }
    }
}

// dL/dx_i = -gphi_i H_i - Hess_phys gH_i with H = -s grad~, Hess_phys = s^2 Hess~, gH = -dn / s.
template <typename real>
__global__ void k_adj_finish_tgt(int64_t N, const int *__restrict__ perm, const real *__restrict__ grad_s,
                                 const real *__restrict__ hess_s, const real *__restrict__ c,
                                 const real2_t<real> *__restrict__ dn, double s, void *__restrict__ dx, int out_f64)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int64_t i = perm[k];
    const double g = (double)c[k];
    const double hx = -(double)dn[k].x / s, hy = -(double)dn[k].y / s;
    const double Hx = -s * (double)grad_s[2 * k], Hy = -s * (double)grad_s[2 * k + 1];
    const double s2 = s * s;
    const double pxx = s2 * (double)hess_s[3 * k], pxy = s2 * (double)hess_s[3 * k + 1];
    const double pyy = s2 * (double)hess_s[3 * k + 2];
    const double ox = -g * Hx - (pxx * hx + pxy * hy);
    const double oy = -g * Hy - (pxy * hx + pyy * hy);
    if (out_f64) {
        ((double *)dx)[2 * i] = ox;
        ((double *)dx)[2 * i + 1] = oy;
    } else {
        ((float *)dx)[2 * i] = (float)ox;
        ((float *)dx)[2 * i + 1] = (float)oy;
    }
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename real>
cudaError_t launch_gather_adj(int64_t N, const int *perm, const void *gphi, const void *gH, int in_f64, double s,
                              double n_os, real *c, void *dn, void *df, double *gsum, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    unsigned b = nblocks(N, 256);
    if (b > 2048)
        b = 2048;
    k_gather_adj<real><<<b, 256, 0, st>>>(N, perm, gphi, gH, in_f64, s, n_os, c, (real2_t<real> *)dn,
                                          (real2_t<real> *)df, gsum);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_near_adj(int64_t M, const int *src_base, const double2 *src_pos, const double2 *tgt_pos,
                            const int *tgt_start, CellGrid cg, const real *c, const void *dn, NearParams<real> np,
                            real *a_s, real *ga_s, real *cg_s, cudaStream_t st)
{
    if (M <= 0)
        return cudaSuccess;
    k_near_adj<real><<<nblocks(M, 256), 256, 0, st>>>(M, src_base, src_pos, tgt_pos, tgt_start, cg, c,
                                                      (const real2_t<real> *)dn, np, a_s, ga_s, cg_s);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_near_hess(int64_t N, const int *tgt_base, const double2 *tgt_pos, const double2 *src_pos,
                             const int *src_start, CellGrid cg, const real *q, NearParams<real> np, real *grad_s,
                             real *hess_s, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near_hess<real><<<nblocks(N, 256), 256, 0, st>>>(N, tgt_base, tgt_pos, src_pos, src_start, cg, q, np, grad_s,
                                                       hess_s);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adj_finish_src(int64_t M, const int *perm, const real *a_s, const real *ga_s, const real *cg_s,
                                  const real *q, double shift, const double *gsum, double s, void *dq, void *dy,
                                  int out_f64, cudaStream_t st)
{
    if (M <= 0)
        return cudaSuccess;
    k_adj_finish_src<real><<<nblocks(M, 256), 256, 0, st>>>(M, perm, a_s, ga_s, cg_s, q, shift, gsum, s, dq, dy,
                                                            out_f64);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adj_finish_tgt(int64_t N, const int *perm, const real *grad_s, const real *hess_s, const real *c,
                                  const void *dn, double s, void *dx, int out_f64, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_adj_finish_tgt<real><<<nblocks(N, 256), 256, 0, st>>>(N, perm, grad_s, hess_s, c, (const real2_t<real> *)dn, s,
                                                            dx, out_f64);
    return cudaGetLastError();
}

#define FS_INST(real)                                                                                           \
    template cudaError_t launch_gather_adj<real>(int64_t, const int *, const void *, const void *, int, double,  \
                                                 double, real *, void *, void *, double *, cudaStream_t);        \
    template cudaError_t launch_near_adj<real>(int64_t, const int *, const double2 *, const double2 *,          \
                                               const int *, CellGrid, const real *, const void *,               \
                                               NearParams<real>, real *, real *, real *, cudaStream_t);         \
    template cudaError_t launch_near_hess<real>(int64_t, const int *, const double2 *, const double2 *,         \
                                                const int *, CellGrid, const real *, NearParams<real>, real *,  \
                                                real *, cudaStream_t);                                          \
    template cudaError_t launch_adj_finish_src<real>(int64_t, const int *, const real *, const real *,          \
                                                     const real *, const real *, double, const double *,        \
                                                     double, void *, void *, int, cudaStream_t);                \
    template cudaError_t launch_adj_finish_tgt<real>(int64_t, const int *, const real *, const real *,          \
                                                     const real *, const void *, double, void *, int,           \
                                                     cudaStream_t);
FS_INST(float)
FS_INST(double)
#undef FS_INST

}  // namespace fs
