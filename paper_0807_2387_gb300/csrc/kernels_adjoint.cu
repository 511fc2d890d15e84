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
//
// Coincident pairs: the direct sum skips them (G(0) := 0, so also grad G(0) := 0 and
// Hess G(0) := 0), while the far field holds the smooth T_I there, with T_I(0) =
// beta_0, grad T_I(0) = 0 and Hess T_I(0) = (2 beta_1 / eps_I^2) I.  The near field
// removes those: -q beta_0 in phi, -q (2 beta_1 / eps_I^2) I in the Hessian and, in
// the source gradient of the adjoint potential, +(2 beta_1 / eps_I^2) dn.
//
// FP64: one thread per point (the comparison path).  FP32: warp items over the
// 8 x 8 sub-cells (near_warp.cuh), the Hessian over the forward's target items and
// the adjoint potential over items of sources against the targets.
#include <cmath>

#include "internal.h"
#include "near_warp.cuh"

namespace fs {

namespace {

template <typename real> using real2_t = typename Cplx<real>::type;

// f = G - T_I, c(w) = (G' - T_I')(r) / r and c'(w) = dc/dw at w = r^2 / eps_I^2 (FP64 sum forms).
__device__ __forceinline__ void near_fcd64(const NearParams<double> &np, double r2, double &f, double &c, double &cp)
{
    const double w = r2 * np.inv_eps2;
    const int p = np.p;
    double t = np.beta[p - 1];
    for (int i = p - 2; i >= 0; --i)
        t = t * w + np.beta[i];
    f = -1.0 / (4.0 * kPi) * log(r2) - t;
    double tp = 0.0, tpp = 0.0;
    for (int k = p - 1; k >= 1; --k)
        tp = tp * w + (double)(2 * k) * np.beta[k];
    for (int k = p - 1; k >= 2; --k)
        tpp = tpp * w + (double)(2 * k * (k - 1)) * np.beta[k];
    const double inv2pi = 1.0 / (2.0 * kPi);
    c = (-inv2pi / w - tp) * np.inv_eps2;
    cp = (inv2pi / (w * w) - tpp) * np.inv_eps2;
}

// Hess T_I(0) = hess0 I.
template <typename real> __host__ __device__ __forceinline__ real self_hessian(const NearParams<real> &np)
{
    return np.p > 1 ? real(2) * np.beta[1] * np.inv_eps2 : real(0);
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
// with respect to the source position, and the coincident gphi.  FP64.
__global__ void __launch_bounds__(256) k_near_adj64(int64_t M, const int *__restrict__ src_base,
                                                    const double2 *__restrict__ src_pos,
                                                    const double2 *__restrict__ tgt_pos,
                                                    const int *__restrict__ tgt_start, CellGrid cg,
                                                    const double *__restrict__ c, const double2 *__restrict__ dn,
                                                    NearParams<double> np, double *__restrict__ a_s,
                                                    double *__restrict__ ga_s, double *__restrict__ cg_s)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= M)
        return;
    const double2 Y = src_pos[j];
    const int packed = src_base[j];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const double two_over_eps2 = 2.0 * np.inv_eps2;
    const double hess0 = self_hessian(np);
    double A = 0, gx = 0, gy = 0, gco = 0;
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
                const double Dx = X.x - Y.x, Dy = X.y - Y.y;
                const double rr2 = Dx * Dx + Dy * Dy;
                if (!(rr2 < np.eps2))
                    continue;
                const double gp = c[i];
                const double2 dd = dn[i];
                if (rr2 == 0.0) {
                    A -= gp * np.beta[0];
                    gco += gp;
                    gx += hess0 * dd.x;
                    gy += hess0 * dd.y;
                    continue;
                }
                double f, cc, cp;
                near_fcd64(np, rr2, f, cc, cp);
                const double dD = dd.x * Dx + dd.y * Dy;
                A += gp * f + dD * cc;
                const double k2 = two_over_eps2 * cp * dD;
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

// Near part of grad phi and Hess phi at the targets (sorted target order), torus units.  FP64.
__global__ void __launch_bounds__(256) k_near_hess64(int64_t N, const int *__restrict__ tgt_base,
                                                     const double2 *__restrict__ tgt_pos,
                                                     const double2 *__restrict__ src_pos,
                                                     const int *__restrict__ src_start, CellGrid cg,
                                                     const double *__restrict__ q, NearParams<double> np,
                                                     double *__restrict__ grad_s, double *__restrict__ hess_s)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const double2 X = tgt_pos[k];
    const int packed = tgt_base[k];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const double two_over_eps2 = 2.0 * np.inv_eps2;
    const double hess0 = self_hessian(np);
    double gx = 0, gy = 0, hxx = 0, hxy = 0, hyy = 0;
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
                const double Dx = X.x - Y.x, Dy = X.y - Y.y;
                const double rr2 = Dx * Dx + Dy * Dy;
                if (!(rr2 < np.eps2))
                    continue;
                const double qj = q[j];
                if (rr2 == 0.0) {
                    hxx -= qj * hess0;
                    hyy -= qj * hess0;
                    continue;
                }
                double f, cc, cp;
                near_fcd64(np, rr2, f, cc, cp);
                gx += qj * cc * Dx;
                gy += qj * cc * Dy;
                const double k2 = qj * two_over_eps2 * cp;
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

// Hessian at the targets (FP32 warp items, own = targets, other = sources, d = x - y):
// grad += q c d, Hess += q (c I + (2 c' / eps_I^2) d d^T), with c = rc c^ and c' = rc c'^;
// the sums over pairs are of the hatted forms with d in units of eps_I (as the traversal
// hands it over, d = eps_I d'), so grad = rc eps_I sum q c^ d' and
// Hess = rc sum q (c^ I + 2 c'^ d' d'^T): rc eps_I and rc are applied at the store.
// For p >= 3 clamping w to 1 masks pairs beyond eps_I (c^ and c'^ vanish there); below, the
// charge is masked.
template <int P> struct NearHess32 {
    static constexpr int kMinBlocks = 5;
    static constexpr int kUnroll = 2;
    static constexpr bool kClamp = P >= 3;
    const float *__restrict__ q;
    float *__restrict__ grad_s;
    float *__restrict__ hess_s;
    float rcoef, geps, self_c;             // rc, eps_I (gradient unit), self_c = Hess T_I(0) / rc
    bool assign;                           // store instead of adding (the far part is added later)
    float qj;
    float2 gx, gy, sI, sxx, sxy, syy;

    __device__ __forceinline__ void init() { gx = gy = sI = sxx = sxy = syy = f2(0.f); }
    // candidate-list traversal: one value per other point (its charge)
    static constexpr int kR = 1;
    __device__ __forceinline__ void fetch(int j, float (&v)[1]) const { v[0] = __ldg(q + j); }
    __device__ __forceinline__ void set_q(const float *v) { qj = v[0]; }
    __device__ __forceinline__ void coincident(const NearParams<float> &, int t) { add_comp(sI, t, -qj * self_c); }
    __device__ __forceinline__ void pair2(const NearParams<float> &np, float2 r2, float2 dx, float2 dy)
    {
        float2 w = r2;
        if constexpr (kClamp)
            w = min1(w);
        float2 c, cp;
        near_c_cp2<P>(w, c, cp);
        float2 qq = f2(qj);
        if constexpr (!kClamp)
            qq = select2(r2, np.eps2, qq);
        const float2 qc = mul2(qq, c), k = mul2(qq, cp);
        gx = fma2(qc, dx, gx);
        gy = fma2(qc, dy, gy);
        sI = add2(sI, qc);
        const float2 kx = mul2(k, dx);
        sxx = fma2(kx, dx, sxx);
        sxy = fma2(kx, dy, sxy);
        syy = fma2(mul2(k, dy), dy, syy);
    }
    __device__ __forceinline__ void row_begin() {}
    __device__ __forceinline__ void row_end() {}
    __device__ __forceinline__ void store(int t, int64_t k)
    {
        // (a select, not a product with 0: the stored-to buffers may hold anything, NaN included)
        const float i0 = comp(sI, t), rg = rcoef * geps;
        const float v[5] = {rg * comp(gx, t), rg * comp(gy, t), rcoef * fmaf(2.f, comp(sxx, t), i0),
                            rcoef * 2.f * comp(sxy, t), rcoef * fmaf(2.f, comp(syy, t), i0)};
        grad_s[2 * k] = assign ? v[0] : grad_s[2 * k] + v[0];
        grad_s[2 * k + 1] = assign ? v[1] : grad_s[2 * k + 1] + v[1];
        hess_s[3 * k] = assign ? v[2] : hess_s[3 * k] + v[2];
        hess_s[3 * k + 1] = assign ? v[3] : hess_s[3 * k + 1] + v[3];
        hess_s[3 * k + 2] = assign ? v[4] : hess_s[3 * k + 2] + v[4];
    }
};

// Adjoint potential at the sources (FP32 warp items, own = sources, other = targets,
// d = y - x = -D):  A += gphi f - (dn . d) c,  grad_y A += c (gphi d - dn) - (2 c' / eps_I^2)(dn . d) d,
// with the hatted c^, c'^ summed.  The traversal hands d over in units of eps_I (d = eps_I d')
// and the dipoles are read as n' = dn / eps_I, so A = sum gphi f - rc eps_I^2 sum (n'.d') c^ and
// grad_y A = rc eps_I sum (c^ (gphi d' - n') - 2 c'^ (n'.d') d'): the factors are applied at the
// store.
template <int P> struct NearAdj32 {
    static constexpr int kMinBlocks = 4;
    static constexpr int kUnroll = 2;
    static constexpr bool kClamp = P >= 3;
    const float *__restrict__ cw;
    const float2 *__restrict__ dnw;
    float *__restrict__ a_s;
    float *__restrict__ ga_s;
    float *__restrict__ cg_s;
    float rcoef, geps, inv_eps, self_c;   // rc, eps_I, 1 / eps_I, self_c = Hess T_I(0) / rc
    bool assign;                           // store instead of adding (the far part is added later)
    float gp;
    float2 dn;
    float2 af, ac, gxc, gyc, gxk, gyk, gco;

    __device__ __forceinline__ void init() { af = ac = gxc = gyc = gxk = gyk = gco = f2(0.f); }
    // candidate-list traversal: three values per other point (gphi and the dipole dn)
    static constexpr int kR = 3;
    __device__ __forceinline__ void fetch(int i, float (&v)[3]) const
    {
        const float2 d = __ldg(dnw + i);
        v[0] = __ldg(cw + i);
        v[1] = d.x * inv_eps;
        v[2] = d.y * inv_eps;
    }
    __device__ __forceinline__ void set_q(const float *v)
    {
        gp = v[0];
        dn = make_float2(v[1], v[2]);
    }
    __device__ __forceinline__ void coincident(const NearParams<float> &np, int t)
    {
        add_comp(af, t, -gp * np.beta[0]);
        add_comp(gco, t, gp);
        add_comp(gxc, t, self_c * dn.x);
        add_comp(gyc, t, self_c * dn.y);
    }
    __device__ __forceinline__ void pair2(const NearParams<float> &np, float2 r2, float2 dx, float2 dy)
    {
        float2 w = r2;
        if constexpr (kClamp)
            w = min1(w);
        float2 c, cp;
        near_c_cp2<P>(w, c, cp);
        const float2 f = near_f2<P>(np, w);
        float2 g = f2(gp), n1 = f2(dn.x), n2 = f2(dn.y);
        if constexpr (!kClamp) {
            g = select2(r2, np.eps2, g);
            n1 = select2(r2, np.eps2, n1);
            n2 = select2(r2, np.eps2, n2);
        }
        const float2 dD = fma2(n1, dx, mul2(n2, dy));
        af = fma2(g, f, af);
        ac = fma2(dD, c, ac);
        gxc = fma2(c, fma2(g, dx, mul2(f2(-1.f), n1)), gxc);
        gyc = fma2(c, fma2(g, dy, mul2(f2(-1.f), n2)), gyc);
        const float2 k = mul2(cp, dD);
        gxk = fma2(k, dx, gxk);
        gyk = fma2(k, dy, gyk);
    }
    __device__ __forceinline__ void row_begin() {}
    __device__ __forceinline__ void row_end() {}
    __device__ __forceinline__ void store(int t, int64_t k)
    {
        const float rg = rcoef * geps;
        const float va = fmaf(-rg * geps, comp(ac, t), comp(af, t));
        const float vx = rg * fmaf(-2.f, comp(gxk, t), comp(gxc, t));
        const float vy = rg * fmaf(-2.f, comp(gyk, t), comp(gyc, t));
        a_s[k] = assign ? va : a_s[k] + va;
        ga_s[2 * k] = assign ? vx : ga_s[2 * k] + vx;
        ga_s[2 * k + 1] = assign ? vy : ga_s[2 * k + 1] + vy;
        cg_s[k] = comp(gco, t);
    }
};

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

cudaError_t launch_near_adj64(int64_t M, const int *src_base, const double2 *src_pos, const double2 *tgt_pos,
                              const int *tgt_start, CellGrid cg, const double *c, const void *dn,
                              NearParams<double> np, double *a_s, double *ga_s, double *cg_s, cudaStream_t st)
{
    if (M <= 0)
        return cudaSuccess;
    k_near_adj64<<<nblocks(M, 256), 256, 0, st>>>(M, src_base, src_pos, tgt_pos, tgt_start, cg, c,
                                                  (const double2 *)dn, np, a_s, ga_s, cg_s);
    return cudaGetLastError();
}

cudaError_t launch_near_hess64(int64_t N, const int *tgt_base, const double2 *tgt_pos, const double2 *src_pos,
                               const int *src_start, CellGrid cg, const double *q, NearParams<double> np,
                               double *grad_s, double *hess_s, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near_hess64<<<nblocks(N, 256), 256, 0, st>>>(N, tgt_base, tgt_pos, src_pos, src_start, cg, q, np, grad_s,
                                                   hess_s);
    return cudaGetLastError();
}

cudaError_t launch_near_adj32(int64_t n_items, const int2 *items, const int *src_base, const float2 *src_hi,
                              const float2 *src_lo, const float2 *tgt_hi, const float2 *tgt_lo, const int *tgt_start,
                              CellGrid cg, const float *c, const void *dn, NearParams<float> np, float *a_s,
                              float *ga_s, float *cg_s, bool assign, cudaStream_t st)
{
    const NearSides sd{src_base, src_hi, src_lo, tgt_hi, tgt_lo, tgt_start};
    return with_degree(np.p, [&](auto pc) {
        NearAdj32<decltype(pc)::value> op{};
        op.assign = assign;
        op.cw = c;
        op.dnw = (const float2 *)dn;
        op.a_s = a_s;
        op.ga_s = ga_s;
        op.cg_s = cg_s;
        op.rcoef = np.rcoef;
        op.geps = (float)std::sqrt((double)np.eps2);
        op.inv_eps = (float)(1.0 / std::sqrt((double)np.eps2));
        op.self_c = self_hessian(np) / np.rcoef;
        return launch_near_list(n_items, items, sd, cg, np, op, st);
    });
}

cudaError_t launch_near_hess32(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                               const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start,
                               CellGrid cg, const float *q, NearParams<float> np, float *grad_s, float *hess_s,
                               bool assign, cudaStream_t st)
{
    const NearSides sd{tgt_base, tgt_hi, tgt_lo, src_hi, src_lo, src_start};
    return with_degree(np.p, [&](auto pc) {
        NearHess32<decltype(pc)::value> op{};
        op.assign = assign;
        op.q = q;
        op.grad_s = grad_s;
        op.hess_s = hess_s;
        op.rcoef = np.rcoef;
        op.geps = (float)std::sqrt((double)np.eps2);
        op.self_c = self_hessian(np) / np.rcoef;
        return launch_near_list(n_items, items, sd, cg, np, op, st);
    });
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
