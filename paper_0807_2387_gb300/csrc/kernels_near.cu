// Near-field correction (step g) and return to physical units.
//
// The far field uses the kernel smoothed inside eps_I ("the price to pay is an
// afterwards correction in the smoothing zone"): for every pair closer than
// eps_I it holds T_I(r) instead of G(r) = -(1/2 pi) log r, so
//     phi_i  += q_j (G(r) - T_I(r))                       0 < r < eps_I
//     grad_i += q_j (-(1/2 pi) / r^2 - T_I'(r)/r) d        d = x~_i - y~_j
//     phi_i  -= q_j T_I(0), coinc_i += q_j                  r = 0 (G(0) := 0)
// Pairs are found among the 3 x 3 cells around the target's cell (cells are
// at least eps_I wide).  The FP32 path reads positions relative to their cell
// corner, so a difference is (offset - offset) + (exact cell step); pairs closer
// than eps_I/8 take their coordinate difference and squared distance from the
// FP64 positions, so r keeps full FP32 relative accuracy when points nearly
// coincide.
//
// The output kernel adds the far and near fields and rescales:
//     phi = phi~ + (log s / 2 pi) (sum_j q_j - coinc_i),   H = -s grad~ phi,
// scattering back to the caller's target order.
#include "internal.h"

namespace fs {

namespace {

template <typename real>
__global__ void __launch_bounds__(256) k_near(int64_t N, const int *__restrict__ tgt_base,
                                              const double2 *__restrict__ tgt_pos, const float2 *__restrict__ tgt_pos32,
                                              const double2 *__restrict__ src_pos, const float2 *__restrict__ src_pos32,
                                              const int *__restrict__ src_start, CellGrid cg, const real *__restrict__ q,
                                              NearParams<real> np, real *__restrict__ phi_s, real *__restrict__ grad_s,
                                              real *__restrict__ coinc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const bool fp32 = sizeof(real) == 4;
    const double2 X = tgt_pos[k];
    real xt, yt;
    if (fp32) {
        const float2 x32 = tgt_pos32[k];
        xt = (real)x32.x;
        yt = (real)x32.y;
    } else {
        xt = (real)X.x;
        yt = (real)X.y;
    }
    const int packed = tgt_base[k];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const real inv4pi = real(1.0 / (4.0 * kPi));
    const real inv2pi = real(1.0 / (2.0 * kPi));
    real phi = 0, gx = 0, gy = 0, qc = 0;
    for (int d1 = -1; d1 <= 1; ++d1) {
        const int e1 = c1 + d1;
        if (e1 < 0 || e1 >= cg.n_c)
            continue;
        for (int d2 = -1; d2 <= 1; ++d2) {
            const int e2 = c2 + d2;
            if (e2 < 0 || e2 >= cg.n_c)
                continue;
            const int key = cg.key(e1, e2);
            const int end = src_start[key + 1];
            // cell-corner offset between the target's and this source cell (exact: dyadic width)
            const real ox = (real)(c1 - e1) * np.hcell, oy = (real)(c2 - e2) * np.hcell;
            for (int j = src_start[key]; j < end; ++j) {
                real dx, dy, r2;
                if (fp32) {
                    const float2 y32 = src_pos32[j];
                    dx = (xt - (real)y32.x) + ox;
                    dy = (yt - (real)y32.y) + oy;
                } else {
                    const double2 Y = src_pos[j];
                    dx = (real)(X.x - Y.x);
                    dy = (real)(X.y - Y.y);
                }
                r2 = dx * dx + dy * dy;
                if (!(r2 < np.eps2))
                    continue;
                const real qj = q[j];
                if (fp32 && (double)r2 < np.close2) {
                    const double2 Y = src_pos[j];
                    const double ddx = X.x - Y.x, ddy = X.y - Y.y;
                    const double rr2 = ddx * ddx + ddy * ddy;
                    dx = (real)ddx;
                    dy = (real)ddy;
                    r2 = (real)rr2;
                    if (rr2 == 0.0)
                        r2 = real(0);
                }
                if (r2 == real(0)) {
                    phi -= qj * np.beta[0];
                    qc += qj;
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
                const real val = -inv4pi * flog<real>(r2) - t;
                const real coef = -inv2pi / r2 - tp;
                phi += qj * val;
                gx += qj * coef * dx;
                gy += qj * coef * dy;
            }
        }
    }
    phi_s[k] += phi;
    grad_s[2 * k] += gx;
    grad_s[2 * k + 1] += gy;
    coinc[k] = qc;
}

template <typename real>
__global__ void k_unpermute(int64_t N, const real *__restrict__ phi_s, const real *__restrict__ grad_s,
                            const real *__restrict__ coinc, const int *__restrict__ perm, double shift,
                            const double *__restrict__ q_sum, double s, void *__restrict__ phi_out,
                            void *__restrict__ H_out, int out_is_f64)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const int64_t i = perm[k];
    const double phi = (double)phi_s[k] + shift * (q_sum[0] - (double)coinc[k]);
    const double hx = -s * (double)grad_s[2 * k];
    const double hy = -s * (double)grad_s[2 * k + 1];
    if (out_is_f64) {
        if (phi_out)
            ((double *)phi_out)[i] = phi;
        if (H_out) {
            ((double *)H_out)[2 * i] = hx;
            ((double *)H_out)[2 * i + 1] = hy;
        }
    } else {
        if (phi_out)
            ((float *)phi_out)[i] = (float)phi;
        if (H_out) {
            ((float *)H_out)[2 * i] = (float)hx;
            ((float *)H_out)[2 * i + 1] = (float)hy;
        }
    }
}

}  // namespace

template <typename real>
cudaError_t launch_near(int64_t N, const int *tgt_base, const double2 *tgt_pos, const float2 *tgt_pos32,
                        const double2 *src_pos, const float2 *src_pos32, const int *src_start, CellGrid cg,
                        const real *q, NearParams<real> np, real *phi_s, real *grad_s, real *coinc, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near<real><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, tgt_base, tgt_pos, tgt_pos32, src_pos, src_pos32,
                                                              src_start, cg, q, np, phi_s, grad_s, coinc);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpermute(int64_t N, const real *phi_s, const real *grad_s, const real *coinc, const int *perm,
                             double shift, const double *q_sum, double s, void *phi_out, void *H_out, int out_is_f64,
                             cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_unpermute<real><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, phi_s, grad_s, coinc, perm, shift, q_sum, s,
                                                                   phi_out, H_out, out_is_f64);
    return cudaGetLastError();
}

template cudaError_t launch_near<float>(int64_t, const int *, const double2 *, const float2 *, const double2 *,
                                        const float2 *, const int *, CellGrid, const float *, NearParams<float>,
                                        float *, float *, float *, cudaStream_t);
template cudaError_t launch_near<double>(int64_t, const int *, const double2 *, const float2 *, const double2 *,
                                         const float2 *, const int *, CellGrid, const double *, NearParams<double>,
                                         double *, double *, double *, cudaStream_t);
template cudaError_t launch_unpermute<float>(int64_t, const float *, const float *, const float *, const int *,
                                             double, const double *, double, void *, void *, int, cudaStream_t);
template cudaError_t launch_unpermute<double>(int64_t, const double *, const double *, const double *, const int *,
                                              double, const double *, double, void *, void *, int, cudaStream_t);

}  // namespace fs
