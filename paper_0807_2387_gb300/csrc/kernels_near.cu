// Near-field correction (step g) and return to physical units.
//
// The far field uses the kernel smoothed inside eps_I ("the price to pay is an
// afterwards correction in the smoothing zone"): for every pair closer than
// eps_I it holds T_I(r) instead of G(r) = -(1/2 pi) log r, so
//     phi_i  += q_j (G(r) - T_I(r))                       0 < r < eps_I
//     grad_i += q_j (-(1/2 pi) / r^2 - T_I'(r)/r) d        d = x~_i - y~_j
//     phi_i  -= q_j T_I(0), coinc_i += q_j                  r = 0 (G(0) := 0)
// Cells are at least eps_I wide, so a target's partners lie in the 3 x 3 cells
// around its own.
//
// FP64 path: one thread per target, direct FP64 formulas (the comparison path).
//
// FP32 path: one warp per work item of at most 64 consecutive targets of one
// cell (two per lane, so each source read serves two targets per lane).  Targets are sorted by cell and, inside a cell, by 8 x 8 sub-cell in
// Morton order; a dense sub-cell gets warps of its own, so a warp's targets are
// spatially compact (and a warp never spans two cells, whose bounding box could
// cross the whole domain).  The warp forms the bounding box of its targets and
// visits only the source sub-cells whose distance to that box is below eps_I
// (a warp-uniform test per sub-cell, so the visited set approximates the union
// of the targets' discs); each source there is read once per warp (a broadcast
// load) and evaluated by all 32 lanes with branch-free masked arithmetic, so no
// lane diverges on the pair test.  With w = r^2 / eps_I^2:
//     G - T_I         = -(ln 2 / 4 pi) log2 w - P(w),   P = T_I - k(eps_I), P(1) = 0
//     (G' - T_I')/r   = c (w - 1)^(p-1) / w,            c = (-1)^p / (2 pi eps_I^2)
// (the numerator has a (p-1)-fold root at w = 1 because G - T_I has a p-fold
// contact there), both free of cancellation near r = eps_I.  Positions are
// FP32 offsets from the cell corner stored as hi + lo: differences use the hi
// parts plus the exact cell step; pairs closer than eps_I/8 refine the
// difference with an exact TwoSum of the hi parts and the lo parts, which
// keeps full FP32 relative accuracy in r for nearly coincident points.
//
// The output kernel adds the far and near fields and rescales:
//     phi = phi~ + (log s / 2 pi) (sum_j q_j - coinc_i),   H = -s grad~ phi,
// scattering back to the caller's target order.
#include "internal.h"

namespace fs {

namespace {

__global__ void __launch_bounds__(256) k_near64(int64_t N, const int *__restrict__ tgt_base,
                                                const double2 *__restrict__ tgt_pos,
                                                const double2 *__restrict__ src_pos, const int *__restrict__ src_start,
                                                CellGrid cg, const double *__restrict__ q, NearParams<double> np,
                                                double *__restrict__ phi_s, double *__restrict__ grad_s,
                                                double *__restrict__ coinc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N)
        return;
    const double2 X = tgt_pos[k];
    const int packed = tgt_base[k];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const double inv4pi = 1.0 / (4.0 * kPi);
    const double inv2pi = 1.0 / (2.0 * kPi);
    double phi = 0, gx = 0, gy = 0, qc = 0;
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
                const double dx = X.x - Y.x, dy = X.y - Y.y;
                const double r2 = dx * dx + dy * dy;
                if (!(r2 < np.eps2))
                    continue;
                const double qj = q[j];
                if (r2 == 0.0) {
                    phi -= qj * np.beta[0];
                    qc += qj;
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
                const double val = -inv4pi * log(r2) - t;
                const double coef = -inv2pi / r2 - tp;
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

template <int E> __device__ __forceinline__ float ipow(float x)
{
    if constexpr (E == 0) {
        return 1.0f;
    } else if constexpr (E == 1) {
        return x;
    } else {
        const float h = ipow<E / 2>(x);
        if constexpr (E % 2 == 0)
            return h * h;
        else
            return h * h * x;
    }
}

__device__ __forceinline__ float warp_min(float v)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// dx from hi parts (a = x_hi - y_hi by TwoSum), the exact cell step and the lo parts.
__device__ __forceinline__ float refine_diff(float xh, float yh, float off, float xl, float yl)
{
    const float a = xh - yh;
    const float bb = a - xh;
    const float e = (xh - (a - bb)) + (-yh - bb);
    return (a + off) + (e + (xl - yl));
}

// Single MUFU operations (approximate, flush-to-zero): log2 with ~2^-22 absolute error on
// (0, 16), and the reciprocal with ~1 ulp error; both arguments here are normal numbers.
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Near-field value and gradient coefficient of one pair from r^2 > 0 (masked by qm = 0
// when the pair is not within eps_I), accumulated into (phi, grad).
template <int P>
__device__ __forceinline__ void near_math(const NearParams<float> &np, float r2, float dx, float dy, float qm,
                                          float &cphi, float &cgx, float &cgy)
{
    const float w = r2 * np.inv_eps2;
    float pw = np.pbeta[P - 1];
#pragma unroll
    for (int i = P - 2; i >= 0; --i)
        pw = fmaf(pw, w, np.pbeta[i]);
    const float c_ln = -0.69314718055994531f / (4.0f * 3.14159265358979324f);   // -(ln 2) / (4 pi)
    const float val = fmaf(c_ln, lg2_approx(w), -pw);
    const float coef = np.rcoef * ipow<P - 1>(w - 1.f) * rcp_approx(w);
    cphi = fmaf(qm, val, cphi);
    const float t = qm * coef;
    cgx = fmaf(t, dx, cgx);
    cgy = fmaf(t, dy, cgy);
}

// Exact coordinate difference for a close pair (both hi parts by TwoSum, the cell step,
// the lo parts); coincident points are reported by dx = dy = 0.
__device__ __forceinline__ void refine_pair(float2 xh, float2 xl, float2 yh, float2 yl, float offx, float offy,
                                            float &dx, float &dy)
{
    dx = refine_diff(xh.x, yh.x, offx, xl.x, yl.x);
    dy = refine_diff(xh.y, yh.y, offy, xl.y, yl.y);
}

// One source against the warp's targets (two per lane): all lanes, no lane-divergent
// branch (the close-pair refinement is taken warp-uniformly when any lane needs it).
template <int P>
__device__ __forceinline__ void near_source(const NearParams<float> &np, const float2 (&xh)[2],
                                            const float2 (&xl)[2], const float2 (&xs)[2], float2 yh, float qj,
                                            const float2 *__restrict__ src_lo, int j, float offx, float offy,
                                            float (&cphi)[2], float (&cgx)[2], float (&cgy)[2], float (&qc)[2])
{
    // xs = xh + (cell step) for this source cell: one subtraction per coordinate; a close pair
    // recomputes its difference exactly from the hi/lo parts
    float dx[2], dy[2], r2[2];
    bool close = false;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        dx[t] = xs[t].x - yh.x;
        dy[t] = xs[t].y - yh.y;
        r2[t] = dx[t] * dx[t] + dy[t] * dy[t];
        close |= r2[t] < np.close2;
    }
    if (__any_sync(0xffffffffu, close)) {
        const float2 yl = __ldg(src_lo + j);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (r2[t] < np.close2) {
                refine_pair(xh[t], xl[t], yh, yl, offx, offy, dx[t], dy[t]);
                r2[t] = dx[t] * dx[t] + dy[t] * dy[t];
                if (dx[t] == 0.f && dy[t] == 0.f) {   // coincident: G(0) := 0 removes the far field's T_I(0)
                    cphi[t] -= qj * np.beta[0];
                    qc[t] += qj;
                    r2[t] = np.eps2;                  // masked out below
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
        near_math<P>(np, r2[t], dx[t], dy[t], r2[t] < np.eps2 ? qj : 0.f, cphi[t], cgx[t], cgy[t]);
}

template <int P>
__global__ void __launch_bounds__(128, 6) k_near32(int64_t n_items, const int2 *__restrict__ items,
                                                const int *__restrict__ tgt_base,
                                                const float2 *__restrict__ tgt_hi, const float2 *__restrict__ tgt_lo,
                                                const float2 *__restrict__ src_hi, const float2 *__restrict__ src_lo,
                                                const int *__restrict__ src_start, CellGrid cg,
                                                const float *__restrict__ q, NearParams<float> np,
                                                float *__restrict__ phi_s, float *__restrict__ grad_s,
                                                float *__restrict__ coinc)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_items)
        return;                                   // whole warp past the end (warp-uniform)
    const int2 item = items[warp];                // (first target, count <= 64), one cell
    const float h = np.hcell, eps = sqrtf(np.eps2);
    const float ginv = h / (float)cg.cell;        // one grid line (1 / n_os)
    bool valid[2];
    int64_t kt[2];
    int cc1[2], cc2[2];
    float2 xh[2], xl[2];
    float tx0 = 3e38f, tx1 = -3e38f, ty0 = 3e38f, ty1 = -3e38f;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        valid[t] = lane + 32 * t < item.y;
        kt[t] = item.x + lane + 32 * t;
        const int64_t kk = valid[t] ? kt[t] : item.x;
        const int packed = tgt_base[kk];
        cc1[t] = base1(packed) / cg.cell;
        cc2[t] = base2(packed) / cg.cell;
        xh[t] = tgt_hi[kk];
        xl[t] = tgt_lo[kk];
        if (valid[t]) {
            const float ax = (float)cc1[t] * h + xh[t].x, ay = (float)cc2[t] * h + xh[t].y;
            tx0 = fminf(tx0, ax);
            tx1 = fmaxf(tx1, ax);
            ty0 = fminf(ty0, ay);
            ty1 = fmaxf(ty1, ay);
        }
    }
    // bounding box of the warp's targets, in "cell * h + offset" coordinates
    tx0 = warp_min(tx0);
    tx1 = warp_max(tx1);
    ty0 = warp_min(ty0);
    ty1 = warp_max(ty1);
    // all targets of an item share one cell
    const int c1 = cc1[0], c2 = cc2[0];
#pragma unroll
    for (int t = 0; t < 2; ++t)
        if (!valid[t])
            xh[t] = make_float2(1e6f, 1e6f);      // idle slots: every pair lands beyond eps_I
    const float reach = eps + ginv;               // eps_I plus one grid line for rounding of positions
    const float reach2 = reach * reach;
    const int cx0 = max(0, (int)floorf((tx0 - reach) / h)), cx1 = min(cg.n_c - 1, (int)floorf((tx1 + reach) / h));
    const int cy0 = max(0, (int)floorf((ty0 - reach) / h)), cy1 = min(cg.n_c - 1, (int)floorf((ty1 + reach) / h));
    float phi[2] = {0.f, 0.f}, gx[2] = {0.f, 0.f}, gy[2] = {0.f, 0.f}, qc[2] = {0.f, 0.f};
    for (int ex = cx0; ex <= cx1; ++ex) {
        const float offx = (float)(c1 - ex) * h;
        const float sx0 = (float)ex * h;
        float2 xs[2];
#pragma unroll
        for (int t = 0; t < 2; ++t)
            xs[t].x = xh[t].x + offx;
        for (int s1 = 0; s1 < kSubEdge; ++s1) {
            // gap between this sub-cell row and the targets' box (warp-uniform)
            const float lo = sx0 + (float)cg.sub_first(s1) * ginv, hi = sx0 + (float)cg.sub_first(s1 + 1) * ginv;
            const float gapx = fmaxf(0.f, fmaxf(lo - tx1, tx0 - hi));
            if (gapx > reach || !(hi > lo))
                continue;
            float rphi[2] = {0.f, 0.f}, rgx[2] = {0.f, 0.f}, rgy[2] = {0.f, 0.f};
            for (int ey = cy0; ey <= cy1; ++ey) {
                const float offy = (float)(c2 - ey) * h;
                const float sy0 = (float)ey * h;
#pragma unroll
                for (int t = 0; t < 2; ++t)
                    xs[t].y = xh[t].y + offy;
                const int kbase = cg.key(ex, ey) * kSub;
                for (int s2 = 0; s2 < kSubEdge; ++s2) {
                    const float ylo = sy0 + (float)cg.sub_first(s2) * ginv;
                    const float yhi = sy0 + (float)cg.sub_first(s2 + 1) * ginv;
                    const float gapy = fmaxf(0.f, fmaxf(ylo - ty1, ty0 - yhi));
                    if (gapx * gapx + gapy * gapy > reach2)
                        continue;                 // no target of this warp is within eps_I of the sub-cell
                    const int sub = morton_sub(s1, s2);
                    const int end = src_start[kbase + sub + 1];
                    for (int j = src_start[kbase + sub]; j < end; ++j)
                        near_source<P>(np, xh, xl, xs, __ldg(src_hi + j), __ldg(q + j), src_lo, j, offx, offy,
                                       rphi, rgx, rgy, qc);
                }
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                phi[t] += rphi[t];
                gx[t] += rgx[t];
                gy[t] += rgy[t];
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (valid[t]) {
            phi_s[kt[t]] += phi[t];
            grad_s[2 * kt[t]] += gx[t];
            grad_s[2 * kt[t] + 1] += gy[t];
            coinc[kt[t]] = qc[t];
        }
    }
}

template <int P>
cudaError_t near32_p(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                     const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start, CellGrid cg,
                     const float *q, NearParams<float> np, float *phi_s, float *grad_s, float *coinc, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n_items + 3) / 4);
    k_near32<P><<<blocks, 128, 0, st>>>(n_items, items, tgt_base, tgt_hi, tgt_lo, src_hi, src_lo, src_start, cg, q,
                                        np, phi_s, grad_s, coinc);
    return cudaGetLastError();
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

cudaError_t launch_near64(int64_t N, const int *tgt_base, const double2 *tgt_pos, const double2 *src_pos,
                          const int *src_start, CellGrid cg, const double *q, NearParams<double> np, double *phi_s,
                          double *grad_s, double *coinc, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near64<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, tgt_base, tgt_pos, src_pos, src_start, cg, q, np, phi_s,
                                                           grad_s, coinc);
    return cudaGetLastError();
}

cudaError_t launch_near32(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                          const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start,
                          CellGrid cg, const float *q, NearParams<float> np, float *phi_s, float *grad_s, float *coinc,
                          cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    switch (np.p) {
#define FS_NEAR_CASE(P)                                                                                          \
    case P:                                                                                                      \
        return near32_p<P>(n_items, items, tgt_base, tgt_hi, tgt_lo, src_hi, src_lo, src_start, cg, q, np, phi_s, \
                           grad_s, coinc, st);
        FS_NEAR_CASE(1)
        FS_NEAR_CASE(2)
        FS_NEAR_CASE(3)
        FS_NEAR_CASE(4)
        FS_NEAR_CASE(5)
        FS_NEAR_CASE(6)
        FS_NEAR_CASE(7)
        FS_NEAR_CASE(8)
        FS_NEAR_CASE(9)
        FS_NEAR_CASE(10)
        FS_NEAR_CASE(11)
        FS_NEAR_CASE(12)
        FS_NEAR_CASE(13)
        FS_NEAR_CASE(14)
        FS_NEAR_CASE(15)
        FS_NEAR_CASE(16)
#undef FS_NEAR_CASE
    default:
        return cudaErrorInvalidValue;
    }
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

template cudaError_t launch_unpermute<float>(int64_t, const float *, const float *, const float *, const int *,
                                             double, const double *, double, void *, void *, int, cudaStream_t);
template cudaError_t launch_unpermute<double>(int64_t, const double *, const double *, const double *, const int *,
                                              double, const double *, double, void *, void *, int, cudaStream_t);

}  // namespace fs
