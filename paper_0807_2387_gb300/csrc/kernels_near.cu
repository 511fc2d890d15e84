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
// cell (two per lane, so each source read serves two targets per lane), over the
// source sub-cells near the item's bounding box (near_warp.cuh).  A dense
// sub-cell gets warps of its own, so a warp's targets are spatially compact (and
// a warp never spans two cells, whose bounding box could cross the whole domain).
// The value and gradient use the cancellation-free forms of G - T_I and of its
// radial derivative over r, c (w - 1)^(p-1) / w with w = r^2 / eps_I^2.
//
// The output kernel adds the far and near fields and rescales:
//     phi = phi~ + (log s / 2 pi) (sum_j q_j - coinc_i),   H = -s grad~ phi,
// scattering back to the caller's target order.
#include <cmath>

#include "internal.h"
#include "output.cuh"
#include "near_warp.cuh"

namespace fs {

namespace {

__device__ __forceinline__ void near64_target(int64_t k, const int *__restrict__ tgt_base,
                                              const double2 *__restrict__ tgt_pos, const double2 *__restrict__ src_pos,
                                              const int *__restrict__ src_start, const CellGrid &cg,
                                              const double *__restrict__ q, const NearParams<double> &np,
                                              double *__restrict__ phi_s, double *__restrict__ grad_s,
                                              double *__restrict__ coinc)
{
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

__global__ void __launch_bounds__(256) k_near64(int64_t N, const int *__restrict__ tgt_base,
                                                const double2 *__restrict__ tgt_pos,
                                                const double2 *__restrict__ src_pos, const int *__restrict__ src_start,
                                                CellGrid cg, const double *__restrict__ q, NearParams<double> np,
                                                double *__restrict__ phi_s, double *__restrict__ grad_s,
                                                double *__restrict__ coinc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N)
        near64_target(k, tgt_base, tgt_pos, src_pos, src_start, cg, q, np, phi_s, grad_s, coinc);
}

// Batched FP64 near field: block -> (instance, block of its targets), blockIdx.y = right-hand side.
__global__ void __launch_bounds__(256) k_batch_near64(const BatchInst<double> *__restrict__ inst, BlockMap bm)
{
    const int i = bm.inst[blockIdx.x];
    const BatchInst<double> &b = inst[i];
    const int64_t k = (int64_t)(blockIdx.x - bm.first[i]) * blockDim.x + threadIdx.x;
    const int64_t N = b.N;
    if (k >= N)
        return;
    const int r = blockIdx.y;
    near64_target(k, b.tgt_base, b.tgt_pos, b.src_pos, b.src_start, b.cg, b.q + (int64_t)r * b.M, b.np,
                  b.phi_s + (int64_t)r * N, b.grad_s + 2 * (int64_t)r * N, b.coinc + (int64_t)r * N);
}

// Forward correction at the targets for R right-hand sides at once (the pair geometry, the
// log and the gradient coefficient are shared): phi += q f, grad += q c d, with the lane's
// two targets as packed pairs and the factor rc eps_I of c applied once at the store (d
// arrives in units of eps_I).  With one right-hand side the sums are split into partial sums
// per list evaluation; with several the registers go to the extra accumulators instead.
// Right-hand side r reads q + r q_stride and writes at r n_stride.
template <int P, int R, bool BATCH = false> struct NearFwd {
    // four blocks per SM (up to 128 registers); the single right-hand-side kernel unrolls its
    // candidate loop eightfold (2.77 -> 2.66 ms at 2^20 points against fourfold at five blocks
    // per SM); the batched kernel holds the instance's constants in registers (the single-plan
    // one reads them from the constant bank) and unrolls less
    static constexpr int kMinBlocks = 4;
    static constexpr int kUnroll = (R == 1 && !BATCH) ? 8 : (R >= 4 ? 1 : 2);
    static constexpr bool kRows = R == 1;
    // the gradient coefficient through exp2 / log2 (single right-hand side: 2.57 -> 2.52 ms at
    // 2^20 points); the batched kernels, with more FMA work per pair and less unrolling, keep the
    // power form, whose dependency chain is shorter (the exp2 form made the batched replay 2 %
    // slower)
    static constexpr bool kExp2 = P >= 2 && R == 1 && !BATCH;
    const float *__restrict__ q;
    float *__restrict__ phi_s;
    float *__restrict__ grad_s;
    float *__restrict__ coinc;
    int64_t q_stride, n_stride;
    float rcoef;   // rc eps_I: the pair differences arrive in units of eps_I
    bool assign;   // store phi_s / grad_s instead of adding (the far field is added later)
    float qj[R];
    float2 phi[R], gx[R], gy[R], qc[R];
    float2 rphi[kRows ? R : 1], rgx[kRows ? R : 1], rgy[kRows ? R : 1];

    __device__ __forceinline__ float2 &acc_phi(int r) { return kRows ? rphi[0] : phi[r]; }
    __device__ __forceinline__ float2 &acc_gx(int r) { return kRows ? rgx[0] : gx[r]; }
    __device__ __forceinline__ float2 &acc_gy(int r) { return kRows ? rgy[0] : gy[r]; }

    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int r = 0; r < R; ++r)
            phi[r] = gx[r] = gy[r] = qc[r] = f2(0.f);
    }
    // candidate-list traversal: the R charges of source j, and those of a listed candidate
    static constexpr int kR = R;
    __device__ __forceinline__ void fetch(int j, float (&v)[R]) const
    {
#pragma unroll
        for (int r = 0; r < R; ++r)
            v[r] = __ldg(q + r * q_stride + j);
    }
    __device__ __forceinline__ void set_q(const float *v)
    {
#pragma unroll
        for (int r = 0; r < R; ++r)
            qj[r] = v[r];
    }
    __device__ __forceinline__ void coincident(const NearParams<float> &np, int t)
    {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            add_comp(acc_phi(r), t, -qj[r] * np.beta[0]);   // G(0) := 0 removes the far field's T_I(0)
            add_comp(qc[r], t, qj[r]);
        }
    }
    __device__ __forceinline__ void pair2(const NearParams<float> &np, float2 r2, float2 dx, float2 dy)
    {
        float2 w = r2;                                    // the traversal works in units of eps_I
        if constexpr (P >= 2)
            w = min1(w);                                  // f(1) = 0 and (w - 1)^(p-1) = 0: masked
        const float2 val = near_f2<P>(np, w);
        float2 coef;
        if constexpr (kExp2) {
            // |w - 1|^(p-1) / w = 2^((p-1) log2(1 - w) - log2 w): two MUFU operations and one FMA
            // instead of a reciprocal and five multiplications; log2 w is shared with val, and
            // the sign (-1)^(p-1) is applied at the store.  w = 1 (masked) gives 2^-inf = 0.
            const float2 lw = lg2_2(w);
            const float2 om = add2(w, f2(-1.f));   // the value's w - 1: 1 - w = -om, no add of its own
            const float2 lo = lg2_2(make_float2(-om.x, -om.y));
            coef = ex2_2(fma2(f2((float)(P - 1)), lo, make_float2(-lw.x, -lw.y)));
        } else {
            coef = rcp_2(w);
            if constexpr (P >= 2)
                coef = mul2(ipow2<P - 1>(add2(w, f2(-1.f))), coef);
        }
        if constexpr (R >= 3 && P >= 2) {
            // three or more right-hand sides: the pair's gradient vector once, then one FMA per
            // component and right-hand side (batched replay 8.01 -> 7.77 ms at three)
            const float2 cdx = mul2(coef, dx), cdy = mul2(coef, dy);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 qq = f2(qj[r]);
                acc_phi(r) = fma2(qq, val, acc_phi(r));
                acc_gx(r) = fma2(qq, cdx, acc_gx(r));
                acc_gy(r) = fma2(qq, cdy, acc_gy(r));
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 qq = f2(qj[r]);
                if constexpr (P == 1)
                    qq = select2(r2, np.eps2, qq);
                acc_phi(r) = fma2(qq, val, acc_phi(r));
                const float2 tq = mul2(qq, coef);
                acc_gx(r) = fma2(tq, dx, acc_gx(r));
                acc_gy(r) = fma2(tq, dy, acc_gy(r));
            }
        }
    }
    // every other far candidate takes the power form, (1 - w)^(p-1) / w (the exp2 form's sign):
    // a reciprocal and five multiplications instead of two MUFU operations and one FMA, so that
    // neither pipe runs alone at its limit (2.44 -> 2.41 ms at 2^20 points)
    static constexpr bool kAlt = kExp2;
    __device__ __forceinline__ void pair2_alt(const NearParams<float> &np, float2 r2, float2 dx, float2 dy)
    {
        float2 w = min1(r2);
        const float2 val = near_f2<P>(np, w);
        const float2 om = add2(w, f2(-1.f));
        float2 coef = mul2(ipow2<P - 1>(make_float2(-om.x, -om.y)), rcp_2(w));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 qq = f2(qj[r]);
            acc_phi(r) = fma2(qq, val, acc_phi(r));
            const float2 tq = mul2(qq, coef);
            acc_gx(r) = fma2(tq, dx, acc_gx(r));
            acc_gy(r) = fma2(tq, dy, acc_gy(r));
        }
    }
    __device__ __forceinline__ void row_begin()
    {
        if constexpr (kRows)
            rphi[0] = rgx[0] = rgy[0] = f2(0.f);
    }
    __device__ __forceinline__ void row_end()
    {
        if constexpr (kRows) {
            phi[0] = add2(phi[0], rphi[0]);
            gx[0] = add2(gx[0], rgx[0]);
            gy[0] = add2(gy[0], rgy[0]);
        }
    }
    __device__ __forceinline__ void store(int t, int64_t k)
    {
        const float rc = (kExp2 && (P - 1) % 2 == 1) ? -rcoef : rcoef;   // the exp2 coef is |w - 1|^(p-1) / w
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t kk = k + r * n_stride;
            if (assign) {
                phi_s[kk] = comp(phi[r], t);
                grad_s[2 * kk] = rc * comp(gx[r], t);
                grad_s[2 * kk + 1] = rc * comp(gy[r], t);
            } else {
                phi_s[kk] += comp(phi[r], t);
                grad_s[2 * kk] += rc * comp(gx[r], t);
                grad_s[2 * kk + 1] += rc * comp(gy[r], t);
            }
            coinc[kk] = comp(qc[r], t);
        }
    }
};

// Plan-time statistics: pairs with r < eps_I and with r < eps_I / 8 (coincident pairs
// included), counted by the same traversal and the same FP32 differences as the field
// kernel.  Each lane adds its counts to one of kCountSlots counter pairs (summed on the host).
static_assert(kNearCountSlots == 64, "counter slots");
constexpr int kCountSlots = kNearCountSlots;
struct NearCount {
    static constexpr int kMinBlocks = 6;
    static constexpr int kUnroll = 2;
    unsigned long long *__restrict__ counts;   // 2 * kCountSlots
    unsigned n_near, n_close;

    __device__ __forceinline__ void init() { n_near = n_close = 0; }
    static constexpr int kR = 1;   // candidate-list traversal: no values per other point
    __device__ __forceinline__ void fetch(int, float (&v)[1]) const { v[0] = 0.f; }
    __device__ __forceinline__ void set_q(const float *) {}
    __device__ __forceinline__ void coincident(const NearParams<float> &, int)
    {
        ++n_near;
        ++n_close;
    }
    __device__ __forceinline__ void pair2(const NearParams<float> &np, float2 r2, float2, float2)
    {
        n_near += (r2.x < np.eps2 ? 1u : 0u) + (r2.y < np.eps2 ? 1u : 0u);
        n_close += (r2.x < np.close2 ? 1u : 0u) + (r2.y < np.close2 ? 1u : 0u);
    }
    __device__ __forceinline__ void row_begin() {}
    __device__ __forceinline__ void row_end() {}
    __device__ __forceinline__ void store(int t, int64_t)
    {
        // both slots' counts are in the lane's totals (an idle slot never lands within eps_I)
        if (t == 0) {
            const int slot = threadIdx.x & (kCountSlots - 1);
            atomicAdd(&counts[2 * slot], (unsigned long long)n_near);
            atomicAdd(&counts[2 * slot + 1], (unsigned long long)n_close);
        }
    }
};

// Batched FP32 near field: one warp per item (first target, count, instance); all R
// right-hand sides in one candidate-list traversal.
template <int P, int R>
__global__ void __launch_bounds__(32 * kNearWarps, NearFwd<P, R, true>::kMinBlocks * 4 / kNearWarps) k_batch_near32(int64_t n_items,
                                                                               const int4 *__restrict__ items,
                                                                               const BatchInst<float> *__restrict__ inst,
                                                                               bool assign)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_items)
        return;
    const int4 it = items[warp];
    const BatchInst<float> &b = inst[it.z];
    const NearSides sd{b.tgt_base, b.tgt_hi, b.tgt_lo, b.src_hi, b.src_lo, b.src_start};
    const CellGrid cg = b.cg;
    const NearParams<float> np = b.np;
    NearFwd<P, R, true> op;
    op.q = b.q;
    op.phi_s = b.phi_s;
    op.grad_s = b.grad_s;
    op.coinc = b.coinc;
    op.q_stride = b.M;
    op.n_stride = b.N;
    op.rcoef = np.rcoef * sqrtf(np.eps2);
    op.assign = assign;
    __shared__ NearLists<R> L;
    const int w = threadIdx.x >> 5;
    near_traverse_list(make_int2(it.x, it.y), lane, sd, cg, np, op, L.xy[w], L.q[w], L.cxy[w], L.cl[w], L.cq[w]);
}

template <typename real>
__device__ __forceinline__ void unpermute_point(int64_t k, const real *__restrict__ phi_s,
                                                const real *__restrict__ grad_s, const real *__restrict__ coinc,
                                                const int *__restrict__ perm, double shift, double q_sum, double s,
                                                void *__restrict__ phi_out, void *__restrict__ H_out, int out_is_f64)
{
    output_point<real>(k, phi_s[k], grad_s[2 * k], grad_s[2 * k + 1], coinc[k], perm, shift, q_sum, s, phi_out, H_out,
                       out_is_f64);
}

template <typename real>
__global__ void k_unpermute(int64_t N, const real *__restrict__ phi_s, const real *__restrict__ grad_s,
                            const real *__restrict__ coinc, const int *__restrict__ perm, double shift,
                            const double *__restrict__ q_sum, double s, void *__restrict__ phi_out,
                            void *__restrict__ H_out, int out_is_f64)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N)
        unpermute_point(k, phi_s, grad_s, coinc, perm, shift, q_sum[0], s, phi_out, H_out, out_is_f64);
}

// Batched output: block -> (instance, block of its targets), blockIdx.y = right-hand side;
// writes the caller's (nrhs, N) and (nrhs, N, 2) buffers of each instance.
template <typename real>
__global__ void k_batch_unpermute(const BatchInst<real> *__restrict__ inst, const BatchIO *__restrict__ io,
                                  BlockMap bm, int out_is_f64)
{
    const int i = bm.inst[blockIdx.x];
    const BatchInst<real> &b = inst[i];
    const int64_t k = (int64_t)(blockIdx.x - bm.first[i]) * blockDim.x + threadIdx.x;
    const int64_t N = b.N;
    if (k >= N)
        return;
    const int r = blockIdx.y;
    const size_t osz = out_is_f64 ? 8 : 4;
    void *po = io[i].phi ? (unsigned char *)io[i].phi + (size_t)r * N * osz : nullptr;
    void *ho = io[i].H ? (unsigned char *)io[i].H + (size_t)r * N * 2 * osz : nullptr;
    unpermute_point(k, b.phi_s + (int64_t)r * N, b.grad_s + 2 * (int64_t)r * N, b.coinc + (int64_t)r * N,
                    b.tgt_perm, b.shift, b.q_sum[r], b.s, po, ho, out_is_f64);
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
                          bool assign, cudaStream_t st)
{
    const NearSides sd{tgt_base, tgt_hi, tgt_lo, src_hi, src_lo, src_start};
    return with_degree(np.p, [&](auto pc) {
        NearFwd<decltype(pc)::value, 1> op{};
        op.q = q;
        op.phi_s = phi_s;
        op.grad_s = grad_s;
        op.coinc = coinc;
        op.q_stride = 0;
        op.n_stride = 0;
        op.rcoef = (float)((double)np.rcoef * std::sqrt((double)np.eps2));
        op.assign = assign;
        return launch_near_list(n_items, items, sd, cg, np, op, st);
    });
}

cudaError_t launch_near_src32(int64_t n_items, const int2 *items, const int *src_base, const float2 *src_hi,
                              const float2 *src_lo, const float2 *tgt_hi, const float2 *tgt_lo, const int *tgt_start,
                              CellGrid cg, const float *q, NearParams<float> np, float *phi_s, float *grad_s,
                              float *coinc, cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    const NearSides sd{src_base, src_hi, src_lo, tgt_hi, tgt_lo, tgt_start};
    const unsigned blocks = (unsigned)((n_items + 3) / 4);
    return with_degree(np.p, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        k_near_src32<P><<<blocks, 128, 0, st>>>(n_items, items, sd, cg, np, q, phi_s, grad_s, coinc);
        return cudaGetLastError();
    });
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

cudaError_t launch_near_count32(int64_t n_items, const int2 *items, const int *tgt_base, const float2 *tgt_hi,
                                const float2 *tgt_lo, const float2 *src_hi, const float2 *src_lo, const int *src_start,
                                CellGrid cg, NearParams<float> np, unsigned long long *counts, cudaStream_t st)
{
    const NearSides sd{tgt_base, tgt_hi, tgt_lo, src_hi, src_lo, src_start};
    NearCount op{};
    op.counts = counts;
    return launch_near_list(n_items, items, sd, cg, np, op, st);
}

cudaError_t launch_batch_near32(int64_t n_items, const int4 *items, const BatchInst<float> *inst, int p, int nrhs,
                                bool assign, cudaStream_t st)
{
    if (n_items <= 0 || nrhs <= 0)
        return cudaSuccess;
    const unsigned blocks = (unsigned)((n_items + kNearWarps - 1) / kNearWarps);
    constexpr int T = 32 * kNearWarps;
    return with_degree(p, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        switch (nrhs) {
        case 1: k_batch_near32<P, 1><<<blocks, T, 0, st>>>(n_items, items, inst, assign); break;
        case 2: k_batch_near32<P, 2><<<blocks, T, 0, st>>>(n_items, items, inst, assign); break;
        case 3: k_batch_near32<P, 3><<<blocks, T, 0, st>>>(n_items, items, inst, assign); break;
        case 4: k_batch_near32<P, 4><<<blocks, T, 0, st>>>(n_items, items, inst, assign); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_batch_near64(const BatchInst<double> *inst, BlockMap bm, int blocks, int nrhs, cudaStream_t st)
{
    if (blocks <= 0 || nrhs <= 0)
        return cudaSuccess;
    k_batch_near64<<<dim3((unsigned)blocks, (unsigned)nrhs), 256, 0, st>>>(inst, bm);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_batch_unpermute(const BatchInst<real> *inst, const BatchIO *io, BlockMap bm, int blocks, int nrhs,
                                   int out_is_f64, cudaStream_t st)
{
    if (blocks <= 0 || nrhs <= 0)
        return cudaSuccess;
    k_batch_unpermute<real><<<dim3((unsigned)blocks, (unsigned)nrhs), 256, 0, st>>>(inst, io, bm, out_is_f64);
    return cudaGetLastError();
}

template cudaError_t launch_batch_unpermute<float>(const BatchInst<float> *, const BatchIO *, BlockMap, int, int, int,
                                                   cudaStream_t);
template cudaError_t launch_batch_unpermute<double>(const BatchInst<double> *, const BatchIO *, BlockMap, int, int,
                                                    int, cudaStream_t);

}  // namespace fs
