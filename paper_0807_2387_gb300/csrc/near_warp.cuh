// Warp-cooperative FP32 near-field traversal, shared by the forward correction
// (phi and grad phi at the targets; one or several charge vectors), the Hessian of phi at
// the targets, the adjoint potential at the sources and the plan's pair statistics.
//
// A work item is at most 64 consecutive "own" points of one cell (two per lane),
// sorted by cell and, inside a cell, by 8 x 8 sub-cell in Morton order, so the item is
// compact.  The warp forms the bounding box of its points, reads the "other" points of the
// neighbour cells within eps_I of that box 32 at a time, keeps those within eps_I of the box
// (ballot) and appends them to candidate lists in shared memory, which all 32 lanes then
// evaluate with branch-free masked arithmetic against both of their points.  Positions are
// FP32 offsets from the cell corner stored as hi + lo; candidates within eps_I / 8 of the box
// go to a second list that carries their position in the item's frame as hi + lo as well, so
// the pair difference keeps full FP32 relative accuracy for nearly coincident points, and
// exactly coincident pairs are detected (G(0) := 0).
//
// With w = r^2 / eps_I^2 and f = G - T_I (T_I the inner polynomial of the
// regularised kernel, p-fold contact with G at r = eps_I):
//     f(w)      = -(ln 2 / 4 pi) log2 w - P(w),      P = T_I - k(eps_I), P(1) = 0
//     c(w)      = f'(r) / r = rc (w - 1)^(p-1) / w,  rc = (-1)^p / (2 pi eps_I^2)
//     c'(w)     = dc/dw = rc (w - 1)^(p-2) ((p - 2) w + 1) / w^2
// (the (p-1)-fold root at w = 1 keeps c free of cancellation near r = eps_I), so
// grad f = c d and Hess f = c I + (2 c' / eps_I^2) d d^T for d = own - other.
//
// The two points of a lane meet the same other point, so their arithmetic is done as
// packed pairs (Blackwell's two-wide FP32 add, multiply and fma: one instruction for
// both).  Pairs beyond eps_I are masked without a select where the forms allow it:
// with w clamped to 1, P(w) = (w - 1) Ptilde(w) and (w - 1)^(p-1) vanish exactly, as
// does log2(1).
#pragma once

#include <type_traits>

#include "internal.h"

namespace fs {

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

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- packed pairs of FP32 values (x: the lane's first point, y: its second)

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 min1(float2 w) { return make_float2(fminf(w.x, 1.f), fminf(w.y, 1.f)); }
__device__ __forceinline__ float2 lg2_2(float2 w) { return make_float2(lg2_approx(w.x), lg2_approx(w.y)); }
__device__ __forceinline__ float2 rcp_2(float2 w) { return make_float2(rcp_approx(w.x), rcp_approx(w.y)); }
__device__ __forceinline__ float2 ex2_2(float2 w) { return make_float2(ex2_approx(w.x), ex2_approx(w.y)); }
__device__ __forceinline__ float2 select2(float2 r2, float eps2, float2 v)
{
    return make_float2(r2.x < eps2 ? v.x : 0.f, r2.y < eps2 ? v.y : 0.f);
}
__device__ __forceinline__ float comp(float2 v, int t) { return t == 0 ? v.x : v.y; }
__device__ __forceinline__ void add_comp(float2 &v, int t, float a)
{
    if (t == 0)
        v.x += a;
    else
        v.y += a;
}

template <int E> __device__ __forceinline__ float2 ipow2(float2 x)
{
    if constexpr (E == 0) {
        return f2(1.f);
    } else if constexpr (E == 1) {
        return x;
    } else {
        const float2 h = ipow2<E / 2>(x);
        if constexpr (E % 2 == 0)
            return mul2(h, h);
        else
            return mul2(mul2(h, h), x);
    }
}

// f = G - T_I at w (clamped to <= 1 by the caller for p >= 2, where f(1) = 0 exactly).
template <int P> __device__ __forceinline__ float2 near_f2(const NearParams<float> &np, float2 w)
{
    const float c_ln = -0.69314718055994531f / (4.0f * 3.14159265358979324f);   // -(ln 2) / (4 pi)
    if constexpr (P == 1) {
        return fma2(f2(c_ln), lg2_2(w), f2(-np.pbeta[0]));
    } else {
        float2 t = f2(np.nptilde[P - 2]);
#pragma unroll
        for (int i = P - 3; i >= 0; --i)
            t = fma2(t, w, f2(np.nptilde[i]));
        return fma2(f2(c_ln), lg2_2(w), mul2(add2(w, f2(-1.f)), t));   // c_ln log2 w - (w - 1) Ptilde(w)
    }
}

// c / rc = (w - 1)^(p-1) / w and c' / rc = (w - 1)^(p-2) ((p - 2) w + 1) / w^2 (rc applied by the caller).
template <int P> __device__ __forceinline__ void near_c_cp2(float2 w, float2 &c, float2 &cp)
{
    const float2 rw = rcp_2(w);
    if constexpr (P == 1) {
        c = rw;
        cp = mul2(f2(-1.f), mul2(rw, rw));
    } else {
        const float2 om = add2(w, f2(-1.f));
        const float2 base = mul2(ipow2<P - 2>(om), rw);
        c = mul2(base, om);
        cp = mul2(mul2(base, fma2(f2((float)(P - 2)), w, f2(1.f))), rw);
    }
}

// The two point sets of a traversal: the item's own points (one per lane slot) and the
// other side's points, visited by sub-cell.
struct NearSides {
    const int *own_base;
    const float2 *own_hi, *own_lo;
    const float2 *oth_hi, *oth_lo;
    const int *oth_start;
};

// ---- candidate-list traversal
//
// The lanes read the other points of each neighbour cell within reach of the box 32 at a time
// (a cell is one contiguous range, so the chunks are full, where sub-cells would hold only a
// few points each), test each against the box (ballot) and append those within reach to the
// warp's lists in shared memory: "far" candidates (beyond eps_I / 8 of the box: no pair can
// need the refined difference) shifted into the item's cell frame and negated,
// (-x, -x, -y, -y), with their Op::kR values (charges, or the adjoint's weights); "close"
// candidates the same way as hi + lo pairs (the TwoSum of the cell step and -y_hi, with -y_lo
// added to the low part), for the refined path.  A list is
// evaluated when it fills and at the end: one shared broadcast load per candidate and no
// per-candidate test or vote in the far loop.  Partial sums are kept per list evaluation
// (op.row_begin / row_end).  An Op provides kMinBlocks, kUnroll, kR, init(), fetch(j, v)
// (the kR values of other point j), set_q(v) (those of the current candidate),
// coincident(np, t) (slot t = 0, 1 coincides with it), pair2(np, r2, dx, dy) (both slots
// packed; dx, dy and r2 in units of eps_I, so w = r2, and np carries eps2 = inv_eps2 = 1 and
// close2 = 1/64; pairs with r2 >= 1 must contribute nothing), row_begin(), row_end() and
// store(t, k).
constexpr int kListCap = 256;    // far candidates per warp
constexpr int kCloseCap = 64;    // close candidates per warp

// Ops with kAlt = true alternate two forms of the pair arithmetic between consecutive far
// candidates (pair2, pair2_alt) whose pipe mixes differ, so that the FMA and MUFU pipes share
// the load; the others evaluate every candidate with pair2.
template <class Op, class = void> struct AltForms : std::false_type {};
template <class Op> struct AltForms<Op, std::void_t<decltype(Op::kAlt)>> : std::bool_constant<Op::kAlt> {};

template <class Op>
__device__ __forceinline__ void near_eval_far(const float4 *s_xy, const float *s_q, int n, float2 X, float2 Y,
                                              const NearParams<float> &np, Op &op)
{
    op.row_begin();
    if constexpr (AltForms<Op>::value) {
        int e = 0;
#pragma unroll(Op::kUnroll / 2)
        for (; e + 1 < n; e += 2) {
            {
                const float4 a = s_xy[e];
                op.set_q(s_q + e * Op::kR);
                const float2 dx = add2(X, make_float2(a.x, a.y));
                const float2 dy = add2(Y, make_float2(a.z, a.w));
                op.pair2(np, fma2(dy, dy, mul2(dx, dx)), dx, dy);
            }
            {
                const float4 a = s_xy[e + 1];
                op.set_q(s_q + (e + 1) * Op::kR);
                const float2 dx = add2(X, make_float2(a.x, a.y));
                const float2 dy = add2(Y, make_float2(a.z, a.w));
                op.pair2_alt(np, fma2(dy, dy, mul2(dx, dx)), dx, dy);
            }
        }
        if (e < n) {
            const float4 a = s_xy[e];
            op.set_q(s_q + e * Op::kR);
            const float2 dx = add2(X, make_float2(a.x, a.y));
            const float2 dy = add2(Y, make_float2(a.z, a.w));
            op.pair2(np, fma2(dy, dy, mul2(dx, dx)), dx, dy);
        }
    } else {
#pragma unroll(Op::kUnroll)
        for (int e = 0; e < n; ++e) {
            const float4 a = s_xy[e];
            op.set_q(s_q + e * Op::kR);
            const float2 dx = add2(X, make_float2(a.x, a.y));
            const float2 dy = add2(Y, make_float2(a.z, a.w));
            op.pair2(np, fma2(dy, dy, mul2(dx, dx)), dx, dy);
        }
    }
    op.row_end();
}

// Close candidates carry their negated position in the item's frame as hi + lo
// (n = -(offset of the cell step) - y, TwoSum-exact at list time), so the difference
// d = (x_hi + n_hi) + (x_lo + n_lo) keeps full FP32 relative accuracy however small it is:
// when x_hi and -n_hi are close the first sum is exact (Sterbenz), and when they are not,
// d is of their size and one rounding is harmless.  Exactly coincident points give d = 0
// (G(0) := 0); they are handled on a warp-uniform branch.  The exact difference is then scaled
// by ie = 1 / eps_I, the unit of every difference handed to the Op.
template <class Op>
__device__ __forceinline__ void near_eval_close(const float4 *s_cxy, const float4 *s_cl, const float *s_cq, int n,
                                                float2 X, float2 Y, float2 XL, float2 YL, float ie,
                                                const NearParams<float> &np, Op &op)
{
    op.row_begin();
    for (int e = 0; e < n; ++e) {
        const float4 c = s_cxy[e];                // (n_hi.x, n_hi.x, n_hi.y, n_hi.y)
        const float4 l = s_cl[e];                 // (n_lo.x, n_lo.x, n_lo.y, n_lo.y)
        op.set_q(s_cq + e * Op::kR);
        const float2 ex = add2(add2(X, make_float2(c.x, c.y)), add2(XL, make_float2(l.x, l.y)));
        const float2 ey = add2(add2(Y, make_float2(c.z, c.w)), add2(YL, make_float2(l.z, l.w)));
        const float2 dx = mul2(ex, f2(ie)), dy = mul2(ey, f2(ie));   // in units of eps_I
        float2 r2 = fma2(dy, dy, mul2(dx, dx));
        const bool z0 = ex.x == 0.f && ey.x == 0.f, z1 = ex.y == 0.f && ey.y == 0.f;
        if (__any_sync(0xffffffffu, z0 || z1)) {
            if (z0) {
                op.coincident(np, 0);
                r2.x = np.eps2;                   // masked out: w = 1
            }
            if (z1) {
                op.coincident(np, 1);
                r2.y = np.eps2;
            }
        }
        op.pair2(np, r2, dx, dy);
    }
    op.row_end();
}

template <class Op>
__device__ __forceinline__ void near_traverse_list(int2 item, int lane, const NearSides &sd, const CellGrid &cg,
                                                   const NearParams<float> &np, Op &op, float4 *s_xy, float *s_q,
                                                   float4 *s_cxy, float4 *s_cl, float *s_cq)
{
    constexpr int R = Op::kR;
    const float h = np.hcell, eps = sqrtf(np.eps2);
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
        const int packed = sd.own_base[kk];
        cc1[t] = base1(packed) / cg.cell;
        cc2[t] = base2(packed) / cg.cell;
        xh[t] = sd.own_hi[kk];
        xl[t] = sd.own_lo[kk];
        if (valid[t]) {
            const float ax = (float)cc1[t] * h + xh[t].x, ay = (float)cc2[t] * h + xh[t].y;
            tx0 = fminf(tx0, ax);
            tx1 = fmaxf(tx1, ax);
            ty0 = fminf(ty0, ay);
            ty1 = fmaxf(ty1, ay);
        }
    }
    tx0 = warp_min(tx0);
    tx1 = warp_max(tx1);
    ty0 = warp_min(ty0);
    ty1 = warp_max(ty1);
    const int c1 = cc1[0], c2 = cc2[0];
#pragma unroll
    for (int t = 0; t < 2; ++t)
        if (!valid[t])
            xh[t] = make_float2(1e6f, 1e6f);      // idle slots: every pair lands beyond eps_I
    const float2 X = make_float2(xh[0].x, xh[1].x), Y = make_float2(xh[0].y, xh[1].y);
    const float2 XL = make_float2(xl[0].x, xl[1].x), YL = make_float2(xl[0].y, xl[1].y);
    // the Op sees differences in units of eps_I, so w = r^2 needs no scaling per pair: the far
    // list holds sources in those units and the item's points are scaled once here
    const float ie = sqrtf(np.inv_eps2);
    const float2 XS = mul2(X, f2(ie)), YS = mul2(Y, f2(ie));
    NearParams<float> nps = np;
    nps.eps2 = 1.f;
    nps.inv_eps2 = 1.f;
    nps.close2 = 1.f / 64.f;
    const float margin = 1e-4f * eps + 1e-5f;
    const float reach = eps + margin;
    const float reach2 = reach * reach;
    const float close_reach = sqrtf(np.close2) + margin;
    const float close_reach2 = close_reach * close_reach;
    const int cx0 = max(0, (int)floorf((tx0 - reach) / h)), cx1 = min(cg.n_c - 1, (int)floorf((tx1 + reach) / h));
    const int cy0 = max(0, (int)floorf((ty0 - reach) / h)), cy1 = min(cg.n_c - 1, (int)floorf((ty1 + reach) / h));
    const unsigned below = (1u << lane) - 1u;
    int nf = 0, nc = 0;
    op.init();
    // whole neighbour cells (contiguous source ranges), read in full chunks of 32
    for (int ex = cx0; ex <= cx1; ++ex) {
        const float offx = (float)(c1 - ex) * h;
        const float sx0 = (float)ex * h;
        const float gapx = fmaxf(0.f, fmaxf(sx0 - tx1, tx0 - (sx0 + h)));
        for (int ey = cy0; ey <= cy1; ++ey) {
            const float offy = (float)(c2 - ey) * h;
            const float sy0 = (float)ey * h;
            const float gapy = fmaxf(0.f, fmaxf(sy0 - ty1, ty0 - (sy0 + h)));
            if (gapx * gapx + gapy * gapy > reach2)
                continue;                           // the whole cell is beyond reach (warp-uniform)
            const int kbase = cg.key(ex, ey) * kSub;
            const int j0 = sd.oth_start[kbase], j1 = sd.oth_start[kbase + kSub];
            for (int jb = j0; jb < j1; jb += 32) {
                const int j = jb + lane;
                const bool in = j < j1;
                float2 yh = make_float2(0.f, 0.f);
                float qv[R];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    qv[r] = 0.f;
                if (in) {
                    yh = __ldg(sd.oth_hi + j);
                    op.fetch(j, qv);
                }
                const float ax = sx0 + yh.x, ay = sy0 + yh.y;
                const float gx = fmaxf(0.f, fmaxf(ax - tx1, tx0 - ax));
                const float gy = fmaxf(0.f, fmaxf(ay - ty1, ty0 - ay));
                const float g2 = gx * gx + gy * gy;
                const bool keep = in && g2 <= reach2;
                const bool close = keep && g2 <= close_reach2;
                const unsigned mf = __ballot_sync(0xffffffffu, keep && !close);
                const unsigned mc = __ballot_sync(0xffffffffu, close);
                if (keep && !close) {
                    const int at = nf + __popc(mf & below);
                    // -(source in the item's frame), in units of eps_I
                    const float nx = (offx - yh.x) * ie, ny = (offy - yh.y) * ie;
                    s_xy[at] = make_float4(nx, nx, ny, ny);
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        s_q[at * R + r] = qv[r];
                }
                if (close) {
                    const int at = nc + __popc(mc & below);
                    const float2 yl = __ldg(sd.oth_lo + j);
                    // -(source in the item's frame) = off - y_hi - y_lo as hi + lo (TwoSum of off and -y_hi)
                    const float hx = offx - yh.x, bx = hx - offx;
                    const float lx = ((offx - (hx - bx)) + (-yh.x - bx)) - yl.x;
                    const float hy = offy - yh.y, by = hy - offy;
                    const float ly = ((offy - (hy - by)) + (-yh.y - by)) - yl.y;
                    s_cxy[at] = make_float4(hx, hx, hy, hy);
                    s_cl[at] = make_float4(lx, lx, ly, ly);
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        s_cq[at * R + r] = qv[r];
                }
                nf += __popc(mf);
                nc += __popc(mc);
                if (nf > kListCap - 32) {
                    __syncwarp();
                    near_eval_far(s_xy, s_q, nf, XS, YS, nps, op);
                    nf = 0;
                    __syncwarp();
                }
                if (nc > kCloseCap - 32) {
                    __syncwarp();
                    near_eval_close(s_cxy, s_cl, s_cq, nc, X, Y, XL, YL, ie, nps, op);
                    nc = 0;
                    __syncwarp();
                }
            }
        }
    }
    __syncwarp();
    near_eval_far(s_xy, s_q, nf, XS, YS, nps, op);
    near_eval_close(s_cxy, s_cl, s_cq, nc, X, Y, XL, YL, ie, nps, op);
#pragma unroll
    for (int t = 0; t < 2; ++t)
        if (valid[t])
            op.store(t, kt[t]);
}

// Warps per block of the candidate-list kernels (a warp per item), and their per-warp lists
// (R charges per candidate).  An Op's kMinBlocks counts blocks of four warps.
constexpr int kNearWarps = 4;
template <int R> struct NearLists {
    float4 xy[kNearWarps][kListCap];
    float q[kNearWarps][kListCap * R];
    float4 cxy[kNearWarps][kCloseCap];
    float4 cl[kNearWarps][kCloseCap];
    float cq[kNearWarps][kCloseCap * R];
};

template <class Op>
__global__ void __launch_bounds__(32 * kNearWarps, Op::kMinBlocks * 4 / kNearWarps) k_near_list(int64_t n_items, const int2 *__restrict__ items,
                                                                   NearSides sd, CellGrid cg, NearParams<float> np,
                                                                   Op op)
{
    __shared__ NearLists<Op::kR> L;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_items)
        return;                                   // whole warp past the end; no block-wide barrier follows
    near_traverse_list(items[warp], lane, sd, cg, np, op, L.xy[w], L.q[w], L.cxy[w], L.cl[w], L.cq[w]);
}

template <class Op> cudaError_t launch_near_list(int64_t n_items, const int2 *items, const NearSides &sd, CellGrid cg,
                                                 const NearParams<float> &np, const Op &op, cudaStream_t st)
{
    if (n_items <= 0)
        return cudaSuccess;
    const unsigned blocks = (unsigned)((n_items + kNearWarps - 1) / kNearWarps);
    k_near_list<Op><<<blocks, 32 * kNearWarps, 0, st>>>(n_items, items, sd, cg, np, op);
    return cudaGetLastError();
}

// ---- source-major forward near field (FP32), for plans with many more sources than targets
//
// FEM plans put several quadrature points around every node, so a cell holds few targets and
// a target item's box spans the whole cell.  Here a warp takes an item of at most 64 sources
// of one cell (compact) and keeps them in shared memory as packed pairs; it reads the targets
// of the neighbour cells within eps_I of the sources' box 32 at a time, lists those within
// reach (a second list for those within eps_I / 8 of the box), and each lane then takes one
// listed target and sums the item's sources on it, two per packed operation; phi, grad phi and
// the coincident charge are added to the target with atomics.  Close pairs are refined from
// the hi and lo parts exactly as in the target-major traversal.
constexpr int kSrcMajorCap = 128;   // listed targets per warp and list

template <int P, bool ALT = false>
__device__ __forceinline__ void near_src_pair(const NearParams<float> &np, float2 r2, float2 dx, float2 dy,
                                              float2 q2, float2 &phi, float2 &gx, float2 &gy)
{
    float2 w = mul2(r2, f2(np.inv_eps2));
    if constexpr (P >= 2)
        w = min1(w);                                      // f(1) = 0 and (w - 1)^(p-1) = 0: masked
    const float2 val = near_f2<P>(np, w);
    float2 coef;
    if constexpr (P >= 2 && ALT) {
        // the power form with the same sign, (1 - w)^(p-1) / w: the caller alternates the two
        // forms between consecutive sources so that the FMA and MUFU pipes share the load
        const float2 om = add2(w, f2(-1.f));
        coef = mul2(ipow2<P - 1>(make_float2(-om.x, -om.y)), rcp_2(w));
    } else if constexpr (P >= 2) {
        // |w - 1|^(p-1) / w = 2^((p-1) log2(1 - w) - log2 w) (log2 w shared with val; the sign
        // (-1)^(p-1) is applied at the store; w = 1 gives 2^-inf = 0)
        const float2 lw = lg2_2(w);
        const float2 om = add2(w, f2(-1.f));   // the value's w - 1: 1 - w = -om, no add of its own
        const float2 lo = lg2_2(make_float2(-om.x, -om.y));
        coef = ex2_2(fma2(f2((float)(P - 1)), lo, make_float2(-lw.x, -lw.y)));
    } else {
        coef = rcp_2(w);
    }
    if constexpr (P == 1)
        q2 = select2(r2, np.eps2, q2);
    phi = fma2(q2, val, phi);
    const float2 tq = mul2(q2, coef);
    gx = fma2(tq, dx, gx);
    gy = fma2(tq, dy, gy);
}

// One round per 32 listed targets.  Far entries: (x, y) in the item's frame and the target
// index; close entries: (hi x, hi y, lo x, lo y) and (cell step x, cell step y, index).
template <int P, bool CLOSE>
__device__ __forceinline__ void near_src_eval(const float4 *s_hi, const float4 *s_lo, const float2 *s_q,
                                              const float4 *ta, const float4 *tb, int n, int lane,
                                              const NearParams<float> &np, float rcoef, float *__restrict__ phi_s,
                                              float *__restrict__ grad_s, float *__restrict__ coinc)
{
    for (int base = 0; base < n; base += 32) {
        const int e = base + lane;
        const bool valid = e < n;
        const float4 A = valid ? ta[e] : make_float4(1e6f, 1e6f, 0.f, 0.f);
        const float4 B = (CLOSE && valid) ? tb[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int k = __float_as_int(CLOSE ? B.z : A.z);
        // frame position of the target (close entries carry hi parts and the cell step)
        const float tx = CLOSE ? A.x + B.x : A.x, ty = CLOSE ? A.y + B.y : A.y;
        const float2 X = f2(tx), Y = f2(ty);
        float2 phi = f2(0.f), gx = f2(0.f), gy = f2(0.f);
        float cq = 0.f;
#pragma unroll 2
        for (int i = 0; i < 32; ++i) {
            const float4 sh = s_hi[i];                    // (xa, xb, ya, yb)
            float2 q2 = s_q[i];
            float2 dx = add2(X, make_float2(-sh.x, -sh.y));
            float2 dy = add2(Y, make_float2(-sh.z, -sh.w));
            float2 r2 = fma2(dy, dy, mul2(dx, dx));
            if constexpr (CLOSE) {
                const float4 sl = s_lo[i];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (valid && (t == 0 ? r2.x : r2.y) < np.close2) {
                        const float ex = refine_diff(A.x, t == 0 ? sh.x : sh.y, B.x, A.z, t == 0 ? sl.x : sl.y);
                        const float ey = refine_diff(A.y, t == 0 ? sh.z : sh.w, B.y, A.w, t == 0 ? sl.z : sl.w);
                        float e2 = ex * ex + ey * ey;
                        if (ex == 0.f && ey == 0.f) {             // coincident: G(0) := 0
                            const float qs = t == 0 ? q2.x : q2.y;
                            add_comp(phi, t, -qs * np.beta[0]);
                            cq += qs;
                            e2 = np.eps2;                          // masked out: w = 1
                        }
                        if (t == 0) {
                            dx.x = ex;
                            dy.x = ey;
                            r2.x = e2;
                        } else {
                            dx.y = ex;
                            dy.y = ey;
                            r2.y = e2;
                        }
                    }
                }
            }
            if (i & 1)
                near_src_pair<P, true>(np, r2, dx, dy, q2, phi, gx, gy);
            else
                near_src_pair<P, false>(np, r2, dx, dy, q2, phi, gx, gy);
        }
        if (valid) {
            const float rc = (P >= 2 && (P - 1) % 2 == 1) ? -rcoef : rcoef;   // near_src_pair's coef is |w - 1|^(p-1) / w
            atomicAdd(phi_s + k, phi.x + phi.y);
            atomicAdd(grad_s + 2 * (int64_t)k, rc * (gx.x + gx.y));
            atomicAdd(grad_s + 2 * (int64_t)k + 1, rc * (gy.x + gy.y));
            if (CLOSE && cq != 0.f)
                atomicAdd(coinc + k, cq);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(128) k_near_src32(int64_t n_items, const int2 *__restrict__ items, NearSides sd,
                                                    CellGrid cg, NearParams<float> np, const float *__restrict__ q,
                                                    float *__restrict__ phi_s, float *__restrict__ grad_s,
                                                    float *__restrict__ coinc)
{
    __shared__ float4 s_hi_all[4][32], s_lo_all[4][32];
    __shared__ float2 s_q_all[4][32];
    __shared__ float4 far_all[4][kSrcMajorCap], ca_all[4][kSrcMajorCap], cb_all[4][kSrcMajorCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_items)
        return;                                   // whole warp past the end; no block-wide barrier follows
    float4 *s_hi = s_hi_all[w], *s_lo = s_lo_all[w], *far = far_all[w], *ca = ca_all[w], *cb = cb_all[w];
    float2 *s_q = s_q_all[w];
    const int2 item = items[warp];
    // the item's sources (own side): slots a = lane, b = lane + 32; idle slots copy the first
    // source with charge 0
    const bool va = lane < item.y, vb = lane + 32 < item.y;
    const int64_t ja = va ? item.x + lane : item.x, jb = vb ? item.x + 32 + lane : item.x;
    const float2 ha = sd.own_hi[ja], hb = sd.own_hi[jb], la = sd.own_lo[ja], lb = sd.own_lo[jb];
    s_hi[lane] = make_float4(ha.x, hb.x, ha.y, hb.y);
    s_lo[lane] = make_float4(la.x, lb.x, la.y, lb.y);
    s_q[lane] = make_float2(va ? __ldg(q + ja) : 0.f, vb ? __ldg(q + jb) : 0.f);
    const int packed = sd.own_base[item.x];
    const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
    const float h = np.hcell, eps = sqrtf(np.eps2);
    // the sources' box in the item's frame (offsets from the item cell's corner)
    const float lx = warp_min(fminf(ha.x, hb.x)), hx = warp_max(fmaxf(ha.x, hb.x));
    const float ly = warp_min(fminf(ha.y, hb.y)), hy = warp_max(fmaxf(ha.y, hb.y));
    const float margin = 1e-4f * eps + 1e-5f;
    const float reach = eps + margin, reach2 = reach * reach;
    const float close_reach = sqrtf(np.close2) + margin, close_reach2 = close_reach * close_reach;
    const unsigned below = (1u << lane) - 1u;
    const float rcoef = np.rcoef;
    __syncwarp();
    int nf = 0, nc = 0;
    for (int e1 = max(c1 - 1, 0); e1 <= min(c1 + 1, cg.n_c - 1); ++e1) {
        const float ox = (float)(e1 - c1) * h;        // cell step into the item's frame
        const float gxc = fmaxf(0.f, fmaxf(ox - hx, lx - (ox + h)));
        for (int e2 = max(c2 - 1, 0); e2 <= min(c2 + 1, cg.n_c - 1); ++e2) {
            const float oy = (float)(e2 - c2) * h;
            const float gyc = fmaxf(0.f, fmaxf(oy - hy, ly - (oy + h)));
            if (gxc * gxc + gyc * gyc > reach2)
                continue;                             // the whole cell is beyond reach (warp-uniform)
            const int kbase = cg.key(e1, e2) * kSub;
            const int j0 = sd.oth_start[kbase], j1 = sd.oth_start[kbase + kSub];
            for (int jb0 = j0; jb0 < j1; jb0 += 32) {
                const int j = jb0 + lane;
                const bool in = j < j1;
                float2 th = make_float2(0.f, 0.f);
                if (in)
                    th = __ldg(sd.oth_hi + j);
                const float tx = th.x + ox, ty = th.y + oy;
                const float dxb = fmaxf(0.f, fmaxf(tx - hx, lx - tx));
                const float dyb = fmaxf(0.f, fmaxf(ty - hy, ly - ty));
                const float g2 = dxb * dxb + dyb * dyb;
                const bool keep = in && g2 <= reach2;
                const bool close = keep && g2 <= close_reach2;
                const unsigned mf = __ballot_sync(0xffffffffu, keep && !close);
                const unsigned mc = __ballot_sync(0xffffffffu, close);
                if (keep && !close)
                    far[nf + __popc(mf & below)] = make_float4(tx, ty, __int_as_float(j), 0.f);
                if (close) {
                    const int at = nc + __popc(mc & below);
                    const float2 tl = __ldg(sd.oth_lo + j);
                    ca[at] = make_float4(th.x, th.y, tl.x, tl.y);
                    cb[at] = make_float4(ox, oy, __int_as_float(j), 0.f);
                }
                nf += __popc(mf);
                nc += __popc(mc);
                if (nf > kSrcMajorCap - 32) {
                    __syncwarp();
                    near_src_eval<P, false>(s_hi, s_lo, s_q, far, nullptr, nf, lane, np, rcoef, phi_s, grad_s, coinc);
                    nf = 0;
                    __syncwarp();
                }
                if (nc > kSrcMajorCap - 32) {
                    __syncwarp();
                    near_src_eval<P, true>(s_hi, s_lo, s_q, ca, cb, nc, lane, np, rcoef, phi_s, grad_s, coinc);
                    nc = 0;
                    __syncwarp();
                }
            }
        }
    }
    __syncwarp();
    near_src_eval<P, false>(s_hi, s_lo, s_q, far, nullptr, nf, lane, np, rcoef, phi_s, grad_s, coinc);
    near_src_eval<P, true>(s_hi, s_lo, s_q, ca, cb, nc, lane, np, rcoef, phi_s, grad_s, coinc);
}

// Calls f(std::integral_constant<int, P>) for the expansion degree p in 1..16.
template <class F> cudaError_t with_degree(int p, F &&f)
{
    switch (p) {
#define FS_P_CASE(P)                                                                                             \
    case P:                                                                                                      \
        return f(std::integral_constant<int, P>{});
        FS_P_CASE(1)
        FS_P_CASE(2)
        FS_P_CASE(3)
        FS_P_CASE(4)
        FS_P_CASE(5)
        FS_P_CASE(6)
        FS_P_CASE(7)
        FS_P_CASE(8)
        FS_P_CASE(9)
        FS_P_CASE(10)
        FS_P_CASE(11)
        FS_P_CASE(12)
        FS_P_CASE(13)
        FS_P_CASE(14)
        FS_P_CASE(15)
        FS_P_CASE(16)
#undef FS_P_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace fs
