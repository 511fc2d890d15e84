// FEM magnetic-charge assembly (step a): the quadrature of Eq. (2).
//
// With M linear in each P1 triangle T (nodes a, b, c), rho = -div M is constant
// on T:  rho_T = -(M_a . grad la_a + M_b . grad la_b + M_c . grad la_c), where
// grad la_a = (y_b - y_c, x_c - x_b) / (2A) (A the signed area, cyclic in a,b,c).
// Three interior points at barycentric (2/3, 1/6, 1/6) and permutations carry
// q = rho_T |T| / 3 each (omega det J = |T|/3).  Each boundary edge e (used by one
// triangle; endpoints lo < hi; `third` the owner's remaining node) carries two
// Gauss-Legendre points t = 1/2 -+ 1/(2 sqrt 3) measured from lo, with
// q = (M(t) . n_e) |e| / 2, n_e the outward unit normal (pointing away from
// `third`) and M(t) = (1-t) M_lo + t M_hi.
//
// Source order: 3 per triangle (triangle-major), then 2 per boundary edge.  For a time loop
// (one plan, many M(t)) the assembly is fused with the gather into cell order
// (k_fem_charges_scatter: each element's charges computed once and written to their sorted
// slots), so a magnetisation becomes sorted charges in one pass.
#include "internal.h"

namespace fs {

namespace {

constexpr double kGaussLo = 0.5 - 0.28867513459481288225457439025097873;   // 1/2 - 1/(2 sqrt 3)
constexpr double kGaussHi = 0.5 + 0.28867513459481288225457439025097873;

__global__ void k_fem_sources(const double2 *__restrict__ nodes, const int *__restrict__ tris, int64_t Nt,
                              const int *__restrict__ bedges, int64_t Ne, double2 *__restrict__ src)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < Nt) {
        const double2 pa = nodes[tris[3 * i]], pb = nodes[tris[3 * i + 1]], pc = nodes[tris[3 * i + 2]];
        const double big = 2.0 / 3.0, small = 1.0 / 6.0;
        src[3 * i] = make_double2(big * pa.x + small * pb.x + small * pc.x, big * pa.y + small * pb.y + small * pc.y);
        src[3 * i + 1] = make_double2(small * pa.x + big * pb.x + small * pc.x, small * pa.y + big * pb.y + small * pc.y);
        src[3 * i + 2] = make_double2(small * pa.x + small * pb.x + big * pc.x, small * pa.y + small * pb.y + big * pc.y);
    } else if (i < Nt + Ne) {
        const int64_t e = i - Nt;
        const double2 p0 = nodes[bedges[3 * e]], p1 = nodes[bedges[3 * e + 1]];
        const int64_t o = 3 * Nt + 2 * e;
        src[o] = make_double2(p0.x + kGaussLo * (p1.x - p0.x), p0.y + kGaussLo * (p1.y - p0.y));
        src[o + 1] = make_double2(p0.x + kGaussHi * (p1.x - p0.x), p0.y + kGaussHi * (p1.y - p0.y));
    }
}

// Charge of one triangle point: rho_T |T| / 3 (the same for its three points).  With
// S = sum_k M_k . (rotated opposite edge) = -rho_T 2A (A the signed area),
// rho_T |T| / 3 = -(S / 2A) |2A| / 6 = -S sign(2A) / 6: no division.
__device__ __forceinline__ double triangle_charge(const double2 *__restrict__ nodes, const int *__restrict__ tris,
                                                  int64_t t, const double2 *__restrict__ mg)
{
    const int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
    const double2 pa = nodes[ia], pb = nodes[ib], pc = nodes[ic];
    const double two_a = (pb.x - pa.x) * (pc.y - pa.y) - (pb.y - pa.y) * (pc.x - pa.x);
    const double2 ma = mg[ia], mb = mg[ib], mc = mg[ic];
    const double S = ma.x * (pb.y - pc.y) + ma.y * (pc.x - pb.x) + mb.x * (pc.y - pa.y) + mb.y * (pa.x - pc.x) +
                     mc.x * (pa.y - pb.y) + mc.y * (pb.x - pa.x);
    return two_a > 0.0 ? S * (-1.0 / 6.0) : S * (1.0 / 6.0);
}

// The triangle's charge as a linear form in its nodal magnetisations: rho_T |T| / 3 =
// sum_k M_k . c_k with c_k the rotated opposite edge times -sign(2A) / 6 (the geometry part of
// triangle_charge, computed once with the plan; a time step then takes 6 FP64 FMAs per triangle).
__global__ void k_fem_tri_coef(const double2 *__restrict__ nodes, const int *__restrict__ tris, int64_t Nt,
                               double2 *__restrict__ coef)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= Nt)
        return;
    const double2 pa = nodes[tris[3 * t]], pb = nodes[tris[3 * t + 1]], pc = nodes[tris[3 * t + 2]];
    const double two_a = (pb.x - pa.x) * (pc.y - pa.y) - (pb.y - pa.y) * (pc.x - pa.x);
    const double s = two_a > 0.0 ? -1.0 / 6.0 : 1.0 / 6.0;
    coef[3 * t] = make_double2(s * (pb.y - pc.y), s * (pc.x - pb.x));
    coef[3 * t + 1] = make_double2(s * (pc.y - pa.y), s * (pa.x - pc.x));
    coef[3 * t + 2] = make_double2(s * (pa.y - pb.y), s * (pb.x - pa.x));
}

// Charge of Gauss point g (0: t = 1/2 - 1/(2 sqrt 3), 1: t = 1/2 + 1/(2 sqrt 3)) of boundary edge e:
// (M(t) . n_e) |e| / 2 with n_e |e| = +-(t_y, -t_x) for the edge vector t (outward sign): no
// square root or division.
__device__ __forceinline__ double edge_charge(const double2 *__restrict__ nodes, const int *__restrict__ bedges,
                                              int64_t e, int g, const double2 *__restrict__ mg)
{
    const int i0 = bedges[3 * e], i1 = bedges[3 * e + 1], i3 = bedges[3 * e + 2];
    const double2 p0 = nodes[i0], p1 = nodes[i1], p3 = nodes[i3];
    const double tx = p1.x - p0.x, ty = p1.y - p0.y;
    double nx = ty, ny = -tx;                      // normal scaled by |e|
    if (nx * (p3.x - p0.x) + ny * (p3.y - p0.y) > 0.0) {
        nx = -nx;
        ny = -ny;
    }
    const double2 m0 = mg[i0], m1 = mg[i1];
    const double t = g == 0 ? kGaussLo : kGaussHi;
    return (((1.0 - t) * m0.x + t * m1.x) * nx + ((1.0 - t) * m0.y + t * m1.y) * ny) * 0.5;
}

__global__ void k_fem_charges(const double2 *__restrict__ nodes, const int *__restrict__ tris, int64_t Nt,
                              const int *__restrict__ bedges, int64_t Ne, const double2 *__restrict__ mag, int64_t Nv,
                              double *__restrict__ q, int64_t M)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const double2 *mg = mag + (int64_t)r * Nv;
    double *qr = q + (int64_t)r * M;
    if (i < Nt) {
        const double qt = triangle_charge(nodes, tris, i, mg);
        qr[3 * i] = qt;
        qr[3 * i + 1] = qt;
        qr[3 * i + 2] = qt;
    } else if (i < Nt + Ne) {
        const int64_t e = i - Nt;
        const int64_t o = 3 * Nt + 2 * e;
        qr[o] = edge_charge(nodes, bedges, e, 0, mg);
        qr[o + 1] = edge_charge(nodes, bedges, e, 1, mg);
    }
}

// Charges straight into cell order (the assembly fused with the gather of fs_set_charges):
// one thread per triangle (or boundary edge) computes its charge once, in FP64, and writes it
// to the sorted slots of its quadrature points (inv_perm: source index -> sorted index, built
// with the plan), in the plan's precision; the block sums go to q_sum.
template <typename real>
__global__ void k_fem_charges_scatter(const double2 *__restrict__ nodes, const int *__restrict__ tris, int64_t Nt,
                                      const double2 *__restrict__ tri_coef, const int *__restrict__ bedges,
                                      int64_t Ne, const double2 *__restrict__ mag, int64_t Nv,
                                      const int *__restrict__ inv_perm, int64_t M, real *__restrict__ q_sorted,
                                      double *__restrict__ q_sum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const double2 *mg = mag + (int64_t)r * Nv;
    real *qs = q_sorted + (int64_t)r * M;
    double v = 0.0;
    if (i < Nt) {
        double qt;
        if (tri_coef) {
            const double2 ma = mg[tris[3 * i]], mb = mg[tris[3 * i + 1]], mc = mg[tris[3 * i + 2]];
            const double2 ca = tri_coef[3 * i], cb = tri_coef[3 * i + 1], cc = tri_coef[3 * i + 2];
            qt = ma.x * ca.x + ma.y * ca.y + mb.x * cb.x + mb.y * cb.y + mc.x * cc.x + mc.y * cc.y;
        } else {
            qt = triangle_charge(nodes, tris, i, mg);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
            qs[inv_perm[3 * i + p]] = (real)qt;
        v = 3.0 * qt;
    } else if (i < Nt + Ne) {
        const int64_t e = i - Nt, o = 3 * Nt + 2 * e;
        const double q0 = edge_charge(nodes, bedges, e, 0, mg), q1 = edge_charge(nodes, bedges, e, 1, mg);
        qs[inv_perm[o]] = (real)q0;
        qs[inv_perm[o + 1]] = (real)q1;
        v = q0 + q1;
    }
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0)
            atomicAdd(&q_sum[r], v);
    }
}

__global__ void k_invert_perm(const int *__restrict__ perm, int64_t n, int *__restrict__ inv)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n)
        inv[perm[k]] = (int)k;
}

// ---------------------------------------------------------------- tetrahedra (d = 3)
//
// The same quadrature with d = 3.  M linear in a P1 tetrahedron (nodes x0..x3) has
// div M = sum_{k=1..3} (M_k - M_0) . grad la_k with grad la_k the rows of J^-1,
// J = [u v w] = [x1 - x0, x2 - x0, x3 - x0]:  J^-1 = [v x w; w x u; u x v] / det J.
// Four points at barycentric (a, b, b, b) and permutations, a = (5 + 3 sqrt 5)/20,
// b = (5 - sqrt 5)/20, carry q = -div M |T| / 4 each (|T| = |det J| / 6).  Each boundary
// face (nodes i0 < i1 < i2 used by one tetrahedron; `opp` its fourth node) carries three
// points at barycentric (2/3, 1/6, 1/6) and permutations with q = (M . n_F) |F| / 3,
// n_F the outward unit normal (pointing away from opp).
// Source order: 4 per tetrahedron (tetrahedron-major), then 3 per boundary face.

constexpr double kTetA = 0.58541019662496845446137605030969143;   // (5 + 3 sqrt 5) / 20
constexpr double kTetB = 0.13819660112501051517954131656343619;   // (5 - sqrt 5) / 20

struct V3 {
    double x, y, z;
};

__device__ __forceinline__ V3 ld3(const double *__restrict__ a, int64_t i)
{
    return V3{a[3 * i], a[3 * i + 1], a[3 * i + 2]};
}
__device__ __forceinline__ V3 sub3(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross3(V3 a, V3 b)
{
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

__global__ void k_fem3_sources(const double *__restrict__ nodes, const int *__restrict__ tets, int64_t Nt,
                               const int *__restrict__ faces, int64_t Nf, double *__restrict__ src)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < Nt) {
        V3 p[4];
        for (int k = 0; k < 4; ++k)
            p[k] = ld3(nodes, tets[4 * i + k]);
        const V3 sum{p[0].x + p[1].x + p[2].x + p[3].x, p[0].y + p[1].y + p[2].y + p[3].y,
                     p[0].z + p[1].z + p[2].z + p[3].z};
        for (int k = 0; k < 4; ++k) {
            double *o = src + 3 * (4 * i + k);
            o[0] = kTetB * sum.x + (kTetA - kTetB) * p[k].x;
            o[1] = kTetB * sum.y + (kTetA - kTetB) * p[k].y;
            o[2] = kTetB * sum.z + (kTetA - kTetB) * p[k].z;
        }
    } else if (i < Nt + Nf) {
        const int64_t f = i - Nt;
        V3 p[3];
        for (int k = 0; k < 3; ++k)
            p[k] = ld3(nodes, faces[4 * f + k]);
        const V3 sum{p[0].x + p[1].x + p[2].x, p[0].y + p[1].y + p[2].y, p[0].z + p[1].z + p[2].z};
        for (int k = 0; k < 3; ++k) {
            double *o = src + 3 * (4 * Nt + 3 * f + k);
            o[0] = sum.x / 6.0 + 0.5 * p[k].x;
            o[1] = sum.y / 6.0 + 0.5 * p[k].y;
            o[2] = sum.z / 6.0 + 0.5 * p[k].z;
        }
    }
}

// Charge of each of the four points of tetrahedron t: -div M |T| / 4.
__device__ __forceinline__ double tet_charge(const double *__restrict__ nodes, const int *__restrict__ tets,
                                             int64_t t, const double *__restrict__ mg)
{
    const int i0 = tets[4 * t], i1 = tets[4 * t + 1], i2 = tets[4 * t + 2], i3 = tets[4 * t + 3];
    const V3 x0 = ld3(nodes, i0);
    const V3 u = sub3(ld3(nodes, i1), x0), v = sub3(ld3(nodes, i2), x0), w = sub3(ld3(nodes, i3), x0);
    const V3 m0 = ld3(mg, i0);
    const V3 vw = cross3(v, w), wu = cross3(w, u), uv = cross3(u, v);
    const double det = dot3(u, vw);
    // div M * det = sum_k (M_k - M_0) . (row k of adj J); q = -div M |det| / 24
    const double num = dot3(sub3(ld3(mg, i1), m0), vw) + dot3(sub3(ld3(mg, i2), m0), wu) +
                       dot3(sub3(ld3(mg, i3), m0), uv);
    return det > 0.0 ? num * (-1.0 / 24.0) : num * (1.0 / 24.0);
}

// The tetrahedron's charge as sum_{k=1..3} (M_k - M_0) . g_k, g_k the rows of adj J times
// -sign(det) / 24 (the geometry of tet_charge, once with the plan; 9 doubles per tetrahedron):
// a time step takes 9 subtractions and 9 FMAs in FP64 instead of ~58 operations, and a uniform
// M still gives exactly zero.
__global__ void k_fem3_tet_coef(const double *__restrict__ nodes, const int *__restrict__ tets, int64_t Nt,
                                double *__restrict__ coef)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= Nt)
        return;
    const int i0 = tets[4 * t], i1 = tets[4 * t + 1], i2 = tets[4 * t + 2], i3 = tets[4 * t + 3];
    const V3 x0 = ld3(nodes, i0);
    const V3 u = sub3(ld3(nodes, i1), x0), v = sub3(ld3(nodes, i2), x0), w = sub3(ld3(nodes, i3), x0);
    const V3 vw = cross3(v, w), wu = cross3(w, u), uv = cross3(u, v);
    const double s = dot3(u, vw) > 0.0 ? -1.0 / 24.0 : 1.0 / 24.0;
    double *c = coef + 9 * t;
    const V3 g[3] = {vw, wu, uv};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c[3 * k] = s * g[k].x;
        c[3 * k + 1] = s * g[k].y;
        c[3 * k + 2] = s * g[k].z;
    }
}

// Charge of point k (the 2/3 weight on node k) of boundary face f: (M . n_F) |F| / 3.
__device__ __forceinline__ double face_charge(const double *__restrict__ nodes, const int *__restrict__ faces,
                                              int64_t f, int k, const double *__restrict__ mg)
{
    const int i0 = faces[4 * f], i1 = faces[4 * f + 1], i2 = faces[4 * f + 2], io = faces[4 * f + 3];
    const V3 p0 = ld3(nodes, i0);
    const V3 c = cross3(sub3(ld3(nodes, i1), p0), sub3(ld3(nodes, i2), p0));   // |c| = 2 |F|
    const double sgn = dot3(c, sub3(ld3(nodes, io), p0)) > 0.0 ? -1.0 : 1.0;   // outward
    const int ik = k == 0 ? i0 : (k == 1 ? i1 : i2);
    const V3 ma = ld3(mg, i0), mb = ld3(mg, i1), mc = ld3(mg, i2), mk = ld3(mg, ik);
    const V3 mp{(ma.x + mb.x + mc.x) / 6.0 + 0.5 * mk.x, (ma.y + mb.y + mc.y) / 6.0 + 0.5 * mk.y,
                (ma.z + mb.z + mc.z) / 6.0 + 0.5 * mk.z};
    // (M . c/|c|) (|c|/2) / 3 = M . c / 6
    return sgn * dot3(mp, c) / 6.0;
}

__device__ __forceinline__ double fem3_point_charge(const double *__restrict__ nodes, const int *__restrict__ tets,
                                                    int64_t Nt, const int *__restrict__ faces, int64_t i,
                                                    const double *__restrict__ mg)
{
    if (i < 4 * Nt)
        return tet_charge(nodes, tets, i >> 2, mg);
    const int64_t j = i - 4 * Nt;
    return face_charge(nodes, faces, j / 3, (int)(j % 3), mg);
}

__global__ void k_fem3_charges(const double *__restrict__ nodes, const int *__restrict__ tets, int64_t Nt,
                               const int *__restrict__ faces, const double *__restrict__ mag, int64_t Nv,
                               double *__restrict__ q, int64_t M)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i < M)
        q[(int64_t)r * M + i] = fem3_point_charge(nodes, tets, Nt, faces, i, mag + (int64_t)r * 3 * Nv);
}

// 3D assembly straight into cell order (as k_fem_charges_scatter): one thread per tetrahedron
// (its four points share one charge) or boundary face (one normal for its three points).
template <typename real>
__global__ void k_fem3_charges_scatter(const double *__restrict__ nodes, const int *__restrict__ tets, int64_t Nt,
                                       const double *__restrict__ tet_coef, const int *__restrict__ faces, int64_t Nf,
                                       const double *__restrict__ mag, int64_t Nv, const int *__restrict__ inv_perm,
                                       int64_t M, real *__restrict__ q_sorted, double *__restrict__ q_sum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const double *mg = mag + (int64_t)r * 3 * Nv;
    real *qs = q_sorted + (int64_t)r * M;
    double v = 0.0;
    if (i < Nt) {
        double qt;
        if (tet_coef) {
            const V3 m0 = ld3(mg, tets[4 * i]);
            const double *c = tet_coef + 9 * i;
            qt = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const V3 d = sub3(ld3(mg, tets[4 * i + 1 + k]), m0);
                qt += d.x * c[3 * k] + d.y * c[3 * k + 1] + d.z * c[3 * k + 2];
            }
        } else {
            qt = tet_charge(nodes, tets, i, mg);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
            qs[inv_perm[4 * i + p]] = (real)qt;
        v = 4.0 * qt;
    } else if (i < Nt + Nf) {
        const int64_t f = i - Nt;
        const int i0 = faces[4 * f], i1 = faces[4 * f + 1], i2 = faces[4 * f + 2], io = faces[4 * f + 3];
        const V3 p0 = ld3(nodes, i0);
        const V3 c = cross3(sub3(ld3(nodes, i1), p0), sub3(ld3(nodes, i2), p0));   // |c| = 2 |F|
        const double sgn = dot3(c, sub3(ld3(nodes, io), p0)) > 0.0 ? -1.0 : 1.0;   // outward
        const V3 ma = ld3(mg, i0), mb = ld3(mg, i1), mc = ld3(mg, i2);
        const double mean6 = dot3(V3{ma.x + mb.x + mc.x, ma.y + mb.y + mc.y, ma.z + mb.z + mc.z}, c) * (1.0 / 6.0);
        const int64_t o = 4 * Nt + 3 * f;
        const V3 mk[3] = {ma, mb, mc};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // (M . n_F) |F| / 3 with M = (Ma + Mb + Mc)/6 + Mk/2 at the point: M . c / 6
            const double qk = sgn * (mean6 + 0.5 * dot3(mk[k], c)) * (1.0 / 6.0);
            qs[inv_perm[o + k]] = (real)qk;
            v += qk;
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0)
            atomicAdd(&q_sum[r], v);
    }
}

}  // namespace

cudaError_t launch_fem3_sources(const double *nodes, const int *tets, int64_t Nt, const int *faces, int64_t Nf,
                                double *src, cudaStream_t st)
{
    const int64_t n = Nt + Nf;
    if (n <= 0)
        return cudaSuccess;
    k_fem3_sources<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nodes, tets, Nt, faces, Nf, src);
    return cudaGetLastError();
}

cudaError_t launch_fem3_charges(const double *nodes, const int *tets, int64_t Nt, const int *faces,
                                const double *mag, int64_t Nv, int nrhs, double *q, int64_t M, cudaStream_t st)
{
    if (M <= 0 || nrhs <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)((M + 255) / 256), nrhs);
    k_fem3_charges<<<grid, 256, 0, st>>>(nodes, tets, Nt, faces, mag, Nv, q, M);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fem3_charges_scatter(const double *nodes, const int *tets, int64_t Nt, const double *tet_coef,
                                        const int *faces, int64_t Nf, const double *mag, int64_t Nv, int nrhs,
                                        const int *inv_perm, int64_t M, real *q_sorted, double *q_sum,
                                        cudaStream_t st)
{
    const int64_t n = Nt + Nf;
    if (n <= 0 || nrhs <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    k_fem3_charges_scatter<real><<<grid, 256, 0, st>>>(nodes, tets, Nt, tet_coef, faces, Nf, mag, Nv, inv_perm, M,
                                                        q_sorted, q_sum);
    return cudaGetLastError();
}

cudaError_t launch_fem3_tet_coef(const double *nodes, const int *tets, int64_t Nt, double *coef, cudaStream_t st)
{
    if (Nt <= 0)
        return cudaSuccess;
    k_fem3_tet_coef<<<(unsigned)((Nt + 255) / 256), 256, 0, st>>>(nodes, tets, Nt, coef);
    return cudaGetLastError();
}

template cudaError_t launch_fem3_charges_scatter<float>(const double *, const int *, int64_t, const double *,
                                                        const int *, int64_t, const double *, int64_t, int,
                                                        const int *, int64_t, float *, double *, cudaStream_t);
template cudaError_t launch_fem3_charges_scatter<double>(const double *, const int *, int64_t, const double *,
                                                         const int *, int64_t, const double *, int64_t, int,
                                                         const int *, int64_t, double *, double *, cudaStream_t);

cudaError_t launch_fem_sources(const double2 *nodes, const int *tris, int64_t Nt, const int *bedges, int64_t Ne,
                               double2 *src, cudaStream_t st)
{
    const int64_t n = Nt + Ne;
    if (n <= 0)
        return cudaSuccess;
    k_fem_sources<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nodes, tris, Nt, bedges, Ne, src);
    return cudaGetLastError();
}

cudaError_t launch_fem_charges(const double2 *nodes, const int *tris, int64_t Nt, const int *bedges, int64_t Ne,
                               const double2 *mag, int64_t Nv, int nrhs, double *q, int64_t M, cudaStream_t st)
{
    const int64_t n = Nt + Ne;
    if (n <= 0 || nrhs <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    k_fem_charges<<<grid, 256, 0, st>>>(nodes, tris, Nt, bedges, Ne, mag, Nv, q, M);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fem_charges_scatter(const double2 *nodes, const int *tris, int64_t Nt, const double2 *tri_coef,
                                       const int *bedges, int64_t Ne, const double2 *mag, int64_t Nv, int nrhs,
                                       const int *inv_perm, int64_t M, real *q_sorted, double *q_sum, cudaStream_t st)
{
    const int64_t n = Nt + Ne;
    if (n <= 0 || nrhs <= 0)
        return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), nrhs);
    k_fem_charges_scatter<real><<<grid, 256, 0, st>>>(nodes, tris, Nt, tri_coef, bedges, Ne, mag, Nv, inv_perm, M,
                                                       q_sorted, q_sum);
    return cudaGetLastError();
}

template cudaError_t launch_fem_charges_scatter<float>(const double2 *, const int *, int64_t, const double2 *,
                                                       const int *, int64_t, const double2 *, int64_t, int,
                                                       const int *, int64_t, float *, double *, cudaStream_t);
template cudaError_t launch_fem_charges_scatter<double>(const double2 *, const int *, int64_t, const double2 *,
                                                        const int *, int64_t, const double2 *, int64_t, int,
                                                        const int *, int64_t, double *, double *, cudaStream_t);

cudaError_t launch_fem_tri_coef(const double2 *nodes, const int *tris, int64_t Nt, double2 *coef, cudaStream_t st)
{
    if (Nt <= 0)
        return cudaSuccess;
    k_fem_tri_coef<<<(unsigned)((Nt + 255) / 256), 256, 0, st>>>(nodes, tris, Nt, coef);
    return cudaGetLastError();
}

cudaError_t launch_invert_perm(const int *perm, int64_t n, int *inv, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_invert_perm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(perm, n, inv);
    return cudaGetLastError();
}

}  // namespace fs
