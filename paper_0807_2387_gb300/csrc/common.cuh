// Device-side building blocks shared by the FEM-NFFT kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

constexpr int kMaxP = 16;        // largest smoothness degree
constexpr int kMaxM = 8;         // largest window half-width; taps per dimension = 2m <= 16
constexpr double kPi = 3.141592653589793238462643383279502884;

template <typename real> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Error codes written by kernels into the plan's device status word.
enum DeviceError : int { kDevOk = 0, kDevDomain = 2, kDevTimeout = 5 };

// Kaiser-Bessel window in grid-cell units x = n_os t, normalised to psi(0) = 1:
//   psi(x) = [m / sinh(b m)] sinh(b tau) / tau,   tau = sqrt(m^2 - x^2),  |x| < m,
// and 0 for |x| >= m.  Written without overflow as
//   psi = S e^{z - b m} (1 - e^{-2z}) / z,   z = b tau,   S = m b / (1 - e^{-2 b m}),
//   psi' = -x b^2 S e^{z - b m} F(z),   F(z) = ((z - 1) + (z + 1) e^{-2z}) / z^3,
// with F(z) = 2 e^{-z} sum_{k>=1} 2k z^{2k-2} / (2k+1)! for small z, and
// z - b m = b (tau - m) = -b x^2 / (tau + m).
template <typename real> struct Window {
    real m;
    real m2;
    real b;
    real bm;
    real S;
};

template <typename real> __device__ __forceinline__ real fexp(real x);
template <> __device__ __forceinline__ float fexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double fexp<double>(double x) { return exp(x); }
template <typename real> __device__ __forceinline__ real fexpm1(real x);
template <> __device__ __forceinline__ float fexpm1<float>(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double fexpm1<double>(double x) { return expm1(x); }
template <typename real> __device__ __forceinline__ real fsqrt(real x);
template <> __device__ __forceinline__ float fsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double fsqrt<double>(double x) { return sqrt(x); }
template <typename real> __device__ __forceinline__ real flog(real x);
template <> __device__ __forceinline__ float flog<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double flog<double>(double x) { return log(x); }

// psi at x = j + frac (j an integer tap offset, frac in [0, 1)).  tau^2 is formed as
// (m - x)(m + x) from exact integer parts, and the exponent z - b m as -b x^2 / (tau + m),
// so no cancellation occurs (e^{z - b m} computed from z ~ b m would lose ~log2(b m) bits).
template <typename real>
__device__ __forceinline__ real kb_value(const Window<real> &w, real frac, int j)
{
    const real t1 = (w.m - real(j)) - frac;   // m - x
    const real t2 = (w.m + real(j)) + frac;   // m + x
    if (!(t1 > real(0)) || !(t2 > real(0)))
        return real(0);
    const real tau = fsqrt<real>(t1 * t2);
    const real x = real(j) + frac;
    const real z = w.b * tau;
    const real e = w.S * fexp<real>(-w.b * x * x / (tau + w.m));
    return e * (-fexpm1<real>(real(-2) * z)) / z;
}

// F(z) = ((z-1) + (z+1) e^{-2z}) / z^3 (the slope factor of psi').
template <typename real>
__device__ __forceinline__ real kb_slope(real z)
{
    if (z < real(1)) {
        // 2 e^{-z} (1/3 + z^2/30 + z^4/840 + ...): coefficients 2k/(2k+1)!, k = 1..10
        const real z2 = z * z;
        real acc = real(20.0 / 51090942171709440000.0);
        acc = acc * z2 + real(18.0 / 121645100408832000.0);
        acc = acc * z2 + real(16.0 / 355687428096000.0);
        acc = acc * z2 + real(14.0 / 1307674368000.0);
        acc = acc * z2 + real(12.0 / 6227020800.0);
        acc = acc * z2 + real(10.0 / 39916800.0);
        acc = acc * z2 + real(8.0 / 362880.0);
        acc = acc * z2 + real(6.0 / 5040.0);
        acc = acc * z2 + real(4.0 / 120.0);
        acc = acc * z2 + real(2.0 / 6.0);
        return real(2) * fexp<real>(-z) * acc;
    }
    const real e = fexp<real>(real(-2) * z);
    return ((z - real(1)) + (z + real(1)) * e) / (z * z * z);
}

// psi and dpsi/dx together, at x = j + frac (see kb_value).
template <typename real>
__device__ __forceinline__ void kb_value_slope(const Window<real> &w, real frac, int j, real &v, real &d)
{
    const real t1 = (w.m - real(j)) - frac;
    const real t2 = (w.m + real(j)) + frac;
    if (!(t1 > real(0)) || !(t2 > real(0))) {
        v = real(0);
        d = real(0);
        return;
    }
    const real tau = fsqrt<real>(t1 * t2);
    const real x = real(j) + frac;
    const real z = w.b * tau;
    const real e = w.S * fexp<real>(-w.b * x * x / (tau + w.m));
    v = e * (-fexpm1<real>(real(-2) * z)) / z;
    d = -x * w.b * w.b * e * kb_slope<real>(z);
}

// FP32 window: per tap a (x = frac + m - 1 - a), a polynomial of degree kPolyD in
// t = frac - 1/2 interpolating psi at Chebyshev points (fitted in FP64 on the host;
// |error| <= 3e-11 of psi(0) for m = 6), and its exact derivative for psi'.  Only
// FMA-pipe work, where the closed form needs five MUFU operations per tap.
constexpr int kPolyD = 12;
struct WindowPoly {
    float c[2 * kMaxM][kPolyD + 1];   // value coefficients, c[a][i] multiplies t^i
    float d[2 * kMaxM][kPolyD];       // slope coefficients (d/dx), d[a][i] multiplies t^i
    float e[2 * kMaxM][kPolyD - 1];   // curvature coefficients (d^2/dx^2), e[a][i] multiplies t^i
};

// psi, psi' and psi'' at x = j + frac (closed form, used by the FP64 path):
//   psi'' = -b^2 S e^{z - bm} [F(z) - b^2 x^2 E(z)],   E(z) = ((z^2-3z+3) - e^{-2z}(z^2+3z+3)) / z^5
// (E = 2 e^{-z} (f'(z)/z) with f(z) = (z cosh z - sinh z)/z^3; series 2 e^{-z}(1/15 + z^2/210 + ...) near 0).
template <typename real>
__device__ __forceinline__ real kb_curv_factor(real z)
{
    if (z < real(1)) {
        // (2k-2)(2k)/(2k+1)! for k = 2..11
        const real z2 = z * z;
        real acc = real(20.0 * 22.0 / 25852016738884976640000.0);
        acc = acc * z2 + real(18.0 * 20.0 / 51090942171709440000.0);
        acc = acc * z2 + real(16.0 * 18.0 / 121645100408832000.0);
        acc = acc * z2 + real(14.0 * 16.0 / 355687428096000.0);
        acc = acc * z2 + real(12.0 * 14.0 / 1307674368000.0);
        acc = acc * z2 + real(10.0 * 12.0 / 6227020800.0);
        acc = acc * z2 + real(8.0 * 10.0 / 39916800.0);
        acc = acc * z2 + real(6.0 * 8.0 / 362880.0);
        acc = acc * z2 + real(4.0 * 6.0 / 5040.0);
        acc = acc * z2 + real(2.0 * 4.0 / 120.0);
        return real(2) * fexp<real>(-z) * acc;
    }
    const real e = fexp<real>(real(-2) * z);
    const real z2 = z * z;
    return ((z2 - real(3) * z + real(3)) - e * (z2 + real(3) * z + real(3))) / (z2 * z2 * z);
}

template <typename real>
__device__ __forceinline__ void kb_value_slope_curv(const Window<real> &w, real frac, int j, real &v, real &d,
                                                    real &dd)
{
    const real t1 = (w.m - real(j)) - frac;
    const real t2 = (w.m + real(j)) + frac;
    if (!(t1 > real(0)) || !(t2 > real(0))) {
        v = d = dd = real(0);
        return;
    }
    const real tau = fsqrt<real>(t1 * t2);
    const real x = real(j) + frac;
    const real z = w.b * tau;
    const real e = w.S * fexp<real>(-w.b * x * x / (tau + w.m));
    const real F = kb_slope<real>(z);
    v = e * (-fexpm1<real>(real(-2) * z)) / z;
    d = -x * w.b * w.b * e * F;
    dd = -w.b * w.b * e * (F - w.b * w.b * x * x * kb_curv_factor<real>(z));
}

template <int DEG> __device__ __forceinline__ float poly_eval(const float *c, float t)
{
    float acc = c[DEG];
#pragma unroll
    for (int i = DEG - 1; i >= 0; --i)
        acc = fmaf(acc, t, c[i]);
    return acc;
}

// Even and odd parts of sum_i c[i] t^i as polynomials in s = t^2: e = sum_j c[2j] s^j,
// o = sum_j c[2j+1] s^j, so that the polynomial at +-t is e +- t o.
template <int DEG> __device__ __forceinline__ void poly_even_odd(const float *c, float s, float &e, float &o)
{
    constexpr int NE = DEG / 2, NO = (DEG - 1) / 2;   // highest even / odd half-index
    e = c[2 * NE];
#pragma unroll
    for (int j = NE - 1; j >= 0; --j)
        e = fmaf(e, s, c[2 * j]);
    o = c[2 * NO + 1];
#pragma unroll
    for (int j = NO - 1; j >= 0; --j)
        o = fmaf(o, s, c[2 * j + 1]);
}

// Spreading tiles in shared memory: a warp's tile holds `rows` x `rows` grid lines at a row
// pitch q >= rows.  The M2 x M2 taps of one source sit at offsets a q + b (a, b < M2) from the
// source's corner; tap (a, b) lies on bank (a q + b) mod 32 relative to the corner.  Dealing the
// taps to lanes by bank makes every read and write of a source conflict-free, provided no bank
// holds more than ceil(M2^2 / 32) taps: spread_pitch picks the smallest such q (q = M2 mod 32
// always qualifies, since the offsets a M2 + b are then consecutive, so q < rows + 32).
__host__ __device__ __forceinline__ int spread_taps_on_bank(int bank, int q, int M2)
{
    int c = 0;
    for (int a = 0; a < M2; ++a)
        c += (((bank - a * q) % 32 + 32) % 32) < M2 ? 1 : 0;
    return c;
}

inline int spread_pitch(int rows, int M2)
{
    const int per = (M2 * M2 + 31) / 32;
    for (int q = rows; q < rows + 32; ++q) {
        int worst = 0;
        for (int bank = 0; bank < 32; ++bank)
            worst = worst > spread_taps_on_bank(bank, q, M2) ? worst : spread_taps_on_bank(bank, q, M2);
        if (worst <= per)
            return q;
    }
    return rows;   // not reached
}

// The same choice made by one warp, each lane counting its own bank.
__device__ __forceinline__ int spread_pitch_warp(int rows, int M2, int lane)
{
    const int per = (M2 * M2 + 31) / 32;
    for (int q = rows; q < rows + 32; ++q)
        if (__reduce_max_sync(0xffffffffu, spread_taps_on_bank(lane, q, M2)) <= per)
            return q;
    return rows;   // not reached
}

// Row groups of the spreading's tap lanes (k_spread, k_batch_spread): G groups of M2 lanes, G the
// largest divisor of M2 with G M2 <= 32; lane (g, b) owns column b of the source's M2 x M2 taps
// and the M2 / G consecutive rows g M2/G .. (g + 1) M2/G - 1.  At every row step the lanes touch
// G runs of M2 consecutive columns, G M2/G rows apart: spread_group_pitch picks the smallest row
// pitch q >= rows at which those runs lie on distinct banks (each step is the first one shifted
// by i q, so checking the first suffices; a pitch within 8 of rows exists for M2 = 4..16).
__host__ __device__ constexpr int spread_groups(int M2)
{
    int G = 1;
    for (int d = 1; d <= M2; ++d)
        if (M2 % d == 0 && d * M2 <= 32)
            G = d;
    return G;
}

__host__ __device__ constexpr bool spread_group_banks_ok(int q, int M2)
{
    const int G = spread_groups(M2), RPL = M2 / G;
    unsigned used = 0u;
    for (int g = 0; g < G; ++g)
        for (int b = 0; b < M2; ++b) {
            const int bank = (g * RPL * q + b) % 32;
            if ((used >> bank) & 1u)
                return false;
            used |= 1u << bank;
        }
    return true;
}

__host__ __device__ constexpr int spread_group_pitch(int rows, int M2)
{
    for (int q = rows; q < rows + 32; ++q)
        if (spread_group_banks_ok(q, M2))
            return q;
    return rows;   // not reached
}

// This lane's taps for pitch q: slot i holds the i-th row a (ascending) whose tap on this lane's
// bank exists, b = (lane - a q) mod 32 < M2.  Slots beyond the count are marked invalid.
template <int M2, int PER>
__device__ __forceinline__ void spread_lane_taps(int lane, int q, int (&ta)[PER], int (&tb)[PER], int (&toff)[PER],
                                                 unsigned &valid)
{
    int g = 0;
    valid = 0u;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        ta[i] = 0;
        tb[i] = 0;
    }
#pragma unroll
    for (int a = 0; a < M2; ++a) {
        const int b = ((lane - a * q) % 32 + 32) % 32;
        if (b < M2) {
#pragma unroll
            for (int i = 0; i < PER; ++i)
                if (g == i) {
                    ta[i] = a;
                    tb[i] = b;
                }
            ++g;
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        toff[i] = ta[i] * q + tb[i];
        if (i < g)
            valid |= 1u << i;
    }
}

// Point record fields in cell-sorted order.
//   base: packed (b1 | b2 << 16), b = floor(u), u = n_os (s x + 1/2) - window_lo
//   frac: u - b in [0, 1), per dimension
__host__ __device__ __forceinline__ int base1(int packed) { return packed & 0xffff; }
__host__ __device__ __forceinline__ int base2(int packed) { return (packed >> 16) & 0xffff; }

// Tile-major cell key: cells of one spreading tile are contiguous, cells row-major inside.
// Points are sorted by key * kSub + sub, where sub is the Morton index of the point's
// 8 x 8 sub-cell, so consecutive points inside a cell are spatially compact; the sorted
// range of cell `key` is [start[key * kSub], start[(key + 1) * kSub]) and that of one
// sub-cell is [start[key * kSub + sub], start[key * kSub + sub + 1]).
constexpr int kSubEdge = 8;
constexpr int kSub = kSubEdge * kSubEdge;

__host__ __device__ __forceinline__ int morton_sub(int s1, int s2)
{
    int r = 0;
#pragma unroll
    for (int bit = 0; bit < 3; ++bit)
        r |= (((s2 >> bit) & 1) << (2 * bit)) | (((s1 >> bit) & 1) << (2 * bit + 1));
    return r;
}

struct CellGrid {
    int cell;      // cell edge in grid cells
    int n_c;       // cells per dimension
    int T;         // cells per tile edge
    int n_t;       // tiles per dimension
    __host__ __device__ __forceinline__ int key(int c1, int c2) const
    {
        const int t1 = c1 / T, t2 = c2 / T;
        return (t1 * n_t + t2) * (T * T) + (c1 - t1 * T) * T + (c2 - t2 * T);
    }
    __host__ __device__ __forceinline__ int n_keys() const { return n_t * n_t * T * T; }
    // sub-cell row of grid line offset o (0 <= o < cell) inside a cell, and the first offset of row s
    __host__ __device__ __forceinline__ int sub_row(int o) const { return (o * kSubEdge) / cell; }
    __host__ __device__ __forceinline__ int sub_first(int s) const { return (s * cell + kSubEdge - 1) / kSubEdge; }
    // Morton index of the sub-cell holding grid line pair (b1, b2) of cell (c1, c2)
    __host__ __device__ __forceinline__ int sub(int b1, int b2, int c1, int c2) const
    {
        return morton_sub(sub_row(b1 - c1 * cell), sub_row(b2 - c2 * cell));
    }
};

}  // namespace fs
