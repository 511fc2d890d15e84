// Oversampled 2D FFT (steps d), diagonal multiply with deconvolution (step e),
// and the FP64 Fourier coefficients b_l of the regularised kernel.
//
// The paper: "perform ... a FFT on the X grid", "divide these numbers by the
// Fourier coefficients of the Gaussian", and the smoothing of G near the
// origin whose coefficients enter the product.  The grid is real and only
// the frequencies l in I_n = {-n/2..n/2-1}^2 are kept, so the transform is
//   rows:    two real rows per complex Stockham FFT of length L = n_os,
//            keeping bins l1 = 0..n/2 (half spectrum, stored column-major);
//   columns: one CTA per kept l1: forward FFT, multiply by the table
//            mul[l1][l2] (b_l / (c(l1)^2 c(l2)^2) with the weights that make
//            the real part of the sum over I_n exact), inverse FFT - no HBM
//            round trip between the two;
//   rows:    Hermitian-extended inverse, two real rows per complex FFT.
// Only the active window of n_a rows/columns that hold points is read or
// written; the rest of the L x L grid is known to be zero and is never stored.
//
// Each 1D transform is a Stockham autosort FFT in shared memory: radix-8
// butterflies held in registers (a final radix-4 or radix-2 pass for the rest of
// log2 L), ping-pong buffers, one __syncthreads per pass.  The twiddles of each
// pass sit together in a table ordered by pass, multiple and butterfly (see
// fft_twiddle_table), which the 2D kernels first copy into shared memory; the
// buffers between two passes are stored with an XOR swizzle of the index so that
// the strided writes of the early passes hit distinct banks.
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace fs {

namespace {

template <typename real> using cplx = typename Cplx<real>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// Multiply by -i (forward) or +i (inverse).
template <bool INV, typename C> __device__ __forceinline__ C rot_i(C a)
{
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

// In-register radix-4 DFT of (v0, v1, v2, v3) (forward e^-, inverse e^+), outputs in order.
template <bool INV, typename C> __device__ __forceinline__ void dft4(C &v0, C &v1, C &v2, C &v3)
{
    const C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = rot_i<INV>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v1 = cadd(a1, a3);
    v2 = csub(a0, a2);
    v3 = csub(a1, a3);
}

// In-register radix-8 DFT: two radix-4 DFTs of the sums and the twiddled differences
// v_k +- v_{k+4}, the differences rotated by e^-+(2 pi i k / 8); X_{2m} from the sums,
// X_{2m+1} from the differences.
template <bool INV, typename real, typename C> __device__ __forceinline__ void dft8(C (&v)[8])
{
    const real h = real(0.70710678118654752440084436210484903928);   // 1 / sqrt 2
    C a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = cadd(v[k], v[k + 4]);
        b[k] = csub(v[k], v[k + 4]);
    }
    // b1 *= e^-+(i pi/4), b2 *= -+i, b3 *= e^-+(3 i pi/4)
    C t;
    if (INV) { t.x = h * (b[1].x - b[1].y); t.y = h * (b[1].x + b[1].y); }
    else { t.x = h * (b[1].x + b[1].y); t.y = h * (b[1].y - b[1].x); }
    b[1] = t;
    b[2] = rot_i<INV>(b[2]);
    if (INV) { t.x = -h * (b[3].x + b[3].y); t.y = h * (b[3].x - b[3].y); }
    else { t.x = h * (b[3].y - b[3].x); t.y = -h * (b[3].x + b[3].y); }
    b[3] = t;
    dft4<INV>(a[0], a[1], a[2], a[3]);
    dft4<INV>(b[0], b[1], b[2], b[3]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        v[2 * m] = a[m];
        v[2 * m + 1] = b[m];
    }
}

// Shared-memory position of element i of a buffer between two passes: the low four bits
// XORed with the next four (a permutation within each aligned run of 16 elements).  Every
// warp-wide access of a pass then touches 16 distinct 8-byte bank pairs per half-warp, where
// the first pass's writes, 8 elements apart, would otherwise fall on two.  m = 15 turns the
// swizzle on, m = 0 leaves the natural order (the line's input and result).
__device__ __forceinline__ int swz(int i, int m) { return i ^ ((i >> 4) & m); }

// One Stockham pass of radix R over the line: butterfly j reads src[j + r L/R], multiplies
// element r by w^(r k) with w = exp(-+2 pi i / (Ns R)) (k = j mod Ns), transforms in
// registers and writes dst[(j - k) R + k + r Ns].  The pass's twiddles are tw[Ns - 1 +
// (r - 1) Ns + k], consecutive in k, so that a warp reads them without bank conflicts.
// LC, NsC and NT, when nonzero, fix L, Ns and the thread count at compile time (the index
// arithmetic then folds to constants); zero takes the run-time L, Ns and blockDim.x.
template <typename real, bool INV, int R, int LC = 0, int NsC = 0, int NT = 0>
__device__ __forceinline__ void stockham_pass(const cplx<real> *src, cplx<real> *dst, int L_rt, int Ns_rt,
                                              const cplx<real> *__restrict__ tw)
{
    using C = cplx<real>;
    const int L = LC ? LC : L_rt;
    const int Ns = NsC ? NsC : Ns_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    const int m_in = Ns > 1 ? 15 : 0, m_out = Ns * R < L ? 15 : 0;
    const int nb = L / R;
    for (int j = threadIdx.x; j < nb; j += nt) {
        const int k = j & (Ns - 1);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            v[r] = src[swz(j + r * nb, m_in)];
        if (Ns > 1 && k) {
            const C *twk = tw + (Ns - 1) + k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C t = twk[(r - 1) * Ns];
                if (INV)
                    t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        if constexpr (R == 8) {
            dft8<INV, real>(v);
        } else if constexpr (R == 4) {
            dft4<INV>(v[0], v[1], v[2], v[3]);
        } else {
            const C t = v[1];
            v[1] = csub(v[0], t);
            v[0] = cadd(v[0], t);
        }
        const int idx = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            dst[swz(idx + r * Ns, m_out)] = v[r];
    }
}

// A pass of compile-time shape (radix R, length L, Ns points combined, NT threads) whose
// operands come from ld(e, it, r) (element e, the thread's butterfly it and operand r) and go
// to st(i, v) (element i): the first pass of a line can read global memory and the last one
// write it, with no shared-memory sweep before or after the transform.
template <typename real, bool INV, int R, int L, int Ns, int NT, class Ld, class St>
__device__ __forceinline__ void pass_io(const cplx<real> *__restrict__ tw, Ld &&ld, St &&st)
{
    using C = cplx<real>;
    constexpr int nb = L / R;
    constexpr int IT = (nb + NT - 1) / NT;   // butterflies per thread
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int j = threadIdx.x + it * NT;
        if (IT * NT > nb && j >= nb)
            break;
        const int k = j & (Ns - 1);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            v[r] = ld(j + r * nb, it, r);
        if (Ns > 1 && k) {
            const C *twk = tw + (Ns - 1) + k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C t = twk[(r - 1) * Ns];
                if (INV)
                    t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        }
        if constexpr (R == 8) {
            dft8<INV, real>(v);
        } else if constexpr (R == 4) {
            dft4<INV>(v[0], v[1], v[2], v[3]);
        } else {
            const C t = v[1];
            v[1] = csub(v[0], t);
            v[0] = cadd(v[0], t);
        }
        const int idx = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            st(idx + r * Ns, v[r]);
    }
}

// Ns of the last pass of a length-L line.
__host__ __device__ constexpr int fft_last_ns(int L)
{
    int Ns = 1;
    while (Ns * fft_pass_radix(L / Ns) < L)
        Ns *= fft_pass_radix(L / Ns);
    return Ns;
}

// The shared-memory passes of a line of compile-time length L from Ns points combined up to
// NsEnd (L: to the end); returns the buffer holding the result.
template <typename real, bool INV, int L, int NT, int Ns, int NsEnd>
__device__ __forceinline__ cplx<real> *fft_mid(cplx<real> *src, cplx<real> *dst, const cplx<real> *__restrict__ tw)
{
    if constexpr (Ns >= NsEnd) {
        return src;
    } else {
        constexpr int R = fft_pass_radix(L / Ns);
        stockham_pass<real, INV, R, L, Ns, NT>(src, dst, L, Ns, tw);
        __syncthreads();
        return fft_mid<real, INV, L, NT, Ns * R, NsEnd>(dst, src, tw);
    }
}

// In-place (via ping-pong) FFT of one line of length L (a power of two) held in shared memory:
// radix-8 passes, then one radix-4 or radix-2 pass for the remaining factor (fft_pass_radix),
// one __syncthreads per pass (2048 points: 4 passes).  Input and result are in natural order,
// the buffers in between swizzled.  tw: the per-pass table of fft_twiddle_table, in shared or
// global memory.  Returns the buffer holding the result (a or b).  All threads of the block
// take part.  LC > 0: L = LC known at compile time, with NT threads (0: blockDim.x).
template <typename real, bool INV, int LC = 0, int NT = 0>
__device__ __forceinline__ cplx<real> *fft_line(cplx<real> *a, cplx<real> *b, int L, const cplx<real> *__restrict__ tw)
{
    if constexpr (LC > 0) {
        return fft_mid<real, INV, LC, NT, 1, LC>(a, b, tw);
    } else {
        cplx<real> *src = a, *dst = b;
        for (int Ns = 1; Ns < L;) {
            const int R = fft_pass_radix(L / Ns);
            if (R == 8)
                stockham_pass<real, INV, 8>(src, dst, L, Ns, tw);
            else if (R == 4)
                stockham_pass<real, INV, 4>(src, dst, L, Ns, tw);
            else
                stockham_pass<real, INV, 2>(src, dst, L, Ns, tw);
            __syncthreads();
            cplx<real> *t = src;
            src = dst;
            dst = t;
            Ns *= R;
        }
        return src;
    }
}

// Loads of data that other blocks of the same launch wrote (the batched transform) go
// through L2 (ld.global.cg); elsewhere plain loads.
template <bool CG, typename T> __device__ __forceinline__ T load(const T *p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}

// ---- Units with the line length L known at compile time (NT threads): the first pass of a
// transform reads its operands from global memory and the last pass of an inverse writes its
// results there, and the spectral multiply rides on the first inverse pass; against the
// run-time units below each line skips one to two shared-memory sweeps and barriers per
// transform.  The twiddles staged by the caller are first read in the second pass, after the
// barrier that ends the first.

template <typename real, int L, int NT>
__device__ __forceinline__ void rows_fwd_fused(int rp, const real *__restrict__ grid, int pitch, int n_a, int n_half,
                                               cplx<real> *__restrict__ spec, int ld,
                                               const cplx<real> *__restrict__ tw, cplx<real> *a, cplx<real> *b)
{
    using C = cplx<real>;
    constexpr int R0 = fft_pass_radix(L);
    const int r = 2 * rp;
    const bool has2 = r + 1 < n_a;
    const real *x0 = grid + (int64_t)r * pitch;
    const real *x1 = grid + (int64_t)(has2 ? r + 1 : r) * pitch;
    pass_io<real, false, R0, L, 1, NT>(
        tw,
        [&](int c, int, int) {
            C z;
            z.x = c < n_a ? x0[c] : real(0);
            z.y = (c < n_a && has2) ? x1[c] : real(0);
            return z;
        },
        [&](int i, const C &v) { b[swz(i, 15)] = v; });
    __syncthreads();
    const C *Z = fft_mid<real, false, L, NT, R0, L>(b, a, tw);
    for (int k = threadIdx.x; k <= n_half; k += NT) {
        const C zk = Z[k];
        const C zc = Z[(L - k) & (L - 1)];
        C X, Y;
        // X = (Z_k + conj Z_{-k}) / 2,  Y = (Z_k - conj Z_{-k}) / (2i)
        X.x = real(0.5) * (zk.x + zc.x);
        X.y = real(0.5) * (zk.y - zc.y);
        Y.x = real(0.5) * (zk.y + zc.y);
        Y.y = real(-0.5) * (zk.x - zc.x);
        if constexpr (sizeof(real) == 4) {
            // the two rows' bins are adjacent (ld and r even): one 16-byte store
            if (has2)
                *reinterpret_cast<float4 *>(spec + (int64_t)k * ld + r) = make_float4(X.x, X.y, Y.x, Y.y);
            else
                spec[(int64_t)k * ld + r] = X;
        } else {
            spec[(int64_t)k * ld + r] = X;
            if (has2)
                spec[(int64_t)k * ld + r + 1] = Y;
        }
    }
}

template <typename real, bool CG, int L, int NT>
__device__ __forceinline__ void cols_fused(int l1, cplx<real> *__restrict__ spec, int ld, int n_a, int n,
                                           const real *__restrict__ mul, const cplx<real> *__restrict__ tw,
                                           cplx<real> *a, cplx<real> *b)
{
    using C = cplx<real>;
    constexpr int R0 = fft_pass_radix(L), NB0 = L / R0, IT0 = (NB0 + NT - 1) / NT;
    constexpr int NSL = fft_last_ns(L), RL = L / NSL;
    cplx<real> *col = spec + (int64_t)l1 * ld;
    // the multipliers of the operands of this thread's first inverse pass, fetched now so that
    // their latency hides behind the forward transform
    const real *mrow = mul + (int64_t)l1 * (n + 1);
    const int h = n / 2;
    real mp[IT0][R0];
#pragma unroll
    for (int it = 0; it < IT0; ++it) {
        const int j = threadIdx.x + it * NT;
#pragma unroll
        for (int q = 0; q < R0; ++q) {
            const int e = j + q * NB0;
            const int l2 = e < L / 2 ? e : e - L;
            mp[it][q] = (j < NB0 && l2 >= -h && l2 <= h) ? mrow[l2 + h] : real(0);
        }
    }
    pass_io<real, false, R0, L, 1, NT>(
        tw,
        [&](int c, int, int) {
            C z;
            if (c < n_a) {
                z = load<CG>(col + c);
            } else {
                z.x = real(0);
                z.y = real(0);
            }
            return z;
        },
        [&](int i, const C &v) { b[swz(i, 15)] = v; });
    __syncthreads();
    C *F = fft_mid<real, false, L, NT, R0, L>(b, a, tw);
    C *other = (F == a) ? b : a;
    pass_io<real, true, R0, L, 1, NT>(
        tw,
        [&](int e, int it, int q) {
            C z = F[e];
            z.x *= mp[it][q];
            z.y *= mp[it][q];
            return z;
        },
        [&](int i, const C &v) { other[swz(i, 15)] = v; });
    __syncthreads();
    const C *Y = fft_mid<real, true, L, NT, R0, NSL>(other, F, tw);
    pass_io<real, true, RL, L, NSL, NT>(
        tw, [&](int e, int, int) { return Y[swz(e, 15)]; },
        [&](int i, const C &v) {
            if (i < n_a)
                col[i] = v;
        });
}

template <typename real, bool CG, int L, int NT>
__device__ __forceinline__ void rows_inv_fused(int rp, const cplx<real> *__restrict__ spec, int ld, int n_a,
                                               int n_half, real *__restrict__ grid, int pitch,
                                               const cplx<real> *__restrict__ tw, cplx<real> *a, cplx<real> *b)
{
    using C = cplx<real>;
    constexpr int R0 = fft_pass_radix(L);
    constexpr int NSL = fft_last_ns(L), RL = L / NSL;
    const int r = 2 * rp;
    const bool has2 = r + 1 < n_a;
    pass_io<real, true, R0, L, 1, NT>(
        tw,
        [&](int c, int, int) {
            // X + i Y from the half spectra of the two rows (Hermitian extension above n_half)
            C X, Y;
            X.x = X.y = Y.x = Y.y = real(0);
            const bool lower = c <= n_half, upper = c >= L - n_half;
            if (lower || upper) {
                const C *at = spec + (int64_t)(lower ? c : L - c) * ld + r;
                if constexpr (sizeof(real) == 4) {
                    if (has2) {
                        const float4 t = load<CG>(reinterpret_cast<const float4 *>(at));
                        X = make_float2(t.x, t.y);
                        Y = make_float2(t.z, t.w);
                    } else {
                        X = load<CG>(at);
                    }
                } else {
                    X = load<CG>(at);
                    if (has2)
                        Y = load<CG>(at + 1);
                }
                if (!lower) {
                    X.y = -X.y;
                    Y.y = -Y.y;
                } else if (c == 0) {
                    X.y = real(0);
                    Y.y = real(0);
                }
            }
            C z;
            z.x = X.x - Y.y;
            z.y = X.y + Y.x;
            return z;
        },
        [&](int i, const C &v) { b[swz(i, 15)] = v; });
    __syncthreads();
    const C *Y = fft_mid<real, true, L, NT, R0, NSL>(b, a, tw);
    real *g0 = grid + (int64_t)r * pitch;
    real *g1 = grid + (int64_t)(r + 1) * pitch;
    pass_io<real, true, RL, L, NSL, NT>(
        tw, [&](int e, int, int) { return Y[swz(e, 15)]; },
        [&](int i, const C &v) {
            if (i < n_a) {
                g0[i] = v.x;
                if (has2)
                    g1[i] = v.y;
            }
        });
}

// Two real rows (2 rp, 2 rp + 1) of the window -> half spectra, bins 0..n_half, written to
// spec[l1 * ld + r].  a, b: 2 L complex values of shared memory.
template <typename real, int LC = 0, int NT = 0, bool FUSED = true>
__device__ __forceinline__ void rows_fwd_unit(int rp, const real *__restrict__ grid, int pitch, int n_a, int L_rt,
                                              int n_half, cplx<real> *__restrict__ spec, int ld,
                                              const cplx<real> *__restrict__ tw, cplx<real> *a, cplx<real> *b)
{
    if constexpr (LC > 0 && FUSED) {
        rows_fwd_fused<real, LC, NT>(rp, grid, pitch, n_a, n_half, spec, ld, tw, a, b);
        return;
    }
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    const int r = 2 * rp;
    const bool has2 = r + 1 < n_a;
    if constexpr (sizeof(real) == 4) {
        // 16-byte loads of four values of each row (n_a and the pitch are multiples of 4),
        // several in flight per thread
        const float4 *r0 = reinterpret_cast<const float4 *>(grid + (int64_t)r * pitch);
        const float4 *r1 = reinterpret_cast<const float4 *>(grid + (int64_t)(has2 ? r + 1 : r) * pitch);
        const int nv = n_a / 4;
#pragma unroll 4
        for (int v = threadIdx.x; v < L / 4; v += nt) {
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
            if (v < nv) {
                x = r0[v];
                if (has2)
                    y = r1[v];
            }
            float4 *dst = reinterpret_cast<float4 *>(a + 4 * v);
            dst[0] = make_float4(x.x, y.x, x.y, y.y);
            dst[1] = make_float4(x.z, y.z, x.w, y.w);
        }
    } else {
        for (int c = threadIdx.x; c < L; c += nt) {
            cplx<real> z;
            z.x = c < n_a ? grid[(int64_t)r * pitch + c] : real(0);
            z.y = (c < n_a && has2) ? grid[(int64_t)(r + 1) * pitch + c] : real(0);
            a[c] = z;
        }
    }
    __syncthreads();
    const cplx<real> *Z = fft_line<real, false, LC, NT>(a, b, L, tw);
    for (int k = threadIdx.x; k <= n_half; k += nt) {
        const cplx<real> zk = Z[k];
        const cplx<real> zc = Z[(L - k) & (L - 1)];
        cplx<real> X, Y;
        // X = (Z_k + conj Z_{-k}) / 2,  Y = (Z_k - conj Z_{-k}) / (2i)
        X.x = real(0.5) * (zk.x + zc.x);
        X.y = real(0.5) * (zk.y - zc.y);
        Y.x = real(0.5) * (zk.y + zc.y);
        Y.y = real(-0.5) * (zk.x - zc.x);
        if constexpr (sizeof(real) == 4) {
            // the two rows' bins are adjacent (ld and r even): one 16-byte store
            if (has2)
                *reinterpret_cast<float4 *>(spec + (int64_t)k * ld + r) = make_float4(X.x, X.y, Y.x, Y.y);
            else
                spec[(int64_t)k * ld + r] = X;
        } else {
            spec[(int64_t)k * ld + r] = X;
            if (has2)
                spec[(int64_t)k * ld + r + 1] = Y;
        }
    }
}

// Column l1: forward FFT over rows, multiply, inverse FFT, keep the window rows.
template <typename real, bool CG, int LC = 0, int NT = 0, bool FUSED = true>
__device__ __forceinline__ void cols_unit(int l1, cplx<real> *__restrict__ spec, int ld, int n_a, int L_rt, int n,
                                          const real *__restrict__ mul, const cplx<real> *__restrict__ tw,
                                          cplx<real> *a, cplx<real> *b)
{
    if constexpr (LC > 0 && FUSED) {
        cols_fused<real, CG, LC, NT>(l1, spec, ld, n_a, n, mul, tw, a, b);
        return;
    }
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    cplx<real> *col = spec + (int64_t)l1 * ld;
    if constexpr (sizeof(real) == 4) {
        // two complex values per 16-byte load (ld and n_a are multiples of 4)
        const float4 *c4 = reinterpret_cast<const float4 *>(col);
#pragma unroll 4
        for (int v = threadIdx.x; v < L / 2; v += nt)
            reinterpret_cast<float4 *>(a)[v] = 2 * v < n_a ? load<CG>(c4 + v) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int r = threadIdx.x; r < L; r += nt) {
            cplx<real> v;
            if (r < n_a) {
                v = load<CG>(col + r);
            } else {
                v.x = real(0);
                v.y = real(0);
            }
            a[r] = v;
        }
    }
    __syncthreads();
    cplx<real> *F = fft_line<real, false, LC, NT>(a, b, L, tw);
    cplx<real> *other = (F == a) ? b : a;
    const real *mrow = mul + (int64_t)l1 * (n + 1);
    const int h = n / 2;
    for (int k2 = threadIdx.x; k2 < L; k2 += nt) {
        const int l2 = k2 < L / 2 ? k2 : k2 - L;
        cplx<real> v = F[k2];
        if (l2 >= -h && l2 <= h) {
            const real f = mrow[l2 + h];
            v.x *= f;
            v.y *= f;
        } else {
            v.x = real(0);
            v.y = real(0);
        }
        F[k2] = v;
    }
    __syncthreads();
    const cplx<real> *G = fft_line<real, true, LC, NT>(F, other, L, tw);
    if constexpr (sizeof(real) == 4) {
        for (int v = threadIdx.x; v < n_a / 2; v += nt)
            reinterpret_cast<float4 *>(col)[v] = reinterpret_cast<const float4 *>(G)[v];
    } else {
        for (int r = threadIdx.x; r < n_a; r += nt)
            col[r] = G[r];
    }
}

// Hermitian-extended inverse of two rows (2 rp, 2 rp + 1): real outputs on the window columns.
template <typename real, bool CG, int LC = 0, int NT = 0, bool FUSED = true>
__device__ __forceinline__ void rows_inv_unit(int rp, const cplx<real> *__restrict__ spec, int ld, int n_a, int L_rt,
                                              int n_half, real *__restrict__ grid, int pitch,
                                              const cplx<real> *__restrict__ tw, cplx<real> *a, cplx<real> *b)
{
    if constexpr (LC > 0 && FUSED) {
        rows_inv_fused<real, CG, LC, NT>(rp, spec, ld, n_a, n_half, grid, pitch, tw, a, b);
        return;
    }
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    const int r = 2 * rp;
    const bool has2 = r + 1 < n_a;
    if constexpr (sizeof(real) == 4) {
        // the two rows' bins are adjacent: one 16-byte load per column, several in flight
#pragma unroll 4
        for (int c = threadIdx.x; c < L; c += nt) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool lower = c <= n_half, upper = c >= L - n_half;
            if (lower || upper) {
                const cplx<real> *at = spec + (int64_t)(lower ? c : L - c) * ld + r;
                if (has2) {
                    t = load<CG>(reinterpret_cast<const float4 *>(at));
                } else {
                    const float2 x = load<CG>(at);
                    t = make_float4(x.x, x.y, 0.f, 0.f);
                }
                if (!lower) {            // the Hermitian half: conjugates
                    t.y = -t.y;
                    t.w = -t.w;
                } else if (c == 0) {
                    t.y = 0.f;
                    t.w = 0.f;
                }
            }
            cplx<real> z;   // X + i Y with X = (t.x, t.y), Y = (t.z, t.w)
            z.x = t.x - t.w;
            z.y = t.y + t.z;
            a[c] = z;
        }
        __syncthreads();
        const cplx<real> *Z = fft_line<real, true, LC, NT>(a, b, L, tw);
        // four columns of both rows per step: 16-byte stores (n_a and the pitch are multiples of 4)
        float4 *r0 = reinterpret_cast<float4 *>(grid + (int64_t)r * pitch);
        float4 *r1 = reinterpret_cast<float4 *>(grid + (int64_t)(r + 1) * pitch);
        for (int v = threadIdx.x; v < n_a / 4; v += nt) {
            const float4 p = reinterpret_cast<const float4 *>(Z)[2 * v];       // Z[4v], Z[4v + 1]
            const float4 q = reinterpret_cast<const float4 *>(Z)[2 * v + 1];   // Z[4v + 2], Z[4v + 3]
            r0[v] = make_float4(p.x, p.z, q.x, q.z);
            if (has2)
                r1[v] = make_float4(p.y, p.w, q.y, q.w);
        }
    } else {
        for (int c = threadIdx.x; c < L; c += nt) {
            cplx<real> X, Y;
            X.x = X.y = Y.x = Y.y = real(0);
            if (c <= n_half) {
                X = load<CG>(spec + (int64_t)c * ld + r);
                if (has2)
                    Y = load<CG>(spec + (int64_t)c * ld + r + 1);
                if (c == 0) {
                    X.y = real(0);
                    Y.y = real(0);
                }
            } else if (c >= L - n_half) {
                X = load<CG>(spec + (int64_t)(L - c) * ld + r);
                X.y = -X.y;
                if (has2) {
                    Y = load<CG>(spec + (int64_t)(L - c) * ld + r + 1);
                    Y.y = -Y.y;
                }
            }
            cplx<real> z;   // X + i Y
            z.x = X.x - Y.y;
            z.y = X.y + Y.x;
            a[c] = z;
        }
        __syncthreads();
        const cplx<real> *Z = fft_line<real, true, LC, NT>(a, b, L, tw);
        for (int c = threadIdx.x; c < n_a; c += nt) {
            grid[(int64_t)r * pitch + c] = Z[c].x;
            if (has2)
                grid[(int64_t)(r + 1) * pitch + c] = Z[c].y;
        }
    }
}

// Copy the twiddle table into shared memory (the caller's next __syncthreads publishes it):
// every pass reads it at scattered indices, which from global memory stalled each pass on
// the load latency.
template <typename real, int LC = 0, int NT = 0>
__device__ __forceinline__ cplx<real> *stage_twiddles(cplx<real> *dst, const cplx<real> *__restrict__ tw, int L_rt)
{
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
#pragma unroll 8
    for (int t = threadIdx.x; t < L; t += nt)
        dst[t] = tw[t];
    return dst;
}

// Threads of the 2D transform kernels for a line of L points: a quarter of L, 32 to 256.
__host__ __device__ constexpr int fft_threads(int L) { return L / 4 > 256 ? 256 : (L / 4 < 32 ? 32 : L / 4); }

// The three 2D kernels.  LC > 0 fixes the line length at compile time (one instance per
// length the plans use, 256 .. 4096 points), LC = 0 takes it at run time.
template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft_rows_fwd(const real *__restrict__ grid, int pitch, int n_a, int L,
                                                      int n_half, cplx<real> *__restrict__ spec, int ld,
                                                      const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    cplx<real> *s_tw = stage_twiddles<real, LC, NT>(a + 2 * L, tw, L);   // published by the unit's first barrier
    rows_fwd_unit<real, LC, NT>(blockIdx.x, grid, pitch, n_a, L, n_half, spec, ld, s_tw, a, a + L);
}

template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft_cols(cplx<real> *__restrict__ spec, int ld, int n_a, int L, int n,
                                                  const real *__restrict__ mul, const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    cplx<real> *s_tw = stage_twiddles<real, LC, NT>(a + 2 * L, tw, L);
    cols_unit<real, false, LC, NT>(blockIdx.x, spec, ld, n_a, L, n, mul, s_tw, a, a + L);
}

template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft_rows_inv(const cplx<real> *__restrict__ spec, int ld, int n_a, int L,
                                                      int n_half, real *__restrict__ grid, int pitch,
                                                      const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    cplx<real> *s_tw = stage_twiddles<real, LC, NT>(a + 2 * L, tw, L);
    rows_inv_unit<real, false, LC, NT>(blockIdx.x, spec, ld, n_a, L, n_half, grid, pitch, s_tw, a, a + L);
}

// Thread 0 waits until *ctr >= target; the wait ends early (failed) when the error word is
// set, and gives up after `spins` polls of ~0.1 us, setting the error word.  Returns the
// outcome to every thread of the block.
__device__ bool block_wait_geq(const int *ctr, int target, int *err, int spins)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const volatile int *vc = ctr;
        const volatile int *ve = err;
        int ok = 1;
        for (int it = 0; *vc < target; ++it) {
            if (*ve != 0) {
                ok = 0;
                break;
            }
            if (it >= spins) {
                atomicCAS(err, 0, 1);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One unit of the batched transform (256 threads) on a line of LC points (0: bi.L at run time).
// The shared-memory sweeps stay (FUSED = false): the fused units' extra registers made this
// kernel, which holds every line length, spill at five blocks per SM, for no measured gain.
template <typename real, int LC>
__device__ __forceinline__ void batch_unit(const FftUnit &fu, const BatchInst<real> &bi, cplx<real> *spec, real *grid,
                                           cplx<real> *a, cplx<real> *b)
{
    const int L = bi.L, n_a = bi.n_a, n = bi.n;
    if (fu.kind == 0)
        rows_fwd_unit<real, LC, 256, false>(fu.index, grid, bi.pitch, n_a, L, n / 2, spec, bi.ld, bi.tw, a, b);
    else if (fu.kind == 1)
        cols_unit<real, true, LC, 256, false>(fu.index, spec, bi.ld, n_a, L, n, bi.mul, bi.tw, a, b);
    else
        rows_inv_unit<real, true, LC, 256, false>(fu.index, spec, bi.ld, n_a, L, n / 2, grid, bi.pitch, bi.tw, a, b);
}

// Batched transform of all instances and right-hand sides in one persistent launch.  Blocks
// take units from a queue in which every row pair precedes every column and every column
// precedes every inverse row pair; a column waits until all forward row pairs of its
// (instance, right-hand side) are done, an inverse row pair until all its columns are.  The
// units a block waits for were taken earlier by blocks that are running and never wait on
// later units, so the waits end; each is bounded all the same (error word on timeout).
template <typename real>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 5 : 3) k_batch_fft(const BatchInst<real> *__restrict__ inst,
                                                   const FftUnit *__restrict__ units, int n_units, int n_inst,
                                                   int nrhs, int L_max, int *counters, int *err, int spins)
{
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    cplx<real> *b = a + L_max;
    __shared__ int s_unit;
    int *head = counters + 2 * n_inst * nrhs;
    for (;;) {
        if (threadIdx.x == 0)
            s_unit = atomicAdd(head, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= n_units)
            return;
        const FftUnit fu = units[u];
        const BatchInst<real> &bi = inst[fu.inst];
        const int slot = fu.inst * nrhs + fu.rhs;
        int *rows_done = counters + slot;
        int *cols_done = counters + n_inst * nrhs + slot;
        const int L = bi.L, n_a = bi.n_a, n = bi.n;
        cplx<real> *spec = bi.spec + (int64_t)fu.rhs * bi.spec_stride;
        real *grid = bi.grid + (int64_t)fu.rhs * bi.grid_stride;
        bool ok = true;
        if (fu.kind == 1)
            ok = block_wait_geq(rows_done, (n_a + 1) / 2, err, spins);
        else if (fu.kind == 2)
            ok = block_wait_geq(cols_done, n / 2 + 1, err, spins);
        if (ok) {
            switch (L) {   // the line lengths of the instances' plans, as compile-time constants
            case 256: batch_unit<real, 256>(fu, bi, spec, grid, a, b); break;
            case 512: batch_unit<real, 512>(fu, bi, spec, grid, a, b); break;
            case 1024: batch_unit<real, 1024>(fu, bi, spec, grid, a, b); break;
            case 2048: batch_unit<real, 2048>(fu, bi, spec, grid, a, b); break;
            default: batch_unit<real, 0>(fu, bi, spec, grid, a, b); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && fu.kind < 2) {
            __threadfence();
            atomicAdd(fu.kind == 0 ? rows_done : cols_done, 1);
        }
    }
}

__global__ void k_wait_selftest(const int *counter, int *err, int spins)
{
    block_wait_geq(counter, 1, err, spins);
}

__device__ double kr_sample(double r, const KernelParams &kp);

// ---- 3D transform on the active window cube g[z][y][x] (x fastest, edge n_a), the five
// passes of the 2D transform with a third axis:
//   A  x rows -> half spectra, per z plane (rows_fwd_unit): spec1[z][l1][y], l1 in [0, n/2]
//   B  y lines forward, keeping l2 in [-n/2, n/2]:         spec2[z][l1][l2 + n/2]
//   C  z lines: forward FFT, multiply by mul3[l1][l2][l3], inverse FFT, window rows kept
//   D  y lines inverse (bins l2 in [-n/2, n/2]) ->          spec1[z][l1][y]
//   E  Hermitian-extended inverse of x rows per plane (rows_inv_unit)
// The multiplier carries the weights that make the real part of the sum over I_n^3 exact.

// LC > 0: the line length L = LC compiled as a constant (NT threads), as in the 2D kernels.
template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft3_x_fwd(const real *__restrict__ grid, int n_a, int L, int n_half,
                                                    cplx<real> *__restrict__ spec1, const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    const int64_t z = blockIdx.y;
    rows_fwd_unit<real, LC, NT>(blockIdx.x, grid + z * n_a * n_a, n_a, n_a, L, n_half,
                                spec1 + z * (int64_t)(n_half + 1) * n_a, n_a, tw, a, a + L);
}

template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft3_y_fwd(const cplx<real> *__restrict__ spec1, int n_a, int L_rt, int n,
                                                    cplx<real> *__restrict__ spec2, const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    const int h = n / 2;
    const int64_t line = (int64_t)blockIdx.y * (h + 1) + blockIdx.x;   // (z, l1)
    const cplx<real> *in = spec1 + line * n_a;
    for (int r = threadIdx.x; r < L; r += nt) {
        cplx<real> v;
        v.x = v.y = real(0);
        if (r < n_a)
            v = in[r];
        a[r] = v;
    }
    __syncthreads();
    const cplx<real> *F = fft_line<real, false, LC, NT>(a, a + L, L, tw);
    cplx<real> *out = spec2 + line * (n + 1);
    for (int k = threadIdx.x; k <= n; k += nt)
        out[k] = F[(k - h + L) & (L - 1)];
}

template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft3_z(cplx<real> *__restrict__ spec2, int n_a, int L_rt, int n,
                                                const real *__restrict__ mul3, const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    cplx<real> *b = a + L;
    const int h = n / 2;
    const int k2 = blockIdx.x, l1 = blockIdx.y;
    const int64_t stride = (int64_t)(h + 1) * (n + 1);
    cplx<real> *col = spec2 + (int64_t)l1 * (n + 1) + k2;
    for (int z = threadIdx.x; z < L; z += nt) {
        cplx<real> v;
        v.x = v.y = real(0);
        if (z < n_a)
            v = col[z * stride];
        a[z] = v;
    }
    __syncthreads();
    cplx<real> *F = fft_line<real, false, LC, NT>(a, b, L, tw);
    cplx<real> *other = (F == a) ? b : a;
    const real *mrow = mul3 + ((int64_t)l1 * (n + 1) + k2) * (n + 1);
    for (int k3 = threadIdx.x; k3 < L; k3 += nt) {
        const int l3 = k3 < L / 2 ? k3 : k3 - L;
        cplx<real> v = F[k3];
        const real f = (l3 >= -h && l3 <= h) ? mrow[l3 + h] : real(0);
        v.x *= f;
        v.y *= f;
        F[k3] = v;
    }
    __syncthreads();
    const cplx<real> *G = fft_line<real, true, LC, NT>(F, other, L, tw);
    for (int z = threadIdx.x; z < n_a; z += nt)
        col[z * stride] = G[z];
}

template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft3_y_inv(const cplx<real> *__restrict__ spec2, int n_a, int L_rt, int n,
                                                    cplx<real> *__restrict__ spec1, const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    const int L = LC ? LC : L_rt;
    const int nt = NT ? NT : (int)blockDim.x;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    const int h = n / 2;
    const int64_t line = (int64_t)blockIdx.y * (h + 1) + blockIdx.x;   // (z, l1)
    for (int r = threadIdx.x; r < L; r += nt) {
        cplx<real> v;
        v.x = v.y = real(0);
        a[r] = v;
    }
    __syncthreads();
    const cplx<real> *in = spec2 + line * (n + 1);
    for (int k = threadIdx.x; k <= n; k += nt)
        a[(k - h + L) & (L - 1)] = in[k];
    __syncthreads();
    const cplx<real> *G = fft_line<real, true, LC, NT>(a, a + L, L, tw);
    cplx<real> *out = spec1 + line * n_a;
    for (int y = threadIdx.x; y < n_a; y += nt)
        out[y] = G[y];
}

template <typename real, int LC>
__global__ void __launch_bounds__(256) k_fft3_x_inv(const cplx<real> *__restrict__ spec1, int n_a, int L, int n_half,
                                                    real *__restrict__ grid, const cplx<real> *__restrict__ tw)
{
    constexpr int NT = LC ? fft_threads(LC) : 0;
    extern __shared__ unsigned char smem_raw[];
    cplx<real> *a = reinterpret_cast<cplx<real> *>(smem_raw);
    const int64_t z = blockIdx.y;
    rows_inv_unit<real, false, LC, NT>(blockIdx.x, spec1 + z * (int64_t)(n_half + 1) * n_a, n_a, n_a, L, n_half,
                                       grid + z * n_a * n_a, n_a, tw, a, a + L);
}

// out[(i3 n + i1) n + i2] = in[(i1 n + i2) n + i3]: the middle axis becomes the fastest.
__global__ void k_rotate3_c64(const double2 *__restrict__ in, double2 *__restrict__ out, int n)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n * n * n;
    if (t >= total)
        return;
    const int i3 = (int)(t % n), i2 = (int)((t / n) % n), i1 = (int)(t / ((int64_t)n * n));
    out[((int64_t)i3 * n + i1) * n + i2] = in[t];
}

__global__ void k_kernel_samples3(double2 *__restrict__ samp, int n, KernelParams kp)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n * n)
        return;
    const int j3 = (int)(t % n), j2 = (int)((t / n) % n), j1 = (int)(t / ((int64_t)n * n));
    const double x1 = (double)(j1 < n / 2 ? j1 : j1 - n) / n;
    const double x2 = (double)(j2 < n / 2 ? j2 : j2 - n) / n;
    const double x3 = (double)(j3 < n / 2 ? j3 : j3 - n) / n;
    samp[t] = make_double2(kr_sample(sqrt(x1 * x1 + x2 * x2 + x3 * x3), kp), 0.0);
}

// mul3[l1][l2 + n/2][l3 + n/2] = V(l) b_l / (c(l1) c(l2) c(l3))^2 with V(l) = ([l in I_n^3] + [-l in I_n^3]) / 2.
template <typename real>
__global__ void k_build_mul3(const double2 *__restrict__ bhat, int n, const double *__restrict__ c_tab,
                             real *__restrict__ mul3)
{
    const int h = n / 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)(h + 1) * (n + 1) * (n + 1);
    if (t >= total)
        return;
    const int k3 = (int)(t % (n + 1)), k2 = (int)((t / (n + 1)) % (n + 1)), l1 = (int)(t / ((int64_t)(n + 1) * (n + 1)));
    const int l2 = k2 - h, l3 = k3 - h;
    auto in_I = [h](int l) { return l >= -h && l <= h - 1; };
    auto in_negI = [h](int l) { return l >= -h + 1 && l <= h; };
    const double v = 0.5 * ((in_I(l1) && in_I(l2) && in_I(l3) ? 1.0 : 0.0) +
                            (in_negI(l1) && in_negI(l2) && in_negI(l3) ? 1.0 : 0.0));
    const int m1 = l1 % n, m2 = ((l2 % n) + n) % n, m3 = ((l3 % n) + n) % n;
    const double b = bhat[((int64_t)m1 * n + m2) * n + m3].x / ((double)n * n * n);
    const double c1 = c_tab[l1], c2 = c_tab[l2 < 0 ? -l2 : l2], c3 = c_tab[l3 < 0 ? -l3 : l3];
    mul3[t] = (real)(v * b / (c1 * c1 * c2 * c2 * c3 * c3));
}

// ---- FP64 coefficients b_l

__device__ double kr_sample(double r, const KernelParams &kp)
{
    const double inv2pi = 1.0 / (2.0 * kPi);
    if (r < kp.eps_I) {
        const double u2 = (r / kp.eps_I) * (r / kp.eps_I);
        double acc = 0.0;
        for (int k = kp.p - 1; k >= 0; --k)
            acc = acc * u2 + kp.beta[k];
        return acc;
    }
    if (r <= 0.5 - kp.eps_B)
        return kp.dim == 3 ? 1.0 / (4.0 * kPi * r) : -log(r) * inv2pi;
    if (r <= 0.5) {
        // two-point Taylor form on v in [0, 1]:
        //   sum_j f0_j v^j (1-v)^p S_{p-1-j}(v) + k(1/2) v^p S_{p-1}(1-v),  S_k(x) = sum_{i<=k} C(p-1+i,i) x^i
        const int p = kp.p;
        const double v = (r - (0.5 - kp.eps_B)) / kp.eps_B;
        const double w = 1.0 - v;
        double wp = 1.0, vp = 1.0;
        for (int i = 0; i < p; ++i) {
            wp *= w;
            vp *= v;
        }
        double total = 0.0, vj = 1.0;
        for (int j = 0; j < p; ++j) {
            double sk = 0.0;
            for (int i = p - 1 - j; i >= 0; --i)
                sk = sk * v + kp.tb_binom[i];
            total += kp.tb_f0[j] * vj * wp * sk;
            vj *= v;
        }
        double sr = 0.0;
        for (int i = p - 1; i >= 0; --i)
            sr = sr * w + kp.tb_binom[i];
        return total + kp.k_half * vp * sr;
    }
    return kp.k_half;
}

__global__ void k_kernel_samples(double2 *__restrict__ samp, int n, KernelParams kp)
{
    const int j2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j1 = blockIdx.y;
    if (j2 >= n)
        return;
    const int s1 = j1 < n / 2 ? j1 : j1 - n;
    const int s2 = j2 < n / 2 ? j2 : j2 - n;
    const double x1 = (double)s1 / n, x2 = (double)s2 / n;
    samp[(int64_t)j1 * n + j2] = make_double2(kr_sample(sqrt(x1 * x1 + x2 * x2), kp), 0.0);
}

__global__ void k_fft_lines_c64(double2 *__restrict__ data, int L, const double2 *__restrict__ tw)
{
    extern __shared__ unsigned char smem_raw[];
    double2 *a = reinterpret_cast<double2 *>(smem_raw);
    double2 *b = a + L;
    double2 *line = data + (int64_t)blockIdx.x * L;
    for (int c = threadIdx.x; c < L; c += blockDim.x)
        a[c] = line[c];
    __syncthreads();
    const double2 *Z = fft_line<double, false>(a, b, L, tw);
    for (int c = threadIdx.x; c < L; c += blockDim.x)
        line[c] = Z[c];
}

__global__ void k_transpose_c64(const double2 *__restrict__ in, double2 *__restrict__ out, int n)
{
    __shared__ double2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = by + i, c = bx + threadIdx.x;
        if (r < n && c < n)
            tile[i][threadIdx.x] = in[(int64_t)r * n + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = bx + i, c = by + threadIdx.x;
        if (r < n && c < n)
            out[(int64_t)r * n + c] = tile[threadIdx.x][i];
    }
}

// mul[l1][l2 + n/2] for l1 in [0, n/2], l2 in [-n/2, n/2].  bhat is the transposed
// unnormalised n x n DFT of the K_R samples: bhat[l2 * n + l1] = n^2 b_(l1,l2).
// c_tab[l] = c(l), l = 0..n/2 (even in l).  Weights: for l1 < n/2 the symmetric
// half weight at l2 = +-n/2; for l1 = n/2 the set -I_n in l2 with the factor 1/2
// that undoes the row inverse's Hermitian doubling.
template <typename real>
__global__ void k_build_mul(const double2 *__restrict__ bhat, int n, const double *__restrict__ c_tab,
                            real *__restrict__ mul)
{
    const int h = n / 2;
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;   // l2 + h
    const int l1 = blockIdx.y;
    if (i2 > n)
        return;
    const int l2 = i2 - h;
    const int m1 = l1 % n, m2 = ((l2 % n) + n) % n;
    const double b = bhat[(int64_t)m2 * n + m1].x / ((double)n * (double)n);
    const double c1 = c_tab[l1], c2 = c_tab[l2 < 0 ? -l2 : l2];
    double wgt;
    if (l1 < h)
        wgt = (l2 == h || l2 == -h) ? 0.5 : 1.0;
    else
        wgt = (l2 == -h) ? 0.0 : 0.5;
    mul[(int64_t)l1 * (n + 1) + i2] = (real)(wgt * b / (c1 * c1 * c2 * c2));
}


template <typename K> cudaError_t set_smem(K kern, size_t bytes)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Calls f with the compile-time line length of L (0 for lengths without an instance of their own).
template <typename F> cudaError_t with_line_length(int L, F &&f)
{
    switch (L) {
    case 256: return f(std::integral_constant<int, 256>{});
    case 512: return f(std::integral_constant<int, 512>{});
    case 1024: return f(std::integral_constant<int, 1024>{});
    case 2048: return f(std::integral_constant<int, 2048>{});
    case 4096: return f(std::integral_constant<int, 4096>{});
    default: return f(std::integral_constant<int, 0>{});
    }
}

template <typename real>
cudaError_t launch_fft_rows_fwd(const real *grid, int pitch, int n_a, int L, int n_half, cplx<real> *spec, int ld,
                                const cplx<real> *tw, cudaStream_t st)
{
    const size_t smem = 3 * (size_t)L * sizeof(cplx<real>);   // two line buffers and the twiddles
    return with_line_length(L, [&](auto lc) {
        constexpr int LC = decltype(lc)::value;
        cudaError_t e = set_smem(k_fft_rows_fwd<real, LC>, smem);
        if (e != cudaSuccess)
            return e;
        k_fft_rows_fwd<real, LC><<<(n_a + 1) / 2, fft_threads(L), smem, st>>>(grid, pitch, n_a, L, n_half, spec, ld,
                                                                              tw);
        return cudaGetLastError();
    });
}

template <typename real>
cudaError_t launch_fft_cols(cplx<real> *spec, int ld, int n_a, int L, int n, const real *mul, const cplx<real> *tw,
                            cudaStream_t st)
{
    const size_t smem = 3 * (size_t)L * sizeof(cplx<real>);   // two line buffers and the twiddles
    return with_line_length(L, [&](auto lc) {
        constexpr int LC = decltype(lc)::value;
        cudaError_t e = set_smem(k_fft_cols<real, LC>, smem);
        if (e != cudaSuccess)
            return e;
        k_fft_cols<real, LC><<<n / 2 + 1, fft_threads(L), smem, st>>>(spec, ld, n_a, L, n, mul, tw);
        return cudaGetLastError();
    });
}

template <typename real>
cudaError_t launch_fft_rows_inv(const cplx<real> *spec, int ld, int n_a, int L, int n_half, real *grid, int pitch,
                                const cplx<real> *tw, cudaStream_t st)
{
    const size_t smem = 3 * (size_t)L * sizeof(cplx<real>);   // two line buffers and the twiddles
    return with_line_length(L, [&](auto lc) {
        constexpr int LC = decltype(lc)::value;
        cudaError_t e = set_smem(k_fft_rows_inv<real, LC>, smem);
        if (e != cudaSuccess)
            return e;
        k_fft_rows_inv<real, LC><<<(n_a + 1) / 2, fft_threads(L), smem, st>>>(spec, ld, n_a, L, n_half, grid, pitch,
                                                                              tw);
        return cudaGetLastError();
    });
}

template <typename real> cudaError_t batch_fft_blocks(int L_max, int *blocks)
{
    const size_t smem = 2 * (size_t)L_max * sizeof(cplx<real>);
    cudaError_t e = set_smem(k_batch_fft<real>, smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_fft<real>, 256, smem)) != cudaSuccess)
        return e;
    *blocks = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

template <typename real>
cudaError_t launch_batch_fft(const BatchInst<real> *inst, const FftUnit *units, int n_units, int n_inst, int nrhs,
                             int L_max, int grid_blocks, int *counters, int *err, int spins, cudaStream_t st)
{
    if (n_units <= 0)
        return cudaSuccess;
    const size_t smem = 2 * (size_t)L_max * sizeof(cplx<real>);
    k_batch_fft<real><<<(unsigned)grid_blocks, 256, smem, st>>>(inst, units, n_units, n_inst, nrhs, L_max, counters,
                                                                err, spins);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int *counter, int *err, int spins, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(counter, err, spins);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fft3(real *grid, int n_a, int L, int n, cplx<real> *spec1, cplx<real> *spec2, const real *mul3,
                        const cplx<real> *tw, cudaStream_t st)
{
    const size_t smem = 2 * (size_t)L * sizeof(cplx<real>);
    return with_line_length(L, [&](auto lc) {
        constexpr int LC = decltype(lc)::value;
        cudaError_t e;
        if ((e = set_smem(k_fft3_x_fwd<real, LC>, smem)) != cudaSuccess ||
            (e = set_smem(k_fft3_y_fwd<real, LC>, smem)) != cudaSuccess ||
            (e = set_smem(k_fft3_z<real, LC>, smem)) != cudaSuccess ||
            (e = set_smem(k_fft3_y_inv<real, LC>, smem)) != cudaSuccess ||
            (e = set_smem(k_fft3_x_inv<real, LC>, smem)) != cudaSuccess)
            return e;
        const int h = n / 2, thr = fft_threads(L);
        k_fft3_x_fwd<real, LC><<<dim3((n_a + 1) / 2, n_a), thr, smem, st>>>(grid, n_a, L, h, spec1, tw);
        k_fft3_y_fwd<real, LC><<<dim3(h + 1, n_a), thr, smem, st>>>(spec1, n_a, L, n, spec2, tw);
        k_fft3_z<real, LC><<<dim3(n + 1, h + 1), thr, smem, st>>>(spec2, n_a, L, n, mul3, tw);
        k_fft3_y_inv<real, LC><<<dim3(h + 1, n_a), thr, smem, st>>>(spec2, n_a, L, n, spec1, tw);
        k_fft3_x_inv<real, LC><<<dim3((n_a + 1) / 2, n_a), thr, smem, st>>>(spec1, n_a, L, h, grid, tw);
        return cudaGetLastError();
    });
}

cudaError_t launch_coeffs3(double2 *samp, double2 *tmp, int n, KernelParams kp, const double2 *tw64,
                           const double *c_tab, void *mul3, int real_is_f64, cudaStream_t st)
{
    const int64_t total = (int64_t)n * n * n;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    k_kernel_samples3<<<blocks, 256, 0, st>>>(samp, n, kp);
    cudaError_t e = launch_fft_lines_c64(samp, n * n, n, tw64, st);
    if (e != cudaSuccess)
        return e;
    k_rotate3_c64<<<blocks, 256, 0, st>>>(samp, tmp, n);
    if ((e = launch_fft_lines_c64(tmp, n * n, n, tw64, st)) != cudaSuccess)
        return e;
    k_rotate3_c64<<<blocks, 256, 0, st>>>(tmp, samp, n);
    if ((e = launch_fft_lines_c64(samp, n * n, n, tw64, st)) != cudaSuccess)
        return e;
    const int h = n / 2;
    const int64_t mt = (int64_t)(h + 1) * (n + 1) * (n + 1);
    const unsigned mb = (unsigned)((mt + 255) / 256);
    if (real_is_f64)
        k_build_mul3<double><<<mb, 256, 0, st>>>(samp, n, c_tab, (double *)mul3);
    else
        k_build_mul3<float><<<mb, 256, 0, st>>>(samp, n, c_tab, (float *)mul3);
    return cudaGetLastError();
}

cudaError_t launch_kernel_samples(double2 *samp, int n, KernelParams kp, cudaStream_t st)
{
    dim3 grid((n + 127) / 128, n);
    k_kernel_samples<<<grid, 128, 0, st>>>(samp, n, kp);
    return cudaGetLastError();
}

cudaError_t launch_fft_lines_c64(double2 *data, int lines, int L, const double2 *tw, cudaStream_t st)
{
    const size_t smem = 2 * (size_t)L * sizeof(double2);
    cudaError_t e = set_smem(k_fft_lines_c64, smem);
    if (e != cudaSuccess)
        return e;
    k_fft_lines_c64<<<lines, fft_threads(L), smem, st>>>(data, L, tw);
    return cudaGetLastError();
}

cudaError_t launch_transpose_c64(const double2 *in, double2 *out, int n, cudaStream_t st)
{
    dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
    k_transpose_c64<<<grid, block, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_build_mul(const double2 *bhat, int n, const double *c_tab, real *mul, cudaStream_t st)
{
    dim3 grid((n + 1 + 127) / 128, n / 2 + 1);
    k_build_mul<real><<<grid, 128, 0, st>>>(bhat, n, c_tab, mul);
    return cudaGetLastError();
}

template <typename real> void fft_twiddle_table(int L, real *re_im)
{
    re_im[2 * (L - 1)] = real(1);
    re_im[2 * (L - 1) + 1] = real(0);
    for (int Ns = 1; Ns < L;) {
        const int R = fft_pass_radix(L / Ns);
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < Ns; ++k) {
                const double ang = 2.0 * kPi * (double)(r * k) / (double)(Ns * R);
                const int t = Ns - 1 + (r - 1) * Ns + k;
                re_im[2 * t] = (real)std::cos(ang);
                re_im[2 * t + 1] = (real)(-std::sin(ang));
            }
        Ns *= R;
    }
}
template void fft_twiddle_table<float>(int, float *);
template void fft_twiddle_table<double>(int, double *);

template cudaError_t launch_fft_rows_fwd<float>(const float *, int, int, int, int, float2 *, int, const float2 *,
                                                cudaStream_t);
template cudaError_t launch_fft_rows_fwd<double>(const double *, int, int, int, int, double2 *, int, const double2 *,
                                                 cudaStream_t);
template cudaError_t launch_fft_cols<float>(float2 *, int, int, int, int, const float *, const float2 *, cudaStream_t);
template cudaError_t launch_fft_cols<double>(double2 *, int, int, int, int, const double *, const double2 *,
                                             cudaStream_t);
template cudaError_t launch_fft_rows_inv<float>(const float2 *, int, int, int, int, float *, int, const float2 *,
                                                cudaStream_t);
template cudaError_t launch_fft_rows_inv<double>(const double2 *, int, int, int, int, double *, int, const double2 *,
                                                 cudaStream_t);
template cudaError_t launch_build_mul<float>(const double2 *, int, const double *, float *, cudaStream_t);
template cudaError_t launch_build_mul<double>(const double2 *, int, const double *, double *, cudaStream_t);

template cudaError_t batch_fft_blocks<float>(int, int *);
template cudaError_t batch_fft_blocks<double>(int, int *);
template cudaError_t launch_batch_fft<float>(const BatchInst<float> *, const FftUnit *, int, int, int, int, int, int *,
                                             int *, int, cudaStream_t);
template cudaError_t launch_batch_fft<double>(const BatchInst<double> *, const FftUnit *, int, int, int, int, int,
                                              int *, int *, int, cudaStream_t);

template cudaError_t launch_fft3<float>(float *, int, int, int, float2 *, float2 *, const float *, const float2 *,
                                        cudaStream_t);
template cudaError_t launch_fft3<double>(double *, int, int, int, double2 *, double2 *, const double *,
                                         const double2 *, cudaStream_t);

}  // namespace fs
