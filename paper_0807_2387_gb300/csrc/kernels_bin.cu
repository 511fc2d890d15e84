// Point binning (cell sort) and per-point records: step (b) of the fast summation.
//
// Points are scaled onto the torus (x~ = s x), placed on the oversampled grid
// in window coordinates u = n_os (x~ + 1/2) - window_lo, and counting-sorted by
// a tile-major cell key (histogram -> exclusive scan -> scatter).  The
// sorted order makes every near-field cell and every spreading tile a
// contiguous range.  Within a cell the order follows the atomic scatter.
#include "internal.h"

namespace fs {

namespace {

__global__ void k_rmax(const double *__restrict__ xy, int64_t n, unsigned long long *out)
{
    double best = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        best = fmax(best, x * x + y * y);
    }
    for (int o = 16; o > 0; o >>= 1)
        best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ double warp_best[32];
    if ((threadIdx.x & 31) == 0)
        warp_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? warp_best[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        // non-negative doubles order like their bit patterns
        if (threadIdx.x == 0)
            atomicMax(out, (unsigned long long)__double_as_longlong(best));
    }
}

// Grid index of one coordinate: base in window coordinates and fraction.
__device__ __forceinline__ void grid_coord(double x, double s, int n_os, int window_lo, int &b, double &frac)
{
    const double v = (double)n_os * (s * x);
    const double fl = floor(v);
    frac = v - fl;
    b = (int)fl + n_os / 2 - window_lo;
}

__device__ __forceinline__ bool clamp_base(int &b, int m, int n_a)
{
    const int lo = m - 1, hi = n_a - 1 - m;
    if (b < lo) { b = lo; return false; }
    if (b > hi) { b = hi; return false; }
    return true;
}

__global__ void k_point_keys(const double *__restrict__ xy, int64_t n, double s, int n_os, int window_lo,
                             int n_a, int m, CellGrid cg, int *__restrict__ key, int *__restrict__ count,
                             int *status)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int b1, b2;
    double f;
    grid_coord(xy[2 * i], s, n_os, window_lo, b1, f);
    grid_coord(xy[2 * i + 1], s, n_os, window_lo, b2, f);
    bool ok = clamp_base(b1, m, n_a);
    ok = clamp_base(b2, m, n_a) && ok;
    if (!ok)
        atomicExch(status, (int)kDevDomain);
    const int c1 = b1 / cg.cell, c2 = b2 / cg.cell;
    const int k = cg.key(c1, c2) * kSub + cg.sub(b1, b2, c1, c2);
    key[i] = k;
    atomicAdd(&count[k], 1);
}

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanBlock = kScanThreads * kScanPer;

// Exclusive scan of up to kScanBlock values per block; block totals to `sums`.
__global__ void k_scan_block(const int *__restrict__ in, int *__restrict__ out, int n, int *__restrict__ sums)
{
    __shared__ int warp_tot[32];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    int v[kScanPer];
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tsum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = tsum;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += t;
        }
        warp_tot[lane] = wi - w;
        if (lane == 31 && sums)
            sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int run = warp_tot[warp] + incl - tsum;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n)
            out[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ offs, int *total_slot,
                           const int *__restrict__ in)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int off = offs ? offs[i / kScanBlock] : 0;
    if (i < n)
        out[i] += off;
    if (i == n - 1)
        *total_slot = out[i] + in[i];
}

__global__ void k_scatter(const int *__restrict__ key, int64_t n, int *__restrict__ fill, int *__restrict__ perm)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int pos = atomicAdd(&fill[key[i]], 1);
    perm[pos] = (int)i;
}

// Sorted records: FP64 torus position, FP32 position relative to the point's cell corner
// (cell differences are then exact multiples of the dyadic cell width), window base and fraction.
template <typename real>
__global__ void k_gather_points(const double *__restrict__ xy, const int *__restrict__ perm, int64_t n, double s,
                                int n_os, int window_lo, int n_a, int m, int cell, double2 *__restrict__ pos,
                                typename Cplx<real>::type *__restrict__ frac, int *__restrict__ base,
                                float2 *__restrict__ pos32, float2 *__restrict__ pos32_lo)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    const int i = perm[k];
    const double x = xy[2 * i], y = xy[2 * i + 1];
    int b1, b2;
    double f1, f2;
    grid_coord(x, s, n_os, window_lo, b1, f1);
    grid_coord(y, s, n_os, window_lo, b2, f2);
    clamp_base(b1, m, n_a);
    clamp_base(b2, m, n_a);
    const double xt = s * x, yt = s * y;
    pos[k] = make_double2(xt, yt);
    typename Cplx<real>::type fr;
    fr.x = (real)f1;
    fr.y = (real)f2;
    frac[k] = fr;
    base[k] = (b1 & 0xffff) | (b2 << 16);
    if (pos32) {
        // torus coordinate of the cell's lower corner: (c * cell + window_lo) / n_os - 1/2
        // offset from the cell corner as an unevaluated sum hi + lo of two floats
        const double c1 = (double)((b1 / cell) * cell + window_lo) / n_os - 0.5;
        const double c2 = (double)((b2 / cell) * cell + window_lo) / n_os - 0.5;
        const double o1 = xt - c1, o2 = yt - c2;
        const float h1 = (float)o1, h2 = (float)o2;
        pos32[k] = make_float2(h1, h2);
        pos32_lo[k] = make_float2((float)(o1 - (double)h1), (float)(o2 - (double)h2));
    }
}

// Sum v over the block (all threads take part) and add the total to *dst.
__device__ __forceinline__ void block_sum_add(double acc, double *dst)
{
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
            atomicAdd(dst, acc);
    }
}

template <typename real>
__global__ void k_gather_charges(const void *__restrict__ q, int q_is_f64, const int *__restrict__ perm,
                                 int64_t M, real *__restrict__ q_sorted, double *__restrict__ q_sum)
{
    const int r = blockIdx.y;
    double acc = 0.0;
#pragma unroll 4
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = (int64_t)r * M + perm[k];
        const double v = q_is_f64 ? ((const double *)q)[src] : (double)((const float *)q)[src];
        q_sorted[(int64_t)r * M + k] = (real)v;
        acc += v;
    }
    block_sum_add(acc, &q_sum[r]);
}

// Batched gather: block -> (instance, block of its sources), blockIdx.y = right-hand side.
template <typename real>
__global__ void k_batch_gather_charges(const BatchInst<real> *__restrict__ inst, const BatchIO *__restrict__ io,
                                       BlockMap bm, int q_is_f64)
{
    const int i = bm.inst[blockIdx.x];
    const BatchInst<real> &b = inst[i];
    const int r = blockIdx.y;
    const int64_t M = b.M;
    const int64_t k = (int64_t)(blockIdx.x - bm.first[i]) * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (k < M) {
        const int64_t src = (int64_t)r * M + b.src_perm[k];
        const void *q = io[i].q;
        v = q_is_f64 ? ((const double *)q)[src] : (double)((const float *)q)[src];
        b.q[(int64_t)r * M + k] = (real)v;
    }
    block_sum_add(v, &b.q_sum[r]);
}

__global__ void k_near_count(const double2 *__restrict__ tgt_pos, const int *__restrict__ tgt_base, int64_t N,
                             const double2 *__restrict__ src_pos, const int *__restrict__ src_start, CellGrid cg,
                             double eps2, double close2, unsigned long long *counts)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long near = 0, close = 0;
    if (k < N) {
        const double2 x = tgt_pos[k];
        const int packed = tgt_base[k];
        const int c1 = base1(packed) / cg.cell, c2 = base2(packed) / cg.cell;
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
                    const double dx = x.x - src_pos[j].x, dy = x.y - src_pos[j].y;
                    const double r2 = dx * dx + dy * dy;
                    if (r2 < eps2) {
                        ++near;
                        if (r2 < close2)
                            ++close;
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        near += __shfl_xor_sync(0xffffffffu, near, o);
        close += __shfl_xor_sync(0xffffffffu, close, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[0], near);
        atomicAdd(&counts[1], close);
    }
}

inline unsigned blocks_for(int64_t n, int threads)
{
    return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

cudaError_t launch_rmax(const double *xy, int64_t n, unsigned long long *out, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const int threads = 256;
    unsigned blocks = blocks_for(n, threads);
    if (blocks > 1024)
        blocks = 1024;
    k_rmax<<<blocks, threads, 0, st>>>(xy, n, out);
    return cudaGetLastError();
}

cudaError_t launch_point_keys(const double *xy, int64_t n, double s, int n_os, int window_lo, int n_a, int m,
                              CellGrid cg, int *key, int *count, int *status, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_point_keys<<<blocks_for(n, 256), 256, 0, st>>>(xy, n, s, n_os, window_lo, n_a, m, cg, key, count, status);
    return cudaGetLastError();
}

// start[0..n] = exclusive scan of count[0..n), start[n] = total.  block_tmp holds
// ceil(n / 4096) + 1 ints; n <= 4096 * 4096.
cudaError_t launch_exclusive_scan(const int *count, int *start, int n, int *block_tmp, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const int nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb > kScanBlock)
        return cudaErrorInvalidValue;
    k_scan_block<<<nb, kScanThreads, 0, st>>>(count, start, n, nb > 1 ? block_tmp : nullptr);
    if (nb > 1)
        k_scan_block<<<1, kScanThreads, 0, st>>>(block_tmp, block_tmp, nb, nullptr);
    k_scan_add<<<blocks_for(n, 256), 256, 0, st>>>(start, n, nb > 1 ? block_tmp : nullptr, start + n, count);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const int *key, int64_t n, int *fill, int *perm, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_scatter<<<blocks_for(n, 256), 256, 0, st>>>(key, n, fill, perm);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gather_points(const double *xy, const int *perm, int64_t n, double s, int n_os, int window_lo,
                                 int n_a, int m, int cell, double2 *pos, void *frac, int *base, float2 *pos32,
                                 float2 *pos32_lo, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_gather_points<real><<<blocks_for(n, 256), 256, 0, st>>>(
        xy, perm, n, s, n_os, window_lo, n_a, m, cell, pos, (typename Cplx<real>::type *)frac, base, pos32,
        pos32_lo);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gather_charges(const void *q, int q_is_f64, const int *perm, int64_t M, int nrhs, real *q_sorted,
                                  double *q_sum, cudaStream_t st)
{
    if (M <= 0 || nrhs <= 0)
        return cudaSuccess;
    // four blocks per SM, each thread with several gathers in flight: fewer blocks also mean
    // fewer FP64 atomics on the charge sum (2^20 charges: 19.9 -> 16.3 us against 2048 blocks)
    static int sms_of[64] = {0};   // per device ordinal (SM counts can differ between GPUs)
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 64 && sms_of[dev] > 0) {
        sms = sms_of[dev];
    } else {
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        if (dev < 64)
            sms_of[dev] = sms;
    }
    unsigned bx = blocks_for(M, 256);
    if (bx > 4u * (unsigned)sms)
        bx = 4u * (unsigned)sms;
    k_gather_charges<real><<<dim3(bx, nrhs), 256, 0, st>>>(q, q_is_f64, perm, M, q_sorted, q_sum);
    return cudaGetLastError();
}

cudaError_t launch_near_count(const double2 *tgt_pos, const int *tgt_base, int64_t N, const double2 *src_pos,
                              const int *src_start, CellGrid cg, double eps2, double close2,
                              unsigned long long *counts, cudaStream_t st)
{
    if (N <= 0)
        return cudaSuccess;
    k_near_count<<<blocks_for(N, 256), 256, 0, st>>>(tgt_pos, tgt_base, N, src_pos, src_start, cg, eps2, close2,
                                                      counts);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_batch_gather_charges(const BatchInst<real> *inst, const BatchIO *io, BlockMap bm, int blocks,
                                        int nrhs, int q_is_f64, cudaStream_t st)
{
    if (blocks <= 0 || nrhs <= 0)
        return cudaSuccess;
    k_batch_gather_charges<real><<<dim3((unsigned)blocks, (unsigned)nrhs), 256, 0, st>>>(inst, io, bm, q_is_f64);
    return cudaGetLastError();
}

template cudaError_t launch_batch_gather_charges<float>(const BatchInst<float> *, const BatchIO *, BlockMap, int, int,
                                                        int, cudaStream_t);
template cudaError_t launch_batch_gather_charges<double>(const BatchInst<double> *, const BatchIO *, BlockMap, int,
                                                         int, int, cudaStream_t);

template cudaError_t launch_gather_points<float>(const double *, const int *, int64_t, double, int, int, int, int, int,
                                                 double2 *, void *, int *, float2 *, float2 *, cudaStream_t);
template cudaError_t launch_gather_points<double>(const double *, const int *, int64_t, double, int, int, int, int,
                                                  int, double2 *, void *, int *, float2 *, float2 *, cudaStream_t);
template cudaError_t launch_gather_charges<float>(const void *, int, const int *, int64_t, int, float *, double *,
                                                  cudaStream_t);
template cudaError_t launch_gather_charges<double>(const void *, int, const int *, int64_t, int, double *, double *,
                                                   cudaStream_t);

}  // namespace fs
