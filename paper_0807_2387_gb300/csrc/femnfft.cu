// C ABI of the FEM-NFFT fast summation: plan, charges, evaluation (host side).
//
// Declared in include/femnfft.h.  Every compute step runs in the kernels of
// this directory; this file validates arguments, sizes the workspace, derives
// the method's constants (torus scale, T_I and T_B, window transform) and
// enqueues the kernels on the plan's stream.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/femnfft.h"
#include "internal.h"
#include "plan.h"

using namespace fs;

namespace fs {

namespace {
thread_local std::string g_last_error;
}

fs_status fail(fs_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

}  // namespace fs

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

// Modified Bessel function I_0 by its power series sum_k (x^2/4)^k / (k!)^2 (all terms positive).
double fs::bessel_i0(double x)
{
    const double y = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= y / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum && k > x)
            break;
    }
    return sum;
}

namespace {

// Solve the p x p system that makes T_I(r) = sum_k beta_k (r/eps)^(2k) match k(r) = -(1/2pi) log r
// and its first p-1 derivatives at r = eps (scaled variable u = r/eps; Gaussian elimination with
// partial pivoting).
bool near_coefficients(double eps, int p, double *beta)
{
    const double inv2pi = 1.0 / (2.0 * kPi);
    std::vector<double> a(p * p, 0.0), rhs(p, 0.0);
    for (int j = 0; j < p; ++j) {
        for (int k = 0; k < p; ++k) {
            const int e = 2 * k;
            if (e < j)
                continue;
            double f = 1.0;
            for (int t = 0; t < j; ++t)
                f *= (double)(e - t);
            a[j * p + k] = f;
        }
        if (j == 0) {
            rhs[j] = -std::log(eps) * inv2pi;
        } else {
            double fact = 1.0;   // (j-1)!
            for (int t = 2; t < j; ++t)
                fact *= t;
            rhs[j] = -((j % 2 == 1) ? 1.0 : -1.0) * fact * inv2pi;   // eps^j k^(j)(eps)
        }
    }
    for (int col = 0; col < p; ++col) {
        int piv = col;
        for (int r = col + 1; r < p; ++r)
            if (std::fabs(a[r * p + col]) > std::fabs(a[piv * p + col]))
                piv = r;
        if (a[piv * p + col] == 0.0)
            return false;
        if (piv != col) {
            for (int c = 0; c < p; ++c)
                std::swap(a[piv * p + c], a[col * p + c]);
            std::swap(rhs[piv], rhs[col]);
        }
        for (int r = col + 1; r < p; ++r) {
            const double f = a[r * p + col] / a[col * p + col];
            if (f == 0.0)
                continue;
            for (int c = col; c < p; ++c)
                a[r * p + c] -= f * a[col * p + c];
            rhs[r] -= f * rhs[col];
        }
    }
    for (int r = p - 1; r >= 0; --r) {
        double s = rhs[r];
        for (int c = r + 1; c < p; ++c)
            s -= a[r * p + c] * beta[c];
        beta[r] = s / a[r * p + r];
    }
    return true;
}

}  // namespace


namespace {

// Per-tap polynomial form of the normalised window for the FP32 kernels: for tap a the
// function frac -> psi(frac + m - 1 - a) on [0, 1) is interpolated at kPolyD + 1 Chebyshev
// points in FP64 and rewritten in monomials of t = frac - 1/2; the slope polynomial is its
// exact derivative.
}  // namespace

void fs::build_window_poly(double sigma, int m, WindowPoly *wp)
{
    const double b = kPi * (2.0 - 1.0 / sigma);
    const int D = kPolyD, K = kPolyD + 1;
    auto psi = [&](double x) {
        const double t = (double)m * m - x * x;
        if (!(t > 0.0))
            return 0.0;
        const double tau = std::sqrt(t);
        return (double)m * std::sinh(b * tau) / (tau * std::sinh(b * m));
    };
    // monomial coefficients of T_n(u), u in [-1, 1]
    std::vector<std::vector<double>> T(K, std::vector<double>(K, 0.0));
    T[0][0] = 1.0;
    if (K > 1)
        T[1][1] = 1.0;
    for (int n = 2; n < K; ++n)
        for (int i = 0; i < K; ++i)
            T[n][i] = (i > 0 ? 2.0 * T[n - 1][i - 1] : 0.0) - T[n - 2][i];
    std::memset(wp, 0, sizeof(*wp));
    for (int a = 0; a < 2 * m; ++a) {
        const int j = m - 1 - a;
        std::vector<double> f(K), cheb(K, 0.0), mono(K, 0.0);
        for (int k = 0; k < K; ++k) {
            const double u = std::cos(kPi * (k + 0.5) / K);
            f[k] = psi(0.5 + 0.5 * u + j);
        }
        for (int n = 0; n < K; ++n) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k)
                acc += f[k] * std::cos(kPi * n * (k + 0.5) / K);
            cheb[n] = acc * (n == 0 ? 1.0 : 2.0) / K;
        }
        for (int n = 0; n < K; ++n)
            for (int i = 0; i < K; ++i)
                mono[i] += cheb[n] * T[n][i];
        // u = 2t: coefficient of t^i is 2^i times that of u^i
        double scale = 1.0;
        for (int i = 0; i < K; ++i) {
            wp->c[a][i] = (float)(mono[i] * scale);
            if (i > 0)
                wp->d[a][i - 1] = (float)(mono[i] * scale * i);
            if (i > 1)
                wp->e[a][i - 2] = (float)(mono[i] * scale * i * (i - 1));
            scale *= 2.0;
        }
    }
    (void)D;
}

namespace {

// Bin one point set: keys, counting sort, per-point records.
template <typename real>
fs_status bin_points(fs_plan *pl, const double *xy, int64_t n, int **perm, int **base, void **frac, double2 **pos,
                     float2 **pos32, float2 **lo32, int **start)
{
    FS_TRY(pl->alloc(perm, n));
    FS_TRY(pl->alloc(base, n));
    FS_TRY(pl->alloc_bytes(frac, (size_t)std::max<int64_t>(n, 1) * 2 * sizeof(real)));
    FS_TRY(pl->alloc(pos, n));
    if (pl->precision == 32) {
        FS_TRY(pl->alloc(pos32, n));
        FS_TRY(pl->alloc(lo32, n));
    } else {
        *pos32 = nullptr;
        *lo32 = nullptr;
    }
    FS_TRY(pl->alloc(start, (size_t)pl->n_keys + 1));
    int *key = nullptr, *count = nullptr, *fill = nullptr, *tmp = nullptr;
    FS_TRY(pl->alloc(&key, n));
    FS_TRY(pl->alloc(&count, pl->n_keys));
    FS_TRY(pl->alloc(&fill, (size_t)pl->n_keys + 1));
    FS_TRY(pl->alloc(&tmp, (size_t)pl->n_keys / 4096 + 2));
    cudaStream_t st = pl->stream;
    FS_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * pl->n_keys, st));
    FS_CUDA(cudaMemsetAsync(*start, 0, sizeof(int) * ((size_t)pl->n_keys + 1), st));
    FS_CUDA(launch_point_keys(xy, n, pl->s, pl->n_os, pl->window_lo, pl->n_a, pl->m, pl->cg, key, count, pl->status,
                              st));
    FS_CUDA(launch_exclusive_scan(count, *start, pl->n_keys, tmp, st));
    FS_CUDA(cudaMemcpyAsync(fill, *start, sizeof(int) * ((size_t)pl->n_keys + 1), cudaMemcpyDeviceToDevice, st));
    FS_CUDA(launch_scatter(key, n, fill, *perm, st));
    FS_CUDA(launch_gather_points<real>(xy, *perm, n, pl->s, pl->n_os, pl->window_lo, pl->n_a, pl->m, pl->cg.cell, *pos,
                                       *frac, *base, *pos32, *lo32, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->release(key);
    pl->release(count);
    pl->release(fill);
    pl->release(tmp);
    return FS_OK;
}

// FP32 near-field warp items over the "own" points (targets for the forward, sources for
// the adjoint): at most 64 consecutive points of one cell (two per lane), in the cell's
// Morton sub-cell order, so an item is compact.  Target items split each cell evenly into
// the fewest items of at most 64; source items give a sub-cell holding 32 or more points
// items of its own (boxes an eighth of a cell wide) and merge sparser sub-cells of the same
// cell up to 64.  On the 2^20-point mixture the even split leaves fewer idle lane slots and
// fewer candidate visits (items 19,884 -> 18,098, evaluated pair slots -4 %), and the
// forward near field fell from 3.28 to 2.87 ms on GB300; the source items, which also serve
// the source-major FEM kernel, keep the rule that kernel was tuned with.  Items are ordered
// by estimated work (points x "other" points in the 3 x 3 cells around the item's cell),
// largest first, so the heavy warps start early and the tail of the launch stays short.
fs_status build_near_items(fs_plan *pl, const int *own_start_d, const int *oth_start_d, bool whole_cells, int2 **out,
                           int64_t *n_out, std::vector<int2> *items_out = nullptr,
                           std::vector<int64_t> *work_out = nullptr)
{
    constexpr int kCap = 64, kOwn = 32;
    std::vector<int> start(pl->n_keys + 1), oth(pl->n_keys + 1);
    FS_CUDA(cudaMemcpy(start.data(), own_start_d, sizeof(int) * start.size(), cudaMemcpyDeviceToHost));
    FS_CUDA(cudaMemcpy(oth.data(), oth_start_d, sizeof(int) * oth.size(), cudaMemcpyDeviceToHost));
    const int n_cells = pl->n_keys / kSub;
    std::vector<int2> items;
    std::vector<int> item_cell;
    for (int key = 0; whole_cells && key < n_cells; ++key) {
        const int a = start[key * kSub], c = start[(key + 1) * kSub] - a;
        const int pieces = (c + kCap - 1) / kCap;
        for (int i = 0; i < pieces; ++i) {
            const int lo = a + (int)((int64_t)c * i / pieces), hi = a + (int)((int64_t)c * (i + 1) / pieces);
            items.push_back(make_int2(lo, hi - lo));
            item_cell.push_back(key);
        }
    }
    for (int key = 0; !whole_cells && key < n_cells; ++key) {
        int open_start = -1, open_count = 0;
        auto flush = [&]() {
            if (open_count > 0) {
                items.push_back(make_int2(open_start, open_count));
                item_cell.push_back(key);
            }
            open_count = 0;
        };
        for (int sub = 0; sub < kSub; ++sub) {
            const int a = start[key * kSub + sub], c = start[key * kSub + sub + 1] - a;
            if (c == 0)
                continue;
            if (c >= kOwn) {
                flush();
                const int pieces = (c + kCap - 1) / kCap;
                for (int i = 0; i < pieces; ++i) {
                    const int lo = a + (int)((int64_t)c * i / pieces), hi = a + (int)((int64_t)c * (i + 1) / pieces);
                    items.push_back(make_int2(lo, hi - lo));
                    item_cell.push_back(key);
                }
                continue;
            }
            if (open_count > 0 && open_count + c > kCap)
                flush();
            if (open_count == 0)
                open_start = a;
            open_count += c;   // contiguous: sub-cells of a cell follow each other in the sorted order
        }
        flush();
    }
    std::vector<int64_t> nb(n_cells, 0);
    const int nc = pl->cg.n_c;
    for (int c1 = 0; c1 < nc; ++c1)
        for (int c2 = 0; c2 < nc; ++c2) {
            int64_t acc = 0;
            for (int d1 = -1; d1 <= 1; ++d1)
                for (int d2 = -1; d2 <= 1; ++d2) {
                    const int e1 = c1 + d1, e2 = c2 + d2;
                    if (e1 < 0 || e2 < 0 || e1 >= nc || e2 >= nc)
                        continue;
                    const int kk = pl->cg.key(e1, e2);
                    acc += oth[(kk + 1) * kSub] - oth[kk * kSub];
                }
            nb[pl->cg.key(c1, c2)] = acc;
        }
    std::vector<std::pair<int64_t, int2>> wi;
    wi.reserve(items.size());
    for (size_t i = 0; i < items.size(); ++i)
        wi.push_back({(int64_t)items[i].y * nb[item_cell[i]], items[i]});
    std::stable_sort(wi.begin(), wi.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    for (size_t i = 0; i < items.size(); ++i)
        items[i] = wi[i].second;
    if (items_out)
        *items_out = items;
    if (work_out) {
        work_out->resize(items.size());
        for (size_t i = 0; i < items.size(); ++i)
            (*work_out)[i] = wi[i].first;
    }
    *n_out = (int64_t)items.size();
    FS_TRY(pl->alloc(out, items.size()));
    if (!items.empty())
        FS_CUDA(cudaMemcpy(*out, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
    return FS_OK;
}

template <typename real> fs_status twiddles(fs_plan *pl, int L, void **out)
{
    std::vector<real> h(2 * (size_t)L);
    fft_twiddle_table<real>(L, h.data());
    FS_TRY(pl->alloc_bytes(out, h.size() * sizeof(real)));
    FS_CUDA(cudaMemcpyAsync(*out, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice, pl->stream));
    FS_CUDA(cudaStreamSynchronize(pl->stream));
    return FS_OK;
}

// b_l on the device in FP64 and the multiplier table in the working precision.
template <typename real> fs_status coefficients(fs_plan *pl)
{
    const int n = pl->n;
    cudaStream_t st = pl->stream;
    double2 *samp = nullptr, *tmp = nullptr;
    void *tw64 = nullptr;
    double *c_tab = nullptr;
    FS_TRY(pl->alloc(&samp, (size_t)n * n));
    FS_TRY(pl->alloc(&tmp, (size_t)n * n));
    FS_TRY(twiddles<double>(pl, n, &tw64));
    FS_CUDA(launch_kernel_samples(samp, n, pl->kp, st));
    FS_CUDA(launch_fft_lines_c64(samp, n, n, (const double2 *)tw64, st));
    FS_CUDA(launch_transpose_c64(samp, tmp, n, st));
    FS_CUDA(launch_fft_lines_c64(tmp, n, n, (const double2 *)tw64, st));
    // window transform c(l) = n_os phi_1-hat(l) / phi_1(0) = I_0(m sqrt(b^2 - (2 pi l / n_os)^2)) pi m / sinh(b m)
    const double b = kPi * (2.0 - 1.0 / pl->sigma);
    const double m = pl->m;
    std::vector<double> c(n / 2 + 1);
    for (int l = 0; l <= n / 2; ++l) {
        const double arg = b * b - std::pow(2.0 * kPi * l / pl->n_os, 2);
        c[l] = bessel_i0(m * std::sqrt(arg)) * kPi * m / std::sinh(b * m);
    }
    FS_TRY(pl->alloc(&c_tab, c.size()));
    FS_CUDA(cudaMemcpyAsync(c_tab, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    FS_TRY(pl->alloc_bytes(&pl->mul, (size_t)(n / 2 + 1) * (n + 1) * sizeof(real)));
    FS_CUDA(launch_build_mul<real>(tmp, n, c_tab, (real *)pl->mul, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->release(samp);
    pl->release(tmp);
    pl->release(tw64);
    pl->release(c_tab);
    return FS_OK;
}

fs_status validate_params(int n_grid, double sigma_os, int m, double eps_I, const fs_opts &o)
{
    if (!is_pow2(n_grid) || n_grid < 8 || n_grid > 2048)
        return fail(FS_EINVAL, "n_grid must be a power of two in [8, 2048]");
    if (!(sigma_os > 1.0))
        return fail(FS_EINVAL, "sigma_os must exceed 1");
    const double nos = sigma_os * n_grid;
    const int n_os = (int)std::lround(nos);
    if (std::fabs(nos - n_os) > 1e-9 || !is_pow2(n_os) || n_os > 4096 || n_os <= n_grid)
        return fail(FS_EINVAL, "sigma_os * n_grid must be a power of two in (n_grid, 4096]");
    if (m < 2 || m > kMaxM || 4 * m >= n_os)
        return fail(FS_EINVAL, "m_window must be in [2, 8] and below n_os / 4");
    if (!(eps_I > 0.0) || !(eps_I < 0.25))
        return fail(FS_EINVAL, "eps_I must be in (0, 1/4) (torus units)");
    if (o.precision != 0 && o.precision != 32 && o.precision != 64)
        return fail(FS_EINVAL, "precision must be 32 or 64");
    if (o.p < 0 || o.p > kMaxP)
        return fail(FS_EINVAL, "p must be in [1, 16] (0 = default)");
    if (o.eps_B < 0.0 || o.eps_B >= 0.25 || std::isnan(o.eps_B))
        return fail(FS_EINVAL, "eps_B must be in (0, 1/4) (0 = default)");
    if (o.cell < 0 || o.tile_cells < 0)
        return fail(FS_EINVAL, "cell and tile_cells must be >= 0");
    return FS_OK;
}

template <typename real>
fs_status plan_init(fs_plan *pl, const double *src, int64_t M, const double *tgt, int64_t N, int n_grid,
                    double sigma_os, int m, double eps_I, const fs_opts &o)
{
    pl->n = n_grid;
    pl->sigma = sigma_os;
    pl->n_os = (int)std::lround(sigma_os * n_grid);
    pl->m = m;
    pl->eps_I = eps_I;
    pl->p = o.p > 0 ? o.p : std::min(kMaxP, std::max(2, (int)std::lround(n_grid * eps_I)));
    pl->eps_B = o.eps_B > 0 ? o.eps_B : eps_I;
    pl->M = M;
    pl->N = N;
    pl->flags = o.flags;
    pl->kahan = !(o.flags & FS_FLAG_NO_KAHAN);
    pl->stream = (cudaStream_t)o.stream;
    FS_CUDA(cudaGetDevice(&pl->device));
    cudaStream_t st = pl->stream;
    FS_TRY(pl->alloc(&pl->status, 1));
    FS_CUDA(cudaMemsetAsync(pl->status, 0, sizeof(int), st));

    // torus scale from the largest radius
    unsigned long long *d_r = nullptr;
    FS_TRY(pl->alloc(&d_r, 1));
    FS_CUDA(cudaMemsetAsync(d_r, 0, sizeof(unsigned long long), st));
    FS_CUDA(launch_rmax(src, M, d_r, st));
    FS_CUDA(launch_rmax(tgt, N, d_r, st));
    unsigned long long r_bits = 0;
    FS_CUDA(cudaMemcpyAsync(&r_bits, d_r, sizeof(r_bits), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->release(d_r);
    double r2max;
    std::memcpy(&r2max, &r_bits, sizeof(double));
    if (!std::isfinite(r2max))
        return fail(FS_EINVAL, "non-finite point coordinates");
    const double rmax = std::sqrt(r2max);
    pl->s = rmax > 0.0 ? (0.25 - 0.5 * pl->eps_B) / rmax : 1.0;

    // active window: grid lines that can hold a tap, with a one-line margin
    const int L = pl->n_os;
    pl->window_lo = (int)std::floor(L * (0.25 + 0.5 * pl->eps_B)) - m - 1;
    const int hi = (int)std::floor(L * (0.75 - 0.5 * pl->eps_B)) + 1;
    int n_a = hi - pl->window_lo + m + 1;
    n_a = (n_a + 3) & ~3;
    if (n_a > L)
        return fail(FS_EINVAL, "window half-width too large for this grid (active window exceeds n_os)");
    pl->n_a = n_a;
    pl->pitch = n_a;
    pl->ld = n_a;

    // cells and tiles
    int cell = o.cell;
    const int min_cell = (int)std::ceil(eps_I * L - 1e-9);
    if (cell == 0)
        cell = std::max(1, min_cell);
    else if (cell < min_cell)
        return fail(FS_EINVAL, "cell narrower than eps_I");
    pl->cg.cell = cell;
    pl->cg.n_c = (n_a + cell - 1) / cell;
    // spreading tiles of about 16 grid lines; plans with three or more sources per target (FEM
    // meshes: the near field then runs over source items beside the spreading) take about 24,
    // fewer and longer items that leave the near field more room (disc mesh time loop 0.185 ->
    // 0.182 ms; the 2^20-point mixture is 2.67 ms with one-cell and 2.74 ms with two-cell tiles)
    const double tile_lines = (N > 0 && M >= 3 * N) ? 24.0 : 16.0;
    int T = o.tile_cells > 0 ? o.tile_cells : std::max(1, (int)std::lround(tile_lines / cell));
    auto smem_for = [&](int t) {   // the larger of the value spreading's and the adjoint's dipole spreading's
        const int P = t * cell + 2 * m - 1;
        const bool comp = pl->kahan && sizeof(real) == 4;
        const size_t dip = (size_t)kSpreadWarps * P * spread_pitch(P, 2 * m) * sizeof(real) * (comp ? 2 : 1) +
                           sizeof(float) * 2 * m * (2 * kPolyD + 1);
        return std::max(dip, spread_smem_bytes<real>(P, 2 * m, comp));
    };
    while (T > 1 && smem_for(T) > 160 * 1024)
        --T;
    if (smem_for(T) > 200 * 1024)
        return fail(FS_EINVAL, "spreading tile does not fit in shared memory (cell too wide)");
    pl->cg.T = T;
    pl->cg.n_t = (pl->cg.n_c + T - 1) / T;
    if ((int64_t)pl->cg.n_keys() * kSub > 4096 * 4096)
        return fail(FS_EINVAL, "too many cells (eps_I too small for this grid)");
    pl->n_keys = pl->cg.n_keys() * kSub;   // cell keys refined by the 8 x 8 sub-cell index

    // regularised kernel data
    pl->kp.eps_I = eps_I;
    pl->kp.eps_B = pl->eps_B;
    pl->kp.p = pl->p;
    if (!near_coefficients(eps_I, pl->p, pl->beta))
        return fail(FS_EINVAL, "singular near-field interpolation system");
    for (int k = 0; k < pl->p; ++k)
        pl->kp.beta[k] = pl->beta[k];
    {
        const double inv2pi = 1.0 / (2.0 * kPi);
        const double r0 = 0.5 - pl->eps_B;
        double fact = 1.0;   // j!
        for (int j = 0; j < pl->p; ++j) {
            double kj;
            if (j == 0) {
                kj = -std::log(r0) * inv2pi;
            } else {
                double f1 = 1.0;   // (j-1)!
                for (int t = 2; t < j; ++t)
                    f1 *= t;
                kj = -((j % 2 == 1) ? 1.0 : -1.0) * f1 * std::pow(r0, -(double)j) * inv2pi;
            }
            if (j > 0)
                fact *= j;
            pl->kp.tb_f0[j] = std::pow(pl->eps_B, (double)j) * kj / fact;
            // C(p-1+j, j)
            double cbin = 1.0;
            for (int t = 1; t <= j; ++t)
                cbin = cbin * (double)(pl->p - 1 + t) / (double)t;
            pl->kp.tb_binom[j] = cbin;
        }
        pl->kp.k_half = std::log(2.0) * inv2pi;
    }

    build_window_poly(pl->sigma, pl->m, &pl->wpoly);

    // binning
    FS_TRY(bin_points<real>(pl, src, M, &pl->src_perm, &pl->src_base, &pl->src_frac, &pl->src_pos, &pl->src_pos32,
                            &pl->src_lo32, &pl->src_start));
    FS_TRY(bin_points<real>(pl, tgt, N, &pl->tgt_perm, &pl->tgt_base, &pl->tgt_frac, &pl->tgt_pos, &pl->tgt_pos32,
                            &pl->tgt_lo32, &pl->tgt_start));
    int dev_status = 0;
    FS_CUDA(cudaMemcpy(&dev_status, pl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_status != 0)
        return fail(FS_EDOMAIN, "a point fell outside the admissible radius after scaling");

    // spreading work items: tiles split into slices of at most kSpreadChunk points (sources
    // for the forward spread, targets for the adjoint one)
    for (int side = 0; side < 2; ++side) {
        std::vector<int> start(pl->n_keys + 1);
        FS_CUDA(cudaMemcpy(start.data(), side == 0 ? pl->src_start : pl->tgt_start, sizeof(int) * start.size(),
                           cudaMemcpyDeviceToHost));
        std::vector<SpreadItem> items;
        const int TT = T * T * kSub;
        const int n_tiles = pl->cg.n_t * pl->cg.n_t;
        for (int t = 0; t < n_tiles; ++t) {
            const int a = start[t * TT], b2 = start[(t + 1) * TT];
            for (int s0 = a; s0 < b2; s0 += kSpreadChunk)
                items.push_back(SpreadItem{t, s0, std::min(kSpreadChunk, b2 - s0), 0});
        }
        if (side == 0)
            pl->items_h = items;
        SpreadItem **dst = side == 0 ? &pl->items : &pl->tgt_items;
        (side == 0 ? pl->n_items : pl->n_tgt_items) = (int)items.size();
        FS_TRY(pl->alloc(dst, items.size()));
        if (!items.empty())
            FS_CUDA(cudaMemcpy(*dst, items.data(), items.size() * sizeof(SpreadItem), cudaMemcpyHostToDevice));
    }

    // spreading mode: shared-memory tiles, or global atomics when the occupied tiles hold so few
    // sources that zeroing and flushing a tile costs more than the atomics it saves
    {
        int occupied = 0, prev = -1;
        for (const SpreadItem &it : pl->items_h)
            if (it.tile != prev) {
                ++occupied;
                prev = it.tile;
            }
        const double per_tile = occupied > 0 ? (double)M / occupied : 0.0;
        if (o.flags & FS_FLAG_SPREAD_DIRECT)
            pl->spread_direct = true;
        else if (o.flags & FS_FLAG_SPREAD_TILES)
            pl->spread_direct = false;
        else
            pl->spread_direct = M > 0 && per_tile < kDirectSpreadBelow;
    }

    if (pl->precision == 32) {
        FS_TRY(build_near_items(pl, pl->tgt_start, pl->src_start, true, &pl->near_items, &pl->n_near_items,
                                &pl->near_items_h, &pl->near_work_h));
        // FEM plans (several quadrature points around every node): a cell holds few targets, so a
        // target item's box would span the whole cell; the forward near field then runs over
        // items of sources, whose boxes stay small
        pl->src_major = N > 0 && M >= 3 * N;
        if (pl->src_major)
            FS_TRY(build_near_items(pl, pl->src_start, pl->tgt_start, false, &pl->src_near_items,
                                    &pl->n_src_near_items));
    }

    // coefficient table and FFT twiddles
    FS_TRY(coefficients<real>(pl));
    FS_TRY(twiddles<real>(pl, L, &pl->tw));

    // grids and per-target intermediates
    FS_TRY(pl->alloc_bytes(&pl->grid, (size_t)n_a * pl->pitch * sizeof(real)));
    if (pl->spread_direct && pl->kahan && sizeof(real) == 4)
        FS_TRY(pl->alloc_bytes(&pl->grid_comp, (size_t)n_a * pl->pitch * sizeof(real)));
    FS_TRY(pl->alloc_bytes(&pl->spec, (size_t)(pl->n / 2 + 1) * pl->ld * 2 * sizeof(real)));
    // the near field's sums in one block (phi_s, grad_s, coinc; each part 16-byte aligned), so
    // that the source-major near field zeroes them with one memset
    pl->sums_n = (std::max<int64_t>(N, 1) + 3) / 4 * 4;
    FS_TRY(pl->alloc_bytes(&pl->phi_s, (size_t)pl->sums_n * 4 * sizeof(real)));
    pl->grad_s = (unsigned char *)pl->phi_s + (size_t)pl->sums_n * sizeof(real);
    pl->coinc = (unsigned char *)pl->phi_s + (size_t)pl->sums_n * 3 * sizeof(real);

    // near-field pair statistics: the FP32 path counts with its own traversal (the pairs its
    // near-field kernel evaluates), the FP64 path with FP64 distances
    {
        unsigned long long *cnt = nullptr;
        FS_TRY(pl->alloc(&cnt, 2 * kNearCountSlots));
        FS_CUDA(cudaMemsetAsync(cnt, 0, 2 * kNearCountSlots * sizeof(unsigned long long), st));
        if constexpr (sizeof(real) == 4)
            FS_CUDA(launch_near_count32(pl->n_near_items, pl->near_items, pl->tgt_base, pl->tgt_pos32, pl->tgt_lo32,
                                        pl->src_pos32, pl->src_lo32, pl->src_start, pl->cg, make_near<float>(pl), cnt,
                                        st));
        else
            FS_CUDA(launch_near_count(pl->tgt_pos, pl->tgt_base, N, pl->src_pos, pl->src_start, pl->cg,
                                      eps_I * eps_I, (eps_I / 8) * (eps_I / 8), cnt, st));
        std::vector<unsigned long long> h(2 * kNearCountSlots, 0);
        FS_CUDA(cudaMemcpyAsync(h.data(), cnt, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        FS_CUDA(cudaStreamSynchronize(st));
        pl->near_pairs = pl->near_pairs_fp64 = 0;
        for (int i = 0; i < kNearCountSlots; ++i) {
            pl->near_pairs += (int64_t)h[2 * i];
            pl->near_pairs_fp64 += (int64_t)h[2 * i + 1];
        }
        pl->release(cnt);
    }

    // FP32 plans overlap the near field with spreading and the transform
    if (sizeof(real) == 4 && N > 0 && !(pl->flags & FS_FLAG_SERIAL)) {
        FS_CUDA(cudaStreamCreateWithFlags(&pl->aux, cudaStreamNonBlocking));
        FS_CUDA(cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming));
        FS_CUDA(cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming));
        pl->overlap = true;
    }
    if (pl->flags & FS_FLAG_TIMING) {
        for (int i = 0; i <= kStages; ++i)
            FS_CUDA(cudaEventCreate(&pl->ev[i]));
        if (pl->overlap) {
            FS_CUDA(cudaEventCreate(&pl->ev_n0));
            FS_CUDA(cudaEventCreate(&pl->ev_n1));
            FS_CUDA(cudaEventCreate(&pl->ev_j));
        }
        FS_CUDA(cudaEventCreate(&pl->ev_q0));
        FS_CUDA(cudaEventCreate(&pl->ev_q1));
        pl->events = true;
    }
    return FS_OK;
}

}  // namespace

namespace fs {

fs_status plan_create_common(const double *src, int64_t M, const double *tgt, int64_t N, int n_grid,
                             double sigma_os, int m, double eps_I, const fs_opts *opts, fs_plan *pl)
{
    fs_opts o{};
    if (opts)
        o = *opts;
    FS_TRY(validate_params(n_grid, sigma_os, m, eps_I, o));
    pl->precision = o.precision == 64 ? 64 : 32;
    if (pl->precision == 64)
        return plan_init<double>(pl, src, M, tgt, N, n_grid, sigma_os, m, eps_I, o);
    return plan_init<float>(pl, src, M, tgt, N, n_grid, sigma_os, m, eps_I, o);
}

void plan_destroy(fs_plan *pl)
{
    if (!pl)
        return;
    cudaStreamSynchronize(pl->stream);
    for (void *p : pl->allocs)
        cudaFree(p);
    for (int i = 0; i <= kStages; ++i)
        if (pl->ev[i])
            cudaEventDestroy(pl->ev[i]);
    if (pl->ev_q0)
        cudaEventDestroy(pl->ev_q0);
    if (pl->ev_q1)
        cudaEventDestroy(pl->ev_q1);
    for (cudaEvent_t e : {pl->ev_fork, pl->ev_join, pl->ev_n0, pl->ev_n1, pl->ev_j})
        if (e)
            cudaEventDestroy(e);
    if (pl->aux) {
        cudaStreamSynchronize(pl->aux);
        cudaStreamDestroy(pl->aux);
    }
    if (pl->status_host)
        cudaFreeHost(pl->status_host);
    delete pl;
}

}  // namespace fs

namespace {

// Sorted-charge storage for nrhs vectors (kept when large enough).
template <typename real> fs_status reserve_charges(fs_plan *pl, int nrhs)
{
    if (nrhs > pl->nrhs_cap) {
        pl->release(pl->q_sorted);
        pl->release(pl->q_sum);
        pl->q_sorted = nullptr;
        pl->q_sum = nullptr;
        FS_TRY(pl->alloc_bytes(&pl->q_sorted, (size_t)std::max<int64_t>(pl->M, 1) * nrhs * sizeof(real)));
        FS_TRY(pl->alloc(&pl->q_sum, nrhs));
        pl->nrhs_cap = nrhs;
    }
    return FS_OK;
}

template <typename real> fs_status set_charges_t(fs_plan *pl, const void *q, fs_dtype dtype, int nrhs)
{
    cudaStream_t st = pl->stream;
    FS_TRY(reserve_charges<real>(pl, nrhs));
    pl->nrhs = nrhs;
    if (pl->events)
        FS_CUDA(cudaEventRecord(pl->ev_q0, st));
    FS_CUDA(cudaMemsetAsync(pl->q_sum, 0, sizeof(double) * nrhs, st));
    FS_CUDA(launch_gather_charges<real>(q, dtype == FS_F64, pl->src_perm, pl->M, nrhs, (real *)pl->q_sorted,
                                        pl->q_sum, st));
    if (pl->events)
        FS_CUDA(cudaEventRecord(pl->ev_q1, st));
    return FS_OK;
}

// Step (c): the grid is zeroed and the charges spread into it, through shared-memory tiles or
// (sparse plans, FS_FLAG_SPREAD_DIRECT) with global atomics and a compensation plane.
template <typename real> fs_status spread_forward(fs_plan *pl, const real *q, const Window<real> &w, cudaStream_t st)
{
    const size_t grid_bytes = (size_t)pl->n_a * pl->pitch * sizeof(real);
    FS_CUDA(cudaMemsetAsync(pl->grid, 0, grid_bytes, st));
    if (!pl->spread_direct) {
        FS_CUDA(launch_spread<real>(pl->items, pl->n_items, pl->cg, pl->m, pl->src_base, pl->src_frac, q, w, pl->wpoly,
                                    (real *)pl->grid, pl->pitch, pl->n_a, pl->kahan, st));
        return FS_OK;
    }
    if (pl->grid_comp)
        FS_CUDA(cudaMemsetAsync(pl->grid_comp, 0, grid_bytes, st));
    FS_CUDA(launch_spread_direct<real>(pl->M, pl->m, pl->src_base, pl->src_frac, q, w, pl->wpoly, (real *)pl->grid,
                                       (real *)pl->grid_comp, pl->pitch, pl->n_a, pl->kahan, st));
    return FS_OK;
}

template <typename real> fs_status eval_t(fs_plan *pl, void *phi, void *H, fs_dtype dtype)
{
    cudaStream_t st = pl->stream;
    const Window<real> w = make_window<real>(pl);
    const NearParams<real> np = make_near<real>(pl);
    using C = typename Cplx<real>::type;
    const double shift = std::log(pl->s) / (2.0 * kPi);
    const size_t osz = dtype == FS_F64 ? 8 : 4;
    for (int r = 0; r < pl->nrhs; ++r) {
        const bool rec = pl->events && r == pl->nrhs - 1;
        const real *q = (const real *)pl->q_sorted + (int64_t)r * pl->M;
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[0], st));
        if (pl->overlap)
            FS_CUDA(cudaEventRecord(pl->ev_fork, st));   // the charges are in
        FS_TRY(spread_forward<real>(pl, q, w, st));
        if (pl->overlap) {
            // the near field (stored, not added) on the second stream, submitted after the
            // spreading so that the spreading's blocks are scheduled first
            FS_CUDA(cudaStreamWaitEvent(pl->aux, pl->ev_fork, 0));
            if (rec)
                FS_CUDA(cudaEventRecord(pl->ev_n0, pl->aux));
            if (pl->src_major) {
                // source items add with atomics: zero the near-field sums first (one block)
                FS_CUDA(cudaMemsetAsync(pl->phi_s, 0, sizeof(float) * 4 * (size_t)pl->sums_n, pl->aux));
                FS_CUDA(launch_near_src32(pl->n_src_near_items, pl->src_near_items, pl->src_base, pl->src_pos32,
                                          pl->src_lo32, pl->tgt_pos32, pl->tgt_lo32, pl->tgt_start, pl->cg,
                                          (const float *)q, make_near<float>(pl), (float *)pl->phi_s,
                                          (float *)pl->grad_s, (float *)pl->coinc, pl->aux));
            } else {
                FS_CUDA(launch_near32(pl->n_near_items, pl->near_items, pl->tgt_base, pl->tgt_pos32, pl->tgt_lo32,
                                      pl->src_pos32, pl->src_lo32, pl->src_start, pl->cg, (const float *)q,
                                      make_near<float>(pl), (float *)pl->phi_s, (float *)pl->grad_s,
                                      (float *)pl->coinc, true, pl->aux));
            }
            if (rec)
                FS_CUDA(cudaEventRecord(pl->ev_n1, pl->aux));
            FS_CUDA(cudaEventRecord(pl->ev_join, pl->aux));
        }
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[1], st));
        FS_CUDA(launch_fft_rows_fwd<real>((const real *)pl->grid, pl->pitch, pl->n_a, pl->n_os, pl->n / 2,
                                          (C *)pl->spec, pl->ld, (const C *)pl->tw, st));
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[2], st));
        FS_CUDA(launch_fft_cols<real>((C *)pl->spec, pl->ld, pl->n_a, pl->n_os, pl->n, (const real *)pl->mul,
                                      (const C *)pl->tw, st));
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[3], st));
        FS_CUDA(launch_fft_rows_inv<real>((const C *)pl->spec, pl->ld, pl->n_a, pl->n_os, pl->n / 2,
                                          (real *)pl->grid, pl->pitch, (const C *)pl->tw, st));
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[4], st));
        void *po = phi ? (unsigned char *)phi + (size_t)r * pl->N * osz : nullptr;
        void *ho = H ? (unsigned char *)H + (size_t)r * pl->N * 2 * osz : nullptr;
        if (pl->overlap) {
            FS_CUDA(cudaStreamWaitEvent(st, pl->ev_join, 0));
            if (rec)
                FS_CUDA(cudaEventRecord(pl->ev_j, st));
            // steps (f) and (h) in one pass: the far field added to the near field's sums and
            // written to the caller's buffers (the output stage's time is in the interpolation's)
            FS_CUDA(launch_interp_out<real>(pl->N, pl->m, pl->tgt_base, pl->tgt_frac, w, pl->wpoly,
                                            (const real *)pl->grid, pl->pitch, (real)pl->n_os,
                                            (const real *)pl->phi_s, (const real *)pl->grad_s,
                                            (const real *)pl->coinc, pl->tgt_perm, shift, pl->q_sum + r, pl->s, po, ho,
                                            dtype == FS_F64, st));
            if (rec) {
                FS_CUDA(cudaEventRecord(pl->ev[5], st));
                FS_CUDA(cudaEventRecord(pl->ev[6], st));
                FS_CUDA(cudaEventRecord(pl->ev[7], st));
            }
            continue;
        }
        FS_CUDA(launch_interp<real>(pl->N, pl->m, pl->tgt_base, pl->tgt_frac, w, pl->wpoly, (const real *)pl->grid, pl->pitch,
                                    (real)pl->n_os, (real *)pl->phi_s, (real *)pl->grad_s, false, st));
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[5], st));
        if constexpr (sizeof(real) == 4) {
            if (pl->src_major) {
                FS_CUDA(cudaMemsetAsync(pl->coinc, 0, sizeof(float) * (size_t)std::max<int64_t>(pl->N, 1), st));
                FS_CUDA(launch_near_src32(pl->n_src_near_items, pl->src_near_items, pl->src_base, pl->src_pos32,
                                          pl->src_lo32, pl->tgt_pos32, pl->tgt_lo32, pl->tgt_start, pl->cg,
                                          (const float *)q, np, (float *)pl->phi_s, (float *)pl->grad_s,
                                          (float *)pl->coinc, st));
            } else {
                FS_CUDA(launch_near32(pl->n_near_items, pl->near_items, pl->tgt_base, pl->tgt_pos32, pl->tgt_lo32,
                                      pl->src_pos32, pl->src_lo32, pl->src_start, pl->cg, (const float *)q, np,
                                      (float *)pl->phi_s, (float *)pl->grad_s, (float *)pl->coinc, false, st));
            }
        } else
            FS_CUDA(launch_near64(pl->N, pl->tgt_base, pl->tgt_pos, pl->src_pos, pl->src_start, pl->cg,
                                  (const double *)q, np, (double *)pl->phi_s, (double *)pl->grad_s,
                                  (double *)pl->coinc, st));
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[6], st));
        FS_CUDA(launch_unpermute<real>(pl->N, (const real *)pl->phi_s, (const real *)pl->grad_s,
                                       (const real *)pl->coinc, pl->tgt_perm, shift, pl->q_sum + r, pl->s, po, ho,
                                       dtype == FS_F64, st));
        if (rec)
            FS_CUDA(cudaEventRecord(pl->ev[7], st));
    }
    return FS_OK;
}

fs_status check_plan(const fs_plan *pl)
{
    if (!pl)
        return fail(FS_EINVAL, "null plan");
    return FS_OK;
}

fs_status check_dtype(fs_dtype d)
{
    if (d != FS_F32 && d != FS_F64)
        return fail(FS_EINVAL, "dtype must be FS_F32 or FS_F64");
    return FS_OK;
}

// Boundary edges (used by one triangle), sorted by (lo, hi), with the owner's third node.
fs_status boundary_edges(const std::vector<int> &tris, int64_t Nt, int64_t Nv, std::vector<int> &out)
{
    struct E {
        int lo, hi, third;
    };
    std::vector<E> e;
    e.reserve(3 * Nt);
    for (int64_t t = 0; t < Nt; ++t) {
        const int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        for (int k = 0; k < 3; ++k) {
            if (v[k] < 0 || v[k] >= Nv)
                return fail(FS_EINVAL, "triangle node index out of range");
        }
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2])
            return fail(FS_EINVAL, "degenerate triangle (repeated node)");
        for (int k = 0; k < 3; ++k) {
            const int a = v[k], b = v[(k + 1) % 3], c = v[(k + 2) % 3];
            e.push_back(E{std::min(a, b), std::max(a, b), c});
        }
    }
    std::sort(e.begin(), e.end(), [](const E &x, const E &y) { return x.lo != y.lo ? x.lo < y.lo : x.hi < y.hi; });
    out.clear();
    size_t i = 0;
    while (i < e.size()) {
        size_t j = i + 1;
        while (j < e.size() && e[j].lo == e[i].lo && e[j].hi == e[i].hi)
            ++j;
        if (j - i == 1) {
            out.push_back(e[i].lo);
            out.push_back(e[i].hi);
            out.push_back(e[i].third);
        } else if (j - i > 2) {
            return fail(FS_EINVAL, "non-manifold mesh: an edge is shared by more than two triangles");
        }
        i = j;
    }
    return FS_OK;
}

// Far-field pipeline on the plan's grid: spread (given launcher) -> FFT rows -> columns x mul -> inverse rows.
template <typename real> fs_status spectral_pipeline(fs_plan *pl)
{
    using C = typename Cplx<real>::type;
    cudaStream_t st = pl->stream;
    FS_CUDA(launch_fft_rows_fwd<real>((const real *)pl->grid, pl->pitch, pl->n_a, pl->n_os, pl->n / 2, (C *)pl->spec,
                                      pl->ld, (const C *)pl->tw, st));
    FS_CUDA(launch_fft_cols<real>((C *)pl->spec, pl->ld, pl->n_a, pl->n_os, pl->n, (const real *)pl->mul,
                                  (const C *)pl->tw, st));
    FS_CUDA(launch_fft_rows_inv<real>((const C *)pl->spec, pl->ld, pl->n_a, pl->n_os, pl->n / 2, (real *)pl->grid,
                                      pl->pitch, (const C *)pl->tw, st));
    return FS_OK;
}

template <typename real>
fs_status adjoint_t(fs_plan *pl, const void *g_phi, const void *g_H, fs_dtype in_dtype, void *dq, void *dsrc,
                    void *dtgt, fs_dtype out_dtype)
{
    cudaStream_t st = pl->stream;
    const int64_t M = pl->M, N = pl->N;
    if (!pl->adj_c) {
        FS_TRY(pl->alloc_bytes(&pl->adj_c, (size_t)std::max<int64_t>(N, 1) * sizeof(real)));
        FS_TRY(pl->alloc_bytes(&pl->adj_dn, (size_t)std::max<int64_t>(N, 1) * 2 * sizeof(real)));
        FS_TRY(pl->alloc_bytes(&pl->adj_df, (size_t)std::max<int64_t>(N, 1) * 2 * sizeof(real)));
        FS_TRY(pl->alloc_bytes(&pl->adj_a, (size_t)std::max<int64_t>(M, 1) * sizeof(real)));
        FS_TRY(pl->alloc_bytes(&pl->adj_ga, (size_t)std::max<int64_t>(M, 1) * 2 * sizeof(real)));
        FS_TRY(pl->alloc_bytes(&pl->adj_cg, (size_t)std::max<int64_t>(M, 1) * sizeof(real)));
        FS_TRY(pl->alloc_bytes(&pl->adj_hess, (size_t)std::max<int64_t>(N, 1) * 3 * sizeof(real)));
        FS_TRY(pl->alloc(&pl->adj_gsum, 1));
        if (pl->precision == 32 && !pl->src_near_items)
            FS_TRY(build_near_items(pl, pl->src_start, pl->tgt_start, false, &pl->src_near_items,
                                    &pl->n_src_near_items));
    }
    const Window<real> w = make_window<real>(pl);
    const NearParams<real> np = make_near<real>(pl);
    const double shift = std::log(pl->s) / (2.0 * kPi);
    const size_t isz = in_dtype == FS_F64 ? 8 : 4, osz = out_dtype == FS_F64 ? 8 : 4;
    const size_t grid_bytes = (size_t)pl->n_a * pl->pitch * sizeof(real);
    for (int r = 0; r < pl->nrhs; ++r) {
        const real *q = (const real *)pl->q_sorted + (int64_t)r * M;
        const void *gp = g_phi ? (const unsigned char *)g_phi + (size_t)r * N * isz : nullptr;
        const void *gh = g_H ? (const unsigned char *)g_H + (size_t)r * N * 2 * isz : nullptr;
        // FP32 plans with a second stream run each near part beside the spreading and transform
        // it does not depend on (stored first; the interpolation adds the far part)
        const bool ovl = sizeof(real) == 4 && pl->aux != nullptr;
        if (dtgt) {
            // forward field and its Hessian at the targets (the grid is recomputed, not stored)
            if constexpr (sizeof(real) == 4) {
                if (ovl) {
                    FS_CUDA(cudaEventRecord(pl->ev_fork, st));
                    FS_CUDA(cudaStreamWaitEvent(pl->aux, pl->ev_fork, 0));
                    FS_CUDA(launch_near_hess32(pl->n_near_items, pl->near_items, pl->tgt_base, pl->tgt_pos32,
                                               pl->tgt_lo32, pl->src_pos32, pl->src_lo32, pl->src_start, pl->cg, q, np,
                                               (float *)pl->grad_s, (float *)pl->adj_hess, true, pl->aux));
                    FS_CUDA(cudaEventRecord(pl->ev_join, pl->aux));
                }
            }
            FS_TRY(spread_forward<real>(pl, q, w, st));
            FS_TRY(spectral_pipeline<real>(pl));
            if (ovl)
                FS_CUDA(cudaStreamWaitEvent(st, pl->ev_join, 0));
            FS_CUDA(launch_interp_hess<real>(N, pl->m, pl->tgt_base, pl->tgt_frac, w, pl->wpoly, (const real *)pl->grid,
                                             pl->pitch, (real)pl->n_os, (real *)pl->grad_s, (real *)pl->adj_hess, ovl,
                                             st));
            if constexpr (sizeof(real) == 4) {
                if (!ovl)
                    FS_CUDA(launch_near_hess32(pl->n_near_items, pl->near_items, pl->tgt_base, pl->tgt_pos32,
                                               pl->tgt_lo32, pl->src_pos32, pl->src_lo32, pl->src_start, pl->cg, q, np,
                                               (float *)pl->grad_s, (float *)pl->adj_hess, false, st));
            } else {
                FS_CUDA(launch_near_hess64(N, pl->tgt_base, pl->tgt_pos, pl->src_pos, pl->src_start, pl->cg, q, np,
                                           (double *)pl->grad_s, (double *)pl->adj_hess, st));
            }
        }
        FS_CUDA(cudaMemsetAsync(pl->adj_gsum, 0, sizeof(double), st));
        FS_CUDA(launch_gather_adj<real>(N, pl->tgt_perm, gp, gh, in_dtype == FS_F64, pl->s, (double)pl->n_os,
                                        (real *)pl->adj_c, pl->adj_dn, pl->adj_df, pl->adj_gsum, st));
        if (dq || dsrc) {
            if constexpr (sizeof(real) == 4) {
                if (ovl) {
                    FS_CUDA(cudaEventRecord(pl->ev_fork, st));   // the adjoint weights are in
                    FS_CUDA(cudaStreamWaitEvent(pl->aux, pl->ev_fork, 0));
                    FS_CUDA(launch_near_adj32(pl->n_src_near_items, pl->src_near_items, pl->src_base, pl->src_pos32,
                                              pl->src_lo32, pl->tgt_pos32, pl->tgt_lo32, pl->tgt_start, pl->cg,
                                              (const float *)pl->adj_c, pl->adj_dn, np, (float *)pl->adj_a,
                                              (float *)pl->adj_ga, (float *)pl->adj_cg, true, pl->aux));
                    FS_CUDA(cudaEventRecord(pl->ev_join, pl->aux));
                }
            }
            FS_CUDA(cudaMemsetAsync(pl->grid, 0, grid_bytes, st));
            FS_CUDA(launch_spread_dip<real>(pl->tgt_items, pl->n_tgt_items, pl->cg, pl->m, pl->tgt_base, pl->tgt_frac,
                                            (const real *)pl->adj_c, pl->adj_df, w, pl->wpoly, (real *)pl->grid,
                                            pl->pitch, pl->n_a, pl->kahan, st));
            FS_TRY(spectral_pipeline<real>(pl));
            if (ovl)
                FS_CUDA(cudaStreamWaitEvent(st, pl->ev_join, 0));
            FS_CUDA(launch_interp<real>(M, pl->m, pl->src_base, pl->src_frac, w, pl->wpoly, (const real *)pl->grid,
                                        pl->pitch, (real)pl->n_os, (real *)pl->adj_a, (real *)pl->adj_ga, ovl, st));
            if constexpr (sizeof(real) == 4) {
                if (!ovl)
                    FS_CUDA(launch_near_adj32(pl->n_src_near_items, pl->src_near_items, pl->src_base, pl->src_pos32,
                                              pl->src_lo32, pl->tgt_pos32, pl->tgt_lo32, pl->tgt_start, pl->cg,
                                              (const float *)pl->adj_c, pl->adj_dn, np, (float *)pl->adj_a,
                                              (float *)pl->adj_ga, (float *)pl->adj_cg, false, st));
            } else
                FS_CUDA(launch_near_adj64(M, pl->src_base, pl->src_pos, pl->tgt_pos, pl->tgt_start, pl->cg,
                                          (const double *)pl->adj_c, pl->adj_dn, np, (double *)pl->adj_a,
                                          (double *)pl->adj_ga, (double *)pl->adj_cg, st));
            void *o_dq = dq ? (unsigned char *)dq + (size_t)r * M * osz : nullptr;
            void *o_dy = dsrc ? (unsigned char *)dsrc + (size_t)r * M * 2 * osz : nullptr;
            FS_CUDA(launch_adj_finish_src<real>(M, pl->src_perm, (const real *)pl->adj_a, (const real *)pl->adj_ga,
                                                (const real *)pl->adj_cg, q, shift, pl->adj_gsum, pl->s, o_dq, o_dy,
                                                out_dtype == FS_F64, st));
        }
        if (dtgt) {
            void *o_dx = (unsigned char *)dtgt + (size_t)r * N * 2 * osz;
            FS_CUDA(launch_adj_finish_tgt<real>(N, pl->tgt_perm, (const real *)pl->grad_s,
                                                (const real *)pl->adj_hess, (const real *)pl->adj_c, pl->adj_dn, pl->s,
                                                o_dx, out_dtype == FS_F64, st));
        }
    }
    return FS_OK;
}

}  // namespace

// The device status word (read back after a synchronisation) as the API's status; a
// non-zero word is reset so that the next call starts clean.
static fs_status status_from_code(fs_plan *plan, int code)
{
    if (code == 0)
        return FS_OK;
    FS_CUDA(cudaMemset(plan->status, 0, sizeof(int)));
    if (code == kDevTimeout)
        return fail(FS_ETIMEOUT, "a bounded device wait gave up");
    return fail(FS_EDOMAIN, "a point fell outside the admissible region");
}

extern "C" {

const char *fs_last_error(void) { return g_last_error.c_str(); }

const char *fs_version(void) { return "femnfft-gb300 0.1 (sm_103a)"; }

fs_status fs_plan_create(const double *src_xy, int64_t M, const double *tgt_xy, int64_t N, int n_grid,
                         double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs_plan **out)
{
    g_last_error.clear();
    if (!out)
        return fail(FS_EINVAL, "out is null");
    *out = nullptr;
    if (M < 0 || N < 0 || M > (int64_t)INT32_MAX || N > (int64_t)INT32_MAX)
        return fail(FS_EINVAL, "M and N must be in [0, 2^31)");
    if ((M > 0 && !src_xy) || (N > 0 && !tgt_xy))
        return fail(FS_EINVAL, "null point array");
    fs_plan *pl = new (std::nothrow) fs_plan();
    if (!pl)
        return fail(FS_ENOMEM, "host allocation failed");
    fs_status st = plan_create_common(src_xy, M, tgt_xy, N, n_grid, sigma_os, m_window, eps_I, opts, pl);
    if (st != FS_OK) {
        const std::string msg = g_last_error;
        plan_destroy(pl);
        g_last_error = msg;
        return st;
    }
    *out = pl;
    return FS_OK;
}

fs_status fs_plan_create_fem(const double *nodes, int64_t Nv, const int32_t *tris, int64_t Nt, int n_grid,
                             double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs_plan **out)
{
    g_last_error.clear();
    if (!out)
        return fail(FS_EINVAL, "out is null");
    *out = nullptr;
    if (Nv <= 0 || Nt <= 0 || !nodes || !tris)
        return fail(FS_EINVAL, "a mesh needs nodes and triangles");
    if (Nv > (int64_t)INT32_MAX || 3 * Nt > (int64_t)INT32_MAX)
        return fail(FS_EINVAL, "mesh too large");
    if ((reinterpret_cast<uintptr_t>(nodes) & 15u) != 0)
        return fail(FS_EINVAL, "nodes must be 16-byte aligned (read as (x, y) pairs)");
    fs_opts o{};
    if (opts)
        o = *opts;
    fs_plan *pl = new (std::nothrow) fs_plan();
    if (!pl)
        return fail(FS_ENOMEM, "host allocation failed");
    auto body = [&]() -> fs_status {
        FS_TRY(validate_params(n_grid, sigma_os, m_window, eps_I, o));
        cudaStream_t st = (cudaStream_t)o.stream;
        std::vector<int> h_tris(3 * Nt), h_edges;
        FS_CUDA(cudaMemcpyAsync(h_tris.data(), tris, sizeof(int) * 3 * Nt, cudaMemcpyDeviceToHost, st));
        FS_CUDA(cudaStreamSynchronize(st));
        FS_TRY(boundary_edges(h_tris, Nt, Nv, h_edges));
        pl->is_fem = true;
        pl->Nv = Nv;
        pl->Nt = Nt;
        pl->Ne = (int64_t)h_edges.size() / 3;
        pl->nodes = (const double2 *)nodes;
        FS_TRY(pl->alloc(&pl->tris, 3 * Nt));
        FS_TRY(pl->alloc(&pl->bedges, std::max<size_t>(h_edges.size(), 1)));
        FS_CUDA(cudaMemcpyAsync(pl->tris, h_tris.data(), sizeof(int) * 3 * Nt, cudaMemcpyHostToDevice, st));
        if (!h_edges.empty())
            FS_CUDA(cudaMemcpyAsync(pl->bedges, h_edges.data(), sizeof(int) * h_edges.size(), cudaMemcpyHostToDevice,
                                    st));
        const int64_t Ms = 3 * Nt + 2 * pl->Ne;
        FS_TRY(pl->alloc(&pl->fem_src, Ms));
        FS_CUDA(launch_fem_sources((const double2 *)nodes, pl->tris, Nt, pl->bedges, pl->Ne, pl->fem_src, st));
        FS_TRY(pl->alloc(&pl->fem_tri_coef, std::max<int64_t>(3 * Nt, 1)));
        FS_CUDA(launch_fem_tri_coef((const double2 *)nodes, pl->tris, Nt, pl->fem_tri_coef, st));
        FS_CUDA(cudaStreamSynchronize(st));
        pl->precision = o.precision == 64 ? 64 : 32;
        if (pl->precision == 64)
            FS_TRY(plan_init<double>(pl, (const double *)pl->fem_src, Ms, nodes, Nv, n_grid, sigma_os, m_window,
                                     eps_I, o));
        else
            FS_TRY(plan_init<float>(pl, (const double *)pl->fem_src, Ms, nodes, Nv, n_grid, sigma_os, m_window,
                                    eps_I, o));
        // source index -> sorted index: the assembly writes each element's charges into cell order
        FS_TRY(pl->alloc(&pl->src_inv_perm, Ms));
        FS_CUDA(launch_invert_perm(pl->src_perm, Ms, pl->src_inv_perm, pl->stream));
        FS_CUDA(cudaStreamSynchronize(pl->stream));
        return FS_OK;
    };
    fs_status st = body();
    if (st != FS_OK) {
        const std::string msg = g_last_error;
        plan_destroy(pl);
        g_last_error = msg;
        return st;
    }
    *out = pl;
    return FS_OK;
}

fs_status fs_set_charges(fs_plan *plan, const void *q, fs_dtype dtype, int nrhs)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    FS_TRY(check_dtype(dtype));
    if (nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "nrhs must be in [1, 65535]");
    if (!q && plan->M > 0)
        return fail(FS_EINVAL, "null charges");
    if (plan->precision == 64)
        return set_charges_t<double>(plan, q, dtype, nrhs);
    return set_charges_t<float>(plan, q, dtype, nrhs);
}

fs_status fs_fem_charges(fs_plan *plan, const double *mag, double *q_out, int nrhs)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!mag || !q_out || nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "bad magnetisation/charge arguments");
    if ((reinterpret_cast<uintptr_t>(mag) & 15u) != 0)
        return fail(FS_EINVAL, "magnetisation must be 16-byte aligned (read as (Mx, My) pairs)");
    FS_CUDA(launch_fem_charges(plan->nodes, plan->tris, plan->Nt, plan->bedges, plan->Ne, (const double2 *)mag,
                               plan->Nv, nrhs, q_out, plan->M, plan->stream));
    return FS_OK;
}

fs_status fs_set_magnetization(fs_plan *plan, const double *mag, int nrhs)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!mag || nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "bad magnetisation arguments");
    if ((reinterpret_cast<uintptr_t>(mag) & 15u) != 0)
        return fail(FS_EINVAL, "magnetisation must be 16-byte aligned (read as (Mx, My) pairs)");
    // assembly fused with the gather: each element's charges go straight into cell order
    cudaStream_t st = plan->stream;
    if (plan->precision == 64)
        FS_TRY(reserve_charges<double>(plan, nrhs));
    else
        FS_TRY(reserve_charges<float>(plan, nrhs));
    plan->nrhs = nrhs;
    if (plan->events)
        FS_CUDA(cudaEventRecord(plan->ev_q0, st));
    FS_CUDA(cudaMemsetAsync(plan->q_sum, 0, sizeof(double) * nrhs, st));
    if (plan->precision == 64)
        FS_CUDA(launch_fem_charges_scatter<double>(plan->nodes, plan->tris, plan->Nt, plan->fem_tri_coef, plan->bedges,
                                                   plan->Ne,
                                                   (const double2 *)mag, plan->Nv, nrhs, plan->src_inv_perm, plan->M,
                                                   (double *)plan->q_sorted, plan->q_sum, st));
    else
        FS_CUDA(launch_fem_charges_scatter<float>(plan->nodes, plan->tris, plan->Nt, plan->fem_tri_coef, plan->bedges,
                                                  plan->Ne,
                                                  (const double2 *)mag, plan->Nv, nrhs, plan->src_inv_perm, plan->M,
                                                  (float *)plan->q_sorted, plan->q_sum, st));
    if (plan->events)
        FS_CUDA(cudaEventRecord(plan->ev_q1, st));
    return FS_OK;
}

fs_status fs_fem_sources(fs_plan *plan, double *src_out)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!src_out)
        return fail(FS_EINVAL, "null output");
    FS_CUDA(cudaMemcpyAsync(src_out, plan->fem_src, sizeof(double2) * plan->M, cudaMemcpyDeviceToDevice,
                            plan->stream));
    return FS_OK;
}

fs_status fs_eval_field(fs_plan *plan, void *phi, void *H, fs_dtype dtype)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    FS_TRY(check_dtype(dtype));
    if (plan->nrhs < 1)
        return fail(FS_EINVAL, "charges not set");
    if (plan->N > 0 && !phi && !H)
        return fail(FS_EINVAL, "no output requested");
    if (plan->precision == 64)
        return eval_t<double>(plan, phi, H, dtype);
    return eval_t<float>(plan, phi, H, dtype);
}

fs_status fs_eval_potential(fs_plan *plan, void *phi, fs_dtype dtype)
{
    if (!phi && plan && plan->N > 0)
        return fail(FS_EINVAL, "null phi");
    return fs_eval_field(plan, phi, nullptr, dtype);
}

fs_status fs_solve_host(fs_plan *plan, const void *q, fs_dtype q_dtype, int nrhs, void *phi, void *H,
                        fs_dtype out_dtype)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    FS_TRY(check_dtype(q_dtype));
    FS_TRY(check_dtype(out_dtype));
    if (nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "nrhs must be in [1, 65535]");
    if ((!q && plan->M > 0) || (!H && plan->N > 0))
        return fail(FS_EINVAL, "null host buffer");
    cudaStream_t st = plan->stream;
    const size_t qb = (size_t)nrhs * plan->M * (q_dtype == FS_F64 ? 8 : 4);
    const size_t ob = (size_t)nrhs * plan->N * (out_dtype == FS_F64 ? 8 : 4);
    if (qb > plan->q_stage_bytes) {
        plan->release(plan->d_q_stage);
        FS_TRY(plan->alloc_bytes(&plan->d_q_stage, qb));
        plan->q_stage_bytes = qb;
    }
    if (ob > plan->phi_stage_bytes) {
        plan->release(plan->d_phi_stage);
        FS_TRY(plan->alloc_bytes(&plan->d_phi_stage, ob));
        plan->phi_stage_bytes = ob;
    }
    if (2 * ob > plan->H_stage_bytes) {
        plan->release(plan->d_H_stage);
        FS_TRY(plan->alloc_bytes(&plan->d_H_stage, 2 * ob));
        plan->H_stage_bytes = 2 * ob;
    }
    if (qb)
        FS_CUDA(cudaMemcpyAsync(plan->d_q_stage, q, qb, cudaMemcpyHostToDevice, st));
    FS_TRY(fs_set_charges(plan, plan->d_q_stage, q_dtype, nrhs));
    FS_TRY(fs_eval_field(plan, phi ? plan->d_phi_stage : nullptr, plan->d_H_stage, out_dtype));
    if (phi && ob)
        FS_CUDA(cudaMemcpyAsync(phi, plan->d_phi_stage, ob, cudaMemcpyDeviceToHost, st));
    if (ob)
        FS_CUDA(cudaMemcpyAsync(H, plan->d_H_stage, 2 * ob, cudaMemcpyDeviceToHost, st));
    // the device status word comes back with the outputs: one synchronisation per call
    if (!plan->status_host)
        FS_CUDA(cudaMallocHost(&plan->status_host, sizeof(int)));
    FS_CUDA(cudaMemcpyAsync(plan->status_host, plan->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    return status_from_code(plan, *plan->status_host);
}

fs_status fs_adjoint(fs_plan *plan, const void *g_phi, const void *g_H, fs_dtype in_dtype, void *dq, void *dsrc,
                     void *dtgt, fs_dtype out_dtype)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    FS_TRY(check_dtype(in_dtype));
    FS_TRY(check_dtype(out_dtype));
    if (plan->nrhs < 1)
        return fail(FS_EINVAL, "charges not set");
    if (!dq && !dsrc && !dtgt)
        return fail(FS_EINVAL, "no gradient requested");
    if (plan->precision == 64)
        return adjoint_t<double>(plan, g_phi, g_H, in_dtype, dq, dsrc, dtgt, out_dtype);
    return adjoint_t<float>(plan, g_phi, g_H, in_dtype, dq, dsrc, dtgt, out_dtype);
}

fs_status fs_sync_status(fs_plan *plan)
{
    FS_TRY(check_plan(plan));
    FS_CUDA(cudaStreamSynchronize(plan->stream));
    int code = 0;
    FS_CUDA(cudaMemcpy(&code, plan->status, sizeof(int), cudaMemcpyDeviceToHost));
    return status_from_code(plan, code);
}

fs_status fs_plan_info(const fs_plan *plan, fs_info *info)
{
    FS_TRY(check_plan(plan));
    if (!info)
        return fail(FS_EINVAL, "null info");
    std::memset(info, 0, sizeof(*info));
    info->n_src = plan->M;
    info->n_tgt = plan->N;
    info->n_grid = plan->n;
    info->n_os = plan->n_os;
    info->m = plan->m;
    info->p = plan->p;
    info->precision = plan->precision;
    info->eps_I = plan->eps_I;
    info->eps_B = plan->eps_B;
    info->scale = plan->s;
    info->window_lo = plan->window_lo;
    info->window_n = plan->n_a;
    info->cell = plan->cg.cell;
    info->cells_per_dim = plan->cg.n_c;
    info->tile_cells = plan->cg.T;
    info->spread_items = plan->n_items;
    info->near_pairs = plan->near_pairs;
    info->near_pairs_fp64 = plan->near_pairs_fp64;
    info->workspace_bytes = plan->bytes;
    info->is_fem = plan->is_fem;
    info->n_nodes = plan->Nv;
    info->n_tris = plan->Nt;
    info->n_bedges = plan->Ne;
    info->spread_direct = plan->spread_direct ? 1 : 0;
    return FS_OK;
}

fs_status fs_stage_times(fs_plan *plan, double *ms, int count)
{
    FS_TRY(check_plan(plan));
    if (!plan->events)
        return fail(FS_EINVAL, "plan created without FS_FLAG_TIMING");
    if (!ms || count < kStages)
        return fail(FS_EINVAL, "need room for 8 stage times");
    FS_CUDA(cudaStreamSynchronize(plan->stream));
    float t = 0.f;
    FS_CUDA(cudaEventElapsedTime(&t, plan->ev_q0, plan->ev_q1));
    ms[0] = t;
    for (int i = 1; i < kStages; ++i) {
        FS_CUDA(cudaEventElapsedTime(&t, plan->ev[i - 1], plan->ev[i]));
        ms[i] = t;
    }
    if (plan->overlap) {
        // interpolation from the join; the near field on its own stream (overlapping stages 1-4)
        FS_CUDA(cudaEventElapsedTime(&t, plan->ev_j, plan->ev[5]));
        ms[5] = t;
        FS_CUDA(cudaEventElapsedTime(&t, plan->ev_n0, plan->ev_n1));
        ms[6] = t;
    }
    return FS_OK;
}

fs_status fs_plan_destroy(fs_plan *plan)
{
    if (!plan)
        return FS_OK;
    plan_destroy(plan);
    return FS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of fs_set_magnetization.
//
// The intermediate FEM charges live in this file-scope device array instead of memory the
// plan allocates.  Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol), so the address is looked up with cudaGetSymbolAddress, with the
// device current, and passed to the kernels.  The lookup is cached per device and keyed on the
// unique id of the device's current CUDA context: after cudaDeviceReset, or under another
// context, the module is loaded again at another address, and the id differs, so the address
// is looked up again instead of reusing a stale one.

namespace {

constexpr int64_t kStaticFemCharges = int64_t(1) << 19;   // doubles (4 MiB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_fem_charge_scratch[kStaticFemCharges];

struct ScratchEntry {
    unsigned long long ctx_id;
    double *addr;
};
std::mutex g_scratch_mutex;
ScratchEntry g_scratch[kMaxDevices] = {};

// Unique id of the calling thread's current context (false when none is current yet).  The
// driver calls are reached through the runtime's entry-point table, so the library does not
// link the driver library itself.
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa{}, qb{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return false;
        get_current = reinterpret_cast<GetCurrent>(a);
        get_id = reinterpret_cast<GetId>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx)
        return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

fs_status static_scratch_address(double **out)
{
    int dev = 0;
    FS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(FS_EUNSUPPORTED, "device index beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (!have_id || !g_scratch[dev].addr || g_scratch[dev].ctx_id != id) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_fem_charge_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(FS_ECUDA, std::string("cudaGetSymbolAddress of the static charge scratch failed: ") +
                                      cudaGetErrorString(e));
        // the lookup made the device's primary context current if none was
        if (!current_context_id(&id))
            return fail(FS_ECUDA, "no current CUDA context after the static scratch lookup");
        g_scratch[dev] = ScratchEntry{id, static_cast<double *>(ptr)};
    }
    *out = g_scratch[dev].addr;
    return FS_OK;
}

template <typename real> fs_status gather_static_charges(fs_plan *pl, const double *q, int nrhs)
{
    cudaStream_t st = pl->stream;
    pl->nrhs = nrhs;
    if (pl->events)
        FS_CUDA(cudaEventRecord(pl->ev_q0, st));
    FS_CUDA(cudaMemsetAsync(pl->q_sum, 0, sizeof(double) * nrhs, st));
    FS_CUDA(launch_gather_charges<real>(q, 1, pl->src_perm, pl->M, nrhs, (real *)pl->q_sorted, pl->q_sum, st));
    if (pl->events)
        FS_CUDA(cudaEventRecord(pl->ev_q1, st));
    return FS_OK;
}

}  // namespace

extern "C" fs_status fs_set_magnetization_static(fs_plan *plan, const double *mag, int nrhs)
{
    g_last_error.clear();
    FS_TRY(check_plan(plan));
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!mag || nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "bad magnetisation arguments");
    if ((reinterpret_cast<uintptr_t>(mag) & 15u) != 0)
        return fail(FS_EINVAL, "magnetisation must be 16-byte aligned (read as (Mx, My) pairs)");
    if ((int64_t)nrhs * plan->M > kStaticFemCharges)
        return fail(FS_EINVAL, "nrhs * n_src = " + std::to_string((int64_t)nrhs * plan->M) +
                                   " exceeds the static scratch limit of 524288 charges");
    if (nrhs > plan->nrhs_cap)
        return fail(FS_EINVAL, "charge storage for " + std::to_string(nrhs) +
                                   " vectors is not reserved: call fs_set_charges or fs_set_magnetization "
                                   "once with at least that many vectors first");
    int dev = 0;
    FS_CUDA(cudaGetDevice(&dev));
    if (dev != plan->device)
        return fail(FS_EINVAL, "the plan's device is not the current device");
    double *scratch = nullptr;
    FS_TRY(static_scratch_address(&scratch));
    FS_CUDA(launch_fem_charges(plan->nodes, plan->tris, plan->Nt, plan->bedges, plan->Ne, (const double2 *)mag,
                               plan->Nv, nrhs, scratch, plan->M, plan->stream));
    if (plan->precision == 64)
        return gather_static_charges<double>(plan, scratch, nrhs);
    return gather_static_charges<float>(plan, scratch, nrhs);
}
