// C ABI of the fast summation for the 3D kernel G(r) = 1/(4 pi r) (host side).
//
// The paper's stated next step: the same pipeline with d = 3.  The plan scales the points
// into the ball of radius 1/4 - eps_B/2 of the torus cube, bins them into cells at least
// eps_I wide, computes the FP64 coefficients b_l of the kernel regularised by T_I (near the
// origin) and T_B (near the cube's inscribed sphere) on the device, and keeps the multiplier
// V(l) b_l / (c(l1) c(l2) c(l3))^2 for l1 in [0, n/2], l2, l3 in [-n/2, n/2].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "plan.h"

using namespace fs;

struct fs3_plan {
    int precision = 32;
    int n = 0, n_os = 0, m = 0, p = 0;
    double sigma = 0, eps_I = 0, eps_B = 0, s = 1.0;
    int64_t M = 0, N = 0;
    int window_lo = 0, n_a = 0;
    CellGrid3 cg{};
    cudaStream_t stream = nullptr;
    KernelParams kp{};
    WindowPoly wpoly{};
    std::vector<void *> allocs;
    int64_t bytes = 0;
    int *status = nullptr;
    int *src_perm = nullptr, *tgt_perm = nullptr, *src_base = nullptr, *tgt_base = nullptr;
    int *src_start = nullptr, *tgt_start = nullptr;
    void *src_frac = nullptr, *tgt_frac = nullptr;
    double *src_pos = nullptr, *tgt_pos = nullptr;
    float4 *src_p32 = nullptr, *tgt_p32 = nullptr;
    void *mul = nullptr, *tw = nullptr;
    void *grid = nullptr, *spec1 = nullptr, *spec2 = nullptr;
    void *phi_s = nullptr, *grad_s = nullptr;
    void *q_sorted = nullptr;
    double *q_sum = nullptr;
    int nrhs = 0, nrhs_cap = 0;
    // FP32 near field: warp items and the coincident-source lists of the targets
    int2 *near_items = nullptr;
    int n_near_items = 0;
    // FP32 spreading through warp-private shared tiles: items of at most kSpread3ItemMax sources
    // of one cell (plans whose tiles fit in shared memory)
    bool spread_tiles = false;
    int2 *spread_items = nullptr;
    int n_spread_items = 0;
    // source-major near field (many more sources than targets): items over the sources
    bool src_major = false;
    int2 *src_items = nullptr;
    int n_src_items = 0;
    int n_coinc = 0;
    // FP32: the near field on a second stream beside spreading and the transform
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int *coinc_start = nullptr, *coinc_src = nullptr;
    // tetrahedral FEM plans: sources are the quadrature points, targets the nodes
    bool is_fem = false;
    int64_t Nv = 0, Nt = 0, Nf = 0;
    int *src_inv_perm = nullptr;      // source index -> sorted index (charges assembled into cell order)
    const double *nodes = nullptr;
    int *tets = nullptr, *faces = nullptr;
    double *fem_tet_coef = nullptr;       // per tetrahedron: 9 charge coefficients (k_fem3_tet_coef)
    double *fem_src = nullptr;

    template <typename T> fs_status alloc(T **out, size_t count)
    {
        *out = nullptr;
        const size_t nbytes = std::max<size_t>(count, 1) * sizeof(T);
        void *ptr = nullptr;
        cudaError_t e = cudaMalloc(&ptr, nbytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FS_ENOMEM, "cudaMalloc of " + std::to_string(nbytes) + " bytes failed: " +
                                       cudaGetErrorString(e));
        }
        allocs.push_back(ptr);
        bytes += (int64_t)nbytes;
        *out = static_cast<T *>(ptr);
        return FS_OK;
    }
    void release(void *ptr)
    {
        auto it = std::find(allocs.begin(), allocs.end(), ptr);
        if (ptr && it != allocs.end()) {
            cudaFree(ptr);
            allocs.erase(it);
        }
    }
};

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// T_I(r) = sum_k beta_k (r/eps)^(2k) with T_I^(j)(eps) = k^(j)(eps), k = 1/(4 pi r), j < p
// (the scaled system eps^j d^j/dr^j: sum_k beta_k (2k)_j = eps^j k^(j)(eps) = (-1)^j j! / (4 pi eps)).
bool near_coefficients3(double eps, int p, double *beta)
{
    std::vector<double> a(p * p, 0.0), rhs(p, 0.0);
    double fact = 1.0;
    for (int j = 0; j < p; ++j) {
        if (j > 0)
            fact *= j;
        for (int k = 0; k < p; ++k) {
            const int e = 2 * k;
            if (e < j)
                continue;
            double f = 1.0;
            for (int t = 0; t < j; ++t)
                f *= (double)(e - t);
            a[j * p + k] = f;
        }
        rhs[j] = ((j % 2 == 0) ? 1.0 : -1.0) * fact / (4.0 * kPi * eps);
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
            for (int c = col; c < p; ++c)
                a[r * p + c] -= f * a[col * p + c];
            rhs[r] -= f * rhs[col];
        }
    }
    for (int r = p - 1; r >= 0; --r) {
        double v = rhs[r];
        for (int c = r + 1; c < p; ++c)
            v -= a[r * p + c] * beta[c];
        beta[r] = v / a[r * p + r];
    }
    return true;
}

template <typename real> fs_status twiddles3(fs3_plan *pl, int L, void **out)
{
    std::vector<real> h(2 * (size_t)L);
    fft_twiddle_table<real>(L, h.data());
    real *d = nullptr;
    FS_TRY(pl->alloc(&d, h.size()));
    FS_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice));
    *out = d;
    return FS_OK;
}

fs_status near_setup3(fs3_plan *pl);

template <typename real> NearParams<real> make_near3(const fs3_plan *pl)
{
    NearParams<real> np{};
    np.p = pl->p;
    np.eps2 = (real)(pl->eps_I * pl->eps_I);
    np.inv_eps2 = (real)(1.0 / (pl->eps_I * pl->eps_I));
    for (int k = 0; k < pl->p; ++k)
        np.beta[k] = (real)pl->kp.beta[k];
    for (int k = 1; k < pl->p; ++k)
        np.dbeta[k - 1] = (real)(2.0 * k * pl->kp.beta[k] / (pl->eps_I * pl->eps_I));
    return np;
}

template <typename real>
fs_status bin3(fs3_plan *pl, const double *xyz, int64_t n, int **perm, int **base, void **frac, double **pos,
               float4 **p32, int **start)
{
    cudaStream_t st = pl->stream;
    const int n_keys = pl->cg.n_keys();
    FS_TRY(pl->alloc(perm, n));
    FS_TRY(pl->alloc(base, n));
    real *fr = nullptr;
    FS_TRY(pl->alloc(&fr, 3 * (size_t)std::max<int64_t>(n, 1)));
    *frac = fr;
    FS_TRY(pl->alloc(pos, 3 * (size_t)std::max<int64_t>(n, 1)));
    *p32 = nullptr;
    if (pl->precision == 32)
        FS_TRY(pl->alloc(p32, n));
    FS_TRY(pl->alloc(start, (size_t)n_keys + 1));
    int *key = nullptr, *count = nullptr, *fill = nullptr, *tmp = nullptr;
    FS_TRY(pl->alloc(&key, n));
    FS_TRY(pl->alloc(&count, n_keys));
    FS_TRY(pl->alloc(&fill, (size_t)n_keys + 1));
    FS_TRY(pl->alloc(&tmp, (size_t)n_keys / 4096 + 2));
    FS_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * n_keys, st));
    FS_CUDA(cudaMemsetAsync(*start, 0, sizeof(int) * ((size_t)n_keys + 1), st));
    FS_CUDA(launch_point_keys3(xyz, n, pl->s, pl->n_os, pl->window_lo, pl->n_a, pl->m, pl->cg, key, count, pl->status,
                               st));
    FS_CUDA(launch_exclusive_scan(count, *start, n_keys, tmp, st));
    FS_CUDA(cudaMemcpyAsync(fill, *start, sizeof(int) * ((size_t)n_keys + 1), cudaMemcpyDeviceToDevice, st));
    FS_CUDA(launch_scatter(key, n, fill, *perm, st));
    FS_CUDA(launch_gather_points3<real>(xyz, *perm, n, pl->s, pl->n_os, pl->window_lo, pl->n_a, pl->m, pl->cg.cell,
                                        1.0 / pl->eps_I, *pos, fr, *base, *p32, pl->status, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->release(key);
    pl->release(count);
    pl->release(fill);
    pl->release(tmp);
    return FS_OK;
}

template <typename real>
fs_status plan3_init(fs3_plan *pl, const double *src, int64_t M, const double *tgt, int64_t N)
{
    using C = typename Cplx<real>::type;
    cudaStream_t st = pl->stream;
    const int n = pl->n, L = pl->n_os, m = pl->m;
    // torus scale
    unsigned long long *d_r = nullptr;
    FS_TRY(pl->alloc(&d_r, 1));
    FS_CUDA(cudaMemsetAsync(d_r, 0, sizeof(unsigned long long), st));
    FS_CUDA(launch_rmax3(src, M, d_r, st));
    FS_CUDA(launch_rmax3(tgt, N, d_r, st));
    unsigned long long bits = 0;
    FS_CUDA(cudaMemcpyAsync(&bits, d_r, sizeof(bits), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->release(d_r);
    double r2max;
    std::memcpy(&r2max, &bits, sizeof(double));
    if (!std::isfinite(r2max))
        return fail(FS_EINVAL, "non-finite point coordinates");
    const double rmax = std::sqrt(r2max);
    pl->s = rmax > 0.0 ? (0.25 - 0.5 * pl->eps_B) / rmax : 1.0;
    // active window and cells
    pl->window_lo = (int)std::floor(L * (0.25 + 0.5 * pl->eps_B)) - m - 1;
    const int hi = (int)std::floor(L * (0.75 - 0.5 * pl->eps_B)) + 1;
    int n_a = hi - pl->window_lo + m + 1;
    n_a = (n_a + 3) & ~3;
    if (n_a > L || n_a > 1023)
        return fail(FS_EINVAL, "window half-width too large for this grid (active window exceeds n_os)");
    pl->n_a = n_a;
    pl->cg.cell = std::max(1, (int)std::ceil(pl->eps_I * L - 1e-9));
    pl->cg.n_c = (n_a + pl->cg.cell - 1) / pl->cg.cell;
    // sub-cells (FP32 near field: compact warp items) while the sort keys stay below 2^24
    pl->cg.sub = 1;
    if (pl->precision == 32)
        for (int sub : {4, 2})
            if ((int64_t)pl->cg.n_c * pl->cg.n_c * pl->cg.n_c * sub * sub * sub <= (int64_t)1 << 24) {
                pl->cg.sub = sub;
                break;
            }
    if ((int64_t)pl->cg.n_c * pl->cg.n_c * pl->cg.n_c * pl->cg.sub3() > (int64_t)1 << 24)
        return fail(FS_EINVAL, "too many near-field cells (eps_I too small for this grid)");
    FS_TRY(pl->alloc(&pl->status, 1));
    FS_CUDA(cudaMemset(pl->status, 0, sizeof(int)));
    FS_TRY(bin3<real>(pl, src, M, &pl->src_perm, &pl->src_base, &pl->src_frac, &pl->src_pos, &pl->src_p32,
                      &pl->src_start));
    FS_TRY(bin3<real>(pl, tgt, N, &pl->tgt_perm, &pl->tgt_base, &pl->tgt_frac, &pl->tgt_pos, &pl->tgt_p32,
                      &pl->tgt_start));
    int dev_status = 0;
    FS_CUDA(cudaMemcpy(&dev_status, pl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_status != 0)
        return fail(FS_EDOMAIN, "a point fell outside the admissible radius after scaling");
    if (pl->precision == 32)
        FS_TRY(near_setup3(pl));
    // kernel regularisation (FP64): T_I and the boundary form's data at 1/2 - eps_B
    KernelParams &kp = pl->kp;
    kp.eps_I = pl->eps_I;
    kp.eps_B = pl->eps_B;
    kp.p = pl->p;
    kp.dim = 3;
    if (!near_coefficients3(pl->eps_I, pl->p, kp.beta))
        return fail(FS_EINVAL, "singular system for the inner smoothing polynomial");
    {
        const double r0 = 0.5 - pl->eps_B;
        double fact = 1.0;
        for (int j = 0; j < pl->p; ++j) {
            if (j > 0)
                fact *= j;
            // eps_B^j k^(j)(r0) / j!,  k^(j)(r) = (-1)^j j! / (4 pi r^(j+1))
            kp.tb_f0[j] = std::pow(pl->eps_B, j) * ((j % 2 == 0) ? 1.0 : -1.0) / (4.0 * kPi * std::pow(r0, j + 1));
            double cbin = 1.0;
            for (int t = 1; t <= j; ++t)
                cbin = cbin * (double)(pl->p - 1 + t) / (double)t;
            kp.tb_binom[j] = cbin;
        }
        (void)fact;
        kp.k_half = 1.0 / (4.0 * kPi * 0.5);
    }
    build_window_poly(pl->sigma, m, &pl->wpoly);
    // coefficients b_l and the multiplier
    {
        double2 *samp = nullptr, *tmp = nullptr;
        double *c_tab = nullptr;
        void *tw64 = nullptr;
        FS_TRY(pl->alloc(&samp, (size_t)n * n * n));
        FS_TRY(pl->alloc(&tmp, (size_t)n * n * n));
        FS_TRY(twiddles3<double>(pl, n, &tw64));
        const double b = kPi * (2.0 - 1.0 / pl->sigma);
        std::vector<double> c(n / 2 + 1);
        for (int l = 0; l <= n / 2; ++l) {
            const double arg = b * b - std::pow(2.0 * kPi * l / L, 2);
            c[l] = bessel_i0(m * std::sqrt(arg)) * kPi * m / std::sinh(b * m);
        }
        FS_TRY(pl->alloc(&c_tab, c.size()));
        FS_CUDA(cudaMemcpy(c_tab, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice));
        real *mul = nullptr;
        FS_TRY(pl->alloc(&mul, (size_t)(n / 2 + 1) * (n + 1) * (n + 1)));
        pl->mul = mul;
        FS_CUDA(launch_coeffs3(samp, tmp, n, kp, (const double2 *)tw64, c_tab, mul, sizeof(real) == 8, st));
        FS_CUDA(cudaStreamSynchronize(st));
        pl->release(samp);
        pl->release(tmp);
        pl->release(tw64);
        pl->release(c_tab);
    }
    FS_TRY(twiddles3<real>(pl, L, &pl->tw));
    // grids and per-target intermediates
    const size_t cube = (size_t)n_a * n_a * n_a;
    real *g = nullptr;
    C *s1 = nullptr, *s2 = nullptr;
    FS_TRY(pl->alloc(&g, cube));
    FS_TRY(pl->alloc(&s1, (size_t)n_a * (n / 2 + 1) * n_a));
    FS_TRY(pl->alloc(&s2, (size_t)n_a * (n / 2 + 1) * (n + 1)));
    pl->grid = g;
    pl->spec1 = s1;
    pl->spec2 = s2;
    real *ph = nullptr, *gr = nullptr;
    FS_TRY(pl->alloc(&ph, (size_t)std::max<int64_t>(N, 1)));
    FS_TRY(pl->alloc(&gr, 3 * (size_t)std::max<int64_t>(N, 1)));
    pl->phi_s = ph;
    pl->grad_s = gr;
    return FS_OK;
}

// FP32 near field: warp items (at most 64 consecutive targets of one cell, split evenly) and,
// per target, the sources at exactly the same FP32 offsets (coincident pairs).
fs_status near_setup3(fs3_plan *pl)
{
    cudaStream_t st = pl->stream;
    if (pl->N > ((int64_t)1 << 24))
        return fail(FS_EINVAL, "FP32 3D plans take at most 2^24 targets");
    const int n_cells = pl->cg.n_cells(), S3 = pl->cg.sub3();
    // the sorted points of each cell, split evenly into pieces of at most 64
    auto make_items = [&](const int *dev_start, int2 **out, int *n_out) -> fs_status {
        std::vector<int> start((size_t)pl->cg.n_keys() + 1);
        FS_CUDA(cudaMemcpyAsync(start.data(), dev_start, sizeof(int) * start.size(), cudaMemcpyDeviceToHost, st));
        FS_CUDA(cudaStreamSynchronize(st));
        std::vector<int2> items;
        for (int c = 0; c < n_cells; ++c) {
            const int a = start[(size_t)c * S3], b = start[(size_t)(c + 1) * S3];
            const int cnt = b - a;
            if (cnt <= 0)
                continue;
            const int pieces = (cnt + 63) / 64;
            for (int k = 0; k < pieces; ++k) {
                const int lo = a + (int)((int64_t)cnt * k / pieces), hi = a + (int)((int64_t)cnt * (k + 1) / pieces);
                items.push_back(make_int2(lo, hi - lo));
            }
        }
        *n_out = (int)items.size();
        FS_TRY(pl->alloc(out, items.size()));
        if (!items.empty())
            FS_CUDA(cudaMemcpyAsync(*out, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st));
        return FS_OK;
    };
    // spreading items: the sources of each cell in pieces of at most kSpread3ItemMax, where
    // the tiles fit in shared memory and the occupied cells are dense enough to pay for them
    std::vector<int> sstart;
    if (spread3_tile_smem(pl->cg.cell, pl->m) > 0 && pl->M > 0) {
        sstart.resize((size_t)pl->cg.n_keys() + 1);
        FS_CUDA(cudaMemcpyAsync(sstart.data(), pl->src_start, sizeof(int) * sstart.size(), cudaMemcpyDeviceToHost,
                                st));
        FS_CUDA(cudaStreamSynchronize(st));
        int64_t occupied = 0;
        for (int c = 0; c < n_cells; ++c)
            occupied += sstart[(size_t)(c + 1) * S3] > sstart[(size_t)c * S3];
        pl->spread_tiles = pl->M >= (int64_t)kSpread3TileMinPerCell * occupied;
    }
    if (pl->spread_tiles) {
        std::vector<int2> sitems;
        for (int c = 0; c < n_cells; ++c) {
            const int a = sstart[(size_t)c * S3], b = sstart[(size_t)(c + 1) * S3];
            for (int lo = a; lo < b; lo += kSpread3ItemMax)
                sitems.push_back(make_int2(lo, std::min(kSpread3ItemMax, b - lo)));
        }
        pl->n_spread_items = (int)sitems.size();
        FS_TRY(pl->alloc(&pl->spread_items, sitems.size()));
        if (!sitems.empty())
            FS_CUDA(cudaMemcpyAsync(pl->spread_items, sitems.data(), sizeof(int2) * sitems.size(),
                                    cudaMemcpyHostToDevice, st));
    }
    // targets much sparser than sources (FEM meshes): near-field items over the sources
    // instead, whose boxes stay small where a cell's few targets would span the whole cell
    pl->src_major = pl->N > 0 && pl->M >= 3 * pl->N;
    if (pl->N > 0) {
        FS_CUDA(cudaStreamCreateWithFlags(&pl->aux, cudaStreamNonBlocking));
        FS_CUDA(cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming));
        FS_CUDA(cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming));
    }
    if (pl->src_major)
        FS_TRY(make_items(pl->src_start, &pl->src_items, &pl->n_src_items));
    else
        FS_TRY(make_items(pl->tgt_start, &pl->near_items, &pl->n_near_items));
    // coincident sources: count, scan, fill
    const int64_t N = pl->N;
    int *count = nullptr, *tmp = nullptr;
    FS_TRY(pl->alloc(&count, (size_t)std::max<int64_t>(N, 1)));
    FS_TRY(pl->alloc(&pl->coinc_start, (size_t)N + 1));
    FS_TRY(pl->alloc(&tmp, (size_t)N / 4096 + 2));
    FS_CUDA(cudaMemsetAsync(pl->coinc_start, 0, sizeof(int) * ((size_t)N + 1), st));
    FS_CUDA(launch_coincident3(N, pl->tgt_base, pl->tgt_pos, pl->src_pos, pl->src_start, pl->cg, count, nullptr,
                               nullptr, st));
    if (N > 0)
        FS_CUDA(launch_exclusive_scan(count, pl->coinc_start, (int)N, tmp, st));
    int total = 0;
    FS_CUDA(cudaMemcpyAsync(&total, pl->coinc_start + N, sizeof(int), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->n_coinc = total;
    FS_TRY(pl->alloc(&pl->coinc_src, (size_t)std::max(total, 1)));
    if (total > 0)
        FS_CUDA(launch_coincident3(N, pl->tgt_base, pl->tgt_pos, pl->src_pos, pl->src_start, pl->cg, nullptr,
                                   pl->coinc_start, pl->coinc_src, st));
    FS_CUDA(cudaStreamSynchronize(st));
    pl->release(count);
    pl->release(tmp);
    return FS_OK;
}

Near3Params make_near3_f32(const fs3_plan *pl)
{
    Near3Params np{};
    const double eps = pl->eps_I;
    np.p = pl->p;
    np.H = (float)((double)pl->cg.cell / pl->n_os / eps);
    np.reach2 = (float)((1.0 + 2e-4) * (1.0 + 2e-4));
    np.close_reach2 = (float)((0.125 + 2e-4) * (0.125 + 2e-4));
    np.inv_eps_d = 1.0 / eps;
    np.c1 = (float)(1.0 / (4.0 * kPi * eps));
    np.inv_eps = (float)(1.0 / eps);
    np.beta0 = (float)pl->kp.beta[0];
    for (int k = 0; k < pl->p; ++k)
        np.nbeta[k] = (float)(-pl->kp.beta[k]);
    for (int k = 0; k + 1 < pl->p; ++k)
        np.dbeta2[k] = (float)(2.0 * (k + 1) * pl->kp.beta[k + 1]);
    return np;
}

// Boundary faces (used by one tetrahedron) as (i0 < i1 < i2, fourth node), sorted by the triple.
fs_status boundary_faces3(const std::vector<int> &tets, int64_t Nt, int64_t Nv, std::vector<int> &out)
{
    struct F {
        int a, b, c, opp;
    };
    std::vector<F> f;
    f.reserve(4 * (size_t)Nt);
    for (int64_t t = 0; t < Nt; ++t) {
        const int *v = &tets[4 * t];
        for (int k = 0; k < 4; ++k)
            if (v[k] < 0 || v[k] >= Nv)
                return fail(FS_EINVAL, "tetrahedron node index out of range");
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j)
                if (v[i] == v[j])
                    return fail(FS_EINVAL, "degenerate tetrahedron (repeated node)");
        for (int skip = 0; skip < 4; ++skip) {
            int w[3], n = 0;
            for (int k = 0; k < 4; ++k)
                if (k != skip)
                    w[n++] = v[k];
            std::sort(w, w + 3);
            f.push_back(F{w[0], w[1], w[2], v[skip]});
        }
    }
    auto key_less = [](const F &x, const F &y) {
        return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.c < y.c);
    };
    std::sort(f.begin(), f.end(), key_less);
    out.clear();
    size_t i = 0;
    while (i < f.size()) {
        size_t j = i + 1;
        while (j < f.size() && f[j].a == f[i].a && f[j].b == f[i].b && f[j].c == f[i].c)
            ++j;
        if (j - i == 1) {
            out.push_back(f[i].a);
            out.push_back(f[i].b);
            out.push_back(f[i].c);
            out.push_back(f[i].opp);
        } else if (j - i > 2) {
            return fail(FS_EINVAL, "non-manifold mesh: a face is shared by more than two tetrahedra");
        }
        i = j;
    }
    return FS_OK;
}

template <typename real> fs_status reserve_charges3(fs3_plan *pl, int nrhs)
{
    if (nrhs > pl->nrhs_cap) {
        pl->release(pl->q_sorted);
        pl->release(pl->q_sum);
        pl->q_sorted = nullptr;
        pl->q_sum = nullptr;
        real *qs = nullptr;
        FS_TRY(pl->alloc(&qs, (size_t)std::max<int64_t>(pl->M, 1) * nrhs));
        pl->q_sorted = qs;
        FS_TRY(pl->alloc(&pl->q_sum, nrhs));
        pl->nrhs_cap = nrhs;
    }
    return FS_OK;
}

template <typename real> fs_status set_magnetization3_t(fs3_plan *pl, const double *mag, int nrhs)
{
    FS_TRY(reserve_charges3<real>(pl, nrhs));
    pl->nrhs = nrhs;
    FS_CUDA(cudaMemsetAsync(pl->q_sum, 0, sizeof(double) * nrhs, pl->stream));
    FS_CUDA(launch_fem3_charges_scatter<real>(pl->nodes, pl->tets, pl->Nt, pl->fem_tet_coef, pl->faces, pl->Nf, mag,
                                              pl->Nv, nrhs,
                                              pl->src_inv_perm, pl->M, (real *)pl->q_sorted, pl->q_sum, pl->stream));
    return FS_OK;
}

template <typename real> fs_status set_charges3_t(fs3_plan *pl, const void *q, fs_dtype dtype, int nrhs)
{
    FS_TRY(reserve_charges3<real>(pl, nrhs));
    pl->nrhs = nrhs;
    FS_CUDA(cudaMemsetAsync(pl->q_sum, 0, sizeof(double) * nrhs, pl->stream));
    FS_CUDA(launch_gather_charges<real>(q, dtype == FS_F64, pl->src_perm, pl->M, nrhs, (real *)pl->q_sorted,
                                        pl->q_sum, pl->stream));
    return FS_OK;
}

template <typename real> fs_status eval3_t(fs3_plan *pl, void *phi, void *H, fs_dtype dtype)
{
    using C = typename Cplx<real>::type;
    cudaStream_t st = pl->stream;
    const Window<real> w = make_window<real>(pl->sigma, pl->m);
    const NearParams<double> np = make_near3<double>(pl);
    const Near3Params np32 = sizeof(real) == 4 ? make_near3_f32(pl) : Near3Params{};
    const size_t osz = dtype == FS_F64 ? 8 : 4;
    const size_t cube = (size_t)pl->n_a * pl->n_a * pl->n_a;
    // FP32 plans run the near field on a second stream beside spreading and the transform: it
    // stores phi_s and grad_s (or adds atomically into zeroed ones) and the interpolation adds
    const bool overlap = sizeof(real) == 4 && pl->aux != nullptr;
    for (int r = 0; r < pl->nrhs; ++r) {
        const real *q = (const real *)pl->q_sorted + (int64_t)r * pl->M;
        if (overlap)
            FS_CUDA(cudaEventRecord(pl->ev_fork, st));   // the charges are in
        FS_CUDA(cudaMemsetAsync(pl->grid, 0, cube * sizeof(real), st));
        if (sizeof(real) == 4 && pl->spread_tiles)
            FS_CUDA(launch_spread3_tile(pl->spread_items, pl->n_spread_items, pl->m, pl->cg.cell, pl->src_base,
                                        (const float *)pl->src_frac, (const float *)q, pl->wpoly, (float *)pl->grid,
                                        pl->n_a, st));
        else
            FS_CUDA(launch_spread3<real>(pl->M, pl->m, pl->src_base, (const real *)pl->src_frac, q, w, pl->wpoly,
                                         (real *)pl->grid, pl->n_a, st));
        if constexpr (sizeof(real) == 4) {
            if (overlap) {
                cudaStream_t sa = pl->aux;
                FS_CUDA(cudaStreamWaitEvent(sa, pl->ev_fork, 0));
                if (pl->src_major) {
                    FS_CUDA(cudaMemsetAsync(pl->phi_s, 0, sizeof(float) * (size_t)pl->N, sa));
                    FS_CUDA(cudaMemsetAsync(pl->grad_s, 0, sizeof(float) * 3 * (size_t)pl->N, sa));
                    FS_CUDA(launch_near3_src(pl->src_items, pl->n_src_items, pl->src_base, pl->src_p32, pl->tgt_p32,
                                             pl->tgt_pos, pl->src_pos, (const float *)q, pl->tgt_start, pl->cg, np32,
                                             pl->N, pl->coinc_start, pl->coinc_src, pl->n_coinc > 0,
                                             (float *)pl->phi_s, (float *)pl->grad_s, sa));
                } else {
                    FS_CUDA(launch_near3_warp(pl->near_items, pl->n_near_items, pl->tgt_base, pl->tgt_p32,
                                              pl->src_p32, pl->tgt_pos, pl->src_pos, (const float *)q, pl->src_start,
                                              pl->cg, np32, pl->coinc_start, pl->coinc_src, (float *)pl->phi_s,
                                              (float *)pl->grad_s, true, sa));
                }
                FS_CUDA(cudaEventRecord(pl->ev_join, sa));
            }
        }
        FS_CUDA(launch_fft3<real>((real *)pl->grid, pl->n_a, pl->n_os, pl->n, (C *)pl->spec1, (C *)pl->spec2,
                                  (const real *)pl->mul, (const C *)pl->tw, st));
        if (overlap)
            FS_CUDA(cudaStreamWaitEvent(st, pl->ev_join, 0));
        FS_CUDA(launch_interp3<real>(pl->N, pl->m, pl->tgt_base, (const real *)pl->tgt_frac, w, pl->wpoly,
                                     (const real *)pl->grid, pl->n_a, (real)pl->n_os, (real *)pl->phi_s,
                                     (real *)pl->grad_s, overlap, st));
        if constexpr (sizeof(real) == 8)
            FS_CUDA(launch_near3_f64(pl->N, pl->tgt_base, pl->tgt_pos, pl->src_pos, pl->src_start, pl->cg,
                                     (const double *)q, np, (double *)pl->phi_s, (double *)pl->grad_s, st));
        void *po = phi ? (unsigned char *)phi + (size_t)r * pl->N * osz : nullptr;
        void *ho = H ? (unsigned char *)H + (size_t)r * pl->N * 3 * osz : nullptr;
        FS_CUDA(launch_unpermute3<real>(pl->N, (const real *)pl->phi_s, (const real *)pl->grad_s, pl->tgt_perm, pl->s,
                                        po, ho, dtype == FS_F64, st));
    }
    return FS_OK;
}

void plan3_free(fs3_plan *pl)
{
    if (!pl)
        return;
    if (pl->stream)
        cudaStreamSynchronize(pl->stream);
    if (pl->aux) {
        cudaStreamSynchronize(pl->aux);
        cudaStreamDestroy(pl->aux);
    }
    for (cudaEvent_t e : {pl->ev_fork, pl->ev_join})
        if (e)
            cudaEventDestroy(e);
    for (void *ptr : pl->allocs)
        cudaFree(ptr);
    delete pl;
}

// Validate the grid parameters and options shared by the point and mesh entry points.
fs_status plan3_new(int n_grid, double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs3_plan **out)
{
    fs_opts o{};
    if (opts)
        o = *opts;
    if (!is_pow2(n_grid) || n_grid < 4 || n_grid > 256)
        return fail(FS_EINVAL, "n_grid must be a power of two in [4, 256]");
    const double nos = sigma_os * n_grid;
    const int n_os = (int)std::lround(nos);
    if (!(sigma_os > 1.0) || std::fabs(nos - n_os) > 1e-9 || !is_pow2(n_os) || n_os > 512 || n_os <= n_grid)
        return fail(FS_EINVAL, "sigma_os * n_grid must be a power of two in (n_grid, 512]");
    if (m_window < 2 || m_window > 5 || 4 * m_window >= n_os)
        return fail(FS_EINVAL, "m_window must be in [2, 5] and below n_os / 4");
    if (!(eps_I > 0.0) || !(eps_I < 0.25))
        return fail(FS_EINVAL, "eps_I must be in (0, 1/4) (torus units)");
    if (o.precision != 0 && o.precision != 32 && o.precision != 64)
        return fail(FS_EINVAL, "precision must be 32 or 64");
    if (o.p < 0 || o.p > kMaxP)
        return fail(FS_EINVAL, "p must be in [1, 16] (0 = default)");
    if (o.eps_B < 0.0 || o.eps_B >= 0.25 || std::isnan(o.eps_B))
        return fail(FS_EINVAL, "eps_B must be in (0, 1/4) (0 = default)");
    fs3_plan *pl = new (std::nothrow) fs3_plan;
    if (!pl)
        return fail(FS_ENOMEM, "host allocation failed");
    pl->precision = o.precision == 64 ? 64 : 32;
    pl->n = n_grid;
    pl->n_os = n_os;
    pl->m = m_window;
    pl->sigma = sigma_os;
    pl->eps_I = eps_I;
    pl->eps_B = o.eps_B > 0.0 ? o.eps_B : eps_I;
    pl->p = o.p > 0 ? o.p : std::max(2, (int)std::lround(n_grid * eps_I));
    pl->stream = (cudaStream_t)o.stream;
    *out = pl;
    return FS_OK;
}

}  // namespace

extern "C" {

fs_status fs3_plan_create(const double *src_xyz, int64_t M, const double *tgt_xyz, int64_t N, int n_grid,
                          double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs3_plan **out)
{
    if (!out)
        return fail(FS_EINVAL, "null output pointer");
    *out = nullptr;
    if (M < 0 || N < 0 || (M > 0 && !src_xyz) || (N > 0 && !tgt_xyz))
        return fail(FS_EINVAL, "bad point arrays");
    fs3_plan *pl = nullptr;
    FS_TRY(plan3_new(n_grid, sigma_os, m_window, eps_I, opts, &pl));
    pl->M = M;
    pl->N = N;
    const fs_status s = pl->precision == 64 ? plan3_init<double>(pl, src_xyz, M, tgt_xyz, N)
                                            : plan3_init<float>(pl, src_xyz, M, tgt_xyz, N);
    if (s != FS_OK) {
        plan3_free(pl);
        return s;
    }
    *out = pl;
    return FS_OK;
}

fs_status fs3_plan_create_fem(const double *nodes, int64_t Nv, const int32_t *tets, int64_t Nt, int n_grid,
                              double sigma_os, int m_window, double eps_I, const fs_opts *opts, fs3_plan **out)
{
    if (!out)
        return fail(FS_EINVAL, "null output pointer");
    *out = nullptr;
    if (Nv <= 0 || Nt <= 0 || !nodes || !tets)
        return fail(FS_EINVAL, "a mesh needs nodes and tetrahedra");
    if (Nv > (int64_t)INT32_MAX || 4 * Nt + 12 * Nt > (int64_t)INT32_MAX)
        return fail(FS_EINVAL, "mesh too large");
    fs3_plan *pl = nullptr;
    FS_TRY(plan3_new(n_grid, sigma_os, m_window, eps_I, opts, &pl));
    auto body = [&]() -> fs_status {
        cudaStream_t st = pl->stream;
        std::vector<int> h_tets(4 * (size_t)Nt), h_faces;
        FS_CUDA(cudaMemcpyAsync(h_tets.data(), tets, sizeof(int) * 4 * Nt, cudaMemcpyDeviceToHost, st));
        FS_CUDA(cudaStreamSynchronize(st));
        FS_TRY(boundary_faces3(h_tets, Nt, Nv, h_faces));
        pl->is_fem = true;
        pl->Nv = Nv;
        pl->Nt = Nt;
        pl->Nf = (int64_t)h_faces.size() / 4;
        pl->nodes = nodes;
        FS_TRY(pl->alloc(&pl->tets, h_tets.size()));
        FS_TRY(pl->alloc(&pl->faces, std::max<size_t>(h_faces.size(), 1)));
        FS_CUDA(cudaMemcpyAsync(pl->tets, h_tets.data(), sizeof(int) * h_tets.size(), cudaMemcpyHostToDevice, st));
        if (!h_faces.empty())
            FS_CUDA(cudaMemcpyAsync(pl->faces, h_faces.data(), sizeof(int) * h_faces.size(), cudaMemcpyHostToDevice,
                                    st));
        const int64_t Ms = 4 * Nt + 3 * pl->Nf;
        FS_TRY(pl->alloc(&pl->fem_src, 3 * (size_t)Ms));
        FS_CUDA(launch_fem3_sources(nodes, pl->tets, Nt, pl->faces, pl->Nf, pl->fem_src, st));
        FS_TRY(pl->alloc(&pl->fem_tet_coef, 9 * (size_t)Nt));
        FS_CUDA(launch_fem3_tet_coef(nodes, pl->tets, Nt, pl->fem_tet_coef, st));
        FS_CUDA(cudaStreamSynchronize(st));
        pl->M = Ms;
        pl->N = Nv;
        FS_TRY(pl->precision == 64 ? plan3_init<double>(pl, pl->fem_src, Ms, nodes, Nv)
                                   : plan3_init<float>(pl, pl->fem_src, Ms, nodes, Nv));
        // source index -> sorted index: the assembly writes each element's charges into cell order
        FS_TRY(pl->alloc(&pl->src_inv_perm, (size_t)Ms));
        FS_CUDA(launch_invert_perm(pl->src_perm, Ms, pl->src_inv_perm, pl->stream));
        FS_CUDA(cudaStreamSynchronize(pl->stream));
        return FS_OK;
    };
    const fs_status s = body();
    if (s != FS_OK) {
        plan3_free(pl);
        return s;
    }
    *out = pl;
    return FS_OK;
}

fs_status fs3_set_magnetization(fs3_plan *plan, const double *mag, int nrhs)
{
    if (!plan)
        return fail(FS_EINVAL, "null plan");
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!mag || nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "bad magnetisation arguments");
    return plan->precision == 64 ? set_magnetization3_t<double>(plan, mag, nrhs)
                                 : set_magnetization3_t<float>(plan, mag, nrhs);
}

fs_status fs3_fem_charges(fs3_plan *plan, const double *mag, double *q_out, int nrhs)
{
    if (!plan)
        return fail(FS_EINVAL, "null plan");
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!mag || !q_out || nrhs < 1 || nrhs > 65535)
        return fail(FS_EINVAL, "bad magnetisation/charge arguments");
    FS_CUDA(launch_fem3_charges(plan->nodes, plan->tets, plan->Nt, plan->faces, mag, plan->Nv, nrhs, q_out, plan->M,
                                plan->stream));
    return FS_OK;
}

fs_status fs3_fem_sources(fs3_plan *plan, double *src_out)
{
    if (!plan)
        return fail(FS_EINVAL, "null plan");
    if (!plan->is_fem)
        return fail(FS_EINVAL, "not a FEM plan");
    if (!src_out)
        return fail(FS_EINVAL, "null output");
    FS_CUDA(cudaMemcpyAsync(src_out, plan->fem_src, sizeof(double) * 3 * plan->M, cudaMemcpyDeviceToDevice,
                            plan->stream));
    return FS_OK;
}

fs_status fs3_set_charges(fs3_plan *plan, const void *q, fs_dtype dtype, int nrhs)
{
    if (!plan)
        return fail(FS_EINVAL, "null plan");
    if ((dtype != FS_F32 && dtype != FS_F64) || nrhs < 1 || nrhs > 65535 || (plan->M > 0 && !q))
        return fail(FS_EINVAL, "bad charge arguments");
    return plan->precision == 64 ? set_charges3_t<double>(plan, q, dtype, nrhs)
                                 : set_charges3_t<float>(plan, q, dtype, nrhs);
}

fs_status fs3_eval_field(fs3_plan *plan, void *phi, void *H, fs_dtype dtype)
{
    if (!plan)
        return fail(FS_EINVAL, "null plan");
    if (dtype != FS_F32 && dtype != FS_F64)
        return fail(FS_EINVAL, "dtype must be FS_F32 or FS_F64");
    if (plan->nrhs < 1)
        return fail(FS_EINVAL, "no charges set");
    if (!phi && !H)
        return fail(FS_EINVAL, "nothing to evaluate");
    return plan->precision == 64 ? eval3_t<double>(plan, phi, H, dtype) : eval3_t<float>(plan, phi, H, dtype);
}

fs_status fs3_sync_status(fs3_plan *plan)
{
    if (!plan)
        return fail(FS_EINVAL, "null plan");
    FS_CUDA(cudaStreamSynchronize(plan->stream));
    return FS_OK;
}

fs_status fs3_plan_info(const fs3_plan *plan, fs_info *info)
{
    if (!plan || !info)
        return fail(FS_EINVAL, "null argument");
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
    info->spread_items = plan->spread_tiles ? plan->n_spread_items : 0;
    info->workspace_bytes = plan->bytes;
    info->is_fem = plan->is_fem;
    info->n_nodes = plan->Nv;
    info->n_tris = plan->Nt;
    info->n_bedges = plan->Nf;
    return FS_OK;
}

fs_status fs3_plan_destroy(fs3_plan *plan)
{
    plan3_free(plan);
    return FS_OK;
}

}  // extern "C"
