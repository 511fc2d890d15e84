// Plan object of the FEM-NFFT fast summation and the host helpers shared by the plan
// entry points (femnfft.cu) and the batched solves (batch.cu).  Private to the library.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/femnfft.h"
#include "internal.h"

namespace fs {

// Records msg as the calling thread's last error and returns st.
fs_status fail(fs_status st, const std::string &msg);

constexpr int kStages = 8;
constexpr int kSpreadChunk = 512;   // sources per spreading work item
// 2D plans whose occupied spreading tiles hold fewer sources than this on average spread with
// global atomics (the plan's choice in plan_init).  Zero: on GB300 the tiles won at every
// density measured, from 1.4 to over 700 sources per occupied tile (uniform discs of 2^10 to
// 2^20 points on n = 128 and 512 grids, m = 5: 12.9 vs 19.9 us at the sparse end, 170 vs
// 545 us at the dense end), so direct spreading is used only when FS_FLAG_SPREAD_DIRECT asks.
constexpr double kDirectSpreadBelow = 0.0;

}  // namespace fs

#define FS_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fs::fail(FS_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_));       \
    } while (0)

#define FS_TRY(expr)                                                                                    \
    do {                                                                                                \
        fs_status s_ = (expr);                                                                          \
        if (s_ != FS_OK)                                                                                \
            return s_;                                                                                  \
    } while (0)

struct fs_plan {
    // parameters
    int precision = 32;
    int n = 0, n_os = 0, m = 0, p = 0;
    double sigma = 0, eps_I = 0, eps_B = 0, s = 1.0;
    int64_t M = 0, N = 0;
    int window_lo = 0, n_a = 0, pitch = 0, ld = 0;
    fs::CellGrid cg{};
    int n_keys = 0;
    unsigned flags = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool kahan = true;
    fs::KernelParams kp{};
    double beta[fs::kMaxP] = {0};
    fs::WindowPoly wpoly{};               // FP32 window polynomials (per tap)
    // device memory
    std::vector<void *> allocs;
    int64_t bytes = 0;
    int *status = nullptr;
    int *status_host = nullptr;           // page-locked copy of *status (fs_solve_host)
    int *src_perm = nullptr, *tgt_perm = nullptr;
    int *src_base = nullptr, *tgt_base = nullptr;
    void *src_frac = nullptr, *tgt_frac = nullptr;
    double2 *src_pos = nullptr, *tgt_pos = nullptr;
    float2 *src_pos32 = nullptr, *tgt_pos32 = nullptr;
    float2 *src_lo32 = nullptr, *tgt_lo32 = nullptr;
    int *src_start = nullptr, *tgt_start = nullptr;
    fs::SpreadItem *items = nullptr;
    int n_items = 0;
    fs::SpreadItem *tgt_items = nullptr;  // adjoint: spreading at the targets
    int n_tgt_items = 0;
    // adjoint workspace (allocated by the first fs_adjoint call)
    void *adj_c = nullptr, *adj_dn = nullptr, *adj_df = nullptr;
    void *adj_a = nullptr, *adj_ga = nullptr, *adj_cg = nullptr, *adj_hess = nullptr;
    double *adj_gsum = nullptr;
    int2 *near_items = nullptr;       // FP32 near field: (first target, count <= 64) per warp
    int64_t n_near_items = 0;
    std::vector<int2> near_items_h;   // host copies (merged into batch work lists)
    std::vector<int64_t> near_work_h; // estimated pair work per near item
    std::vector<fs::SpreadItem> items_h;
    int2 *src_near_items = nullptr;   // FP32 adjoint and source-major near field: (first source, count <= 64)
    int64_t n_src_near_items = 0;
    bool src_major = false;           // FP32 forward near field over source items (many more sources than targets)
    void *mul = nullptr, *tw = nullptr;
    void *grid = nullptr, *spec = nullptr;
    void *grid_comp = nullptr;        // direct spreading (FP32): compensation plane of the grid
    bool spread_direct = false;       // spread with global atomics instead of shared-memory tiles
    void *phi_s = nullptr, *grad_s = nullptr, *coinc = nullptr;   // one allocation, at 0, sums_n and 3 sums_n
    int64_t sums_n = 0;
    // charges
    void *q_sorted = nullptr;
    double *q_sum = nullptr;
    int nrhs = 0, nrhs_cap = 0;
    // FEM
    bool is_fem = false;
    int64_t Nv = 0, Nt = 0, Ne = 0;
    const double2 *nodes = nullptr;   // caller's (valid while the plan is used)
    int *tris = nullptr, *bedges = nullptr;
    double2 *fem_tri_coef = nullptr;      // per triangle: its charge = sum_k M_k . coef_k (k_fem_tri_coef)
    double2 *fem_src = nullptr;
    int *src_inv_perm = nullptr;      // source index -> sorted index (charges assembled into cell order)
    // host staging for fs_solve_host
    void *d_q_stage = nullptr, *d_phi_stage = nullptr, *d_H_stage = nullptr;
    size_t q_stage_bytes = 0, phi_stage_bytes = 0, H_stage_bytes = 0;
    // stats
    int64_t near_pairs = 0, near_pairs_fp64 = 0;
    // timing
    cudaEvent_t ev[fs::kStages + 1] = {};
    cudaEvent_t ev_q0 = nullptr, ev_q1 = nullptr;
    bool events = false;
    // FP32 plans: the near field runs on a second stream beside spreading and the transform
    // (fork after the charges, join before the interpolation adds the far field)
    bool overlap = false;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_n0 = nullptr, ev_n1 = nullptr, ev_j = nullptr;   // timing of the overlapped stages

    template <typename T> fs_status alloc(T **out, size_t count)
    {
        *out = nullptr;
        if (count == 0)
            count = 1;
        void *p_ = nullptr;
        const size_t nbytes = count * sizeof(T);
        cudaError_t e = cudaMalloc(&p_, nbytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fs::fail(FS_ENOMEM, "cudaMalloc of " + std::to_string(nbytes) + " bytes failed: " +
                                       cudaGetErrorString(e));
        }
        allocs.push_back(p_);
        bytes += (int64_t)nbytes;
        *out = static_cast<T *>(p_);
        return FS_OK;
    }
    fs_status alloc_bytes(void **out, size_t nbytes)
    {
        unsigned char *p_ = nullptr;
        FS_TRY(alloc(&p_, nbytes));
        *out = p_;
        return FS_OK;
    }
    void release(void *ptr)
    {
        if (!ptr)
            return;
        auto it = std::find(allocs.begin(), allocs.end(), ptr);
        if (it != allocs.end()) {
            cudaFree(ptr);
            allocs.erase(it);
        }
    }
    size_t rsize() const { return precision == 64 ? 8 : 4; }
};

namespace fs {

// Modified Bessel function I_0 (power series, FP64).
double bessel_i0(double x);
// Per-tap polynomial form of the normalised Kaiser-Bessel window (FP32 kernels) for
// oversampling sigma and half-width m.
void build_window_poly(double sigma, int m, WindowPoly *wp);

// Validates the parameters and builds the plan (binning, tables, items) on its stream.
fs_status plan_create_common(const double *src, int64_t M, const double *tgt, int64_t N, int n_grid,
                             double sigma_os, int m, double eps_I, const fs_opts *opts, fs_plan *pl);
// Waits for the plan's stream and frees everything it owns.
void plan_destroy(fs_plan *pl);

template <typename real> inline Window<real> make_window(double sigma, int m_window)
{
    const double b = kPi * (2.0 - 1.0 / sigma);
    const double m = m_window;
    Window<real> w;
    w.m = (real)m;
    w.m2 = (real)(m * m);
    w.b = (real)b;
    w.bm = (real)(b * m);
    w.S = (real)(m * b / (1.0 - std::exp(-2.0 * b * m)));
    return w;
}

template <typename real> inline Window<real> make_window(const fs_plan *pl)
{
    return make_window<real>(pl->sigma, pl->m);
}

template <typename real> inline NearParams<real> make_near(const fs_plan *pl)
{
    NearParams<real> np{};
    np.p = pl->p;
    np.eps2 = (real)(pl->eps_I * pl->eps_I);
    np.inv_eps2 = (real)(1.0 / (pl->eps_I * pl->eps_I));
    np.close2 = (real)((pl->eps_I / 8.0) * (pl->eps_I / 8.0));
    np.hcell = (real)((double)pl->cg.cell / pl->n_os);
    for (int k = 0; k < pl->p; ++k)
        np.beta[k] = (real)pl->beta[k];
    for (int k = 1; k < pl->p; ++k)
        np.dbeta[k - 1] = (real)(2.0 * k * pl->beta[k] / (pl->eps_I * pl->eps_I));
    // T_I - k(eps_I) vanishes at r = eps_I; and since k - T_I has a zero of order p there, the
    // gradient numerator R(w) = -(1/2pi) - sum_k 2k beta_k w^k (degree p-1) is c (w-1)^(p-1).
    const double k_eps = -std::log(pl->eps_I) / (2.0 * kPi);
    for (int k = 0; k < pl->p; ++k)
        np.pbeta[k] = (real)(k == 0 ? pl->beta[0] - k_eps : pl->beta[k]);
    // synthetic division of P by (w - 1): Ptilde_{p-2} = a_{p-1}, Ptilde_k = a_{k+1} + Ptilde_{k+1}
    // (the remainder P(1) vanishes in exact arithmetic and is dropped)
    {
        double a[kMaxP] = {0}, t[kMaxP] = {0};
        for (int k = 0; k < pl->p; ++k)
            a[k] = k == 0 ? pl->beta[0] - k_eps : pl->beta[k];
        for (int k = pl->p - 2; k >= 0; --k)
            t[k] = a[k + 1] + (k + 1 <= pl->p - 2 ? t[k + 1] : 0.0);
        for (int k = 0; k + 1 < pl->p; ++k)
            np.nptilde[k] = (real)(-t[k]);
    }
    // R(w) = c (w-1)^(p-1) with R(0) = -(1/2pi) gives c = (-1)^p / (2pi), independent of beta
    np.rcoef = (real)(((pl->p % 2 == 0) ? 1.0 : -1.0) / (2.0 * kPi * pl->eps_I * pl->eps_I));
    return np;
}

}  // namespace fs
