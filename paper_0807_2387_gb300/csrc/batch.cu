// Batched solves: many independent fast summations (one per instance, each with its own
// grid size and near-field radius, shared window and oversampling) and several charge
// vectors each, evaluated with one launch per stage over all (instance, right-hand side,
// unit) work items and replayed as one CUDA graph.
//
// Each instance is an ordinary plan (binning, coefficient table, twiddles, work items); the
// batch adds the buffers of every right-hand side, a device table of per-instance
// descriptors (BatchInst) and the merged work lists:
//   spreading  - the plans' tile items, largest first, x right-hand sides;
//   FFT        - one persistent launch over row pairs, then columns, then inverse row pairs
//                of every (instance, right-hand side), ordered by dependency (waits bounded);
//   near field - the plans' warp items ordered by estimated pair work across all instances,
//                every right-hand side in one traversal;
//   per-point stages (charges, interpolation, output) - block maps over the instances.
// With FS_FLAG_AUTOTUNE the tile edge and near-field cell of each (n, log2 N, log2 M) class
// are chosen by timing candidate plans (summation order changes, the sums do not).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "plan.h"

using namespace fs;

namespace {

constexpr int kPointBlock = 256;   // threads (= points) per block of the per-point batched kernels
constexpr size_t kMaxTileSmem = 56 * 1024;   // spreading tiles of tuned batches: >= 4 CTAs per SM
constexpr int kMaxRhs = 4;

struct GraphEntry {
    int q_f64, out_f64;
    cudaGraphExec_t exec;
};

}  // namespace

struct fs_batch {
    int count = 0, nrhs = 0, precision = 32, m = 0, p = 0;
    double sigma = 0;
    bool kahan = true;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<fs_plan *> plans;
    std::vector<void *> allocs;
    int64_t bytes = 0;
    int64_t total_src = 0, total_tgt = 0;
    // device tables
    void *inst = nullptr;                 // BatchInst<real>[count]
    BatchIO *io = nullptr;                // [count]
    std::vector<BatchIO> io_h;
    bool io_set = false;
    SpreadItem *spread_items = nullptr;
    int n_spread_items = 0, max_tile = 0;
    int4 *near_items = nullptr;
    int64_t n_near_items = 0;
    FftUnit *fft_units = nullptr;
    int n_fft_units = 0, fft_blocks = 0, L_max = 0;
    int *counters = nullptr;              // 2 * count * nrhs + 1
    int *err = nullptr;
    int *src_inst = nullptr, *src_first = nullptr, *tgt_inst = nullptr, *tgt_first = nullptr;
    int src_blocks = 0, tgt_blocks = 0;
    // per right-hand side buffers
    void *grids = nullptr, *specs = nullptr, *q_sorted = nullptr, *phi_s = nullptr, *grad_s = nullptr;
    void *coinc = nullptr;
    double *q_sum = nullptr;
    size_t grid_bytes = 0;
    std::vector<GraphEntry> graphs;

    template <typename T> fs_status alloc(T **out, size_t count_)
    {
        *out = nullptr;
        const size_t nbytes = std::max<size_t>(count_, 1) * sizeof(T);
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
};

namespace {

// ---- autotuner: tile edge and near-field cell per instance class

using TuneKey = std::tuple<int, int, double, int, int, int, int, int>;   // n, m, sigma, p, prec, kahan, lgN, lgM
std::map<TuneKey, std::pair<int, int>> g_tuned;
std::mutex g_tune_mu;

int ilog2_round(int64_t v) { return v <= 1 ? 0 : (int)std::lround(std::log2((double)v)); }

// Median-free timing of one candidate: one warm-up evaluation, then the mean of three.
fs_status time_candidate(const fs_instance &in, double sigma, int m, const fs_opts &o, const void *q, void *H,
                         float *ms)
{
    fs_plan *pl = new fs_plan;
    fs_status st = plan_create_common(in.src_xy, in.M, in.tgt_xy, in.N, in.n_grid, sigma, m, in.eps_I, &o, pl);
    if (st != FS_OK) {
        plan_destroy(pl);
        return st;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    st = fs_set_charges(pl, q, FS_F32, 1);
    if (st == FS_OK)
        st = fs_eval_field(pl, nullptr, H, FS_F32);
    if (st == FS_OK) {
        cudaEventRecord(e0, pl->stream);
        for (int k = 0; k < 3 && st == FS_OK; ++k) {
            st = fs_set_charges(pl, q, FS_F32, 1);
            if (st == FS_OK)
                st = fs_eval_field(pl, nullptr, H, FS_F32);
        }
        cudaEventRecord(e1, pl->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            st = fail(FS_ECUDA, "autotune timing failed");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan_destroy(pl);
    return st;
}

// Picks (tile_cells, cell) for the class of `in`: near-field cells of 1, 1.5 and 2 times the
// narrowest admissible width, tiles of about 16, 32 and 64 grid lines whose spreading tile
// fits in kMaxTileSmem, timed on the instance itself with constant charges (the work is
// independent of the charge values).
fs_status tune_instance(const fs_instance &in, double sigma, int m, const fs_opts &base, int *tile_cells, int *cell)
{
    const int L = (int)std::lround(sigma * in.n_grid);
    fs_opts probe = base;
    probe.flags &= ~(unsigned)(FS_FLAG_AUTOTUNE | FS_FLAG_TIMING);
    const int p = base.p > 0 ? base.p : std::max(2, (int)std::lround(in.n_grid * in.eps_I));
    const TuneKey key{in.n_grid, m, sigma, p, base.precision == 64 ? 64 : 32, (base.flags & FS_FLAG_NO_KAHAN) ? 0 : 1,
                      ilog2_round(in.N), ilog2_round(in.M)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *tile_cells = it->second.first;
            *cell = it->second.second;
            return FS_OK;
        }
    }
    const int min_cell = std::max(1, (int)std::ceil(in.eps_I * L - 1e-9));
    std::vector<int> cells{min_cell, (3 * min_cell + 1) / 2, 2 * min_cell};
    cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
    // charges and output for the probes (FP32; 0x3F bytes = 0.747 per charge)
    void *q = nullptr, *H = nullptr;
    if (cudaMalloc(&q, std::max<int64_t>(in.M, 1) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&H, std::max<int64_t>(in.N, 1) * 2 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(q);
        return fail(FS_ENOMEM, "autotune buffers");
    }
    cudaMemset(q, 0x3F, std::max<int64_t>(in.M, 1) * sizeof(float));
    float best = 1e30f;
    int best_t = 0, best_c = 0;
    fs_status st = FS_OK;
    for (int c : cells) {
        std::vector<int> tiles;
        for (int tg : {16, 32, 64})
            tiles.push_back(std::max(1, (int)std::lround((double)tg / c)));
        tiles.erase(std::unique(tiles.begin(), tiles.end()), tiles.end());
        for (int t : tiles) {
            // a batch sizes the spreading kernel's shared memory for its largest tile, so tiles
            // that would leave fewer than four CTAs per SM are not candidates
            const int P = t * c + 2 * m - 1;
            const bool comp = probe.precision != 64 && !(probe.flags & FS_FLAG_NO_KAHAN);
            const size_t bytes = probe.precision == 64 ? spread_smem_bytes<double>(P, 2 * m, false)
                                                       : spread_smem_bytes<float>(P, 2 * m, comp);
            if (bytes > kMaxTileSmem)
                continue;
            fs_opts o = probe;
            o.cell = c;
            o.tile_cells = t;
            float ms = 0.f;
            st = time_candidate(in, sigma, m, o, q, H, &ms);
            if (st == FS_EINVAL) {   // e.g. tile too large for shared memory: not a candidate
                st = FS_OK;
                continue;
            }
            if (st != FS_OK)
                break;
            if (ms < best) {
                best = ms;
                best_t = t;
                best_c = c;
            }
        }
        if (st != FS_OK)
            break;
    }
    cudaFree(q);
    cudaFree(H);
    if (st != FS_OK)
        return st;
    if (best_c == 0)
        return fail(FS_EINVAL, "autotune: no admissible tile / cell candidate");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = {best_t, best_c};
    *tile_cells = best_t;
    *cell = best_c;
    return FS_OK;
}

// ---- creation

template <typename real> fs_status batch_build(fs_batch *b, const fs_instance *in, const fs_opts &o)
{
    using C = typename Cplx<real>::type;
    const int K = b->count, R = b->nrhs;
    cudaStream_t st = b->stream;
    // per-instance plans (tuned or given tile / cell)
    for (int i = 0; i < K; ++i) {
        fs_opts oi = o;
        oi.flags &= ~(unsigned)FS_FLAG_AUTOTUNE;
        oi.stream = st;
        if ((o.flags & FS_FLAG_AUTOTUNE) && o.cell == 0 && o.tile_cells == 0)
            FS_TRY(tune_instance(in[i], b->sigma, b->m, oi, &oi.tile_cells, &oi.cell));
        fs_plan *pl = new fs_plan;
        fs_status s = plan_create_common(in[i].src_xy, in[i].M, in[i].tgt_xy, in[i].N, in[i].n_grid, b->sigma, b->m,
                                         in[i].eps_I, &oi, pl);
        if (s != FS_OK) {
            plan_destroy(pl);
            return s;
        }
        b->plans.push_back(pl);
        if (i == 0) {
            b->p = pl->p;
            b->kahan = pl->kahan;
        } else if (pl->p != b->p) {
            return fail(FS_EINVAL, "instances of a batch must share the smoothness degree p (set fs_opts.p)");
        }
    }
    // buffers of every right-hand side, one allocation per kind, 256-byte aligned slices
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    std::vector<size_t> off_g(K), off_s(K), off_q(K), off_n(K);
    size_t tot_g = 0, tot_s = 0, tot_q = 0, tot_n = 0;
    for (int i = 0; i < K; ++i) {
        const fs_plan *pl = b->plans[i];
        off_g[i] = tot_g;
        tot_g += up((size_t)pl->n_a * pl->pitch * sizeof(real)) * R;
        off_s[i] = tot_s;
        tot_s += up((size_t)(pl->n / 2 + 1) * pl->ld * sizeof(C)) * R;
        off_q[i] = tot_q;
        tot_q += up((size_t)std::max<int64_t>(pl->M, 1) * sizeof(real)) * R;
        off_n[i] = tot_n;
        tot_n += up((size_t)std::max<int64_t>(pl->N, 1) * sizeof(real)) * R;
        b->total_src += pl->M;
        b->total_tgt += pl->N;
        b->L_max = std::max(b->L_max, pl->n_os);
        b->max_tile = std::max(b->max_tile, pl->cg.T * pl->cg.cell);
    }
    unsigned char *grids, *specs, *qs, *phis, *grads, *coincs;
    FS_TRY(b->alloc(&grids, tot_g));
    FS_TRY(b->alloc(&specs, tot_s));
    FS_TRY(b->alloc(&qs, tot_q));
    FS_TRY(b->alloc(&phis, tot_n));
    FS_TRY(b->alloc(&grads, 2 * tot_n));
    FS_TRY(b->alloc(&coincs, tot_n));
    FS_TRY(b->alloc(&b->q_sum, (size_t)K * R));
    b->grids = grids;
    b->specs = specs;
    b->q_sorted = qs;
    b->phi_s = phis;
    b->grad_s = grads;
    b->coinc = coincs;
    b->grid_bytes = tot_g;
    // descriptors
    std::vector<BatchInst<real>> h(K);
    for (int i = 0; i < K; ++i) {
        const fs_plan *pl = b->plans[i];
        BatchInst<real> &d = h[i];
        std::memset(&d, 0, sizeof(d));
        d.n = pl->n;
        d.L = pl->n_os;
        d.n_a = pl->n_a;
        d.pitch = pl->pitch;
        d.ld = pl->ld;
        d.cg = pl->cg;
        d.M = pl->M;
        d.N = pl->N;
        d.src_base = pl->src_base;
        d.tgt_base = pl->tgt_base;
        d.src_frac = pl->src_frac;
        d.tgt_frac = pl->tgt_frac;
        d.src_pos = pl->src_pos;
        d.tgt_pos = pl->tgt_pos;
        d.src_hi = pl->src_pos32;
        d.src_lo = pl->src_lo32;
        d.tgt_hi = pl->tgt_pos32;
        d.tgt_lo = pl->tgt_lo32;
        d.src_start = pl->src_start;
        d.src_perm = pl->src_perm;
        d.tgt_perm = pl->tgt_perm;
        d.mul = (const real *)pl->mul;
        d.tw = (const C *)pl->tw;
        d.grid_stride = (int64_t)(up((size_t)pl->n_a * pl->pitch * sizeof(real)) / sizeof(real));
        d.spec_stride = (int64_t)(up((size_t)(pl->n / 2 + 1) * pl->ld * sizeof(C)) / sizeof(C));
        d.grid = (real *)(grids + off_g[i]);
        d.spec = (C *)(specs + off_s[i]);
        // q, phi_s, grad_s, coinc: right-hand side r at r * M (or r * N) inside the instance's slice
        d.q = (real *)(qs + off_q[i]);
        d.phi_s = (real *)(phis + off_n[i]);
        d.grad_s = (real *)(grads + 2 * off_n[i]);
        d.coinc = (real *)(coincs + off_n[i]);
        d.q_sum = b->q_sum + (size_t)i * R;
        d.s = pl->s;
        d.shift = std::log(pl->s) / (2.0 * kPi);
        d.np = make_near<real>(pl);
    }
    FS_TRY(b->alloc((unsigned char **)&b->inst, sizeof(BatchInst<real>) * K));
    FS_CUDA(cudaMemcpy(b->inst, h.data(), sizeof(BatchInst<real>) * K, cudaMemcpyHostToDevice));
    FS_TRY(b->alloc(&b->io, K));
    b->io_h.assign(K, BatchIO{nullptr, nullptr, nullptr});
    // spreading items: every plan's tiles, most sources first
    std::vector<SpreadItem> si;
    for (int i = 0; i < K; ++i)
        for (SpreadItem it : b->plans[i]->items_h) {
            it.pad = i;
            si.push_back(it);
        }
    std::stable_sort(si.begin(), si.end(), [](const SpreadItem &x, const SpreadItem &y) { return x.count > y.count; });
    b->n_spread_items = (int)si.size();
    FS_TRY(b->alloc(&b->spread_items, si.size()));
    if (!si.empty())
        FS_CUDA(cudaMemcpy(b->spread_items, si.data(), si.size() * sizeof(SpreadItem), cudaMemcpyHostToDevice));
    // near-field items (FP32): all instances, largest estimated work first
    if (b->precision == 32) {
        std::vector<std::pair<int64_t, int4>> ni;
        for (int i = 0; i < K; ++i) {
            const fs_plan *pl = b->plans[i];
            for (size_t k = 0; k < pl->near_items_h.size(); ++k)
                ni.push_back({pl->near_work_h[k], make_int4(pl->near_items_h[k].x, pl->near_items_h[k].y, i, 0)});
        }
        std::stable_sort(ni.begin(), ni.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
        std::vector<int4> items(ni.size());
        for (size_t k = 0; k < ni.size(); ++k)
            items[k] = ni[k].second;
        b->n_near_items = (int64_t)items.size();
        FS_TRY(b->alloc(&b->near_items, items.size()));
        if (!items.empty())
            FS_CUDA(cudaMemcpy(b->near_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    // FFT units: all forward row pairs, then all columns, then all inverse row pairs; larger
    // transforms first inside each phase
    std::vector<int> order(K);
    for (int i = 0; i < K; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->plans[x]->n_os > b->plans[y]->n_os; });
    std::vector<FftUnit> fu;
    for (int kind = 0; kind < 3; ++kind)
        for (int i : order)
            for (int r = 0; r < R; ++r) {
                const fs_plan *pl = b->plans[i];
                const int units = kind == 1 ? pl->n / 2 + 1 : (pl->n_a + 1) / 2;
                for (int u = 0; u < units; ++u)
                    fu.push_back(FftUnit{i, r, kind, u});
            }
    b->n_fft_units = (int)fu.size();
    FS_TRY(b->alloc(&b->fft_units, fu.size()));
    FS_CUDA(cudaMemcpy(b->fft_units, fu.data(), fu.size() * sizeof(FftUnit), cudaMemcpyHostToDevice));
    FS_CUDA(batch_fft_blocks<real>(b->L_max, &b->fft_blocks));
    FS_TRY(b->alloc(&b->counters, 2 * (size_t)K * R + 1));
    FS_TRY(b->alloc(&b->err, 1));
    FS_CUDA(cudaMemset(b->err, 0, sizeof(int)));
    // block maps of the per-point stages
    auto block_map = [&](bool src, int **inst_d, int **first_d, int *blocks) -> fs_status {
        std::vector<int> bi, first(K);
        for (int i = 0; i < K; ++i) {
            first[i] = (int)bi.size();
            const int64_t n = src ? b->plans[i]->M : b->plans[i]->N;
            const int64_t nb = (n + kPointBlock - 1) / kPointBlock;
            for (int64_t k = 0; k < nb; ++k)
                bi.push_back(i);
        }
        *blocks = (int)bi.size();
        FS_TRY(b->alloc(inst_d, bi.size()));
        FS_TRY(b->alloc(first_d, first.size()));
        if (!bi.empty())
            FS_CUDA(cudaMemcpy(*inst_d, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice));
        FS_CUDA(cudaMemcpy(*first_d, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice));
        return FS_OK;
    };
    FS_TRY(block_map(true, &b->src_inst, &b->src_first, &b->src_blocks));
    FS_TRY(block_map(false, &b->tgt_inst, &b->tgt_first, &b->tgt_blocks));
    FS_CUDA(prepare_batch_spread<real>(b->m, b->max_tile, b->kahan));
    return FS_OK;
}

// ---- evaluation

template <typename real> fs_status batch_enqueue(fs_batch *b, int q_f64, int out_f64)
{
    cudaStream_t st = b->stream;
    const int K = b->count, R = b->nrhs;
    const auto *inst = (const BatchInst<real> *)b->inst;
    const fs_plan *p0 = b->plans[0];
    const Window<real> w = make_window<real>(p0);
    const BlockMap src_map{b->src_inst, b->src_first}, tgt_map{b->tgt_inst, b->tgt_first};
    FS_CUDA(cudaMemsetAsync(b->q_sum, 0, sizeof(double) * K * R, st));
    FS_CUDA(cudaMemsetAsync(b->grids, 0, b->grid_bytes, st));
    FS_CUDA(cudaMemsetAsync(b->counters, 0, sizeof(int) * (2 * (size_t)K * R + 1), st));
    FS_CUDA(launch_batch_gather_charges<real>(inst, b->io, src_map, b->src_blocks, R, q_f64, st));
    if constexpr (sizeof(real) == 4) {
        // the near field first, storing its sums (every target lies in one item); the grids are
        // then still in L2 when one pass adds the far field and writes the caller's buffers
        FS_CUDA(launch_batch_near32(b->n_near_items, b->near_items, (const BatchInst<float> *)b->inst, b->p, R, true,
                                    st));
    }
    FS_CUDA(launch_batch_spread<real>(b->spread_items, b->n_spread_items, R, inst, b->m, b->max_tile, w, p0->wpoly,
                                      b->kahan, st));
    FS_CUDA(launch_batch_fft<real>(inst, b->fft_units, b->n_fft_units, K, R, b->L_max, b->fft_blocks, b->counters,
                                   b->err, kWaitSpins, st));
    if constexpr (sizeof(real) == 4) {
        FS_CUDA(launch_batch_interp_out<real>(inst, b->io, tgt_map, b->tgt_blocks, R, b->m, w, p0->wpoly, out_f64, st));
    } else {
        FS_CUDA(launch_batch_interp<real>(inst, tgt_map, b->tgt_blocks, R, b->m, w, p0->wpoly, st));
        FS_CUDA(launch_batch_near64((const BatchInst<double> *)b->inst, tgt_map, b->tgt_blocks, R, st));
        FS_CUDA(launch_batch_unpermute<real>(inst, b->io, tgt_map, b->tgt_blocks, R, out_f64, st));
    }
    return FS_OK;
}

fs_status batch_graph(fs_batch *b, int q_f64, int out_f64, cudaGraphExec_t *out)
{
    for (const GraphEntry &g : b->graphs)
        if (g.q_f64 == q_f64 && g.out_f64 == out_f64) {
            *out = g.exec;
            return FS_OK;
        }
    cudaGraph_t graph = nullptr;
    FS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const fs_status s = b->precision == 64 ? batch_enqueue<double>(b, q_f64, out_f64)
                                           : batch_enqueue<float>(b, q_f64, out_f64);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (s != FS_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess)
        return fail(FS_ECUDA, std::string("stream capture of the batch failed: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess)
        return fail(FS_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e2));
    b->graphs.push_back(GraphEntry{q_f64, out_f64, exec});
    *out = exec;
    return FS_OK;
}

void batch_free(fs_batch *b)
{
    if (!b)
        return;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    for (const GraphEntry &g : b->graphs)
        cudaGraphExecDestroy(g.exec);
    for (fs_plan *pl : b->plans)
        plan_destroy(pl);
    for (void *ptr : b->allocs)
        cudaFree(ptr);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

fs_status fs_batch_create(const fs_instance *inst, int count, double sigma_os, int m_window, int nrhs,
                          const fs_opts *opts, fs_batch **out)
{
    if (!out)
        return fail(FS_EINVAL, "null output pointer");
    *out = nullptr;
    if (!inst || count <= 0)
        return fail(FS_EINVAL, "a batch needs at least one instance");
    if (nrhs < 1 || nrhs > kMaxRhs)
        return fail(FS_EINVAL, "nrhs must be 1.." + std::to_string(kMaxRhs));
    for (int i = 0; i < count; ++i)
        if (inst[i].M < 0 || inst[i].N < 0 || (inst[i].M > 0 && !inst[i].src_xy) ||
            (inst[i].N > 0 && !inst[i].tgt_xy))
            return fail(FS_EINVAL, "instance " + std::to_string(i) + ": bad point arrays");
    fs_opts o{};
    if (opts)
        o = *opts;
    if ((o.cell != 0) != (o.tile_cells != 0) && (o.flags & FS_FLAG_AUTOTUNE))
        return fail(FS_EINVAL, "FS_FLAG_AUTOTUNE chooses cell and tile_cells: leave both 0");
    fs_batch *b = new fs_batch;
    b->count = count;
    b->nrhs = nrhs;
    b->precision = o.precision == 64 ? 64 : 32;
    b->m = m_window;
    b->sigma = sigma_os;
    if (o.stream) {
        b->stream = (cudaStream_t)o.stream;
    } else {
        // the legacy default stream cannot be captured into a graph: use a blocking stream
        // (ordered with the legacy default stream)
        if (cudaStreamCreate(&b->stream) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return fail(FS_ECUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    o.stream = b->stream;
    const fs_status s = b->precision == 64 ? batch_build<double>(b, inst, o) : batch_build<float>(b, inst, o);
    if (s != FS_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return FS_OK;
}

fs_status fs_batch_eval(fs_batch *batch, const void *const *q, fs_dtype q_dtype, void *const *phi, void *const *H,
                        fs_dtype out_dtype)
{
    if (!batch)
        return fail(FS_EINVAL, "null batch");
    if (!q)
        return fail(FS_EINVAL, "null charge pointer array");
    if ((q_dtype != FS_F32 && q_dtype != FS_F64) || (out_dtype != FS_F32 && out_dtype != FS_F64))
        return fail(FS_EINVAL, "dtype must be FS_F32 or FS_F64");
    std::vector<BatchIO> io(batch->count);
    for (int i = 0; i < batch->count; ++i) {
        const fs_plan *pl = batch->plans[i];
        io[i].q = q[i];
        io[i].phi = phi ? phi[i] : nullptr;
        io[i].H = H ? H[i] : nullptr;
        if (pl->M > 0 && !io[i].q)
            return fail(FS_EINVAL, "instance " + std::to_string(i) + ": null charges");
    }
    if (!batch->io_set || std::memcmp(io.data(), batch->io_h.data(), sizeof(BatchIO) * io.size()) != 0) {
        // pageable source: the copy is staged before the call returns, in stream order after
        // every evaluation enqueued before it
        FS_CUDA(cudaMemcpyAsync(batch->io, io.data(), sizeof(BatchIO) * io.size(), cudaMemcpyHostToDevice,
                                batch->stream));
        batch->io_h = io;
        batch->io_set = true;
    }
    cudaGraphExec_t exec = nullptr;
    FS_TRY(batch_graph(batch, q_dtype == FS_F64, out_dtype == FS_F64, &exec));
    FS_CUDA(cudaGraphLaunch(exec, batch->stream));
    return FS_OK;
}

fs_status fs_batch_sync_status(fs_batch *batch)
{
    if (!batch)
        return fail(FS_EINVAL, "null batch");
    FS_CUDA(cudaStreamSynchronize(batch->stream));
    int e = 0;
    FS_CUDA(cudaMemcpy(&e, batch->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        FS_CUDA(cudaMemset(batch->err, 0, sizeof(int)));
        return fail(FS_ETIMEOUT, "a device-side wait of the batched FFT gave up (results of that evaluation are invalid)");
    }
    return FS_OK;
}

fs_status fs_batch_info(const fs_batch *batch, fs_batch_facts *info)
{
    if (!batch || !info)
        return fail(FS_EINVAL, "null argument");
    std::memset(info, 0, sizeof(*info));
    info->count = batch->count;
    info->nrhs = batch->nrhs;
    info->precision = batch->precision;
    info->total_src = batch->total_src;
    info->total_tgt = batch->total_tgt;
    info->spread_items = batch->n_spread_items;
    info->fft_units = batch->n_fft_units;
    info->fft_blocks = batch->fft_blocks;
    info->near_items = batch->n_near_items;
    int64_t bytes = batch->bytes;
    for (const fs_plan *pl : batch->plans)
        bytes += pl->bytes;
    info->workspace_bytes = bytes;
    return FS_OK;
}

fs_status fs_batch_plan(fs_batch *batch, int i, fs_plan **out)
{
    if (!batch || !out)
        return fail(FS_EINVAL, "null argument");
    if (i < 0 || i >= batch->count)
        return fail(FS_EINVAL, "instance index out of range");
    *out = batch->plans[i];
    return FS_OK;
}

fs_status fs_batch_destroy(fs_batch *batch)
{
    batch_free(batch);
    return FS_OK;
}

fs_status fs_wait_selftest(int spins)
{
    if (spins < 1)
        return fail(FS_EINVAL, "spins must be >= 1");
    int *buf = nullptr;
    cudaStream_t st = nullptr;
    FS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t e = cudaMalloc(&buf, 2 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess)
        e = launch_wait_selftest(buf, buf + 1, spins, st);
    int flag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&flag, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaStreamDestroy(st);
    if (e != cudaSuccess)
        return fail(FS_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
    if (flag != 0)
        return fail(FS_ETIMEOUT, "the bounded wait gave up and set the error word (expected)");
    return FS_OK;
}

}  // extern "C"
