// api.cu -- the C ABI of libgmrf (include/gmrf.h): argument validation on the host, device
// memory and layout set-up, the sweep driver (direct launches or captured CUDA graphs), and the
// copy-out of results.  Every compute step runs in the kernels of sweep_kernels.cu,
// csr_build.cu and plain.cu; this file only validates, allocates, launches and copies.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include <atomic>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/gmrf.h"
#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "mbarrier.cuh"

using namespace gmrf;

namespace {

thread_local std::string g_last_error;

gmrf_status fail(gmrf_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

struct CudaFail {
    cudaError_t err;
    std::string where;
};

// Fault injection for tests (gmrf_debug_fail_alloc): device allocations left before one fails
// (0: none fails).  Every device allocation of the library goes through dev_malloc.
std::atomic<int64_t> g_fail_alloc{0};

cudaError_t dev_malloc(void **p, size_t bytes)
{
    int64_t k = g_fail_alloc.load();
    while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

struct HostField {
    int32_t kind = 0;
    int32_t dims[3] = {0, 0, 0};
    int32_t n = 0;
    int32_t ncolors = 0;
    int32_t components = 1;
    bool fused = false;           // sampled by the fused 2-D lattice sweep (ping-pong state)
    std::vector<int32_t> colors;  // CSR: natural-order colouring used
    int32_t max_degree = 0;       // CSR: largest row
    bool weighted = false;        // CSR: weights given
};

// Whether every value is finite: exponent bits not all ones, tested without a branch per value
// (chunks of 4096, so a bad value ends the scan soon).
bool all_finite(const double *v, int64_t n)
{
    constexpr uint64_t kExp = 0x7ff0000000000000ull;
    for (int64_t i0 = 0; i0 < n; i0 += 4096) {
        const int64_t i1 = std::min<int64_t>(n, i0 + 4096);
        uint64_t bad = 0;
        for (int64_t i = i0; i < i1; ++i) {
            uint64_t b;
            std::memcpy(&b, v + i, sizeof(b));
            bad |= static_cast<uint64_t>((b & kExp) == kExp);
        }
        if (bad) return false;
    }
    return true;
}

// Breadth-first order of a graph's vertices, each component from a pseudo-peripheral vertex (the
// last one a breadth-first search from its lowest vertex reaches), neighbours in CSR order.  The
// layout sorts each colour class in this order (the order inside a class is free, Sec. 2.3:
// its sites are conditionally independent), so nearby sites get nearby positions.
std::vector<int32_t> bfs_order(int32_t n, const int32_t *rp, const int32_t *ci)
{
    std::vector<int32_t> order, comp;
    order.reserve(static_cast<size_t>(n));
    std::vector<uint8_t> seen(static_cast<size_t>(n), 0);
    auto search = [&](int32_t src, std::vector<int32_t> &out) {
        size_t head = out.size();
        out.push_back(src);
        seen[src] = 1;
        while (head < out.size()) {
            const int32_t v = out[head++];
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e)
                if (!seen[ci[e]]) {
                    seen[ci[e]] = 1;
                    out.push_back(ci[e]);
                }
        }
    };
    for (int32_t v0 = 0; v0 < n; ++v0) {
        if (seen[v0]) continue;
        comp.clear();
        search(v0, comp);
        for (int32_t v : comp) seen[v] = 0;
        search(comp.back(), order);
    }
    return order;
}

}  // namespace


bool gmrf::pdl_enabled()
{
    static const bool on = [] {
        const char *env = std::getenv("GMRF_PDL");
        return !(env && env[0] == '0');
    }();
    return on;
}

int gmrf::record_error(int st, const char *msg)
{
    g_last_error = msg;
    return st;
}

struct gmrf_sampler {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    // Sweeps with both fused 2-D stages and per-colour stages (disjoint fields) run the per-colour
    // stages on a second stream, forked after the sweep's first stages and joined before the
    // parameter draws.
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    gmrf_model model{};
    gmrf_opts opts{};
    int precision = 0, C = 1, Cp = 1, V = 1;
    int algorithm = GMRF_ALGO_CHROMATIC;
    int nfields = 0;
    int kmax = 0;
    int nparts = 0;
    int64_t slots = 0;
    int64_t max_n = 0;
    std::vector<HostField> hf;
    std::vector<FieldDev> fd;
    std::vector<int32_t> tile_off, tile_cnt;  // per (colour, kind): index colour * 4 + kind
    // Stages of one sweep, in launch order.
    struct Stage {
        int type;    // 0: colour step, 1: fused 2-D lattice sweep, 2: hyperparameter draw,
                     // 3: Polya-Gamma draws (binomial likelihood, first in the sweep)
        int kind;
        int colour;
    };
    std::vector<Stage> stages;
    TileXY *ftiles_dev = nullptr;
    int32_t ftile_off[4] = {0, 0, 0, 0}, ftile_cnt[4] = {0, 0, 0, 0};
    int32_t fTR[4] = {0, 0, 0, 0}, fTC[4] = {0, 0, 0, 0}, fNT[4] = {512, 512, 512, 512};
    // Quad kernel (lattice_quad.cu) for single-chain FP32 8-neighbour lattices: quad columns per
    // staged row (0: not used) and quads per thread.
    int32_t fQCS[4] = {0, 0, 0, 0}, fNQ[4] = {0, 0, 0, 0};
    size_t fsmem_gen[4] = {0, 0, 0, 0};  // the quad tiling's shared memory in lattice_fused_kernel
    size_t fsmem[4] = {0, 0, 0, 0};
    FieldDev *fields_dev = nullptr;
    Tile *tiles_dev = nullptr;
    void *x = nullptr, *y = nullptr, *mean = nullptr, *m2 = nullptr;
    void *x_alt = nullptr;  // second state buffer of fused fields (state of odd sweeps)
    int32_t *rp = nullptr, *ci = nullptr, *perm = nullptr, *perm_inv = nullptr, *coff = nullptr;
    void *w = nullptr, *deg = nullptr;
    double *tau = nullptr, *sig2 = nullptr, *beta = nullptr;
    int32_t *trials = nullptr;  // binomial likelihood: [slots] trials in the colour-split layout
    void *psi = nullptr;        // binomial likelihood: [slots][Cp] Polya-Gamma draws of the sweep
    void *hyp = nullptr;        // [F * Cp][kHypStride] copies in precision T
    Part3 *partials = nullptr;
    double *trace_tau = nullptr, *trace_sig = nullptr, *trace_beta = nullptr;
    SweepCtl *ctl = nullptr;
    double *gpre = nullptr;     // [gpre_batch][F * Cp][4] precomputed variates of a batch
    int32_t gpre_batch = 0;     // sweeps per batch of precomputed variates
    double *staging = nullptr;  // [max_n] doubles for fetch
    double *pool_stage = nullptr;  // [max_n] doubles: the pooled variance of gmrf_fetch_pooled
    double *data_stage = nullptr;    // [max_n][1 + C] doubles: uploads of gmrf_sampler_set_data
    unsigned int *data_flag = nullptr;  // the device checks of those uploads
    int32_t *trials_stage = nullptr; // [max_n] trials uploaded by gmrf_sampler_set_data
    double *diag_work = nullptr;  // [Cp][trace_capacity] scratch of the trace diagnostics
    double *diag_out = nullptr;   // [Cp][4] per-chain results, then the PSRF and a max slot
    void *x_init = nullptr;     // state at creation (for gmrf_sampler_reset)
    double *tau_init = nullptr, *sig2_init = nullptr, *beta_init = nullptr;
    void *hyp_init = nullptr;
    size_t x_bytes = 0, hyp_bytes = 0, nh = 0;
    // plain path
    PlainArgs plain{};
    int32_t *plain_colors = nullptr;
    // graphs: [with_hyper][0: graph_sweeps sweeps, 1: single sweep]
    cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    std::vector<void *> allocs;
    int64_t bytes = 0;
    bool poisoned = false;
    bool test_stall = false;  // GMRF_FLAG_TEST_STALL: the graph cluster kernel's waits run out
    bool restart_pending = false;  // gmrf_sampler_set_data: restart before the state is next used
    int64_t launches_per_sweep = 0;
    // Resident path (lattice_resident.cu): whole sweeps of a small single 2-D lattice field in one
    // launch, one block per chain; 0 when the field takes the per-sweep stages.
    // The 2-D lattice kind whose fused sweep is the only sweep kernel of a sweep (it then starts
    // on a predicted sweep number, see lattice_fused_fast), or -1.
    int early_kind = -1;
    gmrf_tuning tune{};  // launch configuration overrides (zeros: the cost models)
    // 3-D lattice colour steps with every chain of a site in one thread (lattice3d.cu): the
    // padded chain count 4 or 8 when used, 0 when the general colour-step kernel runs them.
    int wide3d = 0;
    // resident: 1 small lattice (one block per chain), 2 graph (a cluster per chain), 3 the quad
    // lattice kernel's tiles kept resident, 4 the fused lattice sweep's tiles kept resident (3, 4:
    // one cooperative launch per batch)
    int resident = 0, res_NI = 0, res_NT = 0, res_batch = 0;
    uint4 *res_nbr = nullptr, *res_nbr2 = nullptr;            // graph: neighbour records
    int res_cluster = 1, res_own_max = 0;                      // graph: blocks per chain, their share
    int res_positions = 0;                                     // graph: 1 = one position per thread
    int32_t res_SR = 0, res_SC = 0;
    size_t res_smem = 0;
    void *res_z = nullptr;  // [res_batch][C][colours][NI][site threads] normals of a batch
    double *res_pm = nullptr;  // fused resident tiles, Cp = 4: the tile partials by field (TileResArgs)

    cudaError_t alloc(void **p, size_t b)
    {
        *p = nullptr;
        if (b == 0) b = 16;
        cudaError_t e = dev_malloc(p, b);
        if (e == cudaSuccess) {
            allocs.push_back(*p);
            bytes += static_cast<int64_t>(b);
        }
        return e;
    }
    template <typename P> cudaError_t alloc_t(P **p, size_t count, size_t elem)
    {
        void *v = nullptr;
        cudaError_t e = alloc(&v, count * elem);
        *p = static_cast<P *>(v);
        return e;
    }
    void release()
    {
        for (auto &row : exec)
            for (auto &g : row)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        if (capture_stream) cudaStreamDestroy(capture_stream);
        capture_stream = nullptr;
        if (side_stream) cudaStreamDestroy(side_stream);
        side_stream = nullptr;
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        ev_fork = ev_join = nullptr;
    }
};

namespace {

size_t tsize(int precision) { return precision == GMRF_FP32 ? sizeof(float) : sizeof(double); }

bool finite(double v) { return std::isfinite(v); }

// ---------------------------------------------------------------------------------------------
// Host validation of a CSR graph: in-range columns, no self-loops, no duplicates, symmetric
// structure and weights, positive finite weights.  Counts connected components (union-find).
// ---------------------------------------------------------------------------------------------
gmrf_status validate_csr(int32_t n, const int32_t *rp, const int32_t *ci, const double *w, int32_t *components)
{
    if (n < 1) return fail(GMRF_E_INVALID, "CSR: n must be >= 1");
    if (!rp || !ci) return fail(GMRF_E_INVALID, "CSR: row_ptr and col_idx are required");
    if (rp[0] != 0) return fail(GMRF_E_INVALID, "CSR: row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return fail(GMRF_E_INVALID, "CSR: row_ptr must be non-decreasing");
    const int64_t nnz = rp[n];
    std::vector<int64_t> keys(static_cast<size_t>(nnz));
    std::vector<int64_t> order(static_cast<size_t>(nnz));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            if (j < 0 || j >= n) return fail(GMRF_E_INVALID, "CSR: column index out of range at row " + std::to_string(i));
            if (j == i) return fail(GMRF_E_INVALID, "CSR: self-loop at row " + std::to_string(i));
            if (w && !(finite(w[e]) && w[e] > 0.0))
                return fail(GMRF_E_INVALID, "CSR: weights must be finite and > 0 (row " + std::to_string(i) + ")");
            keys[e] = static_cast<int64_t>(i) * n + j;
        }
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return keys[a] < keys[b]; });
    for (int64_t k = 1; k < nnz; ++k)
        if (keys[order[k]] == keys[order[k - 1]]) return fail(GMRF_E_INVALID, "CSR: duplicate entry");
    std::vector<int64_t> sorted(static_cast<size_t>(nnz));
    for (int64_t k = 0; k < nnz; ++k) sorted[k] = keys[order[k]];
    for (int64_t k = 0; k < nnz; ++k) {
        const int64_t i = sorted[k] / n, j = sorted[k] % n;
        const int64_t rev = j * n + i;
        auto it = std::lower_bound(sorted.begin(), sorted.end(), rev);
        if (it == sorted.end() || *it != rev) return fail(GMRF_E_INVALID, "CSR: graph is not symmetric");
        if (w && w[order[k]] != w[order[it - sorted.begin()]])
            return fail(GMRF_E_INVALID, "CSR: weights are not symmetric");
    }
    if (components) {
        std::vector<int32_t> parent(static_cast<size_t>(n));
        std::iota(parent.begin(), parent.end(), 0);
        auto find = [&](int32_t v) {
            while (parent[v] != v) {
                parent[v] = parent[parent[v]];
                v = parent[v];
            }
            return v;
        };
        int32_t comps = n;
        for (int32_t i = 0; i < n; ++i)
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
                const int32_t a = find(i), b = find(ci[e]);
                if (a != b) {
                    parent[std::max(a, b)] = std::min(a, b);
                    --comps;
                }
            }
        *components = comps;
    }
    return GMRF_OK;
}

gmrf_status validate_colors(int32_t n, const int32_t *rp, const int32_t *ci, const int32_t *colors, int32_t *k)
{
    int32_t mx = -1;
    for (int32_t i = 0; i < n; ++i) {
        if (colors[i] < 0 || colors[i] >= n) return fail(GMRF_E_INVALID, "colors: value out of range");
        mx = std::max(mx, colors[i]);
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            if (colors[ci[e]] == colors[i]) return fail(GMRF_E_INVALID, "colors: not a proper colouring");
    }
    *k = mx + 1;
    return GMRF_OK;
}

int lattice_colour_host(int kind, const int32_t *dims, int64_t site)
{
    if (kind == GMRF_LATTICE3D_6) {
        const int64_t W = dims[2], H = dims[1];
        return static_cast<int>(((site % W) + ((site / W) % H) + site / (W * H)) & 1);
    }
    const int64_t W = dims[1];
    const int64_t i = site / W, j = site % W;
    if (kind == GMRF_LATTICE2D_8) return static_cast<int>(2 * (i & 1) + (j & 1));
    return static_cast<int>((i + j) & 1);
}

gmrf_status check_model(const gmrf_model *m)
{
    if (!m) return fail(GMRF_E_INVALID, "model is NULL");
    if (m->prior != GMRF_PRIOR_ICAR && m->prior != GMRF_PRIOR_PCAR) return fail(GMRF_E_INVALID, "model.prior");
    if (m->prior == GMRF_PRIOR_PCAR && !(finite(m->rho) && m->rho >= 0.0 && m->rho < 1.0))
        return fail(GMRF_E_INVALID, "model.rho must be in [0, 1) for the proper CAR prior");
    if (!(finite(m->a_tau) && m->a_tau > 0) || !(finite(m->a_sigma) && m->a_sigma > 0))
        return fail(GMRF_E_INVALID, "model: Gamma shapes a_tau, a_sigma must be > 0");
    if (!(finite(m->b_tau) && m->b_tau > 0) || !(finite(m->b_sigma) && m->b_sigma > 0))
        return fail(GMRF_E_INVALID, "model: Gamma rates b_tau, b_sigma must be > 0");
    if (!(finite(m->tau0) && m->tau0 >= 0) || !(finite(m->sigma2_0) && m->sigma2_0 > 0))
        return fail(GMRF_E_INVALID, "model: tau0 >= 0 and sigma2_0 > 0 required");
    if (m->intercept != 0 && m->intercept != 1) return fail(GMRF_E_INVALID, "model.intercept must be 0 or 1");
    if (!finite(m->beta0_0)) return fail(GMRF_E_INVALID, "model.beta0_0 must be finite");
    if (m->likelihood != GMRF_LIKELIHOOD_GAUSSIAN && m->likelihood != GMRF_LIKELIHOOD_BINOMIAL)
        return fail(GMRF_E_INVALID, "model.likelihood");
    if (m->likelihood == GMRF_LIKELIHOOD_BINOMIAL &&
        !(finite(m->beta0_mean) && finite(m->beta0_var) && m->beta0_var > 0))
        return fail(GMRF_E_INVALID, "model: beta0_mean finite and beta0_var > 0 required for binomial data");
    return GMRF_OK;
}

gmrf_status check_opts(const gmrf_opts *o)
{
    if (!o) return fail(GMRF_E_INVALID, "opts is NULL");
    if (o->precision != GMRF_FP32 && o->precision != GMRF_FP64) return fail(GMRF_E_INVALID, "opts.precision");
    if (o->chains < 1 || o->chains > kMaxChains) return fail(GMRF_E_INVALID, "opts.chains must be in 1..64");
    if (o->thin < 1) return fail(GMRF_E_INVALID, "opts.thin must be >= 1");
    if (o->trace_capacity < 1) return fail(GMRF_E_INVALID, "opts.trace_capacity must be >= 1");
    if (o->start_sweep < 0) return fail(GMRF_E_INVALID, "opts.start_sweep must be >= 0");
    if (o->graph_sweeps < 0) return fail(GMRF_E_INVALID, "opts.graph_sweeps must be >= 0");
    if (o->algorithm != GMRF_ALGO_CHROMATIC && o->algorithm != GMRF_ALGO_PLAIN)
        return fail(GMRF_E_INVALID, "opts.algorithm");
    if (const gmrf_tuning *t = o->tuning) {
        int cp = 1;
        while (cp < o->chains) cp <<= 1;
        const int v = t->chains_per_thread;
        if (v != 0 && v != 1 && v != 2 && v != 4) return fail(GMRF_E_INVALID, "tuning.chains_per_thread must be 0, 1, 2 or 4");
        if (v > cp || (o->precision == GMRF_FP64 && v > 2))
            return fail(GMRF_E_INVALID, "tuning.chains_per_thread exceeds the chains (or 2 in FP64)");
        if (t->step_tile != 0 && (t->step_tile < 256 || t->step_tile > 16384))
            return fail(GMRF_E_INVALID, "tuning.step_tile must be 0 or in 256..16384");
        for (int k = 0; k < 2; ++k) {
            const int r = t->fused_rows[k], c = t->fused_cols[k], n = t->fused_threads[k];
            if ((r != 0 && (r < 8 || r > 256)) || (c != 0 && (c < 8 || c > 256)) || ((r == 0) != (c == 0)))
                return fail(GMRF_E_INVALID, "tuning.fused_rows/cols must both be 0 or in 8..256");
            if (n != 0 && n != 512 && n != 1024) return fail(GMRF_E_INVALID, "tuning.fused_threads must be 0, 512 or 1024");
        }
        if (t->quad_config < -1 || t->quad_config > 5) return fail(GMRF_E_INVALID, "tuning.quad_config must be in -1..5");
        if (t->quad_rows != 0 && (t->quad_rows < 8 || (t->quad_rows & 1)))
            return fail(GMRF_E_INVALID, "tuning.quad_rows must be 0 or even and >= 8");
        if (t->wide_3d < -1 || t->wide_3d > 1) return fail(GMRF_E_INVALID, "tuning.wide_3d must be -1, 0 or 1");
        if (t->graph_cluster != 0 && t->graph_cluster != 1 && t->graph_cluster != 2 && t->graph_cluster != 4 &&
            t->graph_cluster != 8 && t->graph_cluster != 16)
            return fail(GMRF_E_INVALID, "tuning.graph_cluster must be 0, 1, 2, 4, 8 or 16");
        if (t->graph_cluster * o->chains > 152) return fail(GMRF_E_INVALID, "tuning.graph_cluster x chains exceeds 152 blocks");
        if (t->wide_3d == 1 && (o->precision != GMRF_FP32 || cp < 4 || cp > 8))
            return fail(GMRF_E_INVALID, "tuning.wide_3d = 1 needs FP32 and 3 to 8 chains");
    }
    return GMRF_OK;
}

gmrf_status check_field(const gmrf_field_desc &f, int idx, int chains, HostField &h)
{
    const std::string at = "field " + std::to_string(idx) + ": ";
    h.kind = f.kind;
    if (f.kind < GMRF_LATTICE2D_4 || f.kind > GMRF_CSR) return fail(GMRF_E_INVALID, at + "unknown kind");
    if (f.kind == GMRF_CSR) {
        h.n = f.n;
        h.dims[0] = f.n;
        gmrf_status st = validate_csr(f.n, f.row_ptr, f.col_idx, f.weights, &h.components);
        if (st != GMRF_OK) return fail(st, at + g_last_error);
        for (int32_t i = 0; i < f.n; ++i) h.max_degree = std::max(h.max_degree, f.row_ptr[i + 1] - f.row_ptr[i]);
        h.weighted = f.weights != nullptr;
        if (f.colors) {
            int32_t k = 0;
            st = validate_colors(f.n, f.row_ptr, f.col_idx, f.colors, &k);
            if (st != GMRF_OK) return fail(st, at + g_last_error);
            h.ncolors = k;
            h.colors.assign(f.colors, f.colors + f.n);
        }
    } else {
        const int nd = f.kind == GMRF_LATTICE3D_6 ? 3 : 2;
        int64_t prod = 1;
        for (int d = 0; d < nd; ++d) {
            if (f.dims[d] < 1) return fail(GMRF_E_INVALID, at + "lattice dims must be >= 1");
            h.dims[d] = f.dims[d];
            prod *= f.dims[d];
        }
        if (prod >= (int64_t(1) << 31)) return fail(GMRF_E_INVALID, at + "lattice has too many sites");
        if (f.n != prod) return fail(GMRF_E_INVALID, at + "n must equal the product of dims");
        h.n = f.n;
        h.ncolors = f.kind == GMRF_LATTICE2D_8 ? 4 : 2;
        h.components = 1;
    }
    if (!f.y) return fail(GMRF_E_INVALID, at + "y is required");
    for (int32_t i = 0; i < h.n; ++i)
        if (!finite(f.y[i])) return fail(GMRF_E_INVALID, at + "y must be finite");
    if (f.x0)
        for (int64_t i = 0; i < static_cast<int64_t>(h.n) * chains; ++i)
            if (!finite(f.x0[i])) return fail(GMRF_E_INVALID, at + "x0 must be finite");
    if (f.tau0)
        for (int c = 0; c < chains; ++c)
            if (!(finite(f.tau0[c]) && f.tau0[c] >= 0)) return fail(GMRF_E_INVALID, at + "tau0 must be >= 0");
    if (f.sigma2_0)
        for (int c = 0; c < chains; ++c)
            if (!(finite(f.sigma2_0[c]) && f.sigma2_0[c] > 0))
                return fail(GMRF_E_INVALID, at + "sigma2_0 must be > 0");
    if (f.beta0)
        for (int c = 0; c < chains; ++c)
            if (!finite(f.beta0[c])) return fail(GMRF_E_INVALID, at + "beta0 must be finite");
    return GMRF_OK;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t _e = (call);                                                                      \
        if (_e != cudaSuccess) throw CudaFail{_e, #call};                                             \
    } while (0)

gmrf_status cuda_status(const CudaFail &f)
{
    const gmrf_status st = (f.err == cudaErrorMemoryAllocation) ? GMRF_E_OOM : GMRF_E_CUDA;
    return fail(st, std::string("CUDA error ") + cudaGetErrorString(f.err) + " in " + f.where);
}

int pow2_at_least(int c)
{
    int p = 1;
    while (p < c) p <<= 1;
    return p;
}

// Upload n doubles from the host into a fresh temporary device buffer (freed by the caller).
double *upload(const double *h, int64_t n, cudaStream_t st, std::vector<void *> &tmp)
{
    void *d = nullptr;
    CK(dev_malloc(&d, sizeof(double) * static_cast<size_t>(n > 0 ? n : 1)));
    tmp.push_back(d);
    CK(cudaMemcpyAsync(d, h, sizeof(double) * static_cast<size_t>(n), cudaMemcpyHostToDevice, st));
    return static_cast<double *>(d);
}

template <typename P> P *upload_t(const P *h, int64_t n, cudaStream_t st, std::vector<void *> &tmp)
{
    void *d = nullptr;
    CK(dev_malloc(&d, sizeof(P) * static_cast<size_t>(n > 0 ? n : 1)));
    tmp.push_back(d);
    if (n > 0) CK(cudaMemcpyAsync(d, h, sizeof(P) * static_cast<size_t>(n), cudaMemcpyHostToDevice, st));
    return static_cast<P *>(d);
}

void free_tmp(std::vector<void *> &tmp)
{
    for (void *p : tmp) cudaFree(p);
    tmp.clear();
}

bool binomial_model(const gmrf_sampler *s) { return s->model.likelihood == GMRF_LIKELIHOOD_BINOMIAL; }
// beta0 is a parameter of the model (the Gaussian intercept, or always with binomial data).
bool has_beta(const gmrf_sampler *s) { return s->model.intercept || binomial_model(s); }

// ---------------------------------------------------------------------------------------------
// Sweep launches
// ---------------------------------------------------------------------------------------------
StepArgs step_args(gmrf_sampler *s, int colour, int kind, int update, int accumulate = 1)
{
    StepArgs a{};
    const size_t slot = static_cast<size_t>(colour) * 4 + kind;
    a.fields = s->fields_dev;
    a.tiles = s->tiles_dev + s->tile_off[slot];
    a.ntiles = s->tile_cnt[slot];
    a.colour = colour;
    a.x = s->x;
    a.y = s->y;
    a.mean = s->mean;
    a.m2 = s->m2;
    a.rp = s->rp;
    a.ci = s->ci;
    a.w = s->w;
    a.deg = s->deg;
    a.perm = s->perm;
    a.coff = s->coff;
    a.hyp = s->hyp;
    a.partials = s->partials;
    a.ctl = s->ctl;
    a.key = philox_key(s->opts.seed);
    philox_round_keys(a.key, a.rk);
    a.Cp = s->Cp;
    a.lanes = std::min(s->Cp, 4);
    a.rho = s->model.prior == GMRF_PRIOR_PCAR ? s->model.rho : 1.0;
    a.burn_in = s->opts.burn_in;
    a.thin = s->opts.thin;
    a.acc_enabled = accumulate;
    a.update = update;
    a.intercept = s->model.intercept ? 1 : 0;
    a.binomial = binomial_model(s) ? 1 : 0;
    a.trials = s->trials;
    a.psi = s->psi;
    return a;
}

HyperArgs hyper_args(gmrf_sampler *s, int draw, int draw_beta, int end_of_sweep)
{
    HyperArgs h{};
    h.fields = s->fields_dev;
    h.nfields = s->nfields;
    h.Cp = s->Cp;
    h.partials = s->partials;
    h.tau = s->tau;
    h.sig2 = s->sig2;
    h.beta = s->beta;
    h.hyp = s->hyp;
    h.trace_tau = s->trace_tau;
    h.trace_sig = s->trace_sig;
    h.trace_beta = has_beta(s) ? s->trace_beta : nullptr;
    h.trace_cap = s->opts.trace_capacity;
    h.ctl = s->ctl;
    h.key = philox_key(s->opts.seed);
    h.a_tau = s->model.a_tau;
    h.b_tau = s->model.b_tau;
    h.a_sig = s->model.a_sigma;
    h.b_sig = s->model.b_sigma;
    h.draw = draw;
    h.draw_beta = has_beta(s) ? draw_beta : 0;
    h.binomial = binomial_model(s) ? 1 : 0;
    h.beta0_mean = s->model.beta0_mean;
    h.beta0_var = s->model.beta0_var;
    h.end_of_sweep = end_of_sweep;
    h.burn_in = s->opts.burn_in;
    h.thin = s->opts.thin;
    h.acc_enabled = 1;
    h.gpre = s->gpre;
    h.max_parts = 0;
    for (int fi = 0; fi < s->nfields; ++fi) h.max_parts = std::max(h.max_parts, s->fd[fi].nparts);
    return h;
}

GammaPreArgs gamma_pre_args(gmrf_sampler *s, int count)
{
    GammaPreArgs g{};
    g.fields = s->fields_dev;
    g.nfields = s->nfields;
    g.Cp = s->Cp;
    g.ctl = s->ctl;
    g.key = philox_key(s->opts.seed);
    g.a_tau = s->model.a_tau;
    g.a_sig = s->model.a_sigma;
    g.count = count;
    g.intercept = has_beta(s) ? 1 : 0;
    g.gpre = s->gpre;
    return g;
}

cudaError_t launch_pre(gmrf_sampler *s, int count, cudaStream_t st)
{
    return launch_gamma_pre(gamma_pre_args(s, count), st);
}

// The resident tile forms, for a single 2-D lattice field whose per-sweep kernel's tiles can all be
// resident at once (one block each): the quad kernel's (single-chain FP32 8-neighbour fields), else
// the fused sweep's when it runs the fast form (FP32, every thread holding all chains).
cudaError_t plan_tile_resident(gmrf_sampler *s)
{
    const int kind = s->fd[0].kind;
    if (kind != GMRF_LATTICE2D_4 && kind != GMRF_LATTICE2D_8) return cudaSuccess;
    bool fits = false;
    if (s->fQCS[kind]) {
        const cudaError_t e = lattice_quad_resident_fits(s->fQCS[kind], s->fNT[kind], s->fNQ[kind], s->fsmem[kind],
                                                         s->ftile_cnt[kind], &fits);
        if (e != cudaSuccess || !fits) return e;
        s->res_batch = std::min(128, std::max(64, s->opts.graph_sweeps));
        s->resident = 3;
        return cudaSuccess;
    }
    if (s->precision != GMRF_FP32 || s->V != s->Cp || (s->Cp != 1 && s->Cp != 2 && s->Cp != 4)) return cudaSuccess;
    const cudaError_t e = lattice_fused_resident_fits(kind, s->fNT[kind], s->Cp, s->fsmem[kind], s->ftile_cnt[kind],
                                                      &fits);
    if (e != cudaSuccess || !fits) return e;
    if (s->Cp == 4) {
        const cudaError_t ea = s->alloc_t(&s->res_pm, static_cast<size_t>(3) * s->Cp * s->ftile_cnt[kind], sizeof(double));
        if (ea != cudaSuccess) return ea;
    }
    s->res_batch = std::min(128, std::max(64, s->opts.graph_sweeps));
    s->resident = 4;
    return cudaSuccess;
}

// The resident path applies to a single fused 2-D lattice field with the Gaussian likelihood whose
// chain fits in shared memory (state, observations, mean and M2 with a ring of zeros: cells below
// 2^16, sites below 2^16) and whose colour classes have at most 2 x 576 (8-neighbour) or 4 x 576
// (4-neighbour) positions; a larger FP32 field takes the resident form of its per-sweep kernel (the
// quad kernel, or the fused sweep's fast form) when its tiles fit in one wave.  It is the default
// for FP32 samplers; GMRF_FLAG_RESIDENT asks for the small-lattice form in FP64 too and
// GMRF_FLAG_NO_RESIDENT switches all off.
cudaError_t plan_resident(gmrf_sampler *s, const std::vector<int32_t> &coff0)
{
    s->resident = 0;
    const int flags = s->opts.flags;
    if (s->algorithm == GMRF_ALGO_PLAIN || s->nfields != 1 || binomial_model(s)) return cudaSuccess;
    if (flags & GMRF_FLAG_NO_RESIDENT) return cudaSuccess;
    if (s->precision != GMRF_FP32 && !(flags & GMRF_FLAG_RESIDENT)) return cudaSuccess;
    const FieldDev &f = s->fd[0];
    const int batch = std::min(128, std::max(64, s->opts.graph_sweeps));
    if (f.kind == GMRF_CSR) {
        // Graph: unit weights, 16-bit positions, at most 16 neighbours and 64 colours, every class
        // within the site threads' positions, and state, mean and M2 in shared memory.
        const HostField &h = s->hf[0];
        if (h.weighted || f.n >= 32768 || h.max_degree > 16 || h.ncolors > 64 || coff0.size() != size_t(h.ncolors) + 1)
            return cudaSuccess;
        // A cluster of CL blocks per chain (at most 152 blocks in all): one block per 2048 sites.
        int cl = 1;
        while (cl < 8 && f.n >= 2048 * 2 * cl && s->C * 2 * cl <= 152) cl *= 2;
        if (s->tune.graph_cluster) cl = s->tune.graph_cluster;
        int own_max = 0, share_max = 0;
        for (int c = 0; c < h.ncolors; ++c) {
            const int len = coff0[c + 1] - coff0[c], q = (len + cl - 1) / cl;
            if (q > csr_resident_max_positions()) return cudaSuccess;
            own_max += q;
            share_max = std::max(share_max, q);
        }
        const size_t smem = (static_cast<size_t>(f.n) + 1 + 2 * static_cast<size_t>(own_max)) * tsize(s->precision);
        if (smem > 220 * 1024) return cudaSuccess;
        cudaError_t e = prepare_csr_resident(s->precision, smem);
        if (e == cudaSuccess) e = s->alloc_t(&s->res_nbr, static_cast<size_t>(f.n), sizeof(uint4));
        if (e == cudaSuccess) e = s->alloc_t(&s->res_nbr2, static_cast<size_t>(f.n), sizeof(uint4));
        if (e == cudaSuccess)
            e = launch_pack_csr_records(f.n, s->rp + f.rp0, s->ci + f.nnz0, s->res_nbr, s->res_nbr2, s->stream);
        if (e == cudaSuccess) e = s->alloc(&s->res_z, static_cast<size_t>(batch) * s->C * f.n * tsize(s->precision));
        if (e != cudaSuccess) return e;
        s->res_batch = batch;
        if (s->test_stall) {
            // After its wait gives up a block no longer announces the bytes the other blocks send it;
            // a launch's unannounced bytes stay below the transaction count's range.
            const int64_t per_sweep = static_cast<int64_t>(f.n) * static_cast<int64_t>(tsize(s->precision));
            s->res_batch = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(batch, (int64_t(1) << 19) / per_sweep)));
        }
        s->res_smem = smem;
        s->res_cluster = cl;
        s->res_own_max = own_max;
        s->res_positions = share_max <= csr_resident_site_threads() ? 1 : 0;
        s->resident = 2;
        return cudaSuccess;
    }
    if (!s->hf[0].fused) return cudaSuccess;
    if (f.kind != GMRF_LATTICE2D_4 && f.kind != GMRF_LATTICE2D_8) return cudaSuccess;
    const bool e8 = f.kind == GMRF_LATTICE2D_8;
    const int K = e8 ? 4 : 2;
    const int64_t SR = f.rows + 2, SC = f.cols + 2, cells = K * SR * SC;
    // positions per colour class: the largest class (8-neighbour) or rows x columns (4-neighbour)
    const int64_t maxq = e8 ? static_cast<int64_t>((f.dims[0] + 1) / 2) * ((f.dims[1] + 1) / 2)
                            : static_cast<int64_t>(f.dims[0]) * f.cols;
    // up to 640 site threads with one position per class each, or 576 with 2 or 4 (4-neighbour
    // lattice only)
    int NI = 0;
    for (int ni : {1, 2, 4})
        if (!NI && (ni < 4 || !e8) && (maxq + ni - 1) / ni <= (ni == 1 ? 640 : 576)) NI = ni;
    if (!NI || cells >= 65536 || f.n >= 65536) return plan_tile_resident(s);
    int NTS = static_cast<int>((maxq + NI - 1) / NI);
    NTS = (NTS + 31) / 32 * 32;
    const size_t smem = 4 * static_cast<size_t>(cells) * tsize(s->precision) + 8 * static_cast<size_t>(K) * NI * NTS;
    if (smem > 220 * 1024) return plan_tile_resident(s);  // with the static reduction scratch, under 227 KiB
    const int NT = NTS + 64;  // and the two drawing warps
    cudaError_t e = prepare_lattice_resident(s->precision, f.kind, NI, smem);
    if (e != cudaSuccess) return e;
    // Sweeps per launch: the Gamma-variate batch, at most 128 (the normals buffer holds a batch).
    e = s->alloc(&s->res_z, static_cast<size_t>(batch) * s->C * K * NI * NTS * tsize(s->precision));
    if (e != cudaSuccess) return e;
    s->res_batch = batch;
    s->resident = 1;
    s->res_NI = NI;
    s->res_NT = NT;
    s->res_SR = static_cast<int32_t>(SR);
    s->res_SC = static_cast<int32_t>(SC);
    s->res_smem = smem;
    return cudaSuccess;
}

ResidentArgs resident_args(gmrf_sampler *s, int count, int draw, int draw_beta)
{
    ResidentArgs r{};
    r.fields = s->fields_dev;
    r.h = hyper_args(s, draw, draw_beta, 1);
    r.x = s->x;
    r.x_alt = s->x_alt;
    r.y = s->y;
    r.mean = s->mean;
    r.m2 = s->m2;
    r.count = count;
    r.SR = s->res_SR;
    r.SC = s->res_SC;
    r.lanes = std::min(s->Cp, 4);
    r.C = s->C;
    r.rho = s->model.prior == GMRF_PRIOR_PCAR ? s->model.rho : 1.0;
    r.zbuf = s->res_z;
    return r;
}

ResCsrArgs csr_resident_args(gmrf_sampler *s, int count, int draw, int draw_beta)
{
    ResCsrArgs r{};
    r.fields = s->fields_dev;
    r.h = hyper_args(s, draw, draw_beta, 1);
    r.x = s->x;
    r.y = s->y;
    r.mean = s->mean;
    r.m2 = s->m2;
    r.nbr = s->res_nbr;
    r.nbr2 = s->res_nbr2;
    r.coff = s->coff + s->fd[0].coff0;
    r.ncolors = s->hf[0].ncolors;
    r.count = count;
    r.C = s->C;
    r.own_max = s->res_own_max;
    r.rho = s->model.prior == GMRF_PRIOR_PCAR ? s->model.rho : 1.0;
    r.zbuf = s->res_z;
    r.extra_bytes = s->test_stall ? 16u : 0u;
    r.wait_ns = s->test_stall ? 1000000ull : kWaitNs;
    return r;
}

// The batch's normals for the resident kernels and, with `gamma`, its Gamma variates (one launch).
cudaError_t launch_res_normals(gmrf_sampler *s, int count, bool gamma, cudaStream_t st)
{
    ResNormArgs r{};
    if (gamma) {
        r.g = gamma_pre_args(s, count);
        r.gamma_blocks = (count * s->nfields * s->Cp * 4 + 63) / 64;
    }
    r.fields = s->fields_dev;
    r.ctl = s->ctl;
    r.key = philox_key(s->opts.seed);
    r.lanes = std::min(s->Cp, 4);
    r.C = s->C;
    r.Cp = s->Cp;
    r.count = count;
    r.NI = s->res_NI;
    r.NTS = s->res_NT - 64;
    r.perm_inv = s->resident == 2 ? s->perm_inv : nullptr;
    r.out = s->res_z;
    const int gs = r.lanes == 4 ? 0 : (r.lanes == 2 ? 1 : 2);
    const int64_t groups = (static_cast<int64_t>(s->fd[0].n) + (1 << gs) - 1) >> gs;
    const int64_t quads = r.lanes == 4 ? s->Cp / 4 : 1;
    return launch_resident_normals(s->precision, r, groups * quads * count, st);
}

FusedArgs fused_args(gmrf_sampler *s, int kind, int update, int accumulate)
{
    FusedArgs a{};
    a.fields = s->fields_dev;
    a.tiles = s->ftiles_dev + s->ftile_off[kind];
    a.ntiles = s->ftile_cnt[kind];
    a.TR = s->fTR[kind];
    a.TC = s->fTC[kind];
    a.threads = s->fNT[kind];
    const int K = kind == GMRF_LATTICE2D_8 ? 4 : 2;
    fast_div_magic(static_cast<uint32_t>(a.TC + 2 * K), a.rc_m, a.rc_s);
    fast_div_magic(static_cast<uint32_t>(a.TC > 0 ? a.TC : 1), a.tc_m, a.tc_s);
    a.lanes = std::min(s->Cp, 4);
    const int gs = a.lanes == 4 ? 0 : (a.lanes == 2 ? 1 : 2);
    fast_div_magic(static_cast<uint32_t>(((a.TC + 2 * K) >> gs) + 2), a.ng_m, a.ng_s);
    a.x = s->x;
    a.x_alt = s->x_alt;
    a.y = s->y;
    a.mean = s->mean;
    a.m2 = s->m2;
    a.hyp = s->hyp;
    a.partials = s->partials;
    a.ctl = s->ctl;
    a.key = philox_key(s->opts.seed);
    a.Cp = s->Cp;
    a.rho = s->model.prior == GMRF_PRIOR_PCAR ? s->model.rho : 1.0;
    a.burn_in = s->opts.burn_in;
    a.thin = s->opts.thin;
    a.acc_enabled = accumulate;
    a.update = update;
    a.early = (update && kind == s->early_kind) ? 1 : 0;
    return a;
}

TileResArgs tile_resident_args(gmrf_sampler *s, int count, int draw, int draw_beta)
{
    TileResArgs r{};
    r.f = fused_args(s, s->fd[0].kind, 1, 1);
    r.h = hyper_args(s, draw, draw_beta, 1);
    r.count = count;
    r.pm = s->res_pm;
    r.extra_arrivals = s->test_stall ? 1u : 0u;
    r.wait_ns = s->test_stall ? 1000000ull : kWaitNs;
    return r;
}

// One stage of a sweep (see gmrf_launch_stage); `draw`, `draw_beta` and `end_of_sweep` only
// matter for the hyperparameter stage.
// Description of stage k of a sweep (also its NVTX range name).
const char *stage_name(const gmrf_sampler *s, size_t k)
{
    static const char *kNames[4][4] = {
        {"colour step, 2-D 4-neighbour lattice", "colour step, 2-D 8-neighbour lattice",
         "colour step, 3-D 6-neighbour lattice", "colour step, CSR graph"},
        {"fused sweep, 2-D 4-neighbour lattice", "fused sweep, 2-D 8-neighbour lattice", "", ""},
        {"hyperparameter draw", "hyperparameter draw", "hyperparameter draw", "hyperparameter draw"},
        {"Polya-Gamma draws", "Polya-Gamma draws", "Polya-Gamma draws", "Polya-Gamma draws"}};
    const gmrf_sampler::Stage &g = s->stages[k];
    if (g.type == 1 && s->fQCS[g.kind]) return "fused quad sweep, 2-D 8-neighbour lattice";
    if (g.type == 0 && g.kind == GMRF_LATTICE3D_6 && s->wide3d)
        return "colour step, 3-D 6-neighbour lattice, all chains of a site per thread";
    return kNames[g.type][g.kind < 0 ? 0 : g.kind];
}

// An NVTX range around the host-side enqueue of a stage (and of a call), for timeline tools.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

cudaError_t enqueue_stage(gmrf_sampler *s, size_t k, int update, int accumulate, int draw, int draw_beta,
                          int end_of_sweep, cudaStream_t st)
{
    const NvtxRange range(stage_name(s, k));
    const gmrf_sampler::Stage &g = s->stages[k];
    if (g.type == 1) {
        FusedArgs fa = fused_args(s, g.kind, update, accumulate);
        if (s->fQCS[g.kind]) {
            if (update) return launch_lattice_quad(s->fQCS[g.kind], s->fNT[g.kind], s->fNQ[g.kind], fa, s->fsmem[g.kind], st);
            fa.threads = 1024;
            return launch_lattice_fused(s->precision, s->V, g.kind, fa, s->fsmem_gen[g.kind], st);
        }
        return launch_lattice_fused(s->precision, s->V, g.kind, fa, s->fsmem[g.kind], st);
    }
    if (g.type == 0 && g.kind == GMRF_LATTICE3D_6 && s->wide3d)
        return launch_lattice3d(s->wide3d, step_args(s, g.colour, g.kind, update, accumulate), st);
    if (g.type == 0)
        return launch_colour_step(s->precision, s->V, g.kind, step_args(s, g.colour, g.kind, update, accumulate), st);
    if (g.type == 3) {
        if (!update) return cudaSuccess;
        PgArgs p{};
        p.fields = s->fields_dev;
        p.nfields = s->nfields;
        p.slots = s->slots;
        p.Cp = s->Cp;
        p.C = s->C;
        p.x = s->x;
        p.hyp = s->hyp;
        p.trials = s->trials;
        p.perm = s->perm;
        p.psi = s->psi;
        p.ctl = s->ctl;
        p.key = philox_key(s->opts.seed);
        return launch_pg_stage(s->precision, p, st);
    }
    return launch_hyper(s->precision, hyper_args(s, draw, draw_beta, end_of_sweep), st);
}

// Sweeps with (with_hyper = 1) or without the draws of tau, sigma^2 (unless fixed) and beta0
// (with the intercept).
cudaError_t enqueue_sweeps(gmrf_sampler *s, int nsweeps, int with_hyper, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    const int draw = (with_hyper && !s->model.fix_hyper) ? 1 : 0;
    const int draw_beta = (with_hyper && has_beta(s)) ? 1 : 0;
    if (s->resident) {
        // Batches of sweeps: the batch's unit-rate Gamma variates and normals, then all its sweeps
        // in one launch.
        static const char *kBatch[5] = {"", "resident batch, lattice", "resident batch, graph",
                                        "resident batch, quad lattice", "resident batch, fused lattice"};
        for (int k = 0; k < nsweeps && e == cudaSuccess;) {
            const NvtxRange range(kBatch[s->resident]);
            const int cnt = std::min(s->res_batch, nsweeps - k);
            if (s->resident >= 3) {
                // the tile kernels draw their own normals
                if (draw || draw_beta) e = launch_pre(s, cnt, st);
                const int kd = s->fd[0].kind;
                const TileResArgs ra = tile_resident_args(s, cnt, draw, draw_beta);
                if (e == cudaSuccess && s->resident == 3)
                    e = launch_lattice_quad_resident(s->fQCS[kd], s->fNT[kd], s->fNQ[kd], ra, s->fsmem[kd], st);
                else if (e == cudaSuccess)
                    e = launch_lattice_fused_resident(kd, s->fNT[kd], s->Cp, ra, s->fsmem[kd], st);
                k += cnt;
                continue;
            }
            // the batch's normals and, when drawn, its Gamma variates
            e = launch_res_normals(s, cnt, draw || draw_beta, st);
            if (e == cudaSuccess && s->resident == 2)
                e = launch_csr_resident(s->precision, s->res_cluster, s->res_positions, s->C,
                                        csr_resident_args(s, cnt, draw, draw_beta), s->res_smem, st);
            else if (e == cudaSuccess)
                e = launch_lattice_resident(s->precision, s->fd[0].kind, s->res_NI, s->res_NT, s->C,
                                            resident_args(s, cnt, draw, draw_beta), s->res_smem, st);
            k += cnt;
        }
        return e;
    }
    for (int k = 0; k < nsweeps && e == cudaSuccess; ++k) {
        // A batch of sweeps starts with the parallel draw of its unit-rate Gamma variates.
        if ((draw || draw_beta) && s->gpre && k % s->gpre_batch == 0)
            e = launch_pre(s, std::min(s->gpre_batch, nsweeps - k), st);
        if (e != cudaSuccess) break;
        if (s->algorithm == GMRF_ALGO_PLAIN) {
            PlainArgs a = s->plain;
            a.draw = draw;
            int64_t l = 0;
            e = launch_plain_sweep(a, st, &l);
            continue;
        }
        if (s->side_stream) {
            // Fused 2-D stages on `st`, per-colour stages (in their order) on the side stream, then
            // the draws after both; a Polya-Gamma stage (all fields) runs before the fork.
            size_t k = 0;
            for (; k < s->stages.size() && e == cudaSuccess && s->stages[k].type == 3; ++k)
                e = enqueue_stage(s, k, 1, 1, draw, draw_beta, 1, st);
            if (e == cudaSuccess) e = cudaEventRecord(s->ev_fork, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side_stream, s->ev_fork, 0);
            for (size_t q = k; q < s->stages.size() && e == cudaSuccess; ++q)
                if (s->stages[q].type == 0) e = enqueue_stage(s, q, 1, 1, draw, draw_beta, 1, s->side_stream);
            for (size_t q = k; q < s->stages.size() && e == cudaSuccess; ++q)
                if (s->stages[q].type == 1) e = enqueue_stage(s, q, 1, 1, draw, draw_beta, 1, st);
            if (e == cudaSuccess) e = cudaEventRecord(s->ev_join, s->side_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->ev_join, 0);
            for (size_t q = k; q < s->stages.size() && e == cudaSuccess; ++q)
                if (s->stages[q].type == 2) e = enqueue_stage(s, q, 1, 1, draw, draw_beta, 1, st);
            continue;
        }
        for (size_t k = 0; k < s->stages.size() && e == cudaSuccess; ++k)
            e = enqueue_stage(s, k, 1, 1, draw, draw_beta, 1, st);
    }
    return e;
}

cudaError_t get_graph(gmrf_sampler *s, int with_hyper, int which, int nsweeps, cudaGraphExec_t *out)
{
    if (s->exec[with_hyper][which]) {
        *out = s->exec[with_hyper][which];
        return cudaSuccess;
    }
    cudaError_t e = cudaStreamBeginCapture(s->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = enqueue_sweeps(s, nsweeps, with_hyper, s->capture_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->capture_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&s->exec[with_hyper][which], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    *out = s->exec[with_hyper][which];
    return cudaSuccess;
}

gmrf_status poison(gmrf_sampler *s, cudaError_t e, const char *where)
{
    s->poisoned = true;
    return cuda_status(CudaFail{e, where});
}

// A bounded device wait that gave up (counted in the sweep control block) makes the results since
// invalid: the call reports it and the sampler is poisoned.
gmrf_status check_waits(gmrf_sampler *s, const SweepCtl &c)
{
    if (c.wait_timeouts == 0) return GMRF_OK;
    s->poisoned = true;
    return fail(GMRF_E_TIMEOUT, "a bounded device wait gave up (" + std::to_string(c.wait_timeouts) +
                                    " times): the results of the sweeps since are invalid");
}

gmrf_status build_plain(gmrf_sampler *s, const gmrf_field_desc &f, std::vector<void *> &tmp)
{
    HostField &h = s->hf[0];
    const int64_t n = h.n;
    PlainArgs &a = s->plain;
    a.n = h.n;
    a.kind = h.kind;
    for (int d = 0; d < 3; ++d) a.dims[d] = h.dims[d];
    a.C = s->C;
    a.lanes = std::min(pow2_at_least(s->C), 4);
    a.rho = s->model.prior == GMRF_PRIOR_PCAR ? s->model.rho : 1.0;
    a.rank = s->model.prior == GMRF_PRIOR_PCAR ? h.n : h.n - h.components;
    a.a_tau = s->model.a_tau;
    a.b_tau = s->model.b_tau;
    a.a_sig = s->model.a_sigma;
    a.b_sig = s->model.b_sigma;
    a.key = philox_key(s->opts.seed);
    a.stream_id = f.stream_id;
    a.trace_cap = s->opts.trace_capacity;
    a.ncolors = h.ncolors;
    double *x = nullptr, *y = nullptr;
    CK(s->alloc_t(&x, static_cast<size_t>(n) * s->C, sizeof(double)));
    CK(s->alloc_t(&y, static_cast<size_t>(n), sizeof(double)));
    CK(cudaMemcpyAsync(y, f.y, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
    for (int c = 0; c < s->C; ++c)
        CK(cudaMemcpyAsync(x + c * n, f.x0 ? f.x0 + c * n : f.y, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
    a.x = x;
    a.y = y;
    if (h.kind == GMRF_CSR) {
        int32_t *rp = nullptr, *ci = nullptr;
        const int64_t nnz = f.row_ptr[h.n];
        CK(s->alloc_t(&rp, static_cast<size_t>(n + 1), sizeof(int32_t)));
        CK(s->alloc_t(&ci, static_cast<size_t>(nnz), sizeof(int32_t)));
        CK(cudaMemcpyAsync(rp, f.row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(ci, f.col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s->stream));
        a.rp = rp;
        a.ci = ci;
        if (f.weights) {
            double *w = nullptr;
            CK(s->alloc_t(&w, static_cast<size_t>(nnz), sizeof(double)));
            CK(cudaMemcpyAsync(w, f.weights, sizeof(double) * nnz, cudaMemcpyHostToDevice, s->stream));
            a.w = w;
        }
        CK(s->alloc_t(&s->plain_colors, static_cast<size_t>(n), sizeof(int32_t)));
        if (h.colors.empty()) {
            void *scratch = nullptr;
            CK(dev_malloc(&scratch, jp_scratch_bytes(h.n)));
            tmp.push_back(scratch);
            int32_t k = 0;
            CK(jp_color(h.n, rp, ci, nullptr, f.color_seed, s->plain_colors, scratch, &k, s->stream,
                        (s->opts.flags & GMRF_FLAG_COLOR_RANDOM) == 0));
            h.ncolors = k;
            a.ncolors = k;
            h.colors.resize(static_cast<size_t>(n));
            CK(cudaMemcpyAsync(h.colors.data(), s->plain_colors, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream));
        } else {
            CK(cudaMemcpyAsync(s->plain_colors, h.colors.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream));
        }
        a.colors = s->plain_colors;
    }
    CK(s->alloc_t(&a.tau, static_cast<size_t>(s->C), sizeof(double)));
    CK(s->alloc_t(&a.sig2, static_cast<size_t>(s->C), sizeof(double)));
    std::vector<double> t0(s->C), s0(s->C);
    for (int c = 0; c < s->C; ++c) {
        t0[c] = f.tau0 ? f.tau0[c] : s->model.tau0;
        s0[c] = f.sigma2_0 ? f.sigma2_0[c] : s->model.sigma2_0;
    }
    CK(cudaMemcpyAsync(a.tau, t0.data(), sizeof(double) * s->C, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(a.sig2, s0.data(), sizeof(double) * s->C, cudaMemcpyHostToDevice, s->stream));
    CK(s->alloc_t(&a.trace_tau, static_cast<size_t>(s->C) * s->opts.trace_capacity, sizeof(double)));
    CK(s->alloc_t(&a.trace_sig, static_cast<size_t>(s->C) * s->opts.trace_capacity, sizeof(double)));
    s->nh = static_cast<size_t>(s->C);
    s->x_bytes = sizeof(double) * static_cast<size_t>(n) * s->C;
    CK(s->alloc(&s->x_init, s->x_bytes));
    CK(cudaMemcpyAsync(s->x_init, x, s->x_bytes, cudaMemcpyDeviceToDevice, s->stream));
    CK(s->alloc_t(&s->tau_init, s->nh, sizeof(double)));
    CK(s->alloc_t(&s->sig2_init, s->nh, sizeof(double)));
    CK(cudaMemcpyAsync(s->tau_init, a.tau, s->nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->sig2_init, a.sig2, s->nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    CK(s->alloc_t(&a.red, static_cast<size_t>(s->C) * 2, sizeof(double)));
    CK(cudaMemsetAsync(a.red, 0, sizeof(double) * 2 * s->C, s->stream));
    a.ctl = s->ctl;
    s->kmax = h.ncolors;
    s->launches_per_sweep = h.ncolors + (s->model.fix_hyper ? 1 : 2);
    s->tau = a.tau;
    s->sig2 = a.sig2;
    s->trace_tau = a.trace_tau;
    s->trace_sig = a.trace_sig;
    return GMRF_OK;
}

gmrf_status build_chromatic(gmrf_sampler *s, const gmrf_field_desc *fields, std::vector<void *> &tmp)
{
    const size_t T = tsize(s->precision);
    // Field geometry and offsets.
    int64_t slots = 0, csr_sites = 0, csr_rp = 0, csr_nnz = 0, coff_n = 0;
    bool any_weights = false;
    s->fd.resize(s->nfields);
    for (int fi = 0; fi < s->nfields; ++fi) {
        HostField &h = s->hf[fi];
        FieldDev &d = s->fd[fi];
        std::memset(&d, 0, sizeof(d));
        d.kind = h.kind;
        d.n = h.n;
        d.stream = fields[fi].stream_id;
        for (int k = 0; k < 3; ++k) d.dims[k] = h.dims[k];
        d.rank = s->model.prior == GMRF_PRIOR_PCAR ? h.n : h.n - h.components;
        d.slot0 = slots;
        if (h.kind == GMRF_CSR) {
            d.nslots = h.n;
            d.csr0 = csr_sites;
            d.rp0 = csr_rp;
            d.nnz0 = csr_nnz;
            d.coff0 = coff_n;
            csr_sites += h.n;
            csr_rp += h.n + 1;
            csr_nnz += fields[fi].row_ptr[h.n];
            coff_n += std::max<int64_t>(h.n, 1) + 1;  // room for up to n colours
            any_weights = any_weights || fields[fi].weights;
        } else {
            if (h.kind == GMRF_LATTICE2D_8) {
                d.rows = (h.dims[0] + 1) / 2;
                d.cols = (h.dims[1] + 1) / 2;
            } else if (h.kind == GMRF_LATTICE3D_6) {
                d.rows = h.dims[0] * h.dims[1];
                d.cols = (h.dims[2] + 1) / 2;
            } else {
                d.rows = h.dims[0];
                d.cols = (h.dims[1] + 1) / 2;
            }
            d.ncolors = h.ncolors;
            d.nslots = static_cast<int64_t>(h.ncolors) * d.rows * d.cols;
            fast_div_magic(static_cast<uint32_t>(d.cols), d.cols_m, d.cols_s);
            fast_div_magic(static_cast<uint32_t>(h.kind == GMRF_LATTICE3D_6 ? h.dims[1] : 1), d.h_m, d.h_s);
        }
        slots += d.nslots;
        s->max_n = std::max<int64_t>(s->max_n, h.n);
        if (d.nslots * s->Cp >= (int64_t(1) << 31))
            return fail(GMRF_E_INVALID, "field " + std::to_string(fi) + ": sites x chains must be < 2^31");
    }
    if (csr_nnz >= (int64_t(1) << 31)) return fail(GMRF_E_INVALID, "total CSR entries must be < 2^31");
    s->slots = slots;
    const size_t Cp = static_cast<size_t>(s->Cp);
    CK(s->alloc(&s->x, static_cast<size_t>(slots) * Cp * T));
    CK(s->alloc(&s->y, static_cast<size_t>(slots) * T));
    CK(s->alloc(&s->mean, static_cast<size_t>(slots) * Cp * T));
    CK(s->alloc(&s->m2, static_cast<size_t>(slots) * Cp * T));
    CK(cudaMemsetAsync(s->x, 0, static_cast<size_t>(slots) * Cp * T, s->stream));
    CK(cudaMemsetAsync(s->y, 0, static_cast<size_t>(slots) * T, s->stream));
    CK(cudaMemsetAsync(s->mean, 0, static_cast<size_t>(slots) * Cp * T, s->stream));
    CK(cudaMemsetAsync(s->m2, 0, static_cast<size_t>(slots) * Cp * T, s->stream));
    if (csr_sites > 0) {
        CK(s->alloc_t(&s->rp, static_cast<size_t>(csr_rp), sizeof(int32_t)));
        CK(s->alloc_t(&s->ci, static_cast<size_t>(csr_nnz), sizeof(int32_t)));
        CK(s->alloc_t(&s->perm, static_cast<size_t>(csr_sites), sizeof(int32_t)));
        CK(s->alloc_t(&s->perm_inv, static_cast<size_t>(csr_sites), sizeof(int32_t)));
        CK(s->alloc_t(&s->coff, static_cast<size_t>(coff_n), sizeof(int32_t)));
        CK(s->alloc(&s->deg, static_cast<size_t>(csr_sites) * T));
        if (any_weights) CK(s->alloc(&s->w, static_cast<size_t>(csr_nnz) * T));
    }
    CK(s->alloc_t(&s->fields_dev, static_cast<size_t>(s->nfields), sizeof(FieldDev)));

    // CSR fields: upload, colour (JP unless given), colour-permuted layout.  Each colour class is
    // ordered breadth-first (neighbouring sites in nearby positions: the per-colour kernels'
    // gathers touch fewer sectors, measured 6 % faster on 15 K- and 50 K-site graphs), except for
    // a single graph small enough for the resident kernel, which measured 3 % faster with the
    // classes in natural order (its shared-memory gathers spread over the banks).
    const bool natural_classes = s->nfields == 1 && s->hf[0].kind == GMRF_CSR && s->hf[0].n < 32768 &&
                                 !binomial_model(s) && !(s->opts.flags & GMRF_FLAG_NO_RESIDENT) &&
                                 (s->precision == GMRF_FP32 || (s->opts.flags & GMRF_FLAG_RESIDENT));
    std::vector<std::vector<int32_t>> coff_host(s->nfields);
    for (int fi = 0; fi < s->nfields; ++fi) {
        HostField &h = s->hf[fi];
        FieldDev &d = s->fd[fi];
        if (h.kind != GMRF_CSR) continue;
        const gmrf_field_desc &f = fields[fi];
        const int64_t nnz = f.row_ptr[h.n];
        int32_t *rp_d = upload_t(f.row_ptr, h.n + 1, s->stream, tmp);
        int32_t *ci_d = upload_t(f.col_idx, nnz, s->stream, tmp);
        double *w_d = f.weights ? upload(f.weights, nnz, s->stream, tmp) : nullptr;
        int32_t *col_d = nullptr;
        {
            void *p = nullptr;
            CK(dev_malloc(&p, sizeof(int32_t) * h.n));
            tmp.push_back(p);
            col_d = static_cast<int32_t *>(p);
        }
        if (h.colors.empty()) {
            void *scratch = nullptr;
            CK(dev_malloc(&scratch, jp_scratch_bytes(h.n)));
            tmp.push_back(scratch);
            int32_t k = 0;
            CK(jp_color(h.n, rp_d, ci_d, nullptr, f.color_seed, col_d, scratch, &k, s->stream,
                        (s->opts.flags & GMRF_FLAG_COLOR_RANDOM) == 0));
            h.ncolors = k;
            h.colors.resize(h.n);
            CK(cudaMemcpyAsync(h.colors.data(), col_d, sizeof(int32_t) * h.n, cudaMemcpyDeviceToHost, s->stream));
        } else {
            CK(cudaMemcpyAsync(col_d, h.colors.data(), sizeof(int32_t) * h.n, cudaMemcpyHostToDevice, s->stream));
        }
        if (h.ncolors > 1024) return fail(GMRF_E_UNSUPPORTED, "CSR colouring with more than 1024 colours");
        d.ncolors = h.ncolors;
        void *scratch = nullptr;
        CK(dev_malloc(&scratch, layout_scratch_bytes(h.n, h.ncolors)));
        tmp.push_back(scratch);
        char *wbase = any_weights && f.weights ? static_cast<char *>(s->w) + d.nnz0 * T : nullptr;
        int32_t *order_d = nullptr;
        if (!natural_classes && h.n > 0) {
            const std::vector<int32_t> order = bfs_order(h.n, f.row_ptr, f.col_idx);
            order_d = upload_t(order.data(), h.n, s->stream, tmp);
        }
        CK(csr_layout(s->precision, h.n, h.ncolors, rp_d, ci_d, w_d, col_d, order_d, scratch, s->perm + d.csr0,
                      s->perm_inv + d.csr0, s->coff + d.coff0, s->rp + d.rp0, s->ci + d.nnz0, wbase,
                      static_cast<char *>(s->deg) + d.csr0 * T, s->stream));
        coff_host[fi].resize(h.ncolors + 1);
        CK(cudaMemcpyAsync(coff_host[fi].data(), s->coff + d.coff0, sizeof(int32_t) * (h.ncolors + 1),
                           cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (!f.weights && any_weights) {
            // Unit weights for this field inside a batch where another field has weights.
            std::vector<char> ones(static_cast<size_t>(nnz) * T);
            for (int64_t k = 0; k < nnz; ++k) {
                if (s->precision == GMRF_FP32) reinterpret_cast<float *>(ones.data())[k] = 1.0f;
                else reinterpret_cast<double *>(ones.data())[k] = 1.0;
            }
            CK(cudaMemcpyAsync(static_cast<char *>(s->w) + d.nnz0 * T, ones.data(), ones.size(), cudaMemcpyHostToDevice,
                               s->stream));
            CK(cudaStreamSynchronize(s->stream));
        }
    }

    // Tiles: per colour, each field's colour class cut into tiles of `target` (site, chain
    // vector) elements, sized so a colour step has several blocks per SM (at least one element
    // per thread, so small classes spread over many SMs, and at most 16384 elements per tile);
    // partial-sum slots are contiguous per field.
    const int CV = s->Cp / s->V;
    // 2-D lattice fields take the fused sweep when a tile of at least 16 x 16 sites with its
    // halo (state, normals and y) fits the 72 KiB shared-memory budget (3 blocks per SM) and it
    // is not switched off.
    bool fused_kind[4] = {false, false, false, false};
    const bool allow_fused = (s->opts.flags & GMRF_FLAG_PER_COLOUR) == 0 && !binomial_model(s);
    for (int kind : {static_cast<int>(GMRF_LATTICE2D_4), static_cast<int>(GMRF_LATTICE2D_8)}) {
        const int K = kind == GMRF_LATTICE2D_8 ? 4 : 2;
        const double per_site = static_cast<double>(T) * (2 * s->Cp + 1);
        int side = static_cast<int>(std::floor(std::sqrt(72.0 * 1024.0 / per_site))) - 2 * K;
        side = std::min(64, side - side % 8);
        if (!allow_fused || side < 16) continue;
        for (auto &h : s->hf)
            if (h.kind == kind) fused_kind[kind] = true;
        // Quad kernel: one chain, FP32, every field of the kind with a row length that is a
        // multiple of 4 (Philox blocks then never straddle rows).
        bool quad_ok = kind == GMRF_LATTICE2D_8 && s->Cp == 1 && s->precision == GMRF_FP32 && fused_kind[kind];
        for (auto &h : s->hf)
            if (h.kind == kind && h.dims[1] % 4 != 0) quad_ok = false;
        if (s->tune.quad_config < 0) quad_ok = false;
        if (quad_ok) {
            // Configurations (quad columns, threads, quads per thread); tile TR x TC with
            // TC = 2 qcs - 8 and (TR/2 + 4) qcs <= threads * quads per thread (68 quad columns:
            // TC = 128, eight tiles across a 1024-wide lattice).  Cost, compared in order (fitted
            // to measured sweeps of 130 x 1000 to 2048 x 2048 lattices): tilings that fit in one
            // wave (one block per SM) first; among those the fewest quads per thread (a thread's
            // quads are its serial path through the latency-bound steps), then more threads per
            // block, then fewer staged quads; with several waves, the fewest waves times staged
            // quads per block (the work of the busiest SM).
            static const int cfg[5][3] = {{64, 768, 3}, {64, 1024, 2}, {32, 1024, 2}, {32, 512, 2}, {68, 704, 3}};
            double best[4] = {1e300, 0, 0, 0};
            int bq = 0, bn = 0, bm = 0, btr = 0;
            for (int ci = 0; ci < 5; ++ci) {
                if (s->tune.quad_config > 0 && ci != s->tune.quad_config - 1) continue;
                const int *cf = cfg[ci];
                const int qcs = cf[0], nt = cf[1], nq = cf[2];
                const int qr_max = nq * nt / qcs;
                const int tc = 2 * qcs - 8;
                for (int tr = 8; (tr / 2 + 4) <= qr_max; tr += 2) {
                    if (lattice_quad_smem(qcs, tr) > 200 * 1024) break;
                    if (s->tune.quad_rows && tr != s->tune.quad_rows) continue;
                    int64_t tiles = 0;
                    for (auto &h : s->hf)
                        if (h.kind == kind) tiles += static_cast<int64_t>((h.dims[0] + tr - 1) / tr) * ((h.dims[1] + tc - 1) / tc);
                    const int quads = (tr / 2 + 4) * qcs;
                    const double waves = std::ceil(static_cast<double>(tiles) / 152.0);
                    const double per_thread = std::ceil(static_cast<double>(quads) / nt);
                    const double cost[4] = {waves > 1 ? 1.0 : 0.0, waves > 1 ? waves * quads : per_thread,
                                            -static_cast<double>(nt), static_cast<double>(quads)};
                    if (std::lexicographical_compare(cost, cost + 4, best, best + 4)) {
                        std::copy(cost, cost + 4, best);
                        bq = qcs;
                        bn = nt;
                        bm = nq;
                        btr = tr;
                    }
                }
            }
            if (bq == 0 && s->tune.quad_rows)
                return fail(GMRF_E_INVALID, "tuning.quad_rows does not fit the quad configuration");
            if (bq > 0) {
                s->fQCS[kind] = bq;
                s->fNQ[kind] = bm;
                s->fNT[kind] = bn;
                s->fTR[kind] = btr;
                s->fTC[kind] = 2 * bq - 8;
                s->fsmem[kind] = lattice_quad_smem(bq, btr);
                CK(prepare_lattice_quad(bq, bn, bm, s->fsmem[kind]));
                // Reduce-only passes (gmrf_hyper_update) run lattice_fused_kernel on the same tiles.
                s->fsmem_gen[kind] = lattice_fused_smem(s->precision, kind, s->Cp, btr, 2 * bq - 8);
                CK(prepare_lattice_fused(s->precision, s->V, kind, s->fsmem_gen[kind]));
                continue;
            }
        }
        if (fused_kind[kind]) {
            int tr = side, tc = side;
            // Cost model over tile shapes and block sizes: waves of blocks (152 SMs, one block of
            // 1024 or two of 512 threads per SM) times the sites a wave computes per SM, halo
            // recomputation included, plus a fixed cost per block (staging, barriers, reduction)
            // worth 1024 site updates (fitted to measured 20 x 22 and 64 x 64 tilings of many
            // small lattices).  Deterministic, so a sampler's tiling (and with it the rounding of
            // the tile partial sums) does not change from run to run.
            double best = 1e300;
            for (int nt : {512, 1024}) {
                // blocks per SM: two of 512 threads where the kernel is compiled for 64 registers
                // (FP32 with up to two chains per thread), else one (four chains keep 128)
                const int bps = (nt == 512 && s->precision == GMRF_FP32 && s->Cp < 4) ? 2 : 1;
                for (int cr = 16; cr <= 160; cr += 2)
                    for (int cc = 16; cc <= 128; cc += 2) {
                        const size_t sm = lattice_fused_smem(s->precision, kind, s->Cp, cr, cc);
                        if (sm * bps > 200 * 1024 || static_cast<int64_t>(cr + 2 * K) * (cc + 2 * K) * s->Cp >= 65536)
                            continue;
                        int64_t tiles = 0;
                        for (auto &h : s->hf)
                            if (h.kind == kind)
                                tiles += static_cast<int64_t>((h.dims[0] + cr - 1) / cr) * ((h.dims[1] + cc - 1) / cc);
                        double work = 1024.0;  // per block: fixed cost + sites computed over the K steps
                        for (int e = 0; e < K; ++e) work += static_cast<double>(cr + 2 * e) * (cc + 2 * e) / K;
                        const double waves = std::ceil(static_cast<double>(tiles) / (152.0 * bps));
                        const double cost = waves * bps * work;
                        if (cost < best * 0.999) {
                            best = cost;
                            tr = cr;
                            tc = cc;
                            s->fNT[kind] = nt;
                        }
                    }
            }
            if (s->tune.fused_rows[kind]) {
                const int r = s->tune.fused_rows[kind] & ~1, c = s->tune.fused_cols[kind] & ~1;
                const int nt = s->tune.fused_threads[kind] ? s->tune.fused_threads[kind] : s->fNT[kind];
                if (lattice_fused_smem(s->precision, kind, s->Cp, r, c) > 200 * 1024 ||
                    static_cast<int64_t>(r + 2 * K) * (c + 2 * K) * (s->Cp / s->V) >= 65536)
                    return fail(GMRF_E_INVALID, "tuning: the fused tile does not fit shared memory");
                tr = r;
                tc = c;
                s->fNT[kind] = nt;
            } else if (s->tune.fused_threads[kind]) {
                s->fNT[kind] = s->tune.fused_threads[kind];
            }
            // The kernel's flattened loops divide indices below 2^16 by one float multiply.
            while (static_cast<int64_t>(tr + 2 * K) * (tc + 2 * K) * (s->Cp / s->V) >= 65536 && tr > 8) tr -= 8;
            s->fTR[kind] = tr;
            s->fTC[kind] = tc;
            s->fsmem[kind] = lattice_fused_smem(s->precision, kind, s->Cp, tr, tc);
            CK(prepare_lattice_fused(s->precision, s->V, kind, s->fsmem[kind]));
        }
    }
    int64_t total_elems = 0;
    for (int fi = 0; fi < s->nfields; ++fi)
        if (!fused_kind[s->hf[fi].kind]) total_elems += static_cast<int64_t>(s->hf[fi].n) * CV;
    const int64_t per_colour = total_elems / 2;
    const int64_t target = s->tune.step_tile ? s->tune.step_tile
                                             : std::min<int64_t>(16384, std::max<int64_t>(kBlock, per_colour / (152 * 4)));
    // 3-D lattices with every chain of a site in one thread: FP32, 4 or 8 chains (padded), the
    // Gaussian likelihood, and either asked for (tuning.wide_3d = 1) or, by default, colour
    // classes of at least one site for each of 256 threads on every SM.  A launch is then one
    // wave of blocks (the blocks resident per SM times the SMs), each field getting blocks in
    // proportion to its sites; block k of a field takes its sub-array rows k, k + nt, k + 2 nt,
    // ... (nt blocks), so that at any time all blocks work on a narrow band of rows and the rows
    // a plane apart that a site reads are read from DRAM once, by whichever block comes first.
    std::vector<int32_t> tiles3d(s->nfields, 0);
    {
        int64_t sites3d = 0;
        for (auto &h : s->hf)
            if (h.kind == GMRF_LATTICE3D_6) sites3d += h.n;
        const bool able = s->precision == GMRF_FP32 && (s->Cp == 4 || s->Cp == 8) && !binomial_model(s) && sites3d > 0;
        int nsm = 0;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device));
        bool use = false;
        if (s->tune.wide_3d == 1) use = able;
        else if (s->tune.wide_3d == 0 && s->tune.chains_per_thread == 0) use = able && sites3d / 2 >= int64_t(nsm) * 256;
        if (use) {
            int bps = 1;
            CK(lattice3d_blocks_per_sm(s->Cp, &bps));
            int64_t units = 0;  // sub-array sites per colour over the 3-D fields
            for (int fi = 0; fi < s->nfields; ++fi)
                if (s->fd[fi].kind == GMRF_LATTICE3D_6) units += static_cast<int64_t>(s->fd[fi].rows) * s->fd[fi].cols;
            // one wave, unless that leaves fewer than one site per thread
            const int64_t goal = std::max<int64_t>(1, std::min<int64_t>(int64_t(nsm) * bps, units / 256));
            for (int fi = 0; fi < s->nfields; ++fi) {
                const FieldDev &d = s->fd[fi];
                if (d.kind != GMRF_LATTICE3D_6) continue;
                const double share = static_cast<double>(d.rows) * d.cols / static_cast<double>(units);
                tiles3d[fi] = static_cast<int32_t>(std::max<int64_t>(
                    1, std::min<int64_t>(d.rows, std::llround(share * static_cast<double>(goal)))));
            }
            s->wide3d = s->Cp;
        }
    }
    s->kmax = 0;
    for (auto &h : s->hf) s->kmax = std::max(s->kmax, h.ncolors);
    std::vector<std::vector<Tile>> by_colour(s->kmax);
    std::vector<TileXY> fz[4];
    int part = 0;
    for (int fi = 0; fi < s->nfields; ++fi) {
        FieldDev &d = s->fd[fi];
        d.part0 = part;
        if (fused_kind[d.kind]) {
            s->hf[fi].fused = true;
            for (int i0 = 0; i0 < d.dims[0]; i0 += s->fTR[d.kind])
                for (int j0 = 0; j0 < d.dims[1]; j0 += s->fTC[d.kind]) {
                    TileXY t{};
                    t.field = fi;
                    t.i0 = i0;
                    t.j0 = j0;
                    t.part = part++;
                    fz[d.kind].push_back(t);
                }
            d.nparts = part - d.part0;
            continue;
        }
        for (int c = 0; c < d.ncolors; ++c) {
            if (d.kind == GMRF_CSR) {
                const int32_t lo = coff_host[fi][c], hi = coff_host[fi][c + 1];
                const int64_t per = std::max<int64_t>(1, target / CV);
                for (int64_t st = lo; st < hi; st += per) {
                    Tile t{};
                    t.field = fi;
                    t.colour = c;
                    t.start = static_cast<int32_t>(st);
                    t.count = static_cast<int32_t>(std::min<int64_t>(per, hi - st));
                    t.part = part++;
                    by_colour[c].push_back(t);
                }
            } else if (tiles3d[fi] > 0) {
                const int32_t nt = tiles3d[fi];
                for (int32_t k = 0; k < nt; ++k) {
                    Tile t{};
                    t.field = fi;
                    t.colour = c;
                    t.start = k;
                    t.count = (d.rows - k + nt - 1) / nt;
                    t.stride = nt;
                    t.part = part++;
                    by_colour[c].push_back(t);
                }
            } else {
                const int64_t per = std::max<int64_t>(1, target / (static_cast<int64_t>(d.cols) * CV));
                for (int64_t st = 0; st < d.rows; st += per) {
                    Tile t{};
                    t.field = fi;
                    t.colour = c;
                    t.start = static_cast<int32_t>(st);
                    t.count = static_cast<int32_t>(std::min<int64_t>(per, d.rows - st));
                    t.part = part++;
                    by_colour[c].push_back(t);
                }
            }
        }
        d.nparts = part - d.part0;
    }
    s->nparts = part;
    // Stages: fused lattice sweeps first (their fields do not interact with the others within a
    // sweep), then colour steps in colour order, one launch per field kind, then the draw.
    s->stages.clear();
    std::vector<TileXY> fall;
    for (int kind = 0; kind < 4; ++kind) {
        s->ftile_off[kind] = static_cast<int32_t>(fall.size());
        s->ftile_cnt[kind] = static_cast<int32_t>(fz[kind].size());
        fall.insert(fall.end(), fz[kind].begin(), fz[kind].end());
        if (!fz[kind].empty()) s->stages.push_back({1, kind, -1});
    }
    std::vector<Tile> all;
    s->tile_off.assign(static_cast<size_t>(s->kmax) * 4, 0);
    s->tile_cnt.assign(static_cast<size_t>(s->kmax) * 4, 0);
    for (int c = 0; c < s->kmax; ++c)
        for (int kind = 0; kind < 4; ++kind) {
            const size_t slot = static_cast<size_t>(c) * 4 + kind;
            s->tile_off[slot] = static_cast<int32_t>(all.size());
            for (const Tile &t : by_colour[c])
                if (s->fd[t.field].kind == kind) all.push_back(t);
            s->tile_cnt[slot] = static_cast<int32_t>(all.size()) - s->tile_off[slot];
            if (s->tile_cnt[slot] > 0) s->stages.push_back({0, kind, c});
        }
    s->stages.push_back({2, -1, -1});
    if (binomial_model(s)) s->stages.insert(s->stages.begin(), {3, -1, -1});
    s->launches_per_sweep = static_cast<int64_t>(s->stages.size());
    {
        int sweep_kernels = 0, kind = -1;
        for (const auto &st : s->stages)
            if (st.type != 2) {
                ++sweep_kernels;
                kind = st.type == 1 ? st.kind : -2;
            }
        s->early_kind = (sweep_kernels == 1 && kind >= 0) ? kind : -1;
    }
    CK(plan_resident(s, coff_host[0]));
    {
        // fused 2-D stages and per-colour stages in one sweep: the latter get a side stream
        bool fused = false, step = false;
        for (const auto &st : s->stages) {
            fused |= st.type == 1;
            step |= st.type == 0;
        }
        if (fused && step && !s->resident) {
            CK(cudaStreamCreateWithFlags(&s->side_stream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
        }
    }
    CK(s->alloc_t(&s->tiles_dev, std::max<size_t>(all.size(), 1), sizeof(Tile)));
    if (!all.empty())
        CK(cudaMemcpyAsync(s->tiles_dev, all.data(), sizeof(Tile) * all.size(), cudaMemcpyHostToDevice, s->stream));
    if (!fall.empty()) CK(s->alloc(&s->x_alt, static_cast<size_t>(slots) * Cp * T));
    CK(s->alloc_t(&s->ftiles_dev, std::max<size_t>(fall.size(), 1), sizeof(TileXY)));
    if (!fall.empty())
        CK(cudaMemcpyAsync(s->ftiles_dev, fall.data(), sizeof(TileXY) * fall.size(), cudaMemcpyHostToDevice,
                           s->stream));
    CK(s->alloc_t(&s->partials, static_cast<size_t>(std::max(part, 1)) * Cp, sizeof(Part3)));
    CK(cudaMemsetAsync(s->partials, 0, static_cast<size_t>(std::max(part, 1)) * Cp * sizeof(Part3), s->stream));
    CK(cudaMemcpyAsync(s->fields_dev, s->fd.data(), sizeof(FieldDev) * s->nfields, cudaMemcpyHostToDevice, s->stream));

    // y and x0 into the colour-split layout.
    for (int fi = 0; fi < s->nfields; ++fi) {
        const gmrf_field_desc &f = fields[fi];
        const HostField &h = s->hf[fi];
        double *y_d = upload(f.y, h.n, s->stream, tmp);
        double *x0_d = f.x0 ? upload(f.x0, static_cast<int64_t>(h.n) * s->C, s->stream, tmp) : nullptr;
        if (!f.x0 && binomial_model(s)) {  // binomial: x0 = 0 (the logit scale) unless given
            const std::vector<double> zeros(static_cast<size_t>(h.n) * s->C, 0.0);
            x0_d = upload(zeros.data(), static_cast<int64_t>(h.n) * s->C, s->stream, tmp);
            CK(cudaStreamSynchronize(s->stream));
        }
        if (binomial_model(s)) {
            if (!s->trials) {
                CK(s->alloc(&s->psi, static_cast<size_t>(std::max<int64_t>(s->slots, 1)) * s->Cp * T));
                CK(s->alloc_t(&s->trials, static_cast<size_t>(std::max<int64_t>(s->slots, 1)), sizeof(int32_t)));
                CK(cudaMemsetAsync(s->trials, 0, sizeof(int32_t) * static_cast<size_t>(std::max<int64_t>(s->slots, 1)),
                                   s->stream));
            }
            int32_t *m_d = upload_t(f.trials, h.n, s->stream, tmp);
            CK(launch_pack_int(s->fields_dev, s->fd[fi], fi, m_d, s->perm_inv, s->trials, s->stream));
        }
        CK(launch_pack(s->precision, s->fields_dev, s->fd[fi], fi, s->C, s->Cp, y_d, x0_d, s->perm_inv, s->x, s->y,
                       s->stream));
    }

    // Hyperparameters and their precision-T copies.
    const size_t nh = static_cast<size_t>(s->nfields) * Cp;
    std::vector<double> t0(nh), s0(nh), b0(nh);
    std::vector<char> hypT(nh * kHypStride * T, 0);
    for (int fi = 0; fi < s->nfields; ++fi)
        for (int c = 0; c < s->Cp; ++c) {
            const size_t k = static_cast<size_t>(fi) * Cp + c;
            const gmrf_field_desc &f = fields[fi];
            t0[k] = (f.tau0 && c < s->C) ? f.tau0[c] : s->model.tau0;
            s0[k] = (f.sigma2_0 && c < s->C) ? f.sigma2_0[c] : s->model.sigma2_0;
            b0[k] = !has_beta(s) ? 0.0 : ((f.beta0 && c < s->C) ? f.beta0[c] : s->model.beta0_0);
            const double v[3] = {t0[k], 1.0 / s0[k], b0[k]};
            for (int q = 0; q < 3; ++q) {
                if (s->precision == GMRF_FP32) reinterpret_cast<float *>(hypT.data())[kHypStride * k + q] = static_cast<float>(v[q]);
                else reinterpret_cast<double *>(hypT.data())[kHypStride * k + q] = v[q];
            }
        }
    CK(s->alloc_t(&s->tau, nh, sizeof(double)));
    CK(s->alloc_t(&s->sig2, nh, sizeof(double)));
    CK(s->alloc_t(&s->beta, nh, sizeof(double)));
    s->gpre_batch = std::max(64, s->opts.graph_sweeps);
    CK(s->alloc_t(&s->gpre, static_cast<size_t>(s->gpre_batch) * nh * 4, sizeof(double)));
    CK(s->alloc(&s->hyp, nh * kHypStride * T));
    CK(cudaMemcpyAsync(s->tau, t0.data(), nh * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->sig2, s0.data(), nh * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->beta, b0.data(), nh * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->hyp, hypT.data(), hypT.size(), cudaMemcpyHostToDevice, s->stream));
    CK(s->alloc_t(&s->trace_tau, nh * s->opts.trace_capacity, sizeof(double)));
    CK(s->alloc_t(&s->trace_sig, nh * s->opts.trace_capacity, sizeof(double)));
    if (has_beta(s)) CK(s->alloc_t(&s->trace_beta, nh * s->opts.trace_capacity, sizeof(double)));
    CK(s->alloc_t(&s->diag_work, static_cast<size_t>(Cp) * s->opts.trace_capacity, sizeof(double)));
    CK(s->alloc_t(&s->diag_out, static_cast<size_t>(Cp) * 4 + 2, sizeof(double)));
    // Initial state kept for gmrf_sampler_reset.
    s->nh = nh;
    s->x_bytes = static_cast<size_t>(slots) * Cp * T;
    s->hyp_bytes = nh * kHypStride * T;
    CK(s->alloc(&s->x_init, s->x_bytes));
    CK(cudaMemcpyAsync(s->x_init, s->x, s->x_bytes, cudaMemcpyDeviceToDevice, s->stream));
    if (s->x_alt) CK(cudaMemcpyAsync(s->x_alt, s->x, s->x_bytes, cudaMemcpyDeviceToDevice, s->stream));
    CK(s->alloc_t(&s->tau_init, nh, sizeof(double)));
    CK(s->alloc_t(&s->sig2_init, nh, sizeof(double)));
    CK(s->alloc_t(&s->beta_init, nh, sizeof(double)));
    CK(s->alloc(&s->hyp_init, s->hyp_bytes));
    CK(cudaMemcpyAsync(s->tau_init, s->tau, nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->sig2_init, s->sig2, nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->beta_init, s->beta, nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->hyp_init, s->hyp, s->hyp_bytes, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return GMRF_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
namespace {

// The restart of gmrf_sampler_reset (stream-ordered): states from x_init, parameters from their
// initial values, running moments and counters cleared.
gmrf_status restart_state(gmrf_sampler *s)
{
    s->restart_pending = false;
    try {
        const bool plain = s->algorithm == GMRF_ALGO_PLAIN;
        void *x = plain ? static_cast<void *>(s->plain.x) : s->x;
        CK(cudaMemcpyAsync(x, s->x_init, s->x_bytes, cudaMemcpyDeviceToDevice, s->stream));
        if (s->x_alt) CK(cudaMemcpyAsync(s->x_alt, s->x_init, s->x_bytes, cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(s->tau, s->tau_init, s->nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(s->sig2, s->sig2_init, s->nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
        if (!plain) {
            CK(cudaMemcpyAsync(s->beta, s->beta_init, s->nh * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
            CK(cudaMemcpyAsync(s->hyp, s->hyp_init, s->hyp_bytes, cudaMemcpyDeviceToDevice, s->stream));
            CK(cudaMemsetAsync(s->mean, 0, s->x_bytes, s->stream));
            CK(cudaMemsetAsync(s->m2, 0, s->x_bytes, s->stream));
        }
        CK(launch_ctl_reset(s->ctl, s->opts.start_sweep, s->stream));
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    return GMRF_OK;
}

// A restart requested by gmrf_sampler_set_data, before a call that uses the sampler's state.
gmrf_status restart_if_pending(gmrf_sampler *s) { return s->restart_pending ? restart_state(s) : GMRF_OK; }

}  // namespace

extern "C" {

const char *gmrf_last_error(void) { return g_last_error.c_str(); }

const char *gmrf_version(void) { return "0.1.0"; }

gmrf_status gmrf_validate_csr(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *weights,
                              int32_t *components)
{
    g_last_error.clear();
    return validate_csr(n, row_ptr, col_idx, weights, components);
}

gmrf_status gmrf_color_graph(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *priorities,
                             uint64_t seed, int32_t *colors, int32_t *num_colors)
{
    g_last_error.clear();
    if (!colors || !num_colors) return fail(GMRF_E_INVALID, "colors and num_colors are required");
    gmrf_status st = validate_csr(n, row_ptr, col_idx, nullptr, nullptr);
    if (st != GMRF_OK) return st;
    std::vector<void *> tmp;
    try {
        cudaStream_t stream = nullptr;
        int32_t *rp = upload_t(row_ptr, n + 1, stream, tmp);
        int32_t *ci = upload_t(col_idx, row_ptr[n], stream, tmp);
        uint32_t *pr = priorities ? upload_t(priorities, n, stream, tmp) : nullptr;
        void *col = nullptr, *scratch = nullptr;
        CK(dev_malloc(&col, sizeof(int32_t) * n));
        tmp.push_back(col);
        CK(dev_malloc(&scratch, jp_scratch_bytes(n)));
        tmp.push_back(scratch);
        int32_t k = 0;
        CK(jp_color(n, rp, ci, pr, seed, static_cast<int32_t *>(col), scratch, &k, stream));
        CK(cudaMemcpy(colors, col, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        *num_colors = k;
    } catch (const CudaFail &f) {
        free_tmp(tmp);
        return cuda_status(f);
    }
    free_tmp(tmp);
    return GMRF_OK;
}

gmrf_status gmrf_sampler_create(gmrf_sampler **out, const gmrf_field_desc *fields, int32_t nfields,
                                const gmrf_model *model, const gmrf_opts *opts, void *cuda_stream)
{
    g_last_error.clear();
    if (!out) return fail(GMRF_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!fields || nfields < 1) return fail(GMRF_E_INVALID, "at least one field is required");
    gmrf_status st = check_model(model);
    if (st != GMRF_OK) return st;
    if ((st = check_opts(opts)) != GMRF_OK) return st;
    std::vector<HostField> hf(nfields);
    for (int i = 0; i < nfields; ++i)
        if ((st = check_field(fields[i], i, opts->chains, hf[i])) != GMRF_OK) return st;
    if (model->likelihood == GMRF_LIKELIHOOD_BINOMIAL)
        for (int i = 0; i < nfields; ++i) {
            const std::string at = "field " + std::to_string(i) + ": ";
            if (!fields[i].trials) return fail(GMRF_E_INVALID, at + "binomial data need trials");
            for (int32_t k = 0; k < hf[i].n; ++k) {
                const int32_t m = fields[i].trials[k];
                if (m < 0 || m > 4095) return fail(GMRF_E_INVALID, at + "trials must be in 0..4095");
                if (!(fields[i].y[k] >= 0.0 && fields[i].y[k] <= m))
                    return fail(GMRF_E_INVALID, at + "successes y must be in [0, trials]");
            }
        }
    if (opts->algorithm == GMRF_ALGO_PLAIN && (nfields != 1 || opts->precision != GMRF_FP64))
        return fail(GMRF_E_UNSUPPORTED, "the plain sweep takes exactly one field in FP64");
    if (opts->algorithm == GMRF_ALGO_PLAIN && (model->intercept || model->likelihood != GMRF_LIKELIHOOD_GAUSSIAN))
        return fail(GMRF_E_UNSUPPORTED, "the plain sweep has neither the intercept nor the binomial likelihood");

    gmrf_sampler *s = new gmrf_sampler();
    s->model = *model;
    s->opts = *opts;
    if (opts->tuning) s->tune = *opts->tuning;
    s->opts.tuning = nullptr;  // no caller memory is retained
    s->test_stall = (opts->flags & GMRF_FLAG_TEST_STALL) != 0;
    s->precision = opts->precision;
    s->C = opts->chains;
    s->Cp = pow2_at_least(opts->chains);
    s->V = std::min(s->Cp, opts->precision == GMRF_FP32 ? 4 : 2);
    {
        // Samplers whose sweeps are per-colour launches only (3-D lattices, graphs): when a step
        // has too few (site, chain group) elements to fill the GPU (below 2048 threads on each of
        // the 152 SMs, four times over), fewer chains per thread give more threads.  (Fused 2-D
        // sweeps keep all chains in a thread: their fast kernel needs it.)
        bool lattice2d = false;
        int64_t sites = 0;
        for (const HostField &h : hf) {
            lattice2d |= (h.kind == GMRF_LATTICE2D_4 || h.kind == GMRF_LATTICE2D_8) &&
                         !(opts->flags & GMRF_FLAG_PER_COLOUR);
            sites += h.n;
        }
        while (!lattice2d && s->V > 1 && sites * s->Cp / s->V < int64_t(152) * 2048 * 4) s->V >>= 1;
    }
    if (s->tune.chains_per_thread) s->V = s->tune.chains_per_thread;
    s->algorithm = opts->algorithm;
    s->nfields = nfields;
    s->hf = std::move(hf);
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    std::vector<void *> tmp;
    try {
        CK(cudaGetDevice(&s->device));
        CK(cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking));
        CK(s->alloc_t(&s->ctl, 1, sizeof(SweepCtl)));
        SweepCtl c0{};
        c0.sweep = opts->start_sweep;
        CK(cudaMemcpyAsync(s->ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, s->stream));
        if (s->algorithm == GMRF_ALGO_PLAIN) st = build_plain(s, fields[0], tmp);
        else st = build_chromatic(s, fields, tmp);
        if (st == GMRF_OK) {
            s->max_n = 0;
            for (auto &h : s->hf) s->max_n = std::max<int64_t>(s->max_n, h.n);
            CK(s->alloc_t(&s->staging, static_cast<size_t>(s->max_n), sizeof(double)));
            if (s->algorithm != GMRF_ALGO_PLAIN)
                CK(s->alloc_t(&s->pool_stage, static_cast<size_t>(s->max_n), sizeof(double)));
            CK(cudaStreamSynchronize(s->stream));
        }
    } catch (const CudaFail &f) {
        st = cuda_status(f);
    }
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_tmp(tmp);
    if (st != GMRF_OK) {
        const std::string msg = g_last_error;
        s->release();
        delete s;
        g_last_error = msg;
        return st;
    }
    *out = s;
    return GMRF_OK;
}

void gmrf_sampler_destroy(gmrf_sampler *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    s->release();
    delete s;
}

gmrf_status gmrf_sweep(gmrf_sampler *s, int32_t nsweeps, int32_t with_hyper)
{
    const NvtxRange range("gmrf_sweep");
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (nsweeps < 0) return fail(GMRF_E_INVALID, "nsweeps must be >= 0");
    const int wh = with_hyper ? 1 : 0;
    cudaError_t e = cudaSuccess;
    const int G = s->opts.graph_sweeps;
    if (G <= 0) {
        e = enqueue_sweeps(s, nsweeps, wh, s->stream);
        if (e != cudaSuccess) return poison(s, e, "sweep launch");
        return GMRF_OK;
    }
    int remaining = nsweeps;
    if (remaining >= G) {
        cudaGraphExec_t g = nullptr;
        if ((e = get_graph(s, wh, 0, G, &g)) != cudaSuccess) return poison(s, e, "graph capture");
        while (remaining >= G) {
            if ((e = cudaGraphLaunch(g, s->stream)) != cudaSuccess) return poison(s, e, "graph launch");
            remaining -= G;
        }
    }
    if (remaining > 0) {
        cudaGraphExec_t g1 = nullptr;
        if ((e = get_graph(s, wh, 1, 1, &g1)) != cudaSuccess) return poison(s, e, "graph capture");
        for (; remaining > 0; --remaining)
            if ((e = cudaGraphLaunch(g1, s->stream)) != cudaSuccess) return poison(s, e, "graph launch");
    }
    return GMRF_OK;
}

gmrf_status gmrf_hyper_update(gmrf_sampler *s)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (s->algorithm == GMRF_ALGO_PLAIN) return fail(GMRF_E_UNSUPPORTED, "hyper_update on the plain sweep");
    if (binomial_model(s)) return fail(GMRF_E_UNSUPPORTED, "hyper_update with the binomial likelihood");
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < s->stages.size() && e == cudaSuccess; ++k)
        if (s->stages[k].type != 2) e = enqueue_stage(s, k, 0, 0, 0, 0, 0, s->stream);
    if (e == cudaSuccess) e = launch_hyper(s->precision, hyper_args(s, 1, 1, 0), s->stream);
    if (e != cudaSuccess) return poison(s, e, "hyper update launch");
    return GMRF_OK;
}

gmrf_status gmrf_fetch_samples(gmrf_sampler *s, int32_t field, int32_t chain, double *x_last, double *x_mean,
                               double *x_var, int64_t trace_cap, double *tau_trace, double *sigma2_trace,
                               int64_t *n_trace, double *tau_now, double *sigma2_now)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (field < 0 || field >= s->nfields || chain < 0 || chain >= s->C)
        return fail(GMRF_E_INVALID, "field or chain out of range");
    if (trace_cap < 0) return fail(GMRF_E_INVALID, "trace_cap must be >= 0");
    const HostField &h = s->hf[field];
    const int64_t n = h.n;
    try {
        SweepCtl c{};
        CK(cudaMemcpyAsync(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (const gmrf_status w = check_waits(s, c)) return w;
        const bool plain = s->algorithm == GMRF_ALGO_PLAIN;
        const int64_t k = plain ? 0 : c.acc_count;
        auto fetch = [&](const void *src, const void *m2, double scale, double *dst) {
            if (plain) {
                CK(cudaMemcpyAsync(dst, s->plain.x + chain * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
                return;
            }
            CK(launch_unpack(s->precision, s->fields_dev, s->fd[field], field, s->Cp, chain, src, m2, scale, s->perm_inv,
                             s->staging, s->stream));
            CK(cudaMemcpyAsync(dst, s->staging, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        };
        // Fused fields keep the state at the start of sweep t in buffer t & 1.
        void *xcur = (h.fused && (c.sweep & 1)) ? s->x_alt : s->x;
        if (x_last) fetch(xcur, nullptr, 1.0, x_last);
        if (x_mean) {
            if (plain || k < 1) std::fill(x_mean, x_mean + n, plain ? NAN : 0.0);
            else fetch(s->mean, nullptr, 1.0, x_mean);
        }
        if (x_var) {
            if (plain || k < 2) std::fill(x_var, x_var + n, NAN);
            else fetch(nullptr, s->m2, 1.0 / static_cast<double>(k - 1), x_var);
        }
        const int64_t cap = s->opts.trace_capacity;
        const int64_t avail = std::min<int64_t>(c.sweep - s->opts.start_sweep, cap);
        if (n_trace) *n_trace = avail;
        const int64_t hc = plain ? chain : static_cast<int64_t>(field) * s->Cp + chain;
        if ((tau_trace || sigma2_trace) && trace_cap > 0 && avail > 0) {
            std::vector<double> rt(static_cast<size_t>(cap)), rs(static_cast<size_t>(cap));
            CK(cudaMemcpyAsync(rt.data(), s->trace_tau + hc * cap, sizeof(double) * cap, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaMemcpyAsync(rs.data(), s->trace_sig + hc * cap, sizeof(double) * cap, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
            const int64_t m = std::min(trace_cap, avail);
            for (int64_t q = 0; q < m; ++q) {
                const int64_t sw = c.sweep - m + q;
                if (tau_trace) tau_trace[q] = rt[sw % cap];
                if (sigma2_trace) sigma2_trace[q] = rs[sw % cap];
            }
        }
        if (tau_now) CK(cudaMemcpyAsync(tau_now, s->tau + hc, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        if (sigma2_now) CK(cudaMemcpyAsync(sigma2_now, s->sig2 + hc, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    return GMRF_OK;
}

gmrf_status gmrf_fetch_pooled(gmrf_sampler *s, int32_t field, double *mean, double *var)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (field < 0 || field >= s->nfields) return fail(GMRF_E_INVALID, "field out of range");
    if (s->algorithm == GMRF_ALGO_PLAIN) return fail(GMRF_E_UNSUPPORTED, "the plain sweep keeps no running moments");
    const int64_t n = s->hf[field].n;
    try {
        SweepCtl c{};
        CK(cudaMemcpyAsync(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (const gmrf_status w = check_waits(s, c)) return w;
        const int64_t k = c.acc_count;
        if (mean && k < 1) std::fill(mean, mean + n, 0.0);
        if (var && s->C * k < 2) std::fill(var, var + n, NAN);
        double *dm = (mean && k >= 1) ? s->staging : nullptr;
        double *dv = (var && s->C * k >= 2) ? s->pool_stage : nullptr;
        if (dm || dv) {
            CK(launch_pool(s->precision, s->fields_dev, s->fd[field], field, s->Cp, s->C, k, s->mean, s->m2,
                           s->perm_inv, dm, dv, s->stream));
            if (dm) CK(cudaMemcpyAsync(mean, dm, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
            if (dv) CK(cudaMemcpyAsync(var, dv, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        }
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    return GMRF_OK;
}

gmrf_status gmrf_fetch_intercept(gmrf_sampler *s, int32_t field, int32_t chain, int64_t trace_cap, double *beta0_trace,
                                 int64_t *n_trace, double *beta0_now)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (!has_beta(s)) return fail(GMRF_E_INVALID, "the model has no intercept");
    if (field < 0 || field >= s->nfields || chain < 0 || chain >= s->C)
        return fail(GMRF_E_INVALID, "field or chain out of range");
    if (trace_cap < 0) return fail(GMRF_E_INVALID, "trace_cap must be >= 0");
    try {
        SweepCtl c{};
        CK(cudaMemcpyAsync(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (const gmrf_status w = check_waits(s, c)) return w;
        const int64_t cap = s->opts.trace_capacity;
        const int64_t avail = std::min<int64_t>(c.sweep - s->opts.start_sweep, cap);
        if (n_trace) *n_trace = avail;
        const int64_t hc = static_cast<int64_t>(field) * s->Cp + chain;
        if (beta0_trace && trace_cap > 0 && avail > 0) {
            std::vector<double> rb(static_cast<size_t>(cap));
            CK(cudaMemcpyAsync(rb.data(), s->trace_beta + hc * cap, sizeof(double) * cap, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
            const int64_t m = std::min(trace_cap, avail);
            for (int64_t q = 0; q < m; ++q) beta0_trace[q] = rb[(c.sweep - m + q) % cap];
        }
        if (beta0_now) CK(cudaMemcpyAsync(beta0_now, s->beta + hc, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    return GMRF_OK;
}

gmrf_status gmrf_trace_diagnostics(gmrf_sampler *s, int32_t field, int32_t param, int64_t n_last, double *iat,
                                   double *ess, double *psrf)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (s->algorithm == GMRF_ALGO_PLAIN) return fail(GMRF_E_UNSUPPORTED, "diagnostics of the plain sweep");
    if (field < 0 || field >= s->nfields) return fail(GMRF_E_INVALID, "field out of range");
    if (param < GMRF_PARAM_TAU2 || param > GMRF_PARAM_TAU) return fail(GMRF_E_INVALID, "param");
    if (param == GMRF_PARAM_BETA0 && !has_beta(s)) return fail(GMRF_E_INVALID, "the model has no intercept");
    if (n_last < 0) return fail(GMRF_E_INVALID, "n_last must be >= 0");
    try {
        SweepCtl c{};
        CK(cudaMemcpyAsync(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (const gmrf_status w = check_waits(s, c)) return w;
        const int64_t cap = s->opts.trace_capacity;
        const int64_t avail = std::min<int64_t>(c.sweep - s->opts.start_sweep, cap);
        const int64_t N = n_last == 0 ? avail : std::min<int64_t>(n_last, avail);
        if (N < 2) return fail(GMRF_E_INVALID, "fewer than 2 trace values available");
        const double *base = param == GMRF_PARAM_SIGMA2 ? s->trace_sig
                             : param == GMRF_PARAM_BETA0 ? s->trace_beta : s->trace_tau;
        DiagArgs a{};
        a.trace = base + static_cast<int64_t>(field) * s->Cp * cap;
        a.cap = cap;
        a.sweep = c.sweep;
        a.N = N;
        a.reciprocal = param == GMRF_PARAM_TAU2 ? 1 : 0;
        a.chains = s->C;
        a.work = s->diag_work;
        a.out = s->diag_out;
        a.psrf = s->diag_out + static_cast<int64_t>(s->Cp) * 4;
        CK(launch_trace_diagnostics(a, s->stream));
        std::vector<double> h(static_cast<size_t>(s->C) * 4 + 1);
        CK(cudaMemcpyAsync(h.data(), s->diag_out, sizeof(double) * s->C * 4, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(h.data() + s->C * 4, a.psrf, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (int q = 0; q < s->C; ++q) {
            if (iat) iat[q] = h[q * 4];
            if (ess) ess[q] = h[q * 4 + 1];
        }
        if (psrf) *psrf = h[s->C * 4];
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    return GMRF_OK;
}

gmrf_status gmrf_site_psrf(gmrf_sampler *s, int32_t field, double *psrf, double *psrf_max)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (s->algorithm == GMRF_ALGO_PLAIN) return fail(GMRF_E_UNSUPPORTED, "diagnostics of the plain sweep");
    if (field < 0 || field >= s->nfields) return fail(GMRF_E_INVALID, "field out of range");
    if (s->C < 2) return fail(GMRF_E_INVALID, "the PSRF needs at least 2 chains");
    try {
        SweepCtl c{};
        CK(cudaMemcpyAsync(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (const gmrf_status w = check_waits(s, c)) return w;
        if (c.acc_count < 2) return fail(GMRF_E_INVALID, "the PSRF needs at least 2 accumulated sweeps");
        unsigned long long *mx = reinterpret_cast<unsigned long long *>(s->diag_out + static_cast<int64_t>(s->Cp) * 4 + 1);
        CK(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s->stream));
        CK(launch_site_psrf(s->precision, s->fields_dev, s->fd[field], field, s->Cp, s->C, s->mean, s->m2, c.acc_count,
                            s->perm_inv, s->staging, mx, s->stream));
        const int64_t n = s->hf[field].n;
        if (psrf) CK(cudaMemcpyAsync(psrf, s->staging, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        if (psrf_max) {
            double v = NAN;
            if (bits) std::memcpy(&v, &bits, sizeof(v));
            *psrf_max = v;
        }
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    return GMRF_OK;
}

gmrf_status gmrf_sampler_reset(gmrf_sampler *s)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    return restart_state(s);
}

gmrf_status gmrf_sampler_set_data(gmrf_sampler *s, int32_t field, const double *y, const int32_t *trials,
                                  const double *x0)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (field < 0 || field >= s->nfields) return fail(GMRF_E_INVALID, "field out of range");
    const int64_t n = s->hf[field].n;
    const bool binomial = binomial_model(s);
    if (!y) return fail(GMRF_E_INVALID, "y is required");
    if (binomial && !trials) return fail(GMRF_E_INVALID, "binomial data need trials");
    // The checks of the values (bad data leave the sampler unchanged): on the device for the
    // staged uploads (a host pass over the caller's arrays took 7 ms for 16.7 M sites), on the
    // host for the plain sweep, which uploads into its buffers directly.
    auto check_data = [&]() -> gmrf_status {
        if (!all_finite(y, n)) return fail(GMRF_E_INVALID, "y must be finite");
        if (binomial)
            for (int64_t i = 0; i < n; ++i) {
                if (trials[i] < 0 || trials[i] > 4095) return fail(GMRF_E_INVALID, "trials must be in 0..4095");
                if (!(y[i] >= 0.0 && y[i] <= trials[i]))
                    return fail(GMRF_E_INVALID, "successes y must be in [0, trials]");
            }
        if (x0 && !all_finite(x0, n * s->C)) return fail(GMRF_E_INVALID, "x0 must be finite");
        return GMRF_OK;
    };
    const bool plain = s->algorithm == GMRF_ALGO_PLAIN;
    if (plain) {
        if (const gmrf_status r = check_data()) return r;
    }
    if (!plain && !s->data_stage) {
        // One staging area for the largest field: y, then x0 (or its default) for every chain.
        int64_t max_n = 1;
        for (const HostField &h : s->hf) max_n = std::max<int64_t>(max_n, h.n);
        cudaError_t e = s->alloc_t(&s->data_stage, static_cast<size_t>(max_n) * (1 + s->C), sizeof(double));
        if (e == cudaSuccess) e = s->alloc_t(&s->data_flag, 1, sizeof(unsigned int));
        if (e == cudaSuccess && binomial)
            e = s->alloc_t(&s->trials_stage, static_cast<size_t>(max_n), sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();  // an allocation failure leaves the context usable
            return cuda_status(CudaFail{e, "staging buffer for gmrf_sampler_set_data"});
        }
    }
    try {
        const size_t yb = sizeof(double) * static_cast<size_t>(n);
        if (plain) {
            CK(cudaMemcpyAsync(const_cast<double *>(s->plain.y), y, yb, cudaMemcpyHostToDevice, s->stream));
            for (int c = 0; c < s->C; ++c)
                CK(cudaMemcpyAsync(static_cast<double *>(s->x_init) + c * n, x0 ? x0 + c * n : y, yb,
                                   cudaMemcpyHostToDevice, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        } else {
            double *y_d = s->data_stage, *x0_d = s->data_stage + n;
            CK(cudaMemcpyAsync(y_d, y, yb, cudaMemcpyHostToDevice, s->stream));
            if (x0) CK(cudaMemcpyAsync(x0_d, x0, yb * s->C, cudaMemcpyHostToDevice, s->stream));
            else if (binomial) CK(cudaMemsetAsync(x0_d, 0, yb * s->C, s->stream));  // all-zero bits: +0.0
            if (binomial)
                CK(cudaMemcpyAsync(s->trials_stage, trials, sizeof(int32_t) * static_cast<size_t>(n),
                                   cudaMemcpyHostToDevice, s->stream));
            CK(launch_check_data(y_d, binomial ? s->trials_stage : nullptr, x0 ? x0_d : nullptr, n,
                                 x0 ? n * s->C : 0, s->data_flag, s->stream));
            unsigned int bad = 0;
            CK(cudaMemcpyAsync(&bad, s->data_flag, sizeof(bad), cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));  // the host arrays may be reused from here on
            // only the staging buffer was written
            if (bad & 1u) return fail(GMRF_E_INVALID, "y must be finite");
            if (bad & 2u) return fail(GMRF_E_INVALID, "trials must be in 0..4095");
            if (bad & 4u) return fail(GMRF_E_INVALID, "successes y must be in [0, trials]");
            if (bad & 8u) return fail(GMRF_E_INVALID, "x0 must be finite");
            if (binomial)
                CK(launch_pack_int(s->fields_dev, s->fd[field], field, s->trials_stage, s->perm_inv, s->trials,
                                   s->stream));
            // The same packing as at creation, into the restart state.
            CK(launch_pack(s->precision, s->fields_dev, s->fd[field], field, s->C, s->Cp, y_d,
                           (x0 || binomial) ? x0_d : nullptr, s->perm_inv, s->x_init, s->y, s->stream));
        }
    } catch (const CudaFail &f) {
        s->poisoned = true;
        return cuda_status(f);
    }
    // The restart runs once before the state is next used (a batch of set_data calls, one per
    // field, restarts the chains once).
    s->restart_pending = true;
    return GMRF_OK;
}

gmrf_status gmrf_launch_stage(gmrf_sampler *s, int32_t stage, int32_t accumulate, const char **name)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    if (s->algorithm == GMRF_ALGO_PLAIN) return fail(GMRF_E_UNSUPPORTED, "stages of the plain sweep");
    if (stage < 0 || stage >= static_cast<int32_t>(s->stages.size())) return fail(GMRF_E_INVALID, "stage out of range");
    if (name) *name = stage_name(s, static_cast<size_t>(stage));
    const int draw = s->model.fix_hyper ? 0 : 1;
    cudaError_t e = enqueue_stage(s, static_cast<size_t>(stage), 1, accumulate ? 1 : 0, draw, 1, 1, s->stream);
    if (e != cudaSuccess) return poison(s, e, "stage launch");
    return GMRF_OK;
}

gmrf_status gmrf_field_colors(gmrf_sampler *s, int32_t field, int32_t *colors, int32_t *num_colors)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    if (field < 0 || field >= s->nfields) return fail(GMRF_E_INVALID, "field out of range");
    const HostField &h = s->hf[field];
    if (colors) {
        if (h.kind == GMRF_CSR) std::copy(h.colors.begin(), h.colors.end(), colors);
        else
            for (int64_t i = 0; i < h.n; ++i) colors[i] = lattice_colour_host(h.kind, h.dims, i);
    }
    if (num_colors) *num_colors = h.ncolors;
    return GMRF_OK;
}

gmrf_status gmrf_sampler_info(gmrf_sampler *s, gmrf_info *out)
{
    g_last_error.clear();
    if (!s || !out) return fail(GMRF_E_INVALID, "sampler and out are required");
    if (s->poisoned) return fail(GMRF_E_STATE, "sampler is poisoned by an earlier CUDA error");
    if (const gmrf_status r = restart_if_pending(s)) return r;
    SweepCtl c{};
    cudaError_t e = cudaMemcpyAsync(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return poison(s, e, "info");
    if (const gmrf_status w = check_waits(s, c)) return w;
    out->nfields = s->nfields;
    out->chains = s->C;
    out->precision = s->precision;
    out->max_colors = s->kmax;
    out->sweeps_done = c.sweep;
    out->accumulated = c.acc_count;
    out->hyper_fallbacks = c.fallbacks;
    out->device_bytes = s->bytes;
    out->launches_per_sweep = s->launches_per_sweep;
    out->early_start_misses = c.fmiss;
    out->resident = s->resident;
    out->wait_timeouts = static_cast<int64_t>(c.wait_timeouts);
    return GMRF_OK;
}

gmrf_status gmrf_normals_timing(uint64_t seed, int64_t sites, int32_t chains, int32_t reps, void *cuda_stream,
                                double *us_per_launch)
{
    g_last_error.clear();
    if (sites < 1 || sites > (int64_t(1) << 31) || chains < 1 || chains > 8 || reps < 1 || !us_per_launch)
        return fail(GMRF_E_INVALID, "sites in 1..2^31, chains in 1..8, reps >= 1 and us_per_launch are required");
    const int cp = chains <= 4 ? 4 : 8;
    const int threads = normals_only_threads(cp);
    if (threads < 1) return cuda_status(CudaFail{cudaErrorInvalidConfiguration, "normals timing grid"});
    void *out = nullptr;
    cudaError_t e = dev_malloc(&out, sizeof(unsigned long long) * static_cast<size_t>(threads));
    if (e == cudaSuccess)
        e = time_normals_only(seed, sites, cp, reps, static_cast<unsigned long long *>(out),
                              static_cast<cudaStream_t>(cuda_stream), us_per_launch);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return cuda_status(CudaFail{e, "normals timing"});
    return GMRF_OK;
}

gmrf_status gmrf_debug_fail_alloc(int64_t nth)
{
    g_last_error.clear();
    if (nth < 0) return fail(GMRF_E_INVALID, "nth must be >= 0");
    g_fail_alloc.store(nth);
    return GMRF_OK;
}

gmrf_status gmrf_debug_poison(gmrf_sampler *s)
{
    g_last_error.clear();
    if (!s) return fail(GMRF_E_INVALID, "sampler is NULL");
    s->poisoned = true;
    return GMRF_OK;
}

gmrf_status gmrf_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count, uint32_t *out,
                              void *cuda_stream)
{
    g_last_error.clear();
    if (count < 0 || (count > 0 && !out)) return fail(GMRF_E_INVALID, "count >= 0 and a device output are required");
    if (count > (int64_t(1) << 32)) return fail(GMRF_E_INVALID, "count must be <= 2^32");
    cudaError_t e = launch_philox_words(seed, c1, c2, c3, count, out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_status(CudaFail{e, "philox_words"});
    return GMRF_OK;
}

gmrf_status gmrf_site_normals(uint64_t seed, uint32_t sweep, uint32_t stream, uint32_t chain, int32_t lanes,
                              int32_t precision, int64_t count, void *out, void *cuda_stream)
{
    g_last_error.clear();
    if (count < 0 || (count > 0 && !out)) return fail(GMRF_E_INVALID, "count >= 0 and a device output are required");
    if (count > (int64_t(1) << 32)) return fail(GMRF_E_INVALID, "count must be <= 2^32");
    if (precision != GMRF_FP32 && precision != GMRF_FP64) return fail(GMRF_E_INVALID, "precision");
    if (lanes != 1 && lanes != 2 && lanes != 4) return fail(GMRF_E_INVALID, "lanes must be 1, 2 or 4");
    if (lanes < 4 && chain >= static_cast<uint32_t>(lanes)) return fail(GMRF_E_INVALID, "chain must be < lanes");
    cudaError_t e = launch_site_normals(seed, sweep, stream, chain, lanes, precision, count, out,
                                        static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_status(CudaFail{e, "site_normals"});
    return GMRF_OK;
}

}  // extern "C"
