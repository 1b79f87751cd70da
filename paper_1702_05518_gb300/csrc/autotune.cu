// autotune.cu -- gmrf_autotune: the launch configuration of a sampler chosen by measurement.
//
// The sweep kernels' work decomposition (chains per thread, the 3-D kernel, the colour-step tile,
// the fused 2-D tile shape and block size, the quad kernel's configuration) changes nothing but the rounding
// of the partial sums, and the library's cost models pick it from the sizes alone.  The
// autotuner measures instead: starting from the cost models' choice it tries each knob's
// candidates in turn (coordinate descent), keeping a candidate when it is at least 2 % faster
// than the best so far, each candidate being a sampler built from the caller's own fields and
// timed over the caller's number of sweeps with CUDA events.  The choice is cached for the
// process by a key of the fields' kinds and sizes, the chains, the precision and the model and
// option switches, so a key is measured once and every sampler built with it decomposes its work
// the same way.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gmrf.h"

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::pair<gmrf_tuning, double>> g_tune_cache;

std::string tune_key(const gmrf_field_desc *fields, int32_t nfields, const gmrf_model *m, const gmrf_opts *o)
{
    std::string k;
    auto add = [&k](long long v) {
        k += std::to_string(v);
        k += ',';
    };
    add(nfields);
    for (int i = 0; i < nfields; ++i) {
        const gmrf_field_desc &f = fields[i];
        add(f.kind);
        add(f.n);
        if (f.kind == GMRF_CSR) {
            add(f.row_ptr ? f.row_ptr[f.n] : -1);
            add(f.weights != nullptr);
        } else {
            add(f.dims[0]);
            add(f.dims[1]);
            add(f.dims[2]);
        }
    }
    add(o->precision);
    add(o->chains);
    add(o->algorithm);
    add(o->graph_sweeps);
    add(o->flags);
    add(m->prior);
    add(m->intercept);
    add(m->likelihood);
    add(m->fix_hyper);
    return k;
}

// Microseconds per sweep of a sampler built with `t`, or +inf when the configuration does not
// apply (the library rejects it); *st receives a failure other than a rejection.
double measure(const gmrf_field_desc *fields, int32_t nfields, const gmrf_model *m, const gmrf_opts *o,
               const gmrf_tuning &t, int32_t sweeps, cudaStream_t stream, gmrf_status *st)
{
    gmrf_opts oo = *o;
    oo.tuning = &t;
    gmrf_sampler *s = nullptr;
    gmrf_status r = gmrf_sampler_create(&s, fields, nfields, m, &oo, stream);
    if (r == GMRF_E_INVALID || r == GMRF_E_UNSUPPORTED) return INFINITY;
    if (r != GMRF_OK) {
        *st = r;
        return INFINITY;
    }
    double best = INFINITY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        *st = GMRF_E_CUDA;
    } else if ((r = gmrf_sweep(s, sweeps < 3 ? sweeps : 3, 1)) != GMRF_OK) {
        *st = r;
    } else {
        for (int rep = 0; rep < 2 && *st == GMRF_OK; ++rep) {
            float ms = 0.0f;
            if (cudaEventRecord(e0, stream) != cudaSuccess || (r = gmrf_sweep(s, sweeps, 1)) != GMRF_OK ||
                cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                *st = r != GMRF_OK ? r : GMRF_E_CUDA;
                break;
            }
            best = std::fmin(best, 1e3 * ms / sweeps);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    gmrf_sampler_destroy(s);
    return *st == GMRF_OK ? best : INFINITY;
}

}  // namespace

extern "C" gmrf_status gmrf_autotune(const gmrf_field_desc *fields, int32_t nfields, const gmrf_model *model,
                                     const gmrf_opts *opts, int32_t sweeps, void *cuda_stream, gmrf_tuning *out,
                                     double *us_per_sweep)
{
    if (!fields || nfields < 1 || !model || !opts || !out || sweeps < 1) {
        // let gmrf_sampler_create describe what is wrong with the arguments it checks
        gmrf_sampler *s = nullptr;
        gmrf_status r = (fields && model && opts) ? gmrf_sampler_create(&s, fields, nfields, model, opts, cuda_stream)
                                                  : GMRF_E_INVALID;
        if (s) gmrf_sampler_destroy(s);
        return r == GMRF_OK ? GMRF_E_INVALID : r;
    }
    const std::string key = tune_key(fields, nfields, model, opts);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
        *out = it->second.first;
        if (us_per_sweep) *us_per_sweep = it->second.second;
        return GMRF_OK;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    gmrf_status st = GMRF_OK;
    gmrf_tuning best{};
    double best_us = measure(fields, nfields, model, opts, best, sweeps, stream, &st);
    if (st != GMRF_OK) return st;
    if (!std::isfinite(best_us)) {  // the automatic configuration itself is rejected: report why
        gmrf_sampler *s = nullptr;
        gmrf_status r = gmrf_sampler_create(&s, fields, nfields, model, opts, cuda_stream);
        if (s) gmrf_sampler_destroy(s);
        return r == GMRF_OK ? GMRF_E_INVALID : r;
    }
    auto consider = [&](const gmrf_tuning &t) {
        if (st != GMRF_OK) return;
        const double us = measure(fields, nfields, model, opts, t, sweeps, stream, &st);
        if (us < 0.98 * best_us) {
            best_us = us;
            best = t;
        }
    };

    bool has_kind[4] = {false, false, false, false};
    for (int i = 0; i < nfields; ++i)
        if (fields[i].kind >= 0 && fields[i].kind < 4) has_kind[fields[i].kind] = true;
    int cp = 1;
    while (cp < opts->chains) cp <<= 1;
    const bool fp32 = opts->precision == GMRF_FP32;

    // 1. chains per thread
    for (int v : {1, 2, 4}) {
        if (v > cp || (!fp32 && v > 2)) continue;
        gmrf_tuning t = best;
        t.chains_per_thread = v;
        consider(t);
    }
    // 1b. 3-D lattices: every chain of a site in one thread, or the general colour-step kernel
    if (has_kind[GMRF_LATTICE3D_6] && fp32 && cp >= 4 && cp <= 8)
        for (int w : {1, -1}) {
            gmrf_tuning t = best;
            t.wide_3d = w;
            consider(t);
        }
    // 1c. a single graph on the resident path: blocks per chain's cluster
    if (nfields == 1 && has_kind[GMRF_CSR])
        for (int cl : {1, 2, 4, 8, 16}) {
            if (cl * opts->chains > 152) continue;
            gmrf_tuning t = best;
            t.graph_cluster = cl;
            consider(t);
        }
    // 2. the colour-step tile (3-D lattices, graphs, and 2-D lattices on per-colour launches)
    if (has_kind[GMRF_LATTICE3D_6] || has_kind[GMRF_CSR] || (opts->flags & GMRF_FLAG_PER_COLOUR))
        for (int tile : {256, 512, 1024, 2048, 4096, 8192, 16384}) {
            gmrf_tuning t = best;
            t.step_tile = tile;
            consider(t);
        }
    // 3. the quad kernel (one chain, FP32, 8-neighbour lattices)
    if (has_kind[GMRF_LATTICE2D_8] && cp == 1 && fp32) {
        for (int q : {-1, 1, 2, 3, 4, 5}) {
            gmrf_tuning t = best;
            t.quad_config = q;
            t.quad_rows = 0;
            consider(t);
        }
        if (best.quad_config >= 0)
            for (int rows : {16, 24, 32, 40, 48, 56, 64, 80, 96, 112}) {
                gmrf_tuning t = best;
                t.quad_rows = rows;
                consider(t);
            }
    }
    // 4. the fused 2-D tile and block size, per kind
    static const int shapes[][2] = {{16, 64}, {24, 64}, {32, 32}, {32, 64}, {32, 96}, {32, 128}, {48, 64},
                                    {48, 120}, {64, 64}, {64, 120}, {64, 128}, {96, 64}, {128, 64}, {16, 128}};
    for (int kind : {static_cast<int>(GMRF_LATTICE2D_4), static_cast<int>(GMRF_LATTICE2D_8)}) {
        if (!has_kind[kind]) continue;
        for (int nt : {512, 1024}) {
            gmrf_tuning t = best;
            t.fused_threads[kind] = nt;
            consider(t);
        }
        for (const auto &sh : shapes) {
            gmrf_tuning t = best;
            t.fused_rows[kind] = sh[0];
            t.fused_cols[kind] = sh[1];
            consider(t);
        }
    }
    if (st != GMRF_OK) return st;
    g_tune_cache[key] = {best, best_us};
    *out = best;
    if (us_per_sweep) *us_per_sweep = best_us;
    return GMRF_OK;
}
