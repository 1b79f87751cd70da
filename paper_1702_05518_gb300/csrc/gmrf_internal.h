// gmrf_internal.h -- declarations shared by the translation units of libgmrf (host side).
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "gmrf_device.cuh"

namespace gmrf {

// Sweep kernels are launched with programmatic stream serialization (see
// pdl_wait_then_release) unless the environment sets GMRF_PDL=0.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_sweep_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Arguments of one colour-step launch (one colour class of every field, or a reduce-only pass
// over the current state when `update` is 0).
struct StepArgs {
    const FieldDev *fields;
    const Tile *tiles;
    int32_t ntiles;
    int32_t colour;
    void *x;             // [slots][Cp]  state, colour-split layout, chains innermost
    const void *y;       // [slots]      observations
    void *mean;          // [slots][Cp]  Welford mean
    void *m2;            // [slots][Cp]  Welford sum of squared deviations
    const int32_t *rp;   // CSR: local row pointers of the permuted graph (n + 1 per field)
    const int32_t *ci;   // CSR: local permuted column indices
    const void *w;       // CSR: edge weights (precision T) or nullptr
    const void *deg;     // CSR: degrees d_i (precision T), permuted order
    const int32_t *perm; // CSR: slot -> natural site
    const int32_t *coff; // CSR: colour offsets (ncolors + 1 per field)
    const void *hyp;     // [F * Cp][kHypStride]: tau, 1/sigma^2, beta0 in precision T
    Part3 *partials;     // [parts][Cp]: per tile and chain sums (S, R, A)
    SweepCtl *ctl;
    uint2 key;
    int32_t Cp;          // chains in the layout (power of two >= chains)
    int32_t lanes;       // normals per site of one Philox block: min(4, Cp)
    double rho;
    long long burn_in;
    int32_t thin;
    int32_t acc_enabled;
    int32_t update;      // 1: draw the colour class; 0: only recompute the partial sums
    int32_t intercept;   // the model has the intercept beta0
    int32_t binomial;    // binomial counts (successes in y) with the logistic link
    const int32_t *trials;  // [slots] binomial trials m_i (binomial model only)
    const void *psi;     // [slots][Cp] Polya-Gamma draws of this sweep (binomial model only)
    uint32_t rk[20];     // Philox round keys of `key` (philox_round_keys), read from the parameters
};

struct HyperArgs {
    const FieldDev *fields;
    int32_t nfields;
    int32_t Cp;
    const Part3 *partials;
    double *tau;          // [F * Cp]
    double *sig2;         // [F * Cp]
    double *beta;         // [F * Cp] intercepts (read and drawn only when draw_beta)
    void *hyp;            // [F * Cp][kHypStride] copies in precision T
    double *trace_tau;    // [F * Cp][cap]
    double *trace_sig;
    double *trace_beta;
    int32_t trace_cap;
    SweepCtl *ctl;
    uint2 key;
    double a_tau, b_tau, a_sig, b_sig;
    int32_t draw;         // 0: keep tau, sigma^2
    int32_t draw_beta;    // 1: draw the intercept beta0 (before sigma^2)
    int32_t binomial;     // binomial model: beta0 from its normal conditional, no sigma^2
    double beta0_mean, beta0_var;  // binomial model: normal prior of beta0
    int32_t end_of_sweep; // 1: sweep counter, traces; 0: extra draw (tags 5 and 6)
    long long burn_in;    // accumulation schedule (to advance the accumulation count)
    int32_t thin;
    int32_t acc_enabled;
    const double *gpre;   // [batch][F * Cp][4]: unit-rate Gamma variates of tau and 1/sigma^2 and
                          // the intercept's standard normal, for the batch's sweeps
    int32_t max_parts;    // the most tile partials of any field
};

// Unit-rate Gamma variates (tau and 1/sigma^2 of every field and chain) for sweeps
// ctl->sweep .. ctl->sweep + count - 1, one thread each; records the batch in ctl.
struct GammaPreArgs {
    const FieldDev *fields;
    int32_t nfields;
    int32_t Cp;
    SweepCtl *ctl;
    uint2 key;
    double a_tau, a_sig;
    int32_t count;
    int32_t intercept;   // 1: also the standard normals of the intercept draws
    double *gpre;
};

// Arguments of one launch of the resident kernel (lattice_resident.cu): `count` whole sweeps of
// the single 2-D lattice field 0, one block per chain, the chain in shared memory.
struct ResidentArgs {
    const FieldDev *fields;
    HyperArgs h;          // the conjugate draws at the end of each sweep (end_of_sweep = 1)
    void *x;              // state buffer 0 (the state at the start of even sweeps)
    void *x_alt;          // state buffer 1 (odd sweeps)
    const void *y;
    void *mean;
    void *m2;
    int32_t count;        // sweeps of this launch
    int32_t SR, SC;       // rows and columns of a shared sub-array: the global ones + a ring of zeros
    int32_t lanes;        // normals per site of one Philox block: min(4, Cp)
    int32_t C;            // chains (one block each)
    double rho;
    const void *zbuf;     // [count][C][colour][NI][site thread] normals of the batch (precision T)
};

// Arguments of the producer of the resident kernels' normals (resident_normals_kernel).
struct ResNormArgs {
    const FieldDev *fields;
    SweepCtl *ctl;        // the batch starts at ctl->sweep
    uint2 key;
    int32_t lanes, C, Cp;
    int32_t count;        // sweeps of the batch
    int32_t NI, NTS;      // lattice: positions per thread and class, site threads
    const int32_t *perm_inv;  // graph: natural site -> permuted position (then out is [count][C][n])
    void *out;
    GammaPreArgs g;           // the batch's Gamma variates, drawn by the first gamma_blocks blocks
    int32_t gamma_blocks;     // (64 threads of each); 0: none
};

// Arguments of one launch of the graph resident kernel (csr_resident.cu): `count` whole sweeps
// of the single graph field 0, one block per chain.
struct ResCsrArgs {
    const FieldDev *fields;
    HyperArgs h;
    void *x;              // [slots][Cp] state (permuted positions)
    const void *y;
    void *mean;
    void *m2;
    const uint4 *nbr;     // [n] eight 16-bit neighbour positions (pad = n; bit 15 of the first:
                          // more in nbr2)
    const uint4 *nbr2;    // [n] neighbours 9..16 of the flagged positions
    const int32_t *coff;  // colour offsets (ncolors + 1)
    int32_t ncolors;
    int32_t count, C;
    int32_t own_max;      // positions a block of a chain's cluster owns (largest share)
    double rho;
    const void *zbuf;     // [count][C][n] normals by permuted position
    uint32_t extra_bytes; // added to every colour step's expected bytes (0; 16 under GMRF_FLAG_TEST_STALL)
    uint64_t wait_ns;     // limit of a colour step's wait
};

// A tile of the fused 2-D lattice sweep: natural coordinates of its first site.
struct TileXY {
    int32_t field;
    int32_t i0, j0;
    int32_t part;       // partial-sum slot
};

// Arguments of one fused-sweep launch (every tile of the fields of one 2-D lattice kind).
struct FusedArgs {
    const FieldDev *fields;
    const TileXY *tiles;
    int32_t ntiles;
    int32_t TR, TC;      // tile rows and columns (natural sites)
    int32_t threads;     // threads per block: 512 or 1024
    uint32_t rc_m, tc_m; // invariant-divisor constants of the staged row length, of TC and of
    int32_t rc_s, tc_s;  // the Philox-group slots per staged row
    uint32_t ng_m;
    int32_t ng_s;
    void *x;             // state buffer 0 (the state at the start of even sweeps)
    void *x_alt;         // state buffer 1 (the state at the start of odd sweeps)
    const void *y;
    void *mean;
    void *m2;
    const void *hyp;     // [F * Cp][kHypStride]
    Part3 *partials;
    SweepCtl *ctl;       // the quad kernel writes ctl->fnext
    uint2 key;
    int32_t Cp;
    int32_t lanes;       // normals per site of one Philox block: min(4, Cp)
    double rho;
    long long burn_in;
    int32_t thin;
    int32_t acc_enabled;
    int32_t update;      // 1: run the colour steps; 0: only recompute the partial sums
    int32_t early;       // the sweep's only sweep kernel: start on a predicted sweep number
};


cudaError_t launch_gamma_pre(const GammaPreArgs &a, cudaStream_t stream);

// Polya-Gamma stage of the binomial model (sweep_kernels.cu): psi[slot][chain] ~ PG(m_i, beta0 +
// x_i) for every site from the state at the start of the sweep, one warp per (slot, chain)
// with the m_i summands spread over the lanes.
struct PgArgs {
    const FieldDev *fields;
    int32_t nfields;
    int64_t slots;         // total slots (every field)
    int32_t Cp, C;
    const void *x;         // [slots][Cp] state (precision T)
    const void *hyp;       // [F * Cp][kHypStride]
    const int32_t *trials; // [slots]
    const int32_t *perm;   // CSR: slot -> natural site
    void *psi;             // [slots][Cp] out (precision T)
    SweepCtl *ctl;
    uint2 key;
};
cudaError_t launch_pg_stage(int precision, const PgArgs &a, cudaStream_t stream);

// Launchers (each enqueues on `stream` and returns the launch status).
// One colour step of the tiles in `a` (all of field kind `kind`).
cudaError_t launch_colour_step(int precision, int V, int kind, const StepArgs &a, cudaStream_t stream);
// 3-D lattice colour step with every chain of a site in one thread (FP32, chains_padded 4 or 8;
// lattice3d.cu), and the blocks of it that are resident on one SM.
cudaError_t launch_lattice3d(int chains_padded, const StepArgs &a, cudaStream_t stream);
cudaError_t lattice3d_blocks_per_sm(int chains_padded, int *blocks);
// Time (CUDA events, `reps` launches after 3 untimed ones) of the 3-D kernel's normals alone for
// `sites` sites and chains_padded (4 or 8) chains, on the kernel's grid.
// (`out`: one 8-byte word per thread of that grid, normals_only_threads).
int normals_only_threads(int chains_padded);
cudaError_t time_normals_only(uint64_t seed, int64_t sites, int chains_padded, int reps, unsigned long long *out,
                              cudaStream_t stream, double *us_per_launch);
cudaError_t launch_hyper(int precision, const HyperArgs &a, cudaStream_t stream);
cudaError_t launch_pack(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx,
                        int32_t C, int32_t Cp, const double *y_nat, const double *x0_nat,
                        const int32_t *perm_inv, void *x, void *y, cudaStream_t stream);
cudaError_t launch_unpack(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx,
                          int32_t Cp, int32_t chain, const void *src, const void *m2, double inv_km1,
                          const int32_t *perm_inv, double *out, cudaStream_t stream);
// Moments pooled over the chains (natural order, FP64; out_var needs C k >= 2, either output may be null).
cudaError_t launch_pool(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, int32_t Cp,
                        int32_t C, int64_t k, const void *mean, const void *m2, const int32_t *perm_inv,
                        double *out_mean, double *out_var, cudaStream_t stream);
// Device checks of data staged by gmrf_sampler_set_data (bits of *flag: 1 y not finite, 2 trials
// outside 0..4095, 4 successes outside [0, trials], 8 x0 not finite); trials, x0 may be null.
cudaError_t launch_check_data(const double *y, const int32_t *trials, const double *x0, int64_t n, int64_t nx0,
                              unsigned int *flag, cudaStream_t stream);
cudaError_t launch_pack_int(const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, const int32_t *v_nat,
                            const int32_t *perm_inv, int32_t *v, cudaStream_t stream);
cudaError_t launch_ctl_reset(SweepCtl *ctl, long long start_sweep, cudaStream_t stream);
cudaError_t launch_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count,
                                uint32_t *out, cudaStream_t stream);
cudaError_t launch_site_normals(uint64_t seed, uint32_t sweep, uint32_t stream_id, uint32_t chain, int lanes,
                                int precision, int64_t count, void *out, cudaStream_t stream);

// Fused 2-D lattice sweep (lattice_fused.cu).
size_t lattice_fused_smem(int precision, int kind, int Cp, int TR, int TC);
cudaError_t prepare_lattice_fused(int precision, int V, int kind, size_t smem);
cudaError_t launch_lattice_fused(int precision, int V, int kind, const FusedArgs &a, size_t smem,
                                 cudaStream_t stream);
// Resident path: NI colour-class positions per thread (1, 2 or 4), `threads` (<= 704) per block, one block per
// chain; prepare_lattice_resident raises the kernel's dynamic shared-memory limit (call once,
// before any capture).
cudaError_t prepare_lattice_resident(int precision, int kind, int NI, size_t smem);
cudaError_t launch_lattice_resident(int precision, int kind, int NI, int threads, int chains, const ResidentArgs &a,
                                    size_t smem, cudaStream_t stream);
// One thread per Philox block of the batch: `blocks_needed` = sweeps x groups x chain quadruples.
cudaError_t launch_resident_normals(int precision, const ResNormArgs &a, int64_t blocks_needed, cudaStream_t stream);
// Graph resident path: the neighbour records from the permuted CSR, the kernel's shared-memory
// limit, and a launch (one cluster of `cluster` (1, 2, 4 or 8) blocks of csr_resident_threads()
// per chain).
int csr_resident_threads();
int csr_resident_max_positions();  // per site thread and colour class
cudaError_t launch_pack_csr_records(int32_t n, const int32_t *rp, const int32_t *ci, uint4 *nbr, uint4 *nbr2,
                                    cudaStream_t stream);
cudaError_t prepare_csr_resident(int precision, size_t smem);
int csr_resident_site_threads();
// positions: 1 when every block's share of every class fits its site threads (then the next
// step's loads are issued ahead), else csr_resident_max_positions() / csr_resident_site_threads().
cudaError_t launch_csr_resident(int precision, int cluster, int positions, int chains, const ResCsrArgs &a,
                                size_t smem, cudaStream_t stream);

// Chain diagnostics (diagnostics.cu): one parameter trace of every chain of one field.
struct DiagArgs {
    const double *trace;   // [chains][cap] ring buffers; the value of sweep t sits at t % cap
    long long cap;
    long long sweep;       // sweeps done: the last N values are those of sweeps sweep-N .. sweep-1
    long long N;           // values used (4 <= N <= min(cap, available) for an IAT)
    int32_t reciprocal;    // 1: use 1 / value (tau^2 from the tau trace)
    int32_t chains;
    double *work;          // [chains][N] scratch
    double *out;           // [chains][4]: IAT, ESS, mean, variance (divisor N - 1)
    double *psrf;          // [1] potential scale reduction factor over the chains
};
cudaError_t launch_trace_diagnostics(const DiagArgs &a, cudaStream_t stream);
// Per-site potential scale reduction from the running means and M2 (count accumulated sweeps),
// natural order into out[n]; the maximum's bit pattern into *max_bits (atomic max, caller zeroes).
cudaError_t launch_site_psrf(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, int32_t Cp,
                             int32_t C, const void *mean, const void *m2, long long count, const int32_t *perm_inv,
                             double *out, unsigned long long *max_bits, cudaStream_t stream);

// Records msg as the calling thread's gmrf_last_error() text and returns st (api.cu).
int record_error(int st, const char *msg);

// Quad kernel for single-chain FP32 8-neighbour lattices (lattice_quad.cu); tiles TR x (2 qcs - 8)
// with TR even and origins at even rows and columns that are multiples of 4.
size_t lattice_quad_smem(int qcs, int TR);
cudaError_t prepare_lattice_quad(int qcs, int nt, int nq, size_t smem);
cudaError_t launch_lattice_quad(int qcs, int nt, int nq, const FusedArgs &a, size_t smem, cudaStream_t stream);
// The resident tile kernels (the quad kernel's and the fused 2-D sweep's resident forms): `count`
// whole sweeps of the single field in one cooperative launch, one block per tile, every block
// resident at once.
struct TileResArgs {
    FusedArgs f;              // the tiling and buffers of the per-sweep kernel (update 1)
    HyperArgs h;              // the conjugate draws at the end of each sweep (end_of_sweep 1)
    int32_t count;            // sweeps of the launch
    double *pm;               // fused tiles with four chains per thread: the tile partials again,
                              // [Cp][S, R, A][tile of the field], so that a warp's reads of one
                              // value over 32 tiles cover consecutive doubles (in the partial
                              // records they fall in 32 lines); null otherwise
    uint32_t extra_arrivals;  // 0; 1 under GMRF_FLAG_TEST_STALL (no grid barrier completes)
    uint64_t wait_ns;         // limit of a wait at the grid barrier
};
cudaError_t lattice_quad_resident_fits(int qcs, int nt, int nq, size_t smem, int ntiles, bool *fits);
// The fused sweep's resident form (lattice_fused_resident.cu; FP32, every thread holding all Cp
// chains as lattice_fused_fast): whether the tiles fit in one wave, and the launch.
cudaError_t lattice_fused_resident_fits(int kind, int threads, int Cp, size_t smem, int ntiles, bool *fits);
cudaError_t launch_lattice_fused_resident(int kind, int threads, int Cp, const TileResArgs &ra, size_t smem,
                                          cudaStream_t stream);
cudaError_t launch_lattice_quad_resident(int qcs, int nt, int nq, const TileResArgs &ra, size_t smem,
                                         cudaStream_t stream);

// Jones-Plassmann colouring and colour-permuted CSR layout (csr_build.cu).
struct CsrBuild {
    int32_t n;
    const int32_t *rp;     // device, natural order
    const int32_t *ci;
    const double *w;       // device or nullptr
    int32_t *colors;       // device [n] (in: given colours, or out: JP colours)
};
// JP colouring on the device; priorities: device [n] or nullptr for Philox(seed).
// Scratch (`scratch_bytes` from jp_scratch_bytes) is caller-provided device memory.
size_t jp_scratch_bytes(int32_t n);
// ldf (with prio == nullptr): largest-degree-first priorities of `seed` instead of the random ones.
cudaError_t jp_color(int32_t n, const int32_t *rp, const int32_t *ci, const uint32_t *prio,
                     uint64_t seed, int32_t *colors, void *scratch, int32_t *num_colors_host,
                     cudaStream_t stream, bool ldf = false);
// Stable counting sort by colour of the sites taken in the sequence `order` (device, n
// vertices; null: natural order), and the permuted CSR (cols remapped, row order kept),
// degrees and weights in precision T.  Outputs are device arrays of the field's block.
size_t layout_scratch_bytes(int32_t n, int32_t ncolors);
cudaError_t csr_layout(int precision, int32_t n, int32_t ncolors, const int32_t *rp, const int32_t *ci,
                       const double *w, const int32_t *colors, const int32_t *order, void *scratch,
                       int32_t *perm, int32_t *perm_inv, int32_t *coff, int32_t *rp_out, int32_t *ci_out,
                       void *w_out, void *deg_out, cudaStream_t stream);

// Plain FP64 baseline sweep (plain.cu): natural layout, one pass per colour over all sites.
struct PlainArgs {
    int32_t n;
    int32_t kind;
    int32_t dims[3];
    const int32_t *rp;     // CSR graphs (natural order) or nullptr for lattices
    const int32_t *ci;
    const double *w;
    const int32_t *colors; // natural order
    int32_t ncolors;
    double *x;             // [C][n] natural order
    const double *y;
    double *tau, *sig2;    // [C]
    double *trace_tau, *trace_sig;
    int32_t trace_cap;
    double *red;           // [C][2] scratch sums
    SweepCtl *ctl;
    uint2 key;
    uint32_t stream_id;
    int32_t C;
    int32_t lanes;         // normals per site of one Philox block: min(4, chains rounded up)
    int32_t rank;
    double rho;
    double a_tau, b_tau, a_sig, b_sig;
    int32_t draw;
};
cudaError_t launch_plain_sweep(const PlainArgs &a, cudaStream_t stream, int64_t *launches);

}  // namespace gmrf
