/*
 * gmrf.h -- C ABI of libgmrf, a GB300 (sm_103a) library for chromatic Gibbs sampling of
 * Gaussian Markov random fields, after Brown, McMahan & Self, "Sampling Strategies for Fast
 * Updating of Gaussian Markov Random Fields" (arXiv 1702.05518).
 *
 * Model (Sec. 2.2, Sec. 3.1; Sec. 3.2 for the proper prior).  A field has n sites on an
 * undirected graph with symmetric weights w_ij > 0 (w_ij = 1 unless given), degrees
 * d_i = sum_j w_ij, observations y = x + eps, eps ~ N(0, sigma^2 I), and the CAR prior with
 * precision tau (D - rho W): rho = 1 is the intrinsic CAR ("IAR"), 0 <= rho < 1 the proper CAR.
 * tau here is a precision: tau = 1 / tau^2 in the paper's notation.  Conjugate priors
 * tau ~ Gamma(a_tau, rate b_tau), 1/sigma^2 ~ Gamma(a_sigma, rate b_sigma).
 *
 * One sweep (Algorithm 1) visits the colour classes A_0..A_{k-1} of a proper colouring in
 * order and draws every site of the class at once from its full conditional
 *     x_i | x_-i ~ N((tau rho s_i + y_i / sigma^2) / P_i, 1 / P_i),
 *     P_i = tau d_i + 1 / sigma^2,  s_i = sum_j w_ij x_j,
 * then (unless the hyperparameters are fixed) draws
 *     tau       ~ Gamma(a_tau + r/2,  rate b_tau + x'(D - rho W)x / 2),
 *     1/sigma^2 ~ Gamma(a_sigma + n/2, rate b_sigma + ||y - x||^2 / 2),
 * with r = n - (connected components) for the intrinsic prior and r = n for the proper one
 * (Sec. 3.1 full conditionals).
 *
 * Random numbers are Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed, with
 * counters that name the draw, so results do not depend on launch shapes or on the order of
 * sites within a colour class:
 *     site update      a block gives normals n0, n1 (cos, sin of Box-Muller(w0, w1)) and n2, n3
 *                      (of (w2, w3)), u = (w + 1/2) 2^-32; with lanes = min(4, chains
 *                      rounded up to a power of two) and G = 4 / lanes it serves G consecutive
 *                      sites: counter (site / G, sweep, stream, (0 << 24) | chain/4), normal
 *                      n[(site mod G) * lanes + chain mod lanes].
 *     tau draw         counter (attempt, sweep, stream, (1 << 24) | chain)   [Marsaglia-Tsang]
 *     1/sigma^2 draw   counter (attempt, sweep, stream, (2 << 24) | chain)
 *     JP priority      word 0 of counter (vertex, 0, 0, 3 << 24)
 *     beta0 draw       Box-Muller cosine of (w0, w1) at counter (0, sweep, stream, (7 << 24) | chain)
 *     extra hyper draw counter (attempt, k, stream, ((5|6) << 24) | chain) and, for beta0,
 *                      (0, k, stream, (8 << 24) | chain), k-th call of gmrf_hyper_update
 * "site" is the natural (row-major for lattices) index, "stream" the field's stream id.
 *
 * Conventions.  Every call returns a gmrf_status and never aborts or prints.  Host pointers
 * are read during the call only and stay owned by the caller; the library owns every device
 * buffer it allocates.  A failed create leaves *out == NULL.  After a CUDA error a sampler is
 * poisoned: later calls on it return GMRF_E_STATE.  gmrf_last_error() describes the last
 * failure of the calling thread.  A sampler is bound to the device current at creation and to
 * one CUDA stream; it is not thread-safe.
 */
#ifndef GMRF_H
#define GMRF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GMRF_OK = 0,
    GMRF_E_INVALID = 1,     /* an argument failed validation; nothing was launched         */
    GMRF_E_CUDA = 2,        /* a CUDA call failed; the sampler is poisoned                 */
    GMRF_E_OOM = 3,         /* device allocation failed                                   */
    GMRF_E_STATE = 4,       /* sampler poisoned by an earlier error, or call out of order  */
    GMRF_E_TIMEOUT = 5,     /* a bounded device wait gave up: the results of the sweeps     */
                            /* since are invalid; reported by the next call that reads the  */
                            /* sampler's counters (fetches, info, diagnostics), which then  */
                            /* poisons the sampler                                          */
    GMRF_E_UNSUPPORTED = 6  /* valid request that the library does not implement          */
} gmrf_status;

typedef enum {
    GMRF_LATTICE2D_4 = 0,   /* H x W lattice, 4 neighbours, 2 colours (i + j) mod 2          */
    GMRF_LATTICE2D_8 = 1,   /* H x W lattice, 8 neighbours, 4 colours 2 (i mod 2) + (j mod 2) */
    GMRF_LATTICE3D_6 = 2,   /* L x H x W lattice, 6 neighbours, 2 colours (l + i + j) mod 2  */
    GMRF_CSR = 3            /* arbitrary graph in compressed sparse rows                   */
} gmrf_field_kind;

typedef enum { GMRF_PRIOR_ICAR = 0, GMRF_PRIOR_PCAR = 1 } gmrf_prior_kind;
typedef enum { GMRF_FP32 = 0, GMRF_FP64 = 1 } gmrf_precision;
typedef enum {
    GMRF_ALGO_CHROMATIC = 0, /* colour-split layout, fused per-colour kernels (the product)   */
    GMRF_ALGO_PLAIN = 1      /* natural layout, one unfused pass over all sites per colour;
                                the plain single-field FP64 reference sweep for speed-ups   */
} gmrf_algorithm;

/*
 * One field.  Lattices (Sec. 2.3, Fig. 1: colourings found by inspection) have free,
 * non-periodic boundaries (Sec. 3.1, edge effects ignored: border sites have fewer
 * neighbours) and sites in row-major order: 2-D site (i, j) = i*W + j with dims = {H, W, 0};
 * 3-D site (l, i, j) = (l*H + i)*W + j with dims = {L, H, W}.  A CSR graph (Sec. 2.3) gives
 * row_ptr[n+1], col_idx[nnz] (int32, host): symmetric, no self-loops, no duplicate entries,
 * rows in any order; weights[nnz] (host, symmetric, > 0) or NULL for w_ij = 1; colors[n]
 * (host) a proper colouring, or NULL to colour on the device by Jones-Plassmann with Philox
 * priorities of `color_seed`.
 */
typedef struct {
    int32_t kind;             /* gmrf_field_kind                                            */
    int32_t dims[3];          /* lattice extents (see above); unused for CSR                */
    int32_t n;                /* sites; must equal the product of dims for lattices         */
    const int32_t *row_ptr;   /* CSR only                                                   */
    const int32_t *col_idx;   /* CSR only                                                   */
    const double *weights;    /* CSR only, may be NULL                                      */
    const int32_t *colors;    /* CSR only, may be NULL                                      */
    uint64_t color_seed;      /* CSR with colors == NULL: priority seed (see GMRF_FLAG_COLOR_RANDOM) */
    const double *y;          /* [n] observations, natural order (host)                     */
    const double *x0;         /* [chains][n] initial states (host) or NULL: x0 = y          */
    const double *tau0;       /* [chains] initial tau or NULL: model.tau0                   */
    const double *sigma2_0;   /* [chains] initial sigma^2 or NULL: model.sigma2_0           */
    uint32_t stream_id;       /* Philox counter word 2 of this field's draws                */
    const double *beta0;      /* [chains] initial intercept or NULL: model.beta0_0           */
    const int32_t *trials;    /* binomial likelihood: [n] trials m_i (0..4095), y = successes */
                              /* (0 <= y_i <= m_i); NULL for the Gaussian likelihood          */
} gmrf_field_desc;

/* Likelihoods.  Gaussian: y_i = [beta0 +] x_i + N(0, sigma^2) (Sec. 3.1).  Binomial:
 * y_i ~ Bin(m_i, logistic(beta0 + x_i)) with beta0 ~ N(beta0_mean, beta0_var) and no sigma^2
 * (Sec. 3.2); each sweep draws psi_i ~ PG(m_i, beta0 + x_i) (Polya-Gamma augmentation, counters
 * (site, sweep, stream, 0xA << 28 | chain << 22 | k << 10 | j) for the k-th PG(1) summand's j-th
 * Philox block) right before site i's update, whose precision is tau d_i + psi_i and mean
 * (tau rho s_i + y_i - m_i/2 - psi_i beta0) / P, then beta0 given x and psi, then tau.  The
 * binomial likelihood runs on the per-colour kernels, with default x0 = 0. */
typedef enum { GMRF_LIKELIHOOD_GAUSSIAN = 0, GMRF_LIKELIHOOD_BINOMIAL = 1 } gmrf_likelihood;

typedef struct {
    int32_t prior;            /* gmrf_prior_kind                                            */
    double rho;               /* proper CAR: 0 <= rho < 1; ignored for the intrinsic prior  */
    double a_tau, b_tau;      /* tau ~ Gamma(a_tau, rate b_tau); a_tau > 0, b_tau >= 0      */
    double a_sigma, b_sigma;  /* 1/sigma^2 ~ Gamma(a_sigma, rate b_sigma)                   */
    int32_t fix_hyper;        /* nonzero: tau, sigma^2 stay at their initial values         */
    double tau0, sigma2_0;    /* default initial values (tau0 >= 0, sigma2_0 > 0)            */
    int32_t intercept;        /* 1: y = beta0 1 + x + noise with a flat prior on beta0 and  */
                              /* beta0 | x, sigma^2 ~ N(1'(y - x)/n, sigma^2/n) drawn before */
                              /* sigma^2 (Sec. 3.1); 0: no intercept                         */
    double beta0_0;           /* default initial intercept (used when intercept = 1)        */
    int32_t likelihood;       /* gmrf_likelihood                                            */
    double beta0_mean, beta0_var; /* binomial likelihood: beta0 ~ N(beta0_mean, beta0_var)   */
} gmrf_model;

/*
 * Launch configuration of a sampler (the kernels' work decomposition; it changes the results only
 * through the rounding of the partial sums).  Zero fields keep the library's cost models; a
 * tuning is usually found by gmrf_autotune.  Invalid values make gmrf_sampler_create return
 * GMRF_E_INVALID.
 */
typedef struct {
    int32_t chains_per_thread;   /* chains one thread updates together: 1, 2 or 4 (FP64: 1 or 2),   */
                                 /* at most the chains rounded up to a power of two; 0: automatic   */
    int32_t step_tile;           /* per-colour kernels (3-D lattices, graphs): (site, chain group)   */
                                 /* elements per block, 256..16384; 0: automatic                     */
    int32_t fused_rows[2];       /* fused 2-D sweep, per kind (index GMRF_LATTICE2D_4, _8): tile rows */
    int32_t fused_cols[2];       /* and columns, 8..256 (made even); 0: automatic                    */
    int32_t fused_threads[2];    /* threads per block, 512 or 1024; 0: automatic                     */
    int32_t quad_config;         /* 8-neighbour lattices, one chain, FP32: quad kernel configuration  */
                                 /* 1..5, -1 for the general fused kernel; 0: automatic               */
    int32_t quad_rows;           /* the quad kernel's tile rows (even, >= 8); 0: automatic            */
    int32_t wide_3d;             /* 3-D lattices, FP32, 3 to 8 chains: 1 updates every chain of a     */
                                 /* site in one thread, -1 keeps chains_per_thread; 0: automatic      */
                                 /* (the former for classes of >= 256 sites per SM when               */
                                 /* chains_per_thread is 0)                                           */
    int32_t graph_cluster;       /* resident graph path: blocks sharing a chain, 1, 2, 4 or 8 (times  */
                                 /* the chains at most 152); a class share that does not fit the      */
                                 /* blocks keeps the per-colour path; 0: automatic (one block per     */
                                 /* 2048 sites, at most 8)                                            */
} gmrf_tuning;

typedef struct {
    int32_t precision;        /* gmrf_precision: state and site arithmetic                  */
    int32_t chains;           /* independent chains per field, 1..64                        */
    uint64_t seed;            /* Philox key                                                 */
    int64_t start_sweep;      /* number of the first sweep (resume); 0 for a fresh run       */
    int64_t burn_in;          /* sweeps numbered < burn_in are not accumulated              */
    int32_t thin;             /* accumulate sweeps burn_in, burn_in + thin, ... (>= 1)       */
    int32_t trace_capacity;   /* tau/sigma^2 trace ring length per chain (>= 1)             */
    int32_t algorithm;        /* gmrf_algorithm                                             */
    int32_t graph_sweeps;     /* sweeps captured per CUDA graph; 0 = launch kernels directly */
    int32_t flags;            /* GMRF_FLAG_* bits; 0 for the defaults                        */
    const gmrf_tuning *tuning; /* launch configuration (host, copied) or NULL: automatic       */
} gmrf_opts;

/* gmrf_opts.flags: GMRF_FLAG_PER_COLOUR makes 2-D lattice fields use one launch per colour
 * class instead of the fused one-launch-per-sweep kernel (same results up to rounding).
 * Resident path: a sampler of one small 2-D lattice field (Gaussian likelihood; each chain's
 * state, observations, mean and M2 fit one block's shared memory; at most 1152 sites per colour
 * class on the 8-neighbour lattice, e.g. 64 x 72, and 72 x 64 sites or the like on the
 * 4-neighbour one), or of one small graph (unit weights, Gaussian likelihood, fewer than 32768
 * sites with state, mean and M2 in shared memory, at most 16 neighbours, 64 colours and 4096
 * sites per colour class), runs a batch of whole sweeps per launch, one block per chain (same
 * draws and counters, results equal up to rounding).  A larger FP32 2-D lattice field whose
 * per-sweep kernel's tiles can all be resident at once also runs a batch of sweeps per launch:
 * one cooperative launch, a block per tile keeping it in shared memory, a grid barrier (bounded
 * wait) per sweep, results bit for bit those of the per-sweep launches -- the quad kernel's tiles
 * for single-chain 8-neighbour fields (1024 x 1024 takes 144 blocks), else the fused sweep's when
 * every thread holds all chains (1, 2 or 4 in the layout).  On by default in FP32;
 * GMRF_FLAG_RESIDENT asks for the small-lattice form in FP64 as well, GMRF_FLAG_NO_RESIDENT keeps
 * the per-sweep launches.
 * gmrf_info.resident tells which path a sampler took. */
#define GMRF_FLAG_PER_COLOUR 1
#define GMRF_FLAG_NO_RESIDENT 2
#define GMRF_FLAG_RESIDENT 4
/* GMRF_FLAG_TEST_STALL (for tests of failure handling only): on the resident graph path with a
 * cluster of two or more blocks per chain (a single graph of 4096 or more sites), every colour
 * step of the cluster kernel expects 16 more bytes than the other blocks send, and on the resident
 * tile paths every grid barrier expects one arrival more than there are blocks, so the bounded
 * wait gives up (after 1 ms with this flag, instead of 1 s), as a lost exchange would make it; the
 * kernel still finishes, and the next call that reads the counters returns GMRF_E_TIMEOUT. */
#define GMRF_FLAG_TEST_STALL 8
/* Graphs that a sampler colours itself (colors == NULL) take Jones-Plassmann with
 * largest-degree-first priorities: min(degree, 255) in the top 8 bits, the top 24 bits of the
 * random priority of color_seed (the priority gmrf_color_graph uses for that seed) below, so
 * vertices of larger degree are coloured first; the colouring equals the greedy colouring in
 * that priority order and usually needs fewer colours, i.e. fewer colour steps per sweep (the
 * 16,384-site Delaunay graph: 6 against 7).  GMRF_FLAG_COLOR_RANDOM takes the random priorities
 * alone, as gmrf_color_graph with that seed does. */
#define GMRF_FLAG_COLOR_RANDOM 16

typedef struct {
    int32_t nfields;
    int32_t chains;
    int32_t precision;
    int32_t max_colors;       /* colour steps per sweep                                     */
    int64_t sweeps_done;      /* sweeps completed (start_sweep included)                    */
    int64_t accumulated;      /* sweeps accumulated into the running mean / variance         */
    int64_t hyper_fallbacks;  /* Gamma draws that hit the 64-attempt limit (normally 0)     */
    int64_t device_bytes;     /* device memory held by the sampler                          */
    int64_t launches_per_sweep; /* kernels launched per sweep                               */
    int64_t early_start_misses; /* sweep kernels that started before their predecessor ended */
                                /* with a wrong sweep-number prediction (normals redrawn)    */
    int64_t resident;         /* sweeps run on the resident path: 1 small lattice, 2 graph,   */
                              /* 3 quad lattice tiles, 4 fused lattice tiles; 0 not          */
    int64_t wait_timeouts;    /* bounded device waits that gave up (then results are invalid) */
} gmrf_info;

typedef struct gmrf_sampler gmrf_sampler;

/*
 * Colour a CSR graph by Jones-Plassmann on the device (Sec. 2.3: a colouring is a one-off
 * pre-computation; the paper's greedy colouring is the special case priority = -index).
 * Round by round, every uncoloured vertex whose (priority, index) is larger than that of all
 * its uncoloured neighbours takes the smallest colour absent among its coloured neighbours;
 * the result equals sequential greedy colouring in decreasing (priority, index) order.
 *   n, row_ptr[n+1], col_idx[nnz]: host CSR, validated as for gmrf_field_desc.
 *   priorities: host [n] or NULL for Philox priorities of `seed`.
 *   colors: host out [n], 0-based; num_colors: out.
 * Device scratch is allocated and freed inside the call; runs on the legacy default stream
 * and synchronises.  Errors: GMRF_E_INVALID (bad CSR / NULL outputs), GMRF_E_CUDA, GMRF_E_OOM.
 */
gmrf_status gmrf_color_graph(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             const uint32_t *priorities, uint64_t seed, int32_t *colors,
                             int32_t *num_colors);

/* Vertex capacity of the static scratch of gmrf_color_graph_noalloc (5 MiB of device memory). */
#define GMRF_NOALLOC_MAX_VERTICES 1048576

/*
 * The colouring of gmrf_color_graph (same rounds, same result) for a CSR graph already on the
 * device, allocating no memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory -- a process whose device memory
 * is held by its own caching allocator (a cudaMalloc inside the call could fail although the
 * pool has room) or a serving loop that must not take the device-wide synchronisation that
 * cudaFree implies.
 *   n: vertices, 1 <= n <= GMRF_NOALLOC_MAX_VERTICES (larger n: GMRF_E_INVALID, nothing runs).
 *   nnz: entries of col_idx.  row_ptr[n+1], col_idx[nnz]: device, caller-owned, read only.
 *   priorities: device [n] or NULL for Philox priorities of `seed`.
 *   colors: device out [n], 0-based, caller-owned; num_colors: host out.
 *   cuda_stream: a cudaStream_t (NULL: legacy default stream); the call synchronises it.
 * Scratch: one fixed file-scope device array (priorities, round flags, counters; 5 MiB).  It is
 * part of the library's device code, which CUDA loads onto a device when the library first runs
 * there (lazy module loading, the default): so make a first call of this function (or any other
 * library call on that device) before the caller's allocator reserves the device's memory, or
 * load modules eagerly (CUDA_MODULE_LOADING=EAGER).  The first call on each device, with that
 * device current, looks up the array's address (cudaGetSymbolAddress) and keeps it for the
 * process; make that first call before any stream capture.  A reset of the device
 * (cudaDeviceReset) unloads the array: do not call this function after one.  Each call clears
 * the counters and the check flag it needs at its start.  Concurrent or overlapping calls on
 * one device share the array and race: serialise them.
 * The structure (row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz, columns in [0, n), no
 * self-loops) is checked on the device before colouring: GMRF_E_INVALID if it fails.  Symmetry
 * is the caller's duty and is not checked: for a non-symmetric graph the call still stays in
 * bounds and terminates, but its result is unspecified (it may differ from run to run and need
 * not be a proper colouring).
 * Errors: GMRF_E_INVALID, GMRF_E_UNSUPPORTED (device ordinal > 63), GMRF_E_CUDA.
 */
gmrf_status gmrf_color_graph_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                     const int32_t *col_idx, const uint32_t *priorities,
                                     uint64_t seed, int32_t *colors, int32_t *num_colors,
                                     void *cuda_stream);

/*
 * Create a sampler over `nfields` independent fields (each with `opts.chains` chains and its
 * own tau, sigma^2 per chain), copy y / x0 / graphs to the device in the colour-split layout
 * (Sec. 3.1: chromatic sampling needs only the lists of sites of each colour), and colour CSR fields that
 * come without colours.  `cuda_stream` (a cudaStream_t, or NULL for the legacy default
 * stream) is the stream every later call enqueues on.  All host inputs are copied; none is
 * retained.  Errors: GMRF_E_INVALID, GMRF_E_UNSUPPORTED (e.g. GMRF_ALGO_PLAIN with more than
 * one field or non-FP64), GMRF_E_OOM, GMRF_E_CUDA.  On error *out is NULL.
 */
gmrf_status gmrf_sampler_create(gmrf_sampler **out, const gmrf_field_desc *fields,
                                int32_t nfields, const gmrf_model *model, const gmrf_opts *opts,
                                void *cuda_stream);

/* Release every device buffer and CUDA graph of the sampler (synchronises its stream). */
void gmrf_sampler_destroy(gmrf_sampler *s);

/*
 * Enqueue `nsweeps` sweeps (Algorithm 1 over all colours of all fields, then -- unless
 * with_hyper == 0 -- the intercept draw (model.intercept) and the conjugate tau, sigma^2 draws
 * (unless model.fix_hyper), then trace and accumulator updates) on the sampler's stream.  Asynchronous: returns before the work finishes.
 * Errors: GMRF_E_INVALID (nsweeps < 0), GMRF_E_STATE, GMRF_E_CUDA.
 */
gmrf_status gmrf_sweep(gmrf_sampler *s, int32_t nsweeps, int32_t with_hyper);

/*
 * One extra draw of tau and sigma^2 (and beta0 first, with the intercept) from their full
 * conditionals (Sec. 3.1) given the current x of every field and chain, without a sweep
 * (counters: tags 5, 6 and 8, k = number of earlier calls).  Asynchronous.  Errors: GMRF_E_STATE, GMRF_E_CUDA.
 */
gmrf_status gmrf_hyper_update(gmrf_sampler *s);

/*
 * Copy results of one (field, chain) to host buffers in natural site order (synchronises the
 * stream).  Any output pointer may be NULL.
 *   x_last[n]: current state;  x_mean[n], x_var[n]: running mean and sample variance
 *   (M2 / (count - 1)) over the accumulated sweeps (zeros / NaN when fewer than 1 / 2);
 *   tau_trace[trace_cap], sigma2_trace[trace_cap]: the last min(trace_cap, available) values,
 *   oldest first; *n_trace: values available (<= opts.trace_capacity);
 *   tau_now, sigma2_now: current hyperparameters.
 * Errors: GMRF_E_INVALID (field/chain out of range), GMRF_E_STATE, GMRF_E_CUDA.
 */
gmrf_status gmrf_fetch_samples(gmrf_sampler *s, int32_t field, int32_t chain, double *x_last,
                               double *x_mean, double *x_var, int64_t trace_cap,
                               double *tau_trace, double *sigma2_trace, int64_t *n_trace,
                               double *tau_now, double *sigma2_now);

/*
 * The intercept of one (field, chain) (model.intercept = 1): the current beta0 and the last
 * min(trace_cap, available) values of its trace (the value after each sweep, oldest first),
 * like the tau/sigma^2 traces of gmrf_fetch_samples.  Synchronises the stream.  Any output
 * pointer may be NULL.  Errors: GMRF_E_INVALID (no intercept, bad indices), GMRF_E_STATE,
 * GMRF_E_CUDA.
 */
gmrf_status gmrf_fetch_intercept(gmrf_sampler *s, int32_t field, int32_t chain, int64_t trace_cap,
                                 double *beta0_trace, int64_t *n_trace, double *beta0_now);

/* Parameters whose traces gmrf_trace_diagnostics reads. */
typedef enum {
    GMRF_PARAM_TAU2 = 0,      /* tau^2 = 1/tau, the paper's variance parameter of the prior  */
    GMRF_PARAM_SIGMA2 = 1,
    GMRF_PARAM_BETA0 = 2,     /* only with model.intercept                                   */
    GMRF_PARAM_TAU = 3        /* the precision tau itself                                    */
} gmrf_param;

/*
 * Chain diagnostics of one parameter of one field (Sec. 3.1 compares samplers by the IAT kappa
 * and effective sample size of the tau^2 chain and by the cost per effective sample
 * CES = kappa T / N, T the run time and N the retained sample).  Over the last n_last values of
 * the trace (0: all available; at most opts.trace_capacity), on the device:
 *   iat[chains]: kappa by Geyer's initial monotone sequence estimator (Geyer 1992, Sec. 3.3):
 *     gamma(k) = (1/N) sum_t (x_t - mean)(x_{t+k} - mean), Gamma_m = gamma(2m) + gamma(2m+1),
 *     kappa = (-gamma(0) + 2 sum_{m<=M} min(Gamma_0..Gamma_m)) / gamma(0), M the last m of the
 *     initial positive sequence, floored at 1/log10(N); NaN for N < 4 or a constant chain;
 *   ess[chains]: N / kappa;
 *   psrf: potential scale reduction factor over the chains (Gelman & Rubin 1992 with the
 *     (m + 1)/m factor of Brooks & Gelman 1998), NaN with one chain.
 * Any output may be NULL.  Synchronises the stream.  Errors: GMRF_E_INVALID (bad field or
 * param, fewer than 2 values), GMRF_E_UNSUPPORTED (plain algorithm), GMRF_E_STATE, GMRF_E_CUDA.
 */
gmrf_status gmrf_trace_diagnostics(gmrf_sampler *s, int32_t field, int32_t param, int64_t n_last,
                                   double *iat, double *ess, double *psrf);

/*
 * Potential scale reduction factor of every site of one field over the chains, from the running
 * means and variances of the accumulated sweeps (same formula as gmrf_trace_diagnostics with N
 * = accumulated sweeps): psrf[n] in natural site order (host, may be NULL) and its maximum over
 * the sites (NaN sites skipped).  Needs >= 2 chains and >= 2 accumulated sweeps (else
 * GMRF_E_INVALID).  Synchronises the stream.
 */
gmrf_status gmrf_site_psrf(gmrf_sampler *s, int32_t field, double *psrf, double *psrf_max);

/*
 * Restart the run: state, tau, sigma^2 and beta0 back to their values at creation, sweep counter back
 * to opts.start_sweep, accumulators cleared.  Asynchronous (device copies on the sampler's
 * stream); lets one sampler run many independent MCMC runs of the same data without re-upload.
 * Errors: GMRF_E_STATE, GMRF_E_CUDA.
 */
gmrf_status gmrf_sampler_reset(gmrf_sampler *s);

/*
 * Autotuner: measure launch configurations for these fields, model and options on the device and
 * return the fastest in *out (and its time per sweep in *us_per_sweep, may be NULL).  Candidates
 * are tried by coordinate descent from the automatic configuration: the chains per thread, the
 * colour-step tile, each 2-D kind's fused tile shape and block size, and the quad kernel's
 * configuration; each one is a sampler built from the same arguments (opts.tuning ignored) and
 * timed with CUDA events over `sweeps` sweeps (>= 1; graphs as in opts) after a warm-up, on
 * `cuda_stream`.  The result is cached for the process by (field kinds and sizes, chains,
 * precision, model and option switches): a later call with the same key returns it without
 * measuring.  Synchronises the stream; the device memory of one sampler at a time.
 * Errors: those of gmrf_sampler_create and gmrf_sweep.
 */
gmrf_status gmrf_autotune(const gmrf_field_desc *fields, int32_t nfields, const gmrf_model *model,
                          const gmrf_opts *opts, int32_t sweeps, void *cuda_stream, gmrf_tuning *out,
                          double *us_per_sweep);

/*
 * Replace the data of one field and restart the run: a sampler built once for a graph then
 * serves many data sets of that graph (the observations y of Sec. 3.1, or the successes and
 * trials of the binomial model of Sec. 3.2) without rebuilding its layout, tiles or graphs.
 *   y: host [n] observations in natural site order (finite; for the binomial likelihood the
 *      successes, 0 <= y[i] <= trials[i]).
 *   trials: host [n], required for the binomial likelihood (0..4095; 0 = site unobserved),
 *      ignored otherwise.
 *   x0: host [chains][n] initial states, or NULL for the creation default (y for the Gaussian
 *      likelihood, 0 for the binomial one).
 * Afterwards the sampler is in the state gmrf_sampler_create with these arrays followed by
 * gmrf_sampler_reset would give (all fields restart, as gmrf_sampler_reset does; the other
 * fields keep their data).  The host arrays are read before the call returns (it synchronises
 * the sampler's stream after its uploads); the rest is enqueued asynchronously.  The restart
 * itself is enqueued by the next call that uses the sampler's state (gmrf_sweep,
 * gmrf_hyper_update, the fetch, diagnostic and stage calls, gmrf_sampler_info), so a set_data call
 * per field restarts the chains once.  The first call
 * allocates a device staging buffer of (1 + chains) doubles (+ one int32 for binomial data) per
 * site of the largest field; later calls allocate nothing.
 * Errors: GMRF_E_INVALID (bad field index or data; nothing changes), GMRF_E_STATE, GMRF_E_OOM,
 * GMRF_E_CUDA.
 */
gmrf_status gmrf_sampler_set_data(gmrf_sampler *s, int32_t field, const double *y, const int32_t *trials,
                                  const double *x0);

/*
 * Diagnostic: enqueue exactly one launch of stage `stage` of a sweep on the sampler's stream.
 * A sweep is gmrf_info.launches_per_sweep stages in order: the fused 2-D lattice sweeps (one
 * per lattice kind present), the colour steps of the other fields (one per colour and field
 * kind), then the hyperparameter draw (the last stage, which also advances the sweep counter).
 * `accumulate` = 0 skips the running-mean update.  For timing one kernel in isolation; the state
 * moves on as in a sweep.  *name (may be NULL) receives a static description of the stage.
 * Errors: GMRF_E_INVALID (stage out of range), GMRF_E_UNSUPPORTED (plain algorithm),
 * GMRF_E_STATE, GMRF_E_CUDA.
 */
gmrf_status gmrf_launch_stage(gmrf_sampler *s, int32_t stage, int32_t accumulate, const char **name);

/* The colouring a field is sampled with (natural order) and its number of colours. */
gmrf_status gmrf_field_colors(gmrf_sampler *s, int32_t field, int32_t *colors,
                              int32_t *num_colors);

/* Sizes and counters of the sampler (synchronises the stream). */
gmrf_status gmrf_sampler_info(gmrf_sampler *s, gmrf_info *out);

/*
 * Host-only check of a CSR graph against the rules of gmrf_field_desc (no CUDA call).
 * Returns GMRF_OK or GMRF_E_INVALID; *components (may be NULL) receives the number of
 * connected components, which sets the rank n - components of the intrinsic prior.
 */
gmrf_status gmrf_validate_csr(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                              const double *weights, int32_t *components);

/*
 * Diagnostics of the device random-number path (same generators the sweep kernels inline).
 * gmrf_philox_words: out[4i..4i+3] = Philox4x32-10 of counter (i, c1, c2, c3) under the key
 *   (seed lo, seed hi), i = 0..count-1.  `out` is a DEVICE pointer of 4*count words.
 * gmrf_site_normals: out[i] = the normal that updates (site i, chain) at `sweep` of a field
 *   with stream id `stream` in a sampler whose Philox blocks serve `lanes` chains (1, 2 or 4:
 *   min(4, chains rounded up to a power of two); see the layout above), in the given precision;
 *   `out` is a DEVICE pointer of `count` floats (GMRF_FP32) or doubles (GMRF_FP64).
 * Both enqueue on `cuda_stream` and return without synchronising.
 */
gmrf_status gmrf_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                              int64_t count, uint32_t *out, void *cuda_stream);
gmrf_status gmrf_site_normals(uint64_t seed, uint32_t sweep, uint32_t stream, uint32_t chain,
                              int32_t lanes, int32_t precision, int64_t count, void *out,
                              void *cuda_stream);

/*
 * The posterior mean and variance of one field pooled over its chains (natural site order, host
 * out [n] each, either may be NULL): mean = the chains' running means averaged; var = the
 * variance of all C k accumulated draws, (sum over chains of M2_c + k (mean_c - mean)^2) / (C k - 1)
 * with k draws per chain (Chan et al.'s pairwise combination of Welford's moments), in FP64 on
 * the device.  The multi-chain estimate of the posterior (Sec. 3.1 runs three chains) in one
 * read-back instead of one per chain.  Synchronises; before any accumulated sweep mean is 0
 * and var NaN.  Errors: GMRF_E_INVALID, GMRF_E_UNSUPPORTED (plain algorithm), GMRF_E_STATE,
 * GMRF_E_TIMEOUT, GMRF_E_CUDA.
 */
gmrf_status gmrf_fetch_pooled(gmrf_sampler *s, int32_t field, double *mean, double *var);

/*
 * Diagnostic: the time of the random numbers of one 3-D lattice colour step alone -- for each
 * of `sites` sites the normals of all its chains (chains <= 4: one Philox4x32-10 block and two
 * Box-Muller pairs; 5..8: two of each), with the counters and arithmetic of the sweep kernel,
 * summed per thread with no state traffic -- on the sweep kernel's grid.  `reps` timed launches
 * (CUDA events on cuda_stream, after 3 untimed ones); *us_per_launch receives their mean.  It
 * bounds the colour step from below the way the HBM roofline does.  Synchronises the stream.
 * Errors: GMRF_E_INVALID, GMRF_E_CUDA, GMRF_E_OOM.
 */
gmrf_status gmrf_normals_timing(uint64_t seed, int64_t sites, int32_t chains, int32_t reps, void *cuda_stream,
                                double *us_per_launch);

/*
 * Fault injection for tests of the error paths (process-wide, not thread-safe; no paper
 * counterpart).  gmrf_debug_fail_alloc: the nth device allocation the library makes from now on
 * (1 = the next) fails as if the device were out of memory (GMRF_E_OOM from the call that made
 * it, with everything that call allocated released); 0 disarms.  gmrf_debug_poison: marks a
 * sampler as after a CUDA error, so that its later calls return GMRF_E_STATE.
 */
gmrf_status gmrf_debug_fail_alloc(int64_t nth);
gmrf_status gmrf_debug_poison(gmrf_sampler *s);

/* Description of the last failure on the calling thread ("" if none). */
const char *gmrf_last_error(void);

/* Library version, "major.minor.patch". */
const char *gmrf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GMRF_H */
