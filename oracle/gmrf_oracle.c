/*
 * gmrf_oracle.c -- the oracle: a plain, slow, single-threaded FP64 CPU statement of the
 * chromatic Gibbs sampler for Gaussian Markov random fields of Brown, McMahan & Self,
 * "Sampling Strategies for Fast Updating of Gaussian Markov Random Fields" (arXiv 1702.05518).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  The product (the CUDA library) neither includes,
 * links nor calls anything here, and nothing here includes or calls the product: the two
 * share no code, no headers and no constants table.  Everything below is written from the
 * paper and from the published definitions of the generators it uses.
 *
 * What is computed, in the paper's order:
 *   - Colouring (Sec. 2.3): a proper colouring f: V -> {0..k-1}.  For graphs it is the
 *     sequential first-fit greedy colouring taken in decreasing (priority, index) order; with
 *     priority decreasing in the index it is the greedy colouring the paper gives (each class
 *     is the lexicographically first maximal independent set of the vertices still uncoloured).
 *     With largest-degree-first priorities (ora_priorities_ldf) higher-degree vertices come
 *     first, which usually needs fewer colours (one per colour step of a sweep).
 *     Lattices use the colourings found "by inspection" (Sec. 2.3, Fig. 1): parity for 4- and
 *     6-neighbour lattices, the 2x2 pattern for the 8-neighbour lattice.
 *   - One Gibbs sweep (Algorithm 1): for colour j = 0..k-1, every site i of colour j is drawn
 *     from its full conditional given the newest values of all other colours.  With the
 *     Gaussian likelihood y = x + eps, eps ~ N(0, sigma^2 I), and a CAR prior with precision
 *     tau (D - rho W) (Sec. 3.1 with tau = 1/tau^2_paper; rho = 1 is the intrinsic CAR, rho < 1
 *     the proper CAR of Sec. 3.2), the local characteristics (Sec. 3.1) are
 *         P_i = tau d_i + 1/sigma^2,  m_i = (tau rho s_i + y_i/sigma^2) / P_i,  s_i = sum_j w_ij x_j
 *     and x_i = m_i + z_i / sqrt(P_i) with z_i ~ N(0, 1).
 *   - Conjugate hyperparameter draws (Sec. 3.1 full conditionals, precision form):
 *         tau | x         ~ Gamma(a_tau + r/2,  rate b_tau + x'(D - rho W)x / 2),
 *         1/sigma^2 | x,y ~ Gamma(a_sig + n/2,  rate b_sig + ||y - x||^2 / 2),
 *     r = n - (number of connected components) for the intrinsic prior, r = n for the proper one.
 *   - Running posterior mean and sum of squared deviations (Welford) of x after burn-in.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), uniforms
 * u = (w + 1/2) 2^-32, normals by Box-Muller (four per Philox block, shared by consecutive sites
 * when there are fewer than four chains), Gamma variates by Marsaglia & Tsang (2000).
 * The counter assignment (which counter feeds which draw) is part of the parity contract with
 * the CUDA path and is stated in the comments of each generator below.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no contraction, so results are identical on
 * x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4): ten rounds of two 32x32->64 multiplications */
/* with the Weyl key schedule.                                                                 */
/* ------------------------------------------------------------------------------------------ */
enum {
    ORA_TAG_X = 0,     /* field-site update normals          */
    ORA_TAG_TAU = 1,   /* Gamma draw of tau                  */
    ORA_TAG_SIG = 2,   /* Gamma draw of 1/sigma^2            */
    ORA_TAG_PRIO = 3,  /* colouring priorities               */
    ORA_TAG_BETA = 7   /* normal of the intercept draw       */
};

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void ora_key_of_seed(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
}

/* Philox over counters (i, c1, c2, c3), i = 0..n-1: out[4i..4i+3]. */
void ora_philox_fill(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n, uint32_t *out)
{
    uint32_t key[2];
    ora_key_of_seed(seed, key);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, c1, c2, c3};
        ora_philox4x32_10(ctr, key, out + 4 * i);
    }
}

/* u = (w + 1/2) 2^-32, exactly representable in double and strictly inside (0, 1). */
double ora_uniform(uint32_t w)
{
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* Box-Muller: r = sqrt(-2 ln u_a), z_cos = r cos(2 pi u_b), z_sin = r sin(2 pi u_b). */
static void ora_box_muller(uint32_t wa, uint32_t wb, double *z_cos, double *z_sin)
{
    double ua = ora_uniform(wa), ub = ora_uniform(wb);
    double r = sqrt(-2.0 * log(ua));
    double th = 2.0 * M_PI * ub;
    *z_cos = r * cos(th);
    *z_sin = r * sin(th);
}

/* The four normals of one Philox block: (w0,w1) -> z0 = cos, z1 = sin; (w2,w3) -> z2, z3. */
void ora_normals4(const uint32_t w[4], double z[4])
{
    ora_box_muller(w[0], w[1], &z[0], &z[1]);
    ora_box_muller(w[2], w[3], &z[2], &z[3]);
}

/* Normals per site of one Philox block: `lanes` = min(4, C rounded up to a power of two) for a
 * sampler with C chains (1, 2 or 4). */
int32_t ora_lanes_for(int32_t chains)
{
    int32_t p = 1;
    while (p < chains) p <<= 1;
    return p < 4 ? p : 4;
}

/* The normal that updates (site, chain) at a given sweep of the field with stream id `stream`.
 * Each Philox block gives four normals n0, n1 (cos, sin of Box-Muller(w0, w1)) and n2, n3 (of
 * (w2, w3)); it serves G = 4 / lanes consecutive sites and `lanes` chains: block counter
 * (site / G, sweep, stream, (TAG_X << 24) | chain / 4), normal n[(site mod G) * lanes + chain mod
 * lanes].  With four or more chains this is one block per site and chain quadruple; with one
 * chain one block per four consecutive sites. */
double ora_site_normal(uint64_t seed, uint32_t site, uint32_t sweep, uint32_t stream, uint32_t chain,
                       int32_t lanes)
{
    uint32_t key[2], w[4];
    ora_key_of_seed(seed, key);
    uint32_t G = 4u / (uint32_t)lanes;
    uint32_t ctr[4] = {site / G, sweep, stream, ((uint32_t)ORA_TAG_X << 24) | (chain >> 2)};
    ora_philox4x32_10(ctr, key, w);
    double z[4];
    ora_normals4(w, z);
    return z[(site % G) * (uint32_t)lanes + chain % (uint32_t)lanes];
}

/* The update normals of sites 0..n-1 of one chain at one sweep (natural order). */
void ora_site_normals(uint64_t seed, int32_t n, uint32_t sweep, uint32_t stream, uint32_t chain,
                      int32_t lanes, double *out)
{
    for (int32_t i = 0; i < n; ++i)
        out[i] = ora_site_normal(seed, (uint32_t)i, sweep, stream, chain, lanes);
}

/* ------------------------------------------------------------------------------------------ */
/* Gamma(shape, rate) by Marsaglia & Tsang, "A simple method for generating gamma variables",  */
/* ACM TOMS 26(3), 2000: d = a - 1/3, c = 1/sqrt(9d); repeat z ~ N(0,1), v = (1 + c z)^3,      */
/* accept d v when v > 0 and ln u < z^2/2 + d - d v + d ln v.  Shapes below one are boosted by */
/* Gamma(a) = Gamma(a + 1) U^(1/a) (same paper, Sec. 6).                                       */
/* Attempt k uses the Philox block at counter (k, sweep, stream, (tag << 24) | chain):         */
/* z from Box-Muller (cos) of (w0, w1), the acceptance uniform from w2, the boost uniform from */
/* w3.  After 64 rejected attempts (probability below 1e-100 for the shapes used) the draw     */
/* returns d / rate and counts a fallback.                                                     */
/* ------------------------------------------------------------------------------------------ */
double ora_gamma_draw(double shape, double rate, uint64_t seed, uint32_t sweep, uint32_t stream,
                      uint32_t tag, uint32_t chain, int32_t *attempts_out)
{
    uint32_t key[2];
    ora_key_of_seed(seed, key);
    int boost = shape < 1.0;
    double a = boost ? shape + 1.0 : shape;
    double d = a - 1.0 / 3.0;
    double c = 1.0 / sqrt(9.0 * d);
    for (uint32_t k = 0; k < 64; ++k) {
        uint32_t ctr[4] = {k, sweep, stream, (tag << 24) | chain};
        uint32_t w[4];
        ora_philox4x32_10(ctr, key, w);
        double z, z_unused;
        ora_box_muller(w[0], w[1], &z, &z_unused);
        double v = 1.0 + c * z;
        if (v <= 0.0)
            continue;
        v = v * v * v;
        double u = ora_uniform(w[2]);
        if (log(u) < 0.5 * z * z + d - d * v + d * log(v)) {
            double g = d * v;
            if (boost)
                g *= pow(ora_uniform(w[3]), 1.0 / shape);
            if (attempts_out)
                *attempts_out = (int32_t)(k + 1);
            return g / rate;
        }
    }
    if (attempts_out)
        *attempts_out = -1;
    return d / rate;
}

/* Standard normal of the intercept draw after sweep `sweep`: the cosine normal of Box-Muller on
 * words (w0, w1) of the Philox block at counter (0, sweep, stream, (tag << 24) | chain). */
double ora_beta_normal(uint64_t seed, uint32_t sweep, uint32_t stream, uint32_t tag, uint32_t chain)
{
    uint32_t ctr[4] = {0u, sweep, stream, (tag << 24) | chain};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    double z[4];
    ora_philox4x32_10(ctr, key, w);
    ora_normals4(w, z);
    return z[0];
}

/* ------------------------------------------------------------------------------------------ */
/* Graphs                                                                                       */
/* ------------------------------------------------------------------------------------------ */
enum { ORA_LAT2D_4 = 0, ORA_LAT2D_8 = 1, ORA_LAT3D_6 = 2 };

/* Sites of a lattice in row-major order: 2-D site (i, j) -> i*W + j with dims = (H, W);
 * 3-D site (l, i, j) -> (l*H + i)*W + j with dims = (L, H, W).  Free (non-periodic) boundary:
 * edge sites simply have fewer neighbours (Sec. 3.1 "ignore edge effects").  Neighbourhoods:
 * 4 (|di| + |dj| = 1), 8 (max(|di|, |dj|) = 1, Sec. 3.1 "eight neighbors"), 6 (one axis step).
 * Returns the number of directed edges; row_ptr/col_idx may be NULL to query the size. */
int64_t ora_lattice_csr(int32_t kind, const int32_t dims[3], int32_t *row_ptr, int32_t *col_idx)
{
    int64_t L = 1, H, W;
    if (kind == ORA_LAT3D_6) { L = dims[0]; H = dims[1]; W = dims[2]; }
    else { H = dims[0]; W = dims[1]; }
    int64_t nnz = 0, site = 0;
    for (int64_t l = 0; l < L; ++l)
        for (int64_t i = 0; i < H; ++i)
            for (int64_t j = 0; j < W; ++j, ++site) {
                if (row_ptr) row_ptr[site] = (int32_t)nnz;
                for (int64_t dl = -1; dl <= 1; ++dl)
                    for (int64_t di = -1; di <= 1; ++di)
                        for (int64_t dj = -1; dj <= 1; ++dj) {
                            int64_t steps = (dl != 0) + (di != 0) + (dj != 0);
                            if (steps == 0) continue;
                            if (kind == ORA_LAT2D_4 && (dl != 0 || steps != 1)) continue;
                            if (kind == ORA_LAT2D_8 && dl != 0) continue;
                            if (kind == ORA_LAT3D_6 && steps != 1) continue;
                            int64_t ll = l + dl, ii = i + di, jj = j + dj;
                            if (ll < 0 || ll >= L || ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                            if (col_idx) col_idx[nnz] = (int32_t)((ll * H + ii) * W + jj);
                            ++nnz;
                        }
            }
    if (row_ptr) row_ptr[site] = (int32_t)nnz;
    return nnz;
}

/* Colourings "by inspection" (Sec. 2.3, Fig. 1): 4-neighbour 2-D and 6-neighbour 3-D lattices
 * take the parity of the coordinate sum (2 colours); the 8-neighbour 2-D lattice takes the 2x2
 * pattern colour = 2 (i mod 2) + (j mod 2) (4 colours).  Returns the number of colours. */
int32_t ora_lattice_colors(int32_t kind, const int32_t dims[3], int32_t *colors)
{
    int64_t L = 1, H, W;
    if (kind == ORA_LAT3D_6) { L = dims[0]; H = dims[1]; W = dims[2]; }
    else { H = dims[0]; W = dims[1]; }
    int64_t site = 0;
    for (int64_t l = 0; l < L; ++l)
        for (int64_t i = 0; i < H; ++i)
            for (int64_t j = 0; j < W; ++j, ++site) {
                if (kind == ORA_LAT2D_8) colors[site] = (int32_t)(2 * (i & 1) + (j & 1));
                else colors[site] = (int32_t)((l + i + j) & 1);
            }
    return kind == ORA_LAT2D_8 ? 4 : 2;
}

/* Colouring priorities: w0 of the Philox block at counter (v, 0, 0, TAG_PRIO << 24). */
void ora_priorities(uint64_t seed, int32_t n, uint32_t *prio)
{
    uint32_t key[2], w[4];
    ora_key_of_seed(seed, key);
    for (int32_t v = 0; v < n; ++v) {
        uint32_t ctr[4] = {(uint32_t)v, 0u, 0u, (uint32_t)ORA_TAG_PRIO << 24};
        ora_philox4x32_10(ctr, key, w);
        prio[v] = w[0];
    }
}

/* Largest-degree-first priorities (the Jones-Plassmann LDF variant, Sec. 2.3 leaves the order
 * of the greedy colouring open): the degree, capped at 255, in the top 8 bits and the top 24
 * bits of the random priority above below it, so vertices of larger degree are coloured first
 * and equal degrees fall back to the random order (then the index). */
void ora_priorities_ldf(uint64_t seed, int32_t n, const int32_t *row_ptr, uint32_t *prio)
{
    ora_priorities(seed, n, prio);
    for (int32_t v = 0; v < n; ++v) {
        int32_t d = row_ptr[v + 1] - row_ptr[v];
        if (d > 255) d = 255;
        prio[v] = ((uint32_t)d << 24) | (prio[v] >> 8);
    }
}

static const uint32_t *ora_sort_prio;
static int ora_cmp_desc(const void *a, const void *b)
{
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    uint32_t pu = ora_sort_prio[u], pv = ora_sort_prio[v];
    if (pu != pv) return pu > pv ? -1 : 1;
    return u > v ? -1 : (u < v ? 1 : 0);
}

/* Sequential first-fit greedy colouring in decreasing (priority, index) order: each vertex
 * takes the smallest colour not used by an already-coloured neighbour.  Returns k. */
int32_t ora_color_greedy(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         const uint32_t *prio, int32_t *colors)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) {
        order[v] = v;
        colors[v] = -1;
        if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
    }
    ora_sort_prio = prio;
    qsort(order, (size_t)n, sizeof(int32_t), ora_cmp_desc);
    unsigned char *used = (unsigned char *)calloc((size_t)maxdeg + 2, 1);
    int32_t k = 0;
    for (int32_t t = 0; t < n; ++t) {
        int32_t v = order[t];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t c = colors[col_idx[e]];
            if (c >= 0 && c <= maxdeg) used[c] = 1;
        }
        int32_t c = 0;
        while (used[c]) ++c;
        colors[v] = c;
        if (c + 1 > k) k = c + 1;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t cu = colors[col_idx[e]];
            if (cu >= 0 && cu <= maxdeg) used[cu] = 0;
        }
    }
    free(used);
    free(order);
    return k;
}

/* Number of connected components (isolated vertices count), by iterative depth-first search. */
int32_t ora_components(int32_t n, const int32_t *row_ptr, const int32_t *col_idx)
{
    int32_t *seen = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t comps = 0;
    for (int32_t s = 0; s < n; ++s) {
        if (seen[s]) continue;
        ++comps;
        int32_t top = 0;
        stack[top++] = s;
        seen[s] = 1;
        while (top > 0) {
            int32_t v = stack[--top];
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                int32_t u = col_idx[e];
                if (!seen[u]) { seen[u] = 1; stack[top++] = u; }
            }
        }
    }
    free(stack);
    free(seen);
    return comps;
}

/* x'(D - rho W)x with D = diag(sum_j w_ij), summed over undirected edges {i, j} (each stored
 * twice in the CSR, taken once where i < j): sum w_ij [rho (x_i - x_j)^2 + (1 - rho)(x_i^2 + x_j^2)].
 * For rho = 1 this is the intrinsic CAR quadratic form of Sec. 3.1. */
double ora_quadform(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *w,
                    double rho, const double *x)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col_idx[e];
            if (j <= i) continue;
            double wij = w ? w[e] : 1.0;
            double dx = x[i] - x[j];
            s += wij * (rho * dx * dx + (1.0 - rho) * (x[i] * x[i] + x[j] * x[j]));
        }
    return s;
}

/* ------------------------------------------------------------------------------------------ */
/* Polya-Gamma variates (Sec. 3.2: binomial data with the logistic link, augmented as in        */
/* Polson, Scott & Windle, JASA 2013).  PG(b, c) for an integer b >= 0 is the sum of b          */
/* independent PG(1, c) = J*(1, |c|/2) / 4 variates, each drawn by Devroye's alternating-series */
/* method (PSW 2013, Sec. 4 and appendix): a proposal from a mixture of an exponential tail on  */
/* (t, inf) and a truncated inverse-Gaussian on (0, t), t = 0.64, accepted by the partial sums  */
/* of the series a_0 - a_1 + a_2 - ...                                                          */
/*                                                                                              */
/* Random numbers: draw k (k < b) of (site, sweep, chain) reads a stream of uniforms            */
/* u = (w + 1/2) 2^-32 from the Philox blocks at counters (site, sweep, stream,                 */
/* 0xA << 28 | chain << 22 | k << 10 | j), j = 0, 1, ..., words w0..w3 in order; a normal takes */
/* two uniforms (Box-Muller cosine).  If a draw exhausts its 1024 blocks (never seen) it       */
/* returns the mean tanh(z)/(4z) and counts a fallback.                                        */
/* ------------------------------------------------------------------------------------------ */
#define ORA_PG_T 0.64
#define ORA_PI 3.14159265358979323846

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t w[4];
    int32_t idx;     /* next word of w (4: fetch a block) */
    int32_t j;       /* next block */
    int32_t exhausted;
} ora_ustream;

static void ora_us_init(ora_ustream *u, uint64_t seed, uint32_t site, uint32_t sweep, uint32_t stream,
                        uint32_t chain, uint32_t k)
{
    ora_key_of_seed(seed, u->key);
    u->ctr[0] = site;
    u->ctr[1] = sweep;
    u->ctr[2] = stream;
    u->ctr[3] = (0xAu << 28) | (chain << 22) | (k << 10);
    u->idx = 4;
    u->j = 0;
    u->exhausted = 0;
}

static double ora_us_next(ora_ustream *u)
{
    if (u->idx == 4) {
        if (u->j >= 1024) {
            u->exhausted = 1;
            return 0.5;
        }
        uint32_t c[4] = {u->ctr[0], u->ctr[1], u->ctr[2], u->ctr[3] | (uint32_t)u->j};
        ora_philox4x32_10(c, u->key, u->w);
        u->j += 1;
        u->idx = 0;
    }
    return ora_uniform(u->w[u->idx++]);
}

static double ora_us_normal(ora_ustream *u)
{
    double a = ora_us_next(u), b = ora_us_next(u);
    return sqrt(-2.0 * log(a)) * cos(2.0 * ORA_PI * b);
}

/* Standard normal CDF. */
static double ora_phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* n-th coefficient of the alternating series of the J*(1, 0) density (Devroye 2009, PSW 2013). */
double ora_pg_term(int32_t n, double x, int32_t form);
static double ora_pg_a(int32_t n, double x) { return ora_pg_term(n, x, x <= ORA_PG_T ? 0 : 1); }

/* Mixture weight of the exponential piece: p / (p + q), with
 *   p = pi / (2K) exp(-K t),  K = pi^2/8 + z^2/2,
 *   q = 2 exp(-z) F_IG(t; mu = 1/z, lambda = 1)  (z > 0),  q = 4 Phi(-1/sqrt(t))  (z = 0),
 * F_IG(t) = Phi((t z - 1)/sqrt(t)) + exp(2z) Phi(-(t z + 1)/sqrt(t)).  For z > 40 the
 * inverse-Gaussian piece (weight below 1e-17) is dropped. */
static double ora_pg_mix(double z)
{
    const double t = ORA_PG_T;
    double K = ORA_PI * ORA_PI / 8.0 + z * z / 2.0;
    double p = ORA_PI / (2.0 * K) * exp(-K * t);
    double q;
    if (z > 40.0) return 1.0;
    if (z == 0.0) q = 4.0 * ora_phi(-1.0 / sqrt(t));
    else q = 2.0 * exp(-z) * (ora_phi((t * z - 1.0) / sqrt(t)) + exp(2.0 * z) * ora_phi(-(t * z + 1.0) / sqrt(t)));
    return p / (p + q);
}

/* Inverse Gaussian IG(mu = 1/z, lambda = 1) truncated to (0, t) (PSW 2013, appendix). */
static double ora_pg_tig(double z, ora_ustream *u)
{
    const double t = ORA_PG_T;
    double x;
    if (z == 0.0 || 1.0 / z > t) {
        for (;;) {
            double e1, e2;
            do {
                e1 = -log(ora_us_next(u));
                e2 = -log(ora_us_next(u));
                if (u->exhausted) return t / 2.0;
            } while (e1 * e1 > 2.0 * e2 / t);
            x = t / ((1.0 + t * e1) * (1.0 + t * e1));
            double alpha = exp(-0.5 * z * z * x);
            if (ora_us_next(u) <= alpha || u->exhausted) return x;
        }
    }
    double mu = 1.0 / z;
    for (;;) {
        double y = ora_us_normal(u);
        y = y * y;
        x = mu + 0.5 * mu * mu * y - 0.5 * mu * sqrt(4.0 * mu * y + (mu * y) * (mu * y));
        if (ora_us_next(u) > mu / (mu + x)) x = mu * mu / x;
        if (x <= t || u->exhausted) return x;
    }
}

/* One J*(1, z) variate (z >= 0); PG(1, c) is J*(1, |c|/2) / 4. */
static double ora_pg_jstar(double z, double mix, ora_ustream *u)
{
    const double t = ORA_PG_T;
    double K = ORA_PI * ORA_PI / 8.0 + z * z / 2.0;
    for (;;) {
        double U = ora_us_next(u), V = ora_us_next(u);
        double x = (U < mix) ? t - log(ora_us_next(u)) / K : ora_pg_tig(z, u);
        if (u->exhausted) return -1.0;
        double S = ora_pg_a(0, x), Y = V * S;
        for (int32_t n = 1; n < 1000; ++n) {
            if (n & 1) {
                S -= ora_pg_a(n, x);
                if (Y <= S) return x;
            } else {
                S += ora_pg_a(n, x);
                if (Y > S) break;
            }
        }
    }
}

/* Term n of the small-x (form 0) or large-x (form 1) series of the J*(1, 0) density:
 *   form 0: pi (n + 1/2) (2 / (pi x))^{3/2} exp(-2 (n + 1/2)^2 / x),
 *   form 1: pi (n + 1/2) exp(-(n + 1/2)^2 pi^2 x / 2);
 * the sampler uses form 0 for x <= t and form 1 above. */
double ora_pg_term(int32_t n, double x, int32_t form)
{
    double k = n + 0.5;
    if (form == 0) return ORA_PI * k * pow(2.0 / (ORA_PI * x), 1.5) * exp(-2.0 * k * k / x);
    return ORA_PI * k * exp(-k * k * ORA_PI * ORA_PI * x / 2.0);
}

/* The exponential-piece weight p / (p + q) (test access). */
double ora_pg_mix_weight(double z) { return ora_pg_mix(z); }

/* PG(b, c) as the sum of b PG(1, c) draws with the counters above; *fallbacks counts draws
 * that exhausted their stream. */
double ora_pg_draw(int32_t b, double c, uint64_t seed, uint32_t site, uint32_t sweep, uint32_t stream,
                   uint32_t chain, int32_t *fallbacks)
{
    double z = fabs(c) / 2.0, mix = ora_pg_mix(z), sum = 0.0;
    for (int32_t k = 0; k < b; ++k) {
        ora_ustream u;
        ora_us_init(&u, seed, site, sweep, stream, chain, (uint32_t)k);
        double j = ora_pg_jstar(z, mix, &u);
        if (j < 0.0) {
            if (fallbacks) ++*fallbacks;
            j = z > 0.0 ? tanh(z) / z : 1.0;
        }
        sum += j / 4.0;
    }
    return sum;
}

/* ------------------------------------------------------------------------------------------ */
/* The sampler                                                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t prior_proper;  /* 0: intrinsic CAR (rho = 1), 1: proper CAR with rho           */
    double rho;
    double a_tau, b_tau;   /* tau ~ Gamma(a_tau, rate b_tau)                             */
    double a_sig, b_sig;   /* 1/sigma^2 ~ Gamma(a_sig, rate b_sig)                       */
    int32_t fix_hyper;     /* 1: tau and sigma^2 stay at their initial values             */
    int32_t intercept;     /* 1: y = beta0 1 + x + noise, flat prior on beta0 (Sec. 3.1)  */
    int32_t binomial;      /* 1: y_i ~ Bin(m_i, logistic(beta0 + x_i)) (Sec. 3.2), beta0 ~  */
    double beta0_mean;     /*    N(beta0_mean, beta0_var), Polya-Gamma augmentation; no     */
    double beta0_var;      /*    sigma^2                                                    */
} ora_model;

typedef struct {
    uint64_t seed;
    uint32_t stream;       /* Philox counter word 2 of this field                           */
    uint32_t start_sweep;  /* number of the first sweep run by this call                    */
    int32_t nsweeps;
    int32_t burn_in;       /* sweeps t < burn_in are not accumulated                        */
    int32_t thin;          /* after burn-in, every thin-th sweep is accumulated             */
} ora_run_opts;

/*
 * Run `nsweeps` sweeps of C independent chains on one field.
 *   x[c*n + i]             in: state before the call, out: state after it (natural order)
 *   tau[c], sig2[c]        in/out: current tau (precision) and sigma^2 of chain c
 *   beta0[c]               in/out: intercept of chain c (read only when model->intercept)
 *   tau_trace/sig2_trace/beta0_trace
 *                          out: [c*nsweeps + t], value after sweep t of this call (may be NULL)
 *   mean, m2, acc_count    in/out Welford accumulators [c*n + i] and the count of accumulated
 *                          sweeps (shared by all chains); NULL disables accumulation
 *   xtrace                 out: [(t*C + c)*n + i] state after every sweep (may be NULL)
 * Returns the number of Gamma draws that hit the attempt limit (normally 0).
 */
int32_t ora_run(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *weights,
                const int32_t *colors, int32_t ncolors, const double *y, const int32_t *trials, int32_t C,
                const ora_model *model, const ora_run_opts *opts, double *x, double *tau,
                double *sig2, double *beta0, double *tau_trace, double *sig2_trace,
                double *beta0_trace, double *mean, double *m2, int64_t *acc_count, double *xtrace)
{
    double rho = model->prior_proper ? model->rho : 1.0;
    double *deg = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) d += weights ? weights[e] : 1.0;
        deg[i] = d;
    }
    int32_t rank = model->prior_proper ? n : n - ora_components(n, row_ptr, col_idx);
    int32_t lanes = ora_lanes_for(C);
    int32_t fallbacks = 0;
    for (int32_t t = 0; t < opts->nsweeps; ++t) {
        uint32_t sweep = opts->start_sweep + (uint32_t)t;
        for (int32_t c = 0; c < C; ++c) {
            double *xc = x + (int64_t)c * n;
            double prec_noise = 1.0 / sig2[c];
            int binom = model->binomial != 0;
            double b0 = (model->intercept || binom) ? beta0[c] : 0.0;
            double sum_psi = 0.0, sum_kx = 0.0; /* binomial: sums of psi_i and kappa_i - psi_i x_i */
            /* Algorithm 1: colour classes in order, every site of the class from its local
             * characteristics given the newest values of the other classes (Sec. 3.1: the
             * observations enter through b = (y - beta0 1) / sigma^2). */
            for (int32_t col = 0; col < ncolors; ++col)
                for (int32_t i = 0; i < n; ++i) {
                    if (colors[i] != col) continue;
                    double s = 0.0;
                    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                        s += (weights ? weights[e] : 1.0) * xc[col_idx[e]];
                    double z = ora_site_normal(opts->seed, (uint32_t)i, sweep, opts->stream, (uint32_t)c, lanes);
                    if (binom) {
                        /* psi_i | beta0, x_i ~ PG(m_i, beta0 + x_i), then x_i given psi_i (Sec. 3.2):
                         * precision tau d_i + psi_i, mean (tau rho s_i + kappa_i - psi_i beta0) / P */
                        double psi = ora_pg_draw(trials[i], b0 + xc[i], opts->seed, (uint32_t)i, sweep,
                                                 opts->stream, (uint32_t)c, &fallbacks);
                        double kappa = y[i] - 0.5 * trials[i];
                        double P = tau[c] * deg[i] + psi;
                        double m = (tau[c] * rho * s + kappa - psi * b0) / P;
                        xc[i] = m + z / sqrt(P);
                        sum_psi += psi;
                        sum_kx += kappa - psi * xc[i];
                        continue;
                    }
                    double P = tau[c] * deg[i] + prec_noise;
                    double m = (tau[c] * rho * s + (y[i] - b0) * prec_noise) / P;
                    xc[i] = m + z / sqrt(P);
                }
            /* Intercept (Sec. 3.1, flat prior): beta0 | y, x, sigma^2 ~ N(1'(y - x) / n, sigma^2 / n),
             * drawn before sigma^2, whose conditional then uses the new beta0. */
            if (binom) {
                /* beta0 | x, psi ~ N(mean, 1/Pb), Pb = 1/v0 + sum psi_i,
                 * mean = (mu0/v0 + sum (kappa_i - psi_i x_i)) / Pb */
                double Pb = 1.0 / model->beta0_var + sum_psi;
                double mb = (model->beta0_mean / model->beta0_var + sum_kx) / Pb;
                double zb = ora_beta_normal(opts->seed, sweep, opts->stream, ORA_TAG_BETA, (uint32_t)c);
                b0 = mb + zb / sqrt(Pb);
                beta0[c] = b0;
            } else if (model->intercept) {
                double A = 0.0;
                for (int32_t i = 0; i < n; ++i) A += y[i] - xc[i];
                double zb = ora_beta_normal(opts->seed, sweep, opts->stream, ORA_TAG_BETA, (uint32_t)c);
                b0 = A / n + sqrt(sig2[c] / n) * zb;
                beta0[c] = b0;
            }
            if (!model->fix_hyper) {
                double S = ora_quadform(n, row_ptr, col_idx, weights, rho, xc);
                double R = 0.0;
                for (int32_t i = 0; i < n; ++i) R += (y[i] - b0 - xc[i]) * (y[i] - b0 - xc[i]);
                int32_t att;
                tau[c] = ora_gamma_draw(model->a_tau + 0.5 * rank, model->b_tau + 0.5 * S,
                                        opts->seed, sweep, opts->stream, ORA_TAG_TAU, (uint32_t)c, &att);
                if (att < 0) ++fallbacks;
                if (!binom) {
                    double prec = ora_gamma_draw(model->a_sig + 0.5 * n, model->b_sig + 0.5 * R, opts->seed,
                                                 sweep, opts->stream, ORA_TAG_SIG, (uint32_t)c, &att);
                    if (att < 0) ++fallbacks;
                    sig2[c] = 1.0 / prec;
                }
            }
            if (tau_trace) tau_trace[(int64_t)c * opts->nsweeps + t] = tau[c];
            if (sig2_trace) sig2_trace[(int64_t)c * opts->nsweeps + t] = sig2[c];
            if (beta0_trace) beta0_trace[(int64_t)c * opts->nsweeps + t] = b0;
            if (xtrace) memcpy(xtrace + ((int64_t)t * C + c) * n, xc, sizeof(double) * (size_t)n);
        }
        if (mean && m2 && acc_count && (int64_t)sweep >= opts->burn_in &&
            ((int64_t)sweep - opts->burn_in) % (opts->thin > 0 ? opts->thin : 1) == 0) {
            int64_t k = ++(*acc_count);
            for (int64_t q = 0; q < (int64_t)C * n; ++q) {
                double delta = x[q] - mean[q];
                mean[q] += delta / (double)k;
                m2[q] += delta * (x[q] - mean[q]);
            }
        }
    }
    free(deg);
    return fallbacks;
}

/* ------------------------------------------------------------------------------------------ */
/* Diagnostics of the chains (Sec. 3.1 reports ESS, IAT and CES = IAT T / N of the tau^2 chain, */
/* and Gelman plots)                                                                            */
/* ------------------------------------------------------------------------------------------ */

/* Integrated autocorrelation time kappa of x[0..N-1] by Geyer's initial monotone sequence
 * estimator (Geyer 1992, Statistical Science 7, Sec. 3.3):
 *   gamma(k) = (1/N) sum_{t=0}^{N-1-k} (x_t - mean)(x_{t+k} - mean),
 *   Gamma_m = gamma(2m) + gamma(2m+1) for 2m+1 <= N-1,
 *   M = the largest m with Gamma_0, ..., Gamma_m all > 0 (M = 0 when Gamma_0 <= 0),
 *   Gamma~_m = min(Gamma_0, ..., Gamma_m),
 *   kappa = (-gamma(0) + 2 sum_{m=0}^{M} Gamma~_m) / gamma(0),
 * floored at 1 / log10(N) (an effective sample size of at most N log10 N).  NaN when N < 4 or
 * the chain is constant. */
double ora_iat(const double *x, int64_t N)
{
    if (N < 4) return NAN;
    double mean = 0.0;
    for (int64_t t = 0; t < N; ++t) mean += x[t];
    mean /= (double)N;
    double g0 = 0.0;
    for (int64_t t = 0; t < N; ++t) g0 += (x[t] - mean) * (x[t] - mean);
    g0 /= (double)N;
    if (!(g0 > 0.0)) return NAN;
    double sum = 0.0, run_min = INFINITY;
    for (int64_t m = 0; 2 * m + 1 <= N - 1; ++m) {
        double G = 0.0;
        for (int64_t k = 2 * m; k <= 2 * m + 1; ++k) {
            double gk = 0.0;
            for (int64_t t = 0; t + k < N; ++t) gk += (x[t] - mean) * (x[t + k] - mean);
            G += gk / (double)N;
        }
        if (m > 0 && !(G > 0.0)) break;
        if (G < run_min) run_min = G;
        sum += run_min;
        if (!(G > 0.0)) break; /* m == 0 with Gamma_0 <= 0 */
    }
    double kappa = (-g0 + 2.0 * sum) / g0;
    double floor_k = 1.0 / log10((double)N);
    return kappa < floor_k ? floor_k : kappa;
}

/* Potential scale reduction factor of m chains of N values each, x[c*N + t] (Gelman & Rubin
 * 1992, with the (m + 1)/m factor of Brooks & Gelman 1998):
 *   W = mean over chains of the within-chain variance (divisor N - 1),
 *   B/N = variance of the chain means (divisor m - 1),
 *   V = (N - 1)/N W + (m + 1)/m B/N,   R = sqrt(V / W).
 * NaN when m < 2, N < 2 or W = 0. */
double ora_psrf_moments(const double *mean, const double *var, int32_t m, int64_t N)
{
    if (m < 2 || N < 2) return NAN;
    double W = 0.0, mm = 0.0;
    for (int32_t c = 0; c < m; ++c) {
        W += var[c];
        mm += mean[c];
    }
    W /= (double)m;
    mm /= (double)m;
    double BN = 0.0;
    for (int32_t c = 0; c < m; ++c) BN += (mean[c] - mm) * (mean[c] - mm);
    BN /= (double)(m - 1);
    if (!(W > 0.0)) return NAN;
    double V = (double)(N - 1) / (double)N * W + (double)(m + 1) / (double)m * BN;
    return sqrt(V / W);
}

double ora_psrf(const double *x, int32_t m, int64_t N)
{
    if (m < 2 || N < 2) return NAN;
    double *mean = (double *)malloc(sizeof(double) * (size_t)m);
    double *var = (double *)malloc(sizeof(double) * (size_t)m);
    for (int32_t c = 0; c < m; ++c) {
        const double *xc = x + (int64_t)c * N;
        double s = 0.0;
        for (int64_t t = 0; t < N; ++t) s += xc[t];
        mean[c] = s / (double)N;
        double v = 0.0;
        for (int64_t t = 0; t < N; ++t) v += (xc[t] - mean[c]) * (xc[t] - mean[c]);
        var[c] = v / (double)(N - 1);
    }
    double r = ora_psrf_moments(mean, var, m, N);
    free(mean);
    free(var);
    return r;
}
