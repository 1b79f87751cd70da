// sweep_kernels.cu -- the per-colour fused update of the chromatic Gibbs sampler (Algorithm 1,
// steps 2-3), the fused reductions behind the conjugate hyperparameter draws (Sec. 3.1), the
// hyperparameter draw itself, and the pack/unpack kernels of the colour-split layout.
//
// One launch of colour_step_kernel covers colour class c of every field: each block takes one
// tile (a range of sub-array rows of a lattice field, or of permuted positions of a CSR field)
// and, for every site i of the tile and every chain,
//     s_i = sum_j w_ij x_j                         (neighbours all have other colours)
//     P_i = tau d_i + 1/sigma^2,  m_i = (tau rho s_i + y_i/sigma^2) / P_i
//     x_i = m_i + z_i / sqrt(P_i),                 z_i Philox/Box-Muller normal of (site, sweep)
// (with the intercept of Sec. 3.1, y_i - beta0 in place of y_i) and accumulates, per chain, the
// sums the conjugate draws need:
//     (1 - rho) d_i x_i^2 + rho sum_{j lower colour} w_ij (x_i - x_j)^2,
//     (y_i - beta0 - x_i)^2  and  y_i - beta0 - x_i,
// so that after the last colour every undirected edge has been counted once, at its endpoint
// of higher colour, with both endpoints final: summed over sites this is x'(D - rho W)x.
// Thread, warp and block partial sums are in the state precision (a tile holds at most a few
// thousand terms); the sums over tiles are FP64; every sum is taken in a fixed order, so
// results are reproducible run to run.  When the sweep is accumulated, the Welford
// running mean and M2 of the site are updated in the same pass.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "gamma_pre.cuh"
#include "hyper_task.cuh"
#include "pg.cuh"

namespace gmrf {
namespace {

template <typename T> struct Arith;
template <> struct Arith<float> {
    // 1/P and 1/sqrt(P) within 1 ulp (P is a normal float): well inside the FP32 parity budget.
    __device__ __forceinline__ static float rcp(float x) { return rcp_approx(x); }
    __device__ __forceinline__ static float rsq(float x) { return rsqrt_approx(x); }
};
template <> struct Arith<double> {
    __device__ __forceinline__ static double rcp(double x) { return 1.0 / x; }
    __device__ __forceinline__ static double rsq(double x) { return 1.0 / sqrt(x); }
};

// Observation models of the colour kernels (compile-time): Gaussian noise without or with the
// intercept beta0 (Sec. 3.1), or binomial counts with the logistic link and Polya-Gamma
// augmentation (Sec. 3.2; y holds the successes, the trials come separately).
enum : int { kModelGauss = 0, kModelGaussIntercept = 1, kModelBinomial = 2 };

template <typename T, int V>
struct SiteCtx {
    T tau[V], isig[V], beta[V];  // per chain of this thread
    T accS[V], accR[V], accA[V]; // thread partial sums
    T inv_k;             // 1 / (accumulated count) when accumulating
    bool acc;
};

// Draw (or, in reduce-only mode, read) the V chain values of one site given its neighbour sum s
// and the neighbour values nb[k] of the neighbours flagged in `lower_mask` (those of lower
// colour), and fold the site's terms into the partial sums.
//
// Binomial model: psi | beta0, x_i ~ PG(m_i, beta0 + x_i) was drawn from the site's value at the
// start of the sweep (the Polya-Gamma stage); x_i gets precision tau d_i + psi and mean
// (tau rho s_i + kappa_i - psi beta0) / P,
// kappa_i = y_i - m_i / 2; the partial sums then collect psi and kappa_i - psi x_i (for beta0)
// in place of the Gaussian residual sums.
template <typename T, int V, int NB, int MODEL>
__device__ __forceinline__ void finish_site(const StepArgs &a, SiteCtx<T, V> &cx, T *xp, T *meanp, T *m2p,
                                            T yv, int mtr, T d, uint32_t site, uint32_t sweep, uint32_t stream,
                                            uint32_t chain0, const T (&s)[V], const T (&nb)[NB][V],
                                            uint32_t lower_mask, const T (&wnb)[NB])
{
    const T rho = static_cast<T>(a.rho);
    T xn[V];
    // Running moments first, so their loads do not wait behind the store of x (possible alias);
    // with four chains per thread the registers are better spent elsewhere.
    T mu[V], mm[V];
    constexpr bool kEarly = V <= 2;
    if (kEarly && cx.acc) {
        Vec<T, V>::ld(meanp, mu);
        Vec<T, V>::ld(m2p, mm);
    }
    T psi[V];
    const T kappa = yv - static_cast<T>(0.5) * static_cast<T>(mtr);
    if (MODEL == kModelBinomial && a.update) {
        T z[V];
        // psi of this site and chain, drawn by the Polya-Gamma stage from the start-of-sweep state
        Vec<T, V>::ld(static_cast<const T *>(a.psi) + (xp - static_cast<T *>(a.x)), psi);
        site_normals<T, V>(a.key, site, sweep, stream, chain0, a.lanes, z);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T P = cx.tau[v] * d + psi[v];
            const T m = (cx.tau[v] * rho * s[v] + kappa - psi[v] * cx.beta[v]) * Arith<T>::rcp(P);
            xn[v] = m + z[v] * Arith<T>::rsq(P);
        }
        Vec<T, V>::st(xp, xn);
    } else if (a.update) {
        T z[V];
        site_normals<T, V>(a.key, site, sweep, stream, chain0, a.lanes, z);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T P = cx.tau[v] * d + cx.isig[v];
            const T m = (cx.tau[v] * rho * s[v] + (yv - cx.beta[v]) * cx.isig[v]) * Arith<T>::rcp(P);
            xn[v] = m + z[v] * Arith<T>::rsq(P);
        }
        Vec<T, V>::st(xp, xn);
    } else {
        Vec<T, V>::ld(xp, xn);
#pragma unroll
        for (int v = 0; v < V; ++v) psi[v] = 0;  // reduce-only passes are not used with this model
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T e = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if ((lower_mask >> k) & 1u) {
                const T df = xn[v] - nb[k][v];
                e += wnb[k] * df * df;
            }
        }
        cx.accS[v] += (static_cast<T>(1) - rho) * d * xn[v] * xn[v] + rho * e;
        if (MODEL == kModelBinomial) {
            cx.accR[v] += psi[v];
            cx.accA[v] += kappa - psi[v] * xn[v];
        } else {
            const T r = (yv - cx.beta[v]) - xn[v];
            cx.accR[v] += r * r;
            cx.accA[v] += r;
        }
    }
    if (cx.acc) {
        if (!kEarly) {
            Vec<T, V>::ld(meanp, mu);
            Vec<T, V>::ld(m2p, mm);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T delta = xn[v] - mu[v];
            mu[v] += delta * cx.inv_k;
            mm[v] += delta * (xn[v] - mu[v]);
        }
        Vec<T, V>::st(meanp, mu);
        Vec<T, V>::st(m2p, mm);
    }
}

// Lattices with parity colourings: 2-D 4-neighbour and 3-D 6-neighbour.  Site of colour c in
// sub-array row r = l*H + i, column h sits at j = 2h + p, p = (c + l + i) & 1; its in-row
// neighbours are columns h - 1 + p and h + p of the other colour's row r, the others column h
// of rows r -+ 1 (i -+ 1) and r -+ H (l -+ 1).  Neighbour k has a fixed position in nb[k];
// missing ones (outside the lattice) are masked.
template <typename T, int V, bool THREE_D, int MODEL>
__device__ void lattice_parity_tile(const StepArgs &a, const FieldDev &f, const Tile &t, SiteCtx<T, V> &cx,
                                    int CV, int cv_shift, uint32_t sweep)
{
    constexpr int NB = THREE_D ? 6 : 4;
    const int L = THREE_D ? f.dims[0] : 1;
    const int H = THREE_D ? f.dims[1] : f.dims[0];
    const int W = THREE_D ? f.dims[2] : f.dims[1];
    const int c = t.colour;
    const int cols = f.cols;
    T *X = static_cast<T *>(a.x);
    const T *Y = static_cast<const T *>(a.y);
    T *MEAN = static_cast<T *>(a.mean);
    T *M2 = static_cast<T *>(a.m2);
    const int Cp = a.Cp;
    const int cvo = (threadIdx.x & (CV - 1)) * V;  // chain offset of this thread (fixed)
    const int64_t self_base = f.slot0 + static_cast<int64_t>(c) * f.rows * cols;
    const int64_t oth_base = f.slot0 + static_cast<int64_t>(1 - c) * f.rows * cols;
    const T *XO = X + oth_base * Cp + cvo;
    T *XS = X + self_base * Cp + cvo;
    T *MS = MEAN + self_base * Cp + cvo;
    T *QS = M2 + self_base * Cp + cvo;
    const T *YS = Y + self_base;
    const uint32_t lower_all = (c == 1) ? 0xffu : 0u;  // all neighbours have the other colour
    const int plane = H * cols;
    const int nelem = t.count * cols * CV;
    for (int e = threadIdx.x; e < nelem; e += kBlock) {
        const int cv = e & (CV - 1);
        const int sr = e >> cv_shift;
        const int rr = fast_div(sr, f.cols_m, f.cols_s);
        const int h = sr - rr * cols;
        const int r = t.start + rr;
        const int l = THREE_D ? fast_div(r, f.h_m, f.h_s) : 0;
        const int i = THREE_D ? r - l * H : r;
        const int p = (c + l + i) & 1;
        const int j = 2 * h + p;
        if (j >= W)
            continue;
        uint32_t valid = (j > 0 ? 1u : 0u) | (j + 1 < W ? 2u : 0u) | (i > 0 ? 4u : 0u) | (i + 1 < H ? 8u : 0u);
        if (THREE_D) valid |= (l > 0 ? 16u : 0u) | (l + 1 < L ? 32u : 0u);
        const int rb = r * cols + h;
        int ns[NB];
        ns[0] = rb - 1 + p;
        ns[1] = rb + p;
        ns[2] = rb - cols;
        ns[3] = rb + cols;
        if (THREE_D) {
            ns[4] = rb - plane;
            ns[5] = rb + plane;
        }
        T nb[NB][V], wnb[NB], s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            wnb[k] = 1;
            if ((valid >> k) & 1u) {
                Vec<T, V>::ld(XO + ns[k] * Cp, nb[k]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) nb[k][v] = 0;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] += nb[k][v];
        }
        const uint32_t site = static_cast<uint32_t>(r * W + j);
        const int mtr = MODEL == kModelBinomial ? a.trials[self_base + rb] : 0;
        finish_site<T, V, NB, MODEL>(a, cx, XS + rb * Cp, MS + rb * Cp, QS + rb * Cp, YS[rb], mtr, static_cast<T>(__popc(valid)),
                              site, sweep, f.stream, static_cast<uint32_t>(cv * V), s, nb, lower_all & valid, wnb);
    }
}

// 2-D 8-neighbour lattice with the 2x2 colouring c = 2 (i & 1) + (j & 1): the site of colour
// c = 2a + b at sub-array (u, v) is (2u + a, 2v + b); neighbour (i + di, j + dj) lives in
// colour 2((a + di) & 1) + ((b + dj) & 1) at sub-array (u + ((a + di) >> 1), v + ((b + dj) >> 1)).
template <typename T, int V, int MODEL>
__device__ void lattice8_tile(const StepArgs &a, const FieldDev &f, const Tile &t, SiteCtx<T, V> &cx, int CV,
                              int cv_shift, uint32_t sweep)
{
    constexpr int NB = 8;
    const int H = f.dims[0], W = f.dims[1];
    const int c = t.colour;
    const int ca = c >> 1, cb = c & 1;
    const int cols = f.cols;
    T *X = static_cast<T *>(a.x);
    const T *Y = static_cast<const T *>(a.y);
    T *MEAN = static_cast<T *>(a.mean);
    T *M2 = static_cast<T *>(a.m2);
    const int Cp = a.Cp;
    const int cvo = (threadIdx.x & (CV - 1)) * V;  // chain offset of this thread (fixed)
    const int sub = f.rows * cols;
    const T *XF = X + f.slot0 * Cp + cvo;
    T *XS = X + (f.slot0 + static_cast<int64_t>(c) * sub) * Cp + cvo;
    T *MS = MEAN + (f.slot0 + static_cast<int64_t>(c) * sub) * Cp + cvo;
    T *QS = M2 + (f.slot0 + static_cast<int64_t>(c) * sub) * Cp + cvo;
    const T *YS = Y + f.slot0 + static_cast<int64_t>(c) * sub;
    // Per direction (block-uniform): offset of the neighbour's slot relative to (u, v) in its
    // colour's sub-array, and whether that colour is lower than c.
    int doff[NB];
    uint32_t lower = 0;
#pragma unroll
    for (int k = 0, q = 0; q < 9; ++q) {
        const int di = q / 3 - 1, dj = q % 3 - 1;
        if (di == 0 && dj == 0) continue;
        const int cc = 2 * ((ca + di) & 1) + ((cb + dj) & 1);
        doff[k] = cc * sub + ((ca + di) >> 1) * cols + ((cb + dj) >> 1);
        if (cc < c) lower |= 1u << k;
        ++k;
    }
    const int nelem = t.count * cols * CV;
    for (int e = threadIdx.x; e < nelem; e += kBlock) {
        const int cv = e & (CV - 1);
        const int sr = e >> cv_shift;
        const int rr = fast_div(sr, f.cols_m, f.cols_s);
        const int vv = sr - rr * cols;
        const int u = t.start + rr;
        const int i = 2 * u + ca, j = 2 * vv + cb;
        if (i >= H || j >= W)
            continue;
        const int base = u * cols + vv;
        uint32_t valid = 0;
#pragma unroll
        for (int k = 0, q = 0; q < 9; ++q) {
            const int di = q / 3 - 1, dj = q % 3 - 1;
            if (di == 0 && dj == 0) continue;
            const bool ok = (i + di >= 0) && (i + di < H) && (j + dj >= 0) && (j + dj < W);
            valid |= ok ? (1u << k) : 0u;
            ++k;
        }
        T nb[NB][V], wnb[NB], s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            wnb[k] = 1;
            if ((valid >> k) & 1u) {
                Vec<T, V>::ld(XF + (doff[k] + base) * Cp, nb[k]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) nb[k][v] = 0;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] += nb[k][v];
        }
        const uint32_t site = static_cast<uint32_t>(i * W + j);
        const int mtr = MODEL == kModelBinomial ? a.trials[f.slot0 + static_cast<int64_t>(c) * sub + base] : 0;
        finish_site<T, V, NB, MODEL>(a, cx, XS + base * Cp, MS + base * Cp, QS + base * Cp, YS[base], mtr,
                              static_cast<T>(__popc(valid)), site, sweep, f.stream, static_cast<uint32_t>(cv * V),
                              s, nb, lower & valid, wnb);
    }
}

// CSR field: permuted positions [start, start + count) of one colour class; neighbours are read
// through the permuted row; a neighbour has lower colour iff its position is below the class's
// first position.
template <typename T, int V, int MODEL>
__device__ void csr_tile(const StepArgs &a, const FieldDev &f, const Tile &t, SiteCtx<T, V> &cx, int CV,
                         int cv_shift, uint32_t sweep)
{
    T *X = static_cast<T *>(a.x);
    const T *Y = static_cast<const T *>(a.y);
    T *MEAN = static_cast<T *>(a.mean);
    T *M2 = static_cast<T *>(a.m2);
    const T *Wt = static_cast<const T *>(a.w);
    const T *DEG = static_cast<const T *>(a.deg);
    const int64_t Cp = a.Cp;
    const int32_t *rp = a.rp + f.rp0;
    const int32_t *ci = a.ci + f.nnz0;
    const T *wr = Wt ? Wt + f.nnz0 : nullptr;
    const int32_t lo = a.coff[f.coff0 + t.colour];
    const T rho = static_cast<T>(a.rho);
    const int nelem = t.count * CV;
    for (int e = threadIdx.x; e < nelem; e += kBlock) {
        const int cv = e & (CV - 1);
        const int pos = t.start + (e >> cv_shift);
        const int rb = rp[pos], re = rp[pos + 1];
        // The first R neighbours stay in registers: their loads are all issued before any is
        // used, and the lower-colour terms of the prior sum need no second pass over them.
        constexpr int R = V == 4 ? 6 : 8;
        T nb[R][V], wnb[R], s[V];
        uint32_t lower = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int k = rb + q;
            if (k < re) {
                const int jn = ci[k];
                Vec<T, V>::ld(X + (f.slot0 + jn) * Cp + cv * V, nb[q]);
                wnb[q] = wr ? wr[k] : static_cast<T>(1);
                lower |= (jn < lo ? 1u : 0u) << q;
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) nb[q][v] = 0;
                wnb[q] = 0;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] += wnb[q] * nb[q][v];
        }
        for (int k = rb + R; k < re; ++k) {  // rows longer than R
            T xv[V];
            Vec<T, V>::ld(X + (f.slot0 + ci[k]) * Cp + cv * V, xv);
            const T wv = wr ? wr[k] : static_cast<T>(1);
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] += wv * xv[v];
        }
        const int64_t self = f.slot0 + pos;
        const T yv = Y[self];
        const T d = DEG[f.csr0 + pos];
        const uint32_t site = static_cast<uint32_t>(a.perm[f.csr0 + pos]);
        const int mtr = MODEL == kModelBinomial ? a.trials[self] : 0;
        finish_site<T, V, R, MODEL>(a, cx, X + self * Cp + cv * V, MEAN + self * Cp + cv * V, M2 + self * Cp + cv * V, yv,
                                    mtr, d, site, sweep, f.stream, static_cast<uint32_t>(cv * V), s, nb, lower, wnb);
        if (re - rb > R) {
            // the lower-colour edges beyond the first R
            T xn[V], e2[V];
            Vec<T, V>::ld(X + self * Cp + cv * V, xn);
#pragma unroll
            for (int v = 0; v < V; ++v) e2[v] = 0;
            for (int k = rb + R; k < re; ++k) {
                const int jn = ci[k];
                if (jn >= lo) continue;
                T xv[V];
                Vec<T, V>::ld(X + (f.slot0 + jn) * Cp + cv * V, xv);
                const T wv = wr ? wr[k] : static_cast<T>(1);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const T df = xn[v] - xv[v];
                    e2[v] += wv * df * df;
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) cx.accS[v] += rho * e2[v];
        }
    }
}

// MODEL: the observation model; without the intercept beta0 = 0 and the third sum is not
// needed, which the compiler then removes, registers included.
template <typename T, int V, int KIND, int MODEL>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? (KIND == kCsr ? 2 : 3) : 1) colour_step_kernel(const StepArgs a)
{
    pdl_wait_then_release();
    const Tile t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const int CV = a.Cp / V;
    const int cv = threadIdx.x % CV;  // fixed per thread: kBlock is a multiple of CV
    const long long sweep_ll = a.ctl->sweep;
    const uint32_t sweep = static_cast<uint32_t>(sweep_ll);

    SiteCtx<T, V> cx;
    const T *hyp = static_cast<const T *>(a.hyp);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int64_t hc = (static_cast<int64_t>(t.field) * a.Cp + cv * V + v) * kHypStride;
        cx.tau[v] = hyp[hc];
        cx.isig[v] = hyp[hc + 1];
        cx.beta[v] = MODEL != kModelGauss ? hyp[hc + 2] : static_cast<T>(0);
        cx.accS[v] = 0;
        cx.accR[v] = 0;
        cx.accA[v] = 0;
    }
    cx.acc = false;
    cx.inv_k = 0;
    if (a.update && a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin)) {
        cx.acc = true;
        cx.inv_k = static_cast<T>(1) / static_cast<T>(a.ctl->acc_count + 1);
    }

    const int cv_shift = __ffs(CV) - 1;
    if constexpr (KIND == kLat2D4) lattice_parity_tile<T, V, false, MODEL>(a, f, t, cx, CV, cv_shift, sweep);
    else if constexpr (KIND == kLat3D6) lattice_parity_tile<T, V, true, MODEL>(a, f, t, cx, CV, cv_shift, sweep);
    else if constexpr (KIND == kLat2D8) lattice8_tile<T, V, MODEL>(a, f, t, cx, CV, cv_shift, sweep);
    else csr_tile<T, V, MODEL>(a, f, t, cx, CV, cv_shift, sweep);

    // Deterministic block reduction of the 3 V partial sums of each chain in the state precision:
    // a shuffle tree over the lanes that share a chain vector (lanes equal mod CV), then the
    // warps' sums in order; the tile's sum is stored in FP64 and summed over tiles in FP64.
    __shared__ T red[kBlock / 32][kMaxChains][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T sS = cx.accS[v];
        T sR = cx.accR[v];
        T sA = MODEL != kModelGauss ? cx.accA[v] : static_cast<T>(0);
        for (int off = 16; off >= CV; off >>= 1) {
            sS += __shfl_xor_sync(0xffffffffu, sS, off);
            sR += __shfl_xor_sync(0xffffffffu, sR, off);
            if (MODEL != kModelGauss) sA += __shfl_xor_sync(0xffffffffu, sA, off);
        }
        if (lane < CV) {
            red[warp][lane * V + v][0] = sS;
            red[warp][lane * V + v][1] = sR;
            red[warp][lane * V + v][2] = sA;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.Cp * 3; q += kBlock) {
        const int chain = q / 3, k = q - 3 * chain;
        T acc = 0;
        for (int w = 0; w < kBlock / 32; ++w) acc += red[w][chain][k];
        double *dst = reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * a.Cp + chain);
        dst[k] = static_cast<double>(acc);
    }
}

// The hyperparameter stage: one warp per task of hyper_task (eight per block).  With a single
// block its thread 0 advances the counters after a barrier; with several, the last block to
// finish does (ticket counter; no block waits for another).
constexpr int kHyperWarps = 8;

template <typename T, bool BATCH>
__global__ void __launch_bounds__(kHyperWarps * 32) hyper_kernel(const HyperArgs a)
{
    // Let the next sweep kernel be scheduled now: it does its own early work (observations,
    // predicted normals) while this draw waits for and runs after the current sweep.
    pdl_release();
    pdl_wait();
    const int task = blockIdx.x * kHyperWarps + (threadIdx.x >> 5);
    const long long sweep = a.ctl->sweep;
    if (task < a.nfields * a.Cp * 2) hyper_task<T, BATCH>(a, task, sweep);
    bool last = gridDim.x == 1;
    __syncthreads();
    if (!last && threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&a.ctl->ticket, 1ull) == gridDim.x - 1;
    }
    if (threadIdx.x == 0 && last) {
        hyper_advance(a, sweep);
        a.ctl->ticket = 0;
    }
}

// The Polya-Gamma stage of the binomial model: one warp per (slot, chain).  The slot's natural
// site gives the counters; lane l draws the PG(1, c) summands k = l, l + 32, ... < m_i and the
// warp adds them in a fixed order (shuffle tree); psi = 0 for sites without trials and for
// padding slots.
template <typename T>
__global__ void pg_stage_kernel(const PgArgs a)
{
    pdl_wait_then_release();
    const int lane = threadIdx.x & 31;
    const uint32_t sweep = static_cast<uint32_t>(a.ctl->sweep);
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const T *X = static_cast<const T *>(a.x);
    const T *hyp = static_cast<const T *>(a.hyp);
    T *PSI = static_cast<T *>(a.psi);
    int fb = 0;
    for (int64_t task = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; task < a.slots * a.C;
         task += warps) {
        const int64_t slot = task / a.C;
        const int chain = static_cast<int>(task - slot * a.C);
        int fi = 0;  // field of the slot (fields are few; their slot ranges are in order)
        while (fi + 1 < a.nfields && a.fields[fi + 1].slot0 <= slot) ++fi;
        const FieldDev &f = a.fields[fi];
        const int64_t rel = slot - f.slot0;
        // natural site of the slot (padding slots of the lattice layouts have none)
        int64_t site = -1;
        if (f.kind == kCsr) {
            site = a.perm[f.csr0 + rel];
        } else {
            const int64_t sub = static_cast<int64_t>(f.rows) * f.cols;
            const int64_t c = rel / sub, r = (rel - c * sub) / f.cols, h = rel - c * sub - r * f.cols;
            if (f.kind == kLat2D8) {
                const int64_t i = 2 * r + (c >> 1), j = 2 * h + (c & 1);
                if (i < f.dims[0] && j < f.dims[1]) site = i * f.dims[1] + j;
            } else if (f.kind == kLat2D4) {
                const int64_t j = 2 * h + ((c + r) & 1);
                if (j < f.dims[1]) site = r * f.dims[1] + j;
            } else {
                const int64_t l = r / f.dims[1], i = r - l * f.dims[1], j = 2 * h + ((c + l + i) & 1);
                if (j < f.dims[2]) site = r * f.dims[2] + j;
            }
        }
        const int m = site >= 0 ? a.trials[slot] : 0;
        // the sampler's arithmetic follows the state precision (pg.cuh)
        T sum = 0;
        if (m > 0) {
            const T eta = hyp[(static_cast<int64_t>(fi) * a.Cp + chain) * kHypStride + 2] + X[slot * a.Cp + chain];
            const T z = static_cast<T>(0.5) * fabs(eta);
            // the proposal's mixture weight, once per warp (the special functions are costly)
            T wexp = lane == 0 ? pg_exp_weight<T>(z) : static_cast<T>(0);
            wexp = __shfl_sync(0xffffffffu, wexp, 0);
            for (int k = lane; k < m; k += 32) {
                PgStream st;
                pg_stream_init(st, a.key, static_cast<uint32_t>(site), sweep, f.stream, static_cast<uint32_t>(chain),
                               static_cast<uint32_t>(k));
                T j = pg_jstar<T>(z, wexp, st);
                if (j < static_cast<T>(0)) {
                    ++fb;
                    j = z > static_cast<T>(0) ? tanh(z) / z : static_cast<T>(1);
                }
                sum += static_cast<T>(0.25) * j;
            }
        }
        for (int off = 16; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0) PSI[slot * a.Cp + chain] = sum;
    }
    if (fb) atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->fallbacks), static_cast<unsigned long long>(fb));
}

// Natural order -> colour-split layout: y and the chains' initial states (x0 = y by default;
// chains >= C of the padded layout start at y too).
template <typename T>
__global__ void pack_kernel(const FieldDev *fields, int32_t fidx, int32_t C, int32_t Cp, const double *y_nat,
                            const double *x0_nat, const int32_t *perm_inv, T *x, T *y)
{
    const FieldDev f = fields[fidx];
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < f.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t slot = f.slot0 + (f.kind == kCsr ? perm_inv[f.csr0 + i] : lattice_slot_of_site(f, i));
        const double yv = y_nat[i];
        y[slot] = static_cast<T>(yv);
        for (int c = 0; c < Cp; ++c)
            x[slot * Cp + c] = static_cast<T>((x0_nat && c < C) ? x0_nat[static_cast<int64_t>(c) * f.n + i] : yv);
    }
}

// Natural order -> colour-split layout of a per-site integer array (binomial trials).
__global__ void pack_int_kernel(const FieldDev *fields, int32_t fidx, const int32_t *v_nat, const int32_t *perm_inv,
                                int32_t *v)
{
    const FieldDev f = fields[fidx];
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < f.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t slot = f.slot0 + (f.kind == kCsr ? perm_inv[f.csr0 + i] : lattice_slot_of_site(f, i));
        v[slot] = v_nat[i];
    }
}

// Colour-split layout -> natural order for one chain: out[i] = src (or m2 * inv_km1).
template <typename T>
__global__ void unpack_kernel(const FieldDev *fields, int32_t fidx, int32_t Cp, int32_t chain, const T *src,
                              const T *m2, double inv_km1, const int32_t *perm_inv, double *out)
{
    const FieldDev f = fields[fidx];
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < f.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t slot = f.slot0 + (f.kind == kCsr ? perm_inv[f.csr0 + i] : lattice_slot_of_site(f, i));
        if (m2) out[i] = static_cast<double>(m2[slot * Cp + chain]) * inv_km1;
        else out[i] = static_cast<double>(src[slot * Cp + chain]);
    }
}

// Running moments pooled over the C chains of one field, natural order, FP64: mean = the chains'
// means averaged; var = the sum over chains of M2_c + k (mean_c - mean)^2, over C k - 1 (the
// variance of all C k draws).  k >= 1 accumulated draws per chain.
template <typename T>
__global__ void pool_kernel(const FieldDev *fields, int32_t fidx, int32_t Cp, int32_t C, int64_t k, const T *mean,
                            const T *m2, const int32_t *perm_inv, double *out_mean, double *out_var)
{
    const FieldDev f = fields[fidx];
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < f.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t slot = f.slot0 + (f.kind == kCsr ? perm_inv[f.csr0 + i] : lattice_slot_of_site(f, i));
        double mu = 0.0;
        for (int c = 0; c < C; ++c) mu += static_cast<double>(mean[slot * Cp + c]);
        mu /= static_cast<double>(C);
        if (out_mean) out_mean[i] = mu;
        if (out_var) {
            double ss = 0.0;
            for (int c = 0; c < C; ++c) {
                const double d = static_cast<double>(mean[slot * Cp + c]) - mu;
                ss += static_cast<double>(m2[slot * Cp + c]) + static_cast<double>(k) * d * d;
            }
            out_var[i] = ss / static_cast<double>(C * k - 1);
        }
    }
}

__global__ void philox_words_kernel(uint2 key, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count, uint4 *out)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = philox4x32_10(make_uint4(static_cast<uint32_t>(i), c1, c2, c3), key);
}

template <typename T>
__global__ void site_normals_kernel(uint2 key, uint32_t sweep, uint32_t stream, uint32_t chain, int lanes,
                                    int64_t count, T *out)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        T z[1];
        site_normals<T, 1>(key, static_cast<uint32_t>(i), sweep, stream, chain, lanes, z);
        out[i] = z[0];
    }
}

// One thread per (sweep of the batch, field, chain, variate): the unit-rate Marsaglia-Tsang
// variates of tau and 1/sigma^2 and the intercept's standard normal, with the counters of that
// sweep's draws.  They are independent of the state, so a whole batch runs in parallel and the
// per-sweep draw reduces to a division by the rate (and a shift for the intercept).
__global__ void gamma_pre_kernel(const GammaPreArgs a)
{
    pdl_wait_then_release();
    const long long base = a.ctl->sweep;
    const int total = gamma_pre_tasks(a);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) gamma_pre_task(a, q, base);
    if (blockIdx.x == 0 && threadIdx.x == 0) gamma_pre_record(a, base);
}

__global__ void ctl_reset_kernel(SweepCtl *ctl, long long start_sweep)
{
    SweepCtl c{};
    c.sweep = start_sweep;
    c.fnext = start_sweep;
    *ctl = c;
}

int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return static_cast<int>(g);
}

}  // namespace

template <int KIND, int MODEL>
cudaError_t launch_model(int precision, int V, const StepArgs &a, cudaStream_t stream)
{
    const dim3 grid(a.ntiles), block(kBlock);
    if (precision == 0) {
        if (V == 4) return launch_sweep_kernel(colour_step_kernel<float, 4, KIND, MODEL>, grid, block, 0, stream, a);
        if (V == 2) return launch_sweep_kernel(colour_step_kernel<float, 2, KIND, MODEL>, grid, block, 0, stream, a);
        return launch_sweep_kernel(colour_step_kernel<float, 1, KIND, MODEL>, grid, block, 0, stream, a);
    }
    if (V == 2) return launch_sweep_kernel(colour_step_kernel<double, 2, KIND, MODEL>, grid, block, 0, stream, a);
    return launch_sweep_kernel(colour_step_kernel<double, 1, KIND, MODEL>, grid, block, 0, stream, a);
}

template <int KIND>
cudaError_t launch_kind(int precision, int V, const StepArgs &a, cudaStream_t stream)
{
    if (a.binomial) return launch_model<KIND, kModelBinomial>(precision, V, a, stream);
    if (a.intercept) return launch_model<KIND, kModelGaussIntercept>(precision, V, a, stream);
    return launch_model<KIND, kModelGauss>(precision, V, a, stream);
}

cudaError_t launch_colour_step(int precision, int V, int kind, const StepArgs &a, cudaStream_t stream)
{
    if (a.ntiles <= 0) return cudaSuccess;
    switch (kind) {
    case kLat2D4: return launch_kind<kLat2D4>(precision, V, a, stream);
    case kLat2D8: return launch_kind<kLat2D8>(precision, V, a, stream);
    case kLat3D6: return launch_kind<kLat3D6>(precision, V, a, stream);
    default: return launch_kind<kCsr>(precision, V, a, stream);
    }
}

cudaError_t launch_hyper(int precision, const HyperArgs &a, cudaStream_t stream)
{
    const int grid = (a.nfields * a.Cp * 2 + kHyperWarps - 1) / kHyperWarps;
    if (a.max_parts >= 256) {  // batched partial-sum loads (fields of many tiles)
        if (precision == 0) return launch_sweep_kernel(hyper_kernel<float, true>, grid, kHyperWarps * 32, 0, stream, a);
        return launch_sweep_kernel(hyper_kernel<double, true>, grid, kHyperWarps * 32, 0, stream, a);
    }
    if (precision == 0) return launch_sweep_kernel(hyper_kernel<float, false>, grid, kHyperWarps * 32, 0, stream, a);
    return launch_sweep_kernel(hyper_kernel<double, false>, grid, kHyperWarps * 32, 0, stream, a);
}

cudaError_t launch_pack(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, int32_t C,
                        int32_t Cp, const double *y_nat, const double *x0_nat, const int32_t *perm_inv, void *x,
                        void *y, cudaStream_t stream)
{
    const int grid = grid_for(f.n, 256);
    if (precision == 0)
        pack_kernel<float><<<grid, 256, 0, stream>>>(fields_dev, fidx, C, Cp, y_nat, x0_nat, perm_inv,
                                                     static_cast<float *>(x), static_cast<float *>(y));
    else
        pack_kernel<double><<<grid, 256, 0, stream>>>(fields_dev, fidx, C, Cp, y_nat, x0_nat, perm_inv,
                                                      static_cast<double *>(x), static_cast<double *>(y));
    return cudaGetLastError();
}

cudaError_t launch_pg_stage(int precision, const PgArgs &a, cudaStream_t stream)
{
    const int64_t tasks = a.slots * a.C;
    int64_t blocks = (tasks + 7) / 8;  // eight warps per block
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    if (precision == 0) return launch_sweep_kernel(pg_stage_kernel<float>, static_cast<int>(blocks), 256, 0, stream, a);
    return launch_sweep_kernel(pg_stage_kernel<double>, static_cast<int>(blocks), 256, 0, stream, a);
}

namespace {

// The checks of data uploaded for gmrf_sampler_set_data, on the device: bit 0 of *flag when a y
// is not finite, bit 1 a trials count outside 0..4095, bit 2 a success count outside
// [0, trials], bit 3 an x0 not finite (x0 may be null; trials null unless binomial).
__global__ void check_data_kernel(const double *y, const int32_t *trials, const double *x0, int64_t n, int64_t nx0,
                                  unsigned int *flag)
{
    unsigned int bad = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        const double v = y[i];
        if (!isfinite(v)) bad |= 1u;
        if (trials) {
            const int32_t m = trials[i];
            if (m < 0 || m > 4095) bad |= 2u;
            if (!(v >= 0.0 && v <= static_cast<double>(m))) bad |= 4u;
        }
    }
    if (x0)
        for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nx0; i += stride)
            if (!isfinite(x0[i])) bad |= 8u;
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, bad);
}

}  // namespace

cudaError_t launch_check_data(const double *y, const int32_t *trials, const double *x0, int64_t n, int64_t nx0,
                              unsigned int *flag, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    check_data_kernel<<<grid_for(n > nx0 ? n : nx0, 256), 256, 0, stream>>>(y, trials, x0, n, nx0, flag);
    return cudaGetLastError();
}

cudaError_t launch_pack_int(const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, const int32_t *v_nat,
                            const int32_t *perm_inv, int32_t *v, cudaStream_t stream)
{
    pack_int_kernel<<<grid_for(f.n, 256), 256, 0, stream>>>(fields_dev, fidx, v_nat, perm_inv, v);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, int32_t Cp,
                          int32_t chain, const void *src, const void *m2, double inv_km1, const int32_t *perm_inv,
                          double *out, cudaStream_t stream)
{
    const int grid = grid_for(f.n, 256);
    if (precision == 0)
        unpack_kernel<float><<<grid, 256, 0, stream>>>(fields_dev, fidx, Cp, chain, static_cast<const float *>(src),
                                                       static_cast<const float *>(m2), inv_km1, perm_inv, out);
    else
        unpack_kernel<double><<<grid, 256, 0, stream>>>(fields_dev, fidx, Cp, chain, static_cast<const double *>(src),
                                                        static_cast<const double *>(m2), inv_km1, perm_inv, out);
    return cudaGetLastError();
}

cudaError_t launch_pool(int precision, const FieldDev *fields_dev, const FieldDev &f, int32_t fidx, int32_t Cp,
                        int32_t C, int64_t k, const void *mean, const void *m2, const int32_t *perm_inv,
                        double *out_mean, double *out_var, cudaStream_t stream)
{
    const int grid = grid_for(f.n, 256);
    if (precision == 0)
        pool_kernel<float><<<grid, 256, 0, stream>>>(fields_dev, fidx, Cp, C, k, static_cast<const float *>(mean),
                                                     static_cast<const float *>(m2), perm_inv, out_mean, out_var);
    else
        pool_kernel<double><<<grid, 256, 0, stream>>>(fields_dev, fidx, Cp, C, k, static_cast<const double *>(mean),
                                                      static_cast<const double *>(m2), perm_inv, out_mean, out_var);
    return cudaGetLastError();
}

cudaError_t launch_gamma_pre(const GammaPreArgs &a, cudaStream_t stream)
{
    const int total = a.count * a.nfields * a.Cp * 4;
    if (total <= 0) return cudaSuccess;
    return launch_sweep_kernel(gamma_pre_kernel, (total + 127) / 128, 128, 0, stream, a);
}

cudaError_t launch_ctl_reset(SweepCtl *ctl, long long start_sweep, cudaStream_t stream)
{
    ctl_reset_kernel<<<1, 1, 0, stream>>>(ctl, start_sweep);
    return cudaGetLastError();
}

cudaError_t launch_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count, uint32_t *out,
                                cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    philox_words_kernel<<<grid_for(count, 256), 256, 0, stream>>>(philox_key(seed), c1, c2, c3, count,
                                                                   reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_site_normals(uint64_t seed, uint32_t sweep, uint32_t stream_id, uint32_t chain, int lanes,
                                int precision, int64_t count, void *out, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    if (precision == 0)
        site_normals_kernel<float><<<grid_for(count, 256), 256, 0, stream>>>(philox_key(seed), sweep, stream_id, chain,
                                                                            lanes, count, static_cast<float *>(out));
    else
        site_normals_kernel<double><<<grid_for(count, 256), 256, 0, stream>>>(philox_key(seed), sweep, stream_id, chain,
                                                                             lanes, count, static_cast<double *>(out));
    return cudaGetLastError();
}

}  // namespace gmrf
