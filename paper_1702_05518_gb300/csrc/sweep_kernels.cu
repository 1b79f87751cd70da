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
// and accumulates, per chain, the two sums the conjugate draws need:
//     (1 - rho) d_i x_i^2 + rho sum_{j lower colour} w_ij (x_i - x_j)^2,   (y_i - x_i)^2,
// so that after the last colour every undirected edge has been counted once, at its endpoint
// of higher colour, with both endpoints final: summed over sites this is x'(D - rho W)x.
// Thread partial sums are in the state precision; warps and blocks reduce in FP64 in a fixed
// order, so results are reproducible run to run.  When the sweep is accumulated, the Welford
// running mean and M2 of the site are updated in the same pass.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {
namespace {

template <typename T> struct AccOf { using type = T; };

template <typename T, int V>
struct SiteCtx {
    T tau[V], isig[V];   // per chain of this thread
    T accS[V], accR[V];  // thread partial sums
    T inv_k;             // 1 / (accumulated count) when accumulating
    bool acc;
};

// Draw (or, in reduce-only mode, read) the V chain values of one site given the neighbour
// values nb[0..nnb), and fold the site's terms into the partial sums.
template <typename T, int V, int NB>
__device__ __forceinline__ void finish_site(const StepArgs &a, SiteCtx<T, V> &cx, T *xp, T *meanp, T *m2p,
                                            T yv, T d, uint32_t site, uint32_t sweep, uint32_t stream,
                                            uint32_t chain0, const T (&s)[V], const T (&nb)[NB][V],
                                            uint32_t lower_mask, const T (&wnb)[NB], int nnb)
{
    const T rho = static_cast<T>(a.rho);
    T xn[V];
    if (a.update) {
        T z[V];
        site_normals<T, V>(a.key, site, sweep, stream, chain0, z);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T P = cx.tau[v] * d + cx.isig[v];
            const T m = (cx.tau[v] * rho * s[v] + yv * cx.isig[v]) / P;
            xn[v] = m + z[v] / sqrt(P);
        }
        Vec<T, V>::st(xp, xn);
    } else {
        Vec<T, V>::ld(xp, xn);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T q = (static_cast<T>(1) - rho) * d * xn[v] * xn[v];
        T e = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (k < nnb && ((lower_mask >> k) & 1u)) {
                const T df = xn[v] - nb[k][v];
                e += wnb[k] * df * df;
            }
        }
        cx.accS[v] += q + rho * e;
        const T r = yv - xn[v];
        cx.accR[v] += r * r;
    }
    if (cx.acc) {
        T mu[V], mm[V];
        Vec<T, V>::ld(meanp, mu);
        Vec<T, V>::ld(m2p, mm);
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
// of rows r -+ 1 (i -+ 1) and r -+ H (l -+ 1).
template <typename T, int V, bool THREE_D>
__device__ void lattice_parity_tile(const StepArgs &a, const FieldDev &f, const Tile &t, SiteCtx<T, V> &cx,
                                    int CV, uint32_t sweep)
{
    constexpr int NB = THREE_D ? 6 : 4;
    const int L = THREE_D ? f.dims[0] : 1;
    const int H = THREE_D ? f.dims[1] : f.dims[0];
    const int W = THREE_D ? f.dims[2] : f.dims[1];
    const int c = t.colour;
    T *X = static_cast<T *>(a.x);
    const T *Y = static_cast<const T *>(a.y);
    T *MEAN = static_cast<T *>(a.mean);
    T *M2 = static_cast<T *>(a.m2);
    const int64_t Cp = a.Cp;
    const int64_t self_base = f.slot0 + static_cast<int64_t>(c) * f.rows * f.cols;
    const int64_t oth_base = f.slot0 + static_cast<int64_t>(1 - c) * f.rows * f.cols;
    const bool lower = (c == 1);  // all neighbours have the other colour
    const int64_t nelem = static_cast<int64_t>(t.count) * f.cols * CV;
    for (int64_t e = threadIdx.x; e < nelem; e += kBlock) {
        const int cv = static_cast<int>(e % CV);
        const int64_t sr = e / CV;
        const int r = t.start + static_cast<int>(sr / f.cols);
        const int h = static_cast<int>(sr % f.cols);
        const int l = THREE_D ? r / H : 0;
        const int i = THREE_D ? r - l * H : r;
        const int p = (c + l + i) & 1;
        const int j = 2 * h + p;
        if (j >= W)
            continue;
        int64_t ns[NB];
        int nnb = 0;
        if (j > 0) ns[nnb++] = static_cast<int64_t>(r) * f.cols + (h - 1 + p);
        if (j + 1 < W) ns[nnb++] = static_cast<int64_t>(r) * f.cols + (h + p);
        if (i > 0) ns[nnb++] = static_cast<int64_t>(r - 1) * f.cols + h;
        if (i + 1 < H) ns[nnb++] = static_cast<int64_t>(r + 1) * f.cols + h;
        if (THREE_D) {
            if (l > 0) ns[nnb++] = static_cast<int64_t>(r - H) * f.cols + h;
            if (l + 1 < L) ns[nnb++] = static_cast<int64_t>(r + H) * f.cols + h;
        }
        T nb[NB][V], wnb[NB], s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            wnb[k] = 1;
            if (k < nnb) {
                Vec<T, V>::ld(X + (oth_base + ns[k]) * Cp + cv * V, nb[k]);
#pragma unroll
                for (int v = 0; v < V; ++v) s[v] += nb[k][v];
            }
        }
        const int64_t self = self_base + static_cast<int64_t>(r) * f.cols + h;
        const uint32_t site = static_cast<uint32_t>(static_cast<int64_t>(r) * W + j);
        finish_site<T, V, NB>(a, cx, X + self * Cp + cv * V, MEAN + self * Cp + cv * V, M2 + self * Cp + cv * V,
                              Y[self], static_cast<T>(nnb), site, sweep, f.stream, static_cast<uint32_t>(cv * V),
                              s, nb, lower ? 0xffu : 0u, wnb, nnb);
    }
}

// 2-D 8-neighbour lattice with the 2x2 colouring c = 2 (i & 1) + (j & 1): the site of colour
// c = 2a + b at sub-array (u, v) is (2u + a, 2v + b); neighbour (i + di, j + dj) lives in
// colour 2((i + di) & 1) + ((j + dj) & 1) at ((i + di) >> 1, (j + dj) >> 1).
template <typename T, int V>
__device__ void lattice8_tile(const StepArgs &a, const FieldDev &f, const Tile &t, SiteCtx<T, V> &cx, int CV,
                              uint32_t sweep)
{
    constexpr int NB = 8;
    const int H = f.dims[0], W = f.dims[1];
    const int c = t.colour;
    const int ca = c >> 1, cb = c & 1;
    T *X = static_cast<T *>(a.x);
    const T *Y = static_cast<const T *>(a.y);
    T *MEAN = static_cast<T *>(a.mean);
    T *M2 = static_cast<T *>(a.m2);
    const int64_t Cp = a.Cp;
    const int64_t sub = static_cast<int64_t>(f.rows) * f.cols;
    const int64_t nelem = static_cast<int64_t>(t.count) * f.cols * CV;
    for (int64_t e = threadIdx.x; e < nelem; e += kBlock) {
        const int cv = static_cast<int>(e % CV);
        const int64_t sr = e / CV;
        const int u = t.start + static_cast<int>(sr / f.cols);
        const int vv = static_cast<int>(sr % f.cols);
        const int i = 2 * u + ca, j = 2 * vv + cb;
        if (i >= H || j >= W)
            continue;
        int64_t ns[NB];
        uint32_t lower = 0;
        int nnb = 0;
#pragma unroll
        for (int di = -1; di <= 1; ++di)
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj) {
                if (di == 0 && dj == 0) continue;
                const int ii = i + di, jj = j + dj;
                if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                const int cc = 2 * (ii & 1) + (jj & 1);
                ns[nnb] = f.slot0 + cc * sub + static_cast<int64_t>(ii >> 1) * f.cols + (jj >> 1);
                if (cc < c) lower |= 1u << nnb;
                ++nnb;
            }
        T nb[NB][V], wnb[NB], s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            wnb[k] = 1;
            if (k < nnb) {
                Vec<T, V>::ld(X + ns[k] * Cp + cv * V, nb[k]);
#pragma unroll
                for (int v = 0; v < V; ++v) s[v] += nb[k][v];
            }
        }
        const int64_t self = f.slot0 + c * sub + static_cast<int64_t>(u) * f.cols + vv;
        const uint32_t site = static_cast<uint32_t>(static_cast<int64_t>(i) * W + j);
        finish_site<T, V, NB>(a, cx, X + self * Cp + cv * V, MEAN + self * Cp + cv * V, M2 + self * Cp + cv * V,
                              Y[self], static_cast<T>(nnb), site, sweep, f.stream, static_cast<uint32_t>(cv * V),
                              s, nb, lower, wnb, nnb);
    }
}

// CSR field: permuted positions [start, start + count) of one colour class; neighbours are read
// through the permuted row; a neighbour has lower colour iff its position is below the class's
// first position.  The lower-colour terms of the reduction take a second pass over the row.
template <typename T, int V>
__device__ void csr_tile(const StepArgs &a, const FieldDev &f, const Tile &t, SiteCtx<T, V> &cx, int CV,
                         uint32_t sweep)
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
    const int64_t nelem = static_cast<int64_t>(t.count) * CV;
    for (int64_t e = threadIdx.x; e < nelem; e += kBlock) {
        const int cv = static_cast<int>(e % CV);
        const int pos = t.start + static_cast<int>(e / CV);
        const int rb = rp[pos], re = rp[pos + 1];
        T s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = 0;
        for (int k = rb; k < re; ++k) {
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
        T nb0[1][V];
        T w0[1] = {0};
        finish_site<T, V, 1>(a, cx, X + self * Cp + cv * V, MEAN + self * Cp + cv * V, M2 + self * Cp + cv * V, yv,
                             d, site, sweep, f.stream, static_cast<uint32_t>(cv * V), s, nb0, 0u, w0, 0);
        // finish_site added (1 - rho) d x^2 and the likelihood term; add the lower-colour edges.
        T xn[V];
        Vec<T, V>::ld(X + self * Cp + cv * V, xn);
        T e2[V];
#pragma unroll
        for (int v = 0; v < V; ++v) e2[v] = 0;
        for (int k = rb; k < re; ++k) {
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

template <typename T, int V>
__global__ void __launch_bounds__(kBlock) colour_step_kernel(const StepArgs a)
{
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
        const int64_t hc = (static_cast<int64_t>(t.field) * a.Cp + cv * V + v) * 2;
        cx.tau[v] = hyp[hc];
        cx.isig[v] = hyp[hc + 1];
        cx.accS[v] = 0;
        cx.accR[v] = 0;
    }
    cx.acc = false;
    cx.inv_k = 0;
    if (a.update && a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin)) {
        cx.acc = true;
        cx.inv_k = static_cast<T>(1) / static_cast<T>(a.ctl->acc_count + 1);
    }

    if (f.kind == kLat2D4) lattice_parity_tile<T, V, false>(a, f, t, cx, CV, sweep);
    else if (f.kind == kLat3D6) lattice_parity_tile<T, V, true>(a, f, t, cx, CV, sweep);
    else if (f.kind == kLat2D8) lattice8_tile<T, V>(a, f, t, cx, CV, sweep);
    else csr_tile<T, V>(a, f, t, cx, CV, sweep);

    // Deterministic block reduction of the 2 V partial sums of each chain: FP64 shuffle tree
    // over the lanes that share a chain vector (lanes equal mod CV), then warps in order.
    __shared__ double red[kBlock / 32][kMaxChains][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        double sS = static_cast<double>(cx.accS[v]);
        double sR = static_cast<double>(cx.accR[v]);
        for (int off = 16; off >= CV; off >>= 1) {
            sS += __shfl_xor_sync(0xffffffffu, sS, off);
            sR += __shfl_xor_sync(0xffffffffu, sR, off);
        }
        if (lane < CV) {
            red[warp][lane * V + v][0] = sS;
            red[warp][lane * V + v][1] = sR;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.Cp * 2; q += kBlock) {
        const int chain = q >> 1, k = q & 1;
        double acc = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) acc += red[w][chain][k];
        double *dst = reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * a.Cp + chain);
        dst[k] = acc;
    }
}

// One block per (field, chain): the block sums the field's tile partials in a fixed order (thread
// strides, then a shuffle tree, then warps in order) and thread 0 draws tau and 1/sigma^2 from
// their Gamma full conditionals (Sec. 3.1), refreshes the precision-T copies the colour kernels
// read, and records the traces.  The last block to finish (ticket counter; no block waits for
// another) advances the sweep counter, the accumulation count, or the extra-draw counter.
template <typename T>
__global__ void __launch_bounds__(256) hyper_kernel(const HyperArgs a)
{
    __shared__ double red[8][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long sweep = a.ctl->sweep;
    const long long extra = a.ctl->extra;
    const int pidx = blockIdx.x;
    const int fi = pidx / a.Cp, chain = pidx - fi * a.Cp;
    const FieldDev f = a.fields[fi];
    double S = 0.0, R = 0.0;
    if (a.draw) {
        for (int k = threadIdx.x; k < f.nparts; k += blockDim.x) {
            const double2 p = a.partials[static_cast<int64_t>(f.part0 + k) * a.Cp + chain];
            S += p.x;
            R += p.y;
        }
        for (int off = 16; off >= 1; off >>= 1) {
            S += __shfl_xor_sync(0xffffffffu, S, off);
            R += __shfl_xor_sync(0xffffffffu, R, off);
        }
        if (lane == 0) {
            red[warp][0] = S;
            red[warp][1] = R;
        }
        __syncthreads();
        S = 0.0;
        R = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            S += red[w][0];
            R += red[w][1];
        }
    }
    if (threadIdx.x == 0) {
        const int64_t hc = static_cast<int64_t>(fi) * a.Cp + chain;
        double tau = a.tau[hc], sig2 = a.sig2[hc];
        if (a.draw) {
            const uint32_t word1 = static_cast<uint32_t>(a.end_of_sweep ? sweep : extra);
            const uint32_t ttag = (a.end_of_sweep ? kTagTau : kTagTauExtra) << 24;
            const uint32_t stag = (a.end_of_sweep ? kTagSig : kTagSigExtra) << 24;
            int fb1 = 0, fb2 = 0;
            tau = gamma_mt(a.a_tau + 0.5 * f.rank, a.b_tau + 0.5 * S, a.key, word1, f.stream,
                           ttag | static_cast<uint32_t>(chain), fb1);
            const double prec = gamma_mt(a.a_sig + 0.5 * f.n, a.b_sig + 0.5 * R, a.key, word1, f.stream,
                                         stag | static_cast<uint32_t>(chain), fb2);
            sig2 = 1.0 / prec;
            if (fb1 + fb2)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->fallbacks),
                          static_cast<unsigned long long>(fb1 + fb2));
            a.tau[hc] = tau;
            a.sig2[hc] = sig2;
            T *hyp = static_cast<T *>(a.hyp);
            hyp[hc * 2] = static_cast<T>(tau);
            hyp[hc * 2 + 1] = static_cast<T>(prec);
        }
        if (a.end_of_sweep && a.trace_cap > 0) {
            const int64_t slot = hc * a.trace_cap + (sweep % a.trace_cap);
            a.trace_tau[slot] = tau;
            a.trace_sig[slot] = sig2;
        }
        __threadfence();
        const unsigned long long done = atomicAdd(&a.ctl->ticket, 1ull);
        if (done == gridDim.x - 1) {
            if (a.end_of_sweep) {
                if (a.acc_enabled && sweep_accumulated(sweep, a.burn_in, a.thin)) a.ctl->acc_count += 1;
                a.ctl->sweep = sweep + 1;
            } else {
                a.ctl->extra = extra + 1;
            }
            a.ctl->ticket = 0;
        }
    }
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

__global__ void philox_words_kernel(uint2 key, uint32_t c1, uint32_t c2, uint32_t c3, int64_t count, uint4 *out)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = philox4x32_10(make_uint4(static_cast<uint32_t>(i), c1, c2, c3), key);
}

template <typename T>
__global__ void site_normals_kernel(uint2 key, uint32_t sweep, uint32_t stream, uint32_t chain, int64_t count, T *out)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        T z[1];
        site_normals<T, 1>(key, static_cast<uint32_t>(i), sweep, stream, chain, z);
        out[i] = z[0];
    }
}

__global__ void ctl_reset_kernel(SweepCtl *ctl, long long start_sweep)
{
    SweepCtl c{};
    c.sweep = start_sweep;
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

cudaError_t launch_colour_step(int precision, int V, const StepArgs &a, cudaStream_t stream)
{
    if (a.ntiles <= 0) return cudaSuccess;
    const dim3 grid(a.ntiles), block(kBlock);
    if (precision == 0) {
        if (V == 4) colour_step_kernel<float, 4><<<grid, block, 0, stream>>>(a);
        else if (V == 2) colour_step_kernel<float, 2><<<grid, block, 0, stream>>>(a);
        else colour_step_kernel<float, 1><<<grid, block, 0, stream>>>(a);
    } else {
        if (V == 2) colour_step_kernel<double, 2><<<grid, block, 0, stream>>>(a);
        else colour_step_kernel<double, 1><<<grid, block, 0, stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_hyper(int precision, const HyperArgs &a, cudaStream_t stream)
{
    const int grid = a.nfields * a.Cp;
    if (precision == 0) hyper_kernel<float><<<grid, 256, 0, stream>>>(a);
    else hyper_kernel<double><<<grid, 256, 0, stream>>>(a);
    return cudaGetLastError();
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

cudaError_t launch_site_normals(uint64_t seed, uint32_t sweep, uint32_t stream_id, uint32_t chain, int precision,
                                int64_t count, void *out, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    if (precision == 0)
        site_normals_kernel<float><<<grid_for(count, 256), 256, 0, stream>>>(philox_key(seed), sweep, stream_id, chain,
                                                                            count, static_cast<float *>(out));
    else
        site_normals_kernel<double><<<grid_for(count, 256), 256, 0, stream>>>(philox_key(seed), sweep, stream_id, chain,
                                                                             count, static_cast<double *>(out));
    return cudaGetLastError();
}

}  // namespace gmrf
