// lattice_fused.cu -- one launch per sweep for 2-D lattice fields: all k colour steps of
// Algorithm 1 run inside the kernel on a shared-memory copy of the block's tile.
//
// A block owns a TR x TC tile of natural sites.  It stages the tile plus a halo of width k
// (k = 2 colours for the 4-neighbour lattice, 4 for the 8-neighbour one) from the colour-split
// state into shared memory, draws the normals of every site it will update (phase A, no
// barriers), then performs colour steps c = 0..k-1 in place: step c draws the colour-c sites
// of the tile grown by k-1-c rings.  Each step reads only values the previous
// steps made final, so after the last step the owned sites hold exactly the sweep's result
// (Sec. 2.3: the sites of one colour are conditionally independent given the others).  Sites
// of the halo are drawn by every block that overlaps them; the counter-based generator makes
// those draws identical, so no block needs another's results within a sweep.  The owned sites
// are then written to the other of two state buffers (so no block stages a neighbour's new
// values), folded into the two sums of the hyperparameter conditionals (each edge counted at
// its endpoint of higher colour) and, when the sweep is accumulated, into the running mean
// and M2.
#include <cuda_runtime.h>

#include <type_traits>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "lattice_common.cuh"

namespace gmrf {
namespace {

template <typename T, int V, int KIND, int kFusedBlock>
__global__ void __launch_bounds__(kFusedBlock, (kFusedBlock == 512 && sizeof(T) == 4 && V <= 2) ? 2 : 1)
    lattice_fused_kernel(const FusedArgs a)
{
    pdl_wait_then_release();
    using D = Dirs<KIND>;
    constexpr bool E8 = (KIND == kLat2D8);
    constexpr int K = E8 ? 4 : 2;   // colours = halo width
    constexpr int NS = E8 ? 4 : 2;  // sub-arrays
    constexpr int NW = kFusedBlock / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileXY t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const int Hl = f.dims[0], Wl = f.dims[1];
    const int TR = a.TR, TC = a.TC, RR = TR + 2 * K, RC = TC + 2 * K;
    const int SR = E8 ? (RR >> 1) : RR, SC = RC >> 1, SUB = SR * SC;
    const int Cp = a.Cp, CV = Cp / V, cv_shift = __ffs(CV) - 1;
    const int tx = threadIdx.x & 31;
    const int cvo = (tx & (CV - 1)) * V;  // chain offset of this thread (fixed: 32 % CV == 0)
    T *xs = reinterpret_cast<T *>(smem_raw);  // [NS][SR][SC][Cp] state
    T *zs = xs + NS * SUB * Cp;               // [NS][SR][SC][Cp] normals of this sweep
    T *ys = zs + NS * SUB * Cp;               // [NS][SR][SC] observations
    const int gi0 = t.i0 - K, gj0 = t.j0 - K;
    const int gu0 = E8 ? (gi0 >> 1) : gi0, gv0 = gj0 >> 1;  // staged origin in the global sub-arrays
    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + RR <= Hl && gj0 + RC <= Wl;
    // Ping-pong state: sweep t reads buffer t & 1 and writes the other, so no block can see a
    // neighbour's new values while staging its halo.
    const long long sweep_ll = a.ctl->sweep;
    const void *xsrc = (sweep_ll & 1) ? a.x_alt : a.x;
    void *xdst = (sweep_ll & 1) ? a.x : a.x_alt;
    const int64_t gsub = static_cast<int64_t>(f.rows) * f.cols;  // sites per global sub-array
    const T *X = static_cast<const T *>(xsrc) + f.slot0 * Cp + cvo;
    const T *Y = static_cast<const T *>(a.y) + f.slot0;
    const uint32_t sweep = static_cast<uint32_t>(sweep_ll);
    const T rho = static_cast<T>(a.rho);

    T tau[V], isig[V], beta[V];
    const T *hyp = static_cast<const T *>(a.hyp);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int64_t hc = (static_cast<int64_t>(t.field) * Cp + cvo + v) * kHypStride;
        tau[v] = hyp[hc];
        isig[v] = hyp[hc + 1];
        beta[v] = hyp[hc + 2];
    }

    // Stage: rows of the NS sub-arrays; slots outside a global sub-array read as zero, and the
    // global padding slots (sites beyond an odd extent) hold zero, so every position outside
    // the lattice is zero.
    {
        const int rowu = SC << cv_shift;  // work units per staged row
        const float rcp_rowu = __frcp_rn(static_cast<float>(rowu)), rcp_sr = __frcp_rn(static_cast<float>(SR));
        // Four loads per thread in flight before their stores (the loads come from L2 or HBM).
        constexpr int UNR = 4;
        const int total = NS * SR * rowu;
        for (int q0 = threadIdx.x; q0 < total; q0 += UNR * kFusedBlock) {
            T val[UNR][V], yv[UNR];
            int si[UNR];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int q = q0 + k * kFusedBlock;
                si[k] = -1;
                if (q >= total) continue;
                const int rr = div_small(q, rcp_rowu), u = q - rr * rowu;
                const int sa = div_small(rr, rcp_sr), r = rr - sa * SR;
                const int v = u >> cv_shift, gu = gu0 + r, gv = gv0 + v;
                const bool ok = interior || (gu >= 0 && gu < f.rows && gv >= 0 && gv < f.cols);
                const int64_t go = sa * gsub + static_cast<int64_t>(gu) * f.cols + gv;
                si[k] = rr * SC + v;
                if (ok) {
                    Vec<T, V>::ld(X + go * Cp, val[k]);
                    yv[k] = Y[go];
                } else {
#pragma unroll
                    for (int w = 0; w < V; ++w) val[k][w] = 0;
                    yv[k] = 0;
                }
            }
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                if (si[k] < 0) continue;
                Vec<T, V>::st(xs + si[k] * Cp + cvo, val[k]);
                if (cvo == 0) ys[si[k]] = yv[k];
            }
        }
    }

    // Region of the colour-c sites drawn by this block: the tile grown by K - 1 - c rings,
    // clipped to the lattice.  Calls fn(i, j, idx) with idx the site's shared-memory index.
    auto for_region = [&](int c, auto &&fn) {
        const int e = K - 1 - c;
        const int lo_i = max(0, t.i0 - e), hi_i = min(Hl, t.i0 + TR + e);
        const int lo_j = max(0, t.j0 - e), hi_j = min(Wl, t.j0 + TC + e);
        if (E8) {
            const int ca = c >> 1, cb = c & 1;
            const int u_lo = (lo_i - gi0 - ca + 1) >> 1, u_hi = (hi_i - gi0 - ca + 1) >> 1;
            const int v_lo = (lo_j - gj0 - cb + 1) >> 1, v_hi = (hi_j - gj0 - cb + 1) >> 1;
            const int nu = (v_hi - v_lo) << cv_shift;
            if (u_hi <= u_lo || nu <= 0) return;
            const float rcp = __frcp_rn(static_cast<float>(nu));
            for (int q = threadIdx.x; q < (u_hi - u_lo) * nu; q += kFusedBlock) {
                const int ru = div_small(q, rcp), w = q - ru * nu;
                const int u = u_lo + ru, v = v_lo + (w >> cv_shift);
                fn(gi0 + 2 * u + ca, gj0 + 2 * v + cb, (c * SR + u) * SC + v);
            }
        } else {
            // Colour-c sites of row i sit at columns of parity (c + i) & 1: at most nv per row.
            const int nv = (hi_j - lo_j + 1) >> 1, nu = nv << cv_shift;
            if (hi_i <= lo_i || nu <= 0) return;
            const float rcp = __frcp_rn(static_cast<float>(nu));
            for (int q = threadIdx.x; q < (hi_i - lo_i) * nu; q += kFusedBlock) {
                const int ri = div_small(q, rcp), w = q - ri * nu;
                const int i = lo_i + ri, p = (c + i) & 1;
                const int v = ((lo_j - gj0 - p + 1) >> 1) + (w >> cv_shift);
                const int j = gj0 + 2 * v + p;
                if (j >= hi_j) continue;
                fn(i, j, (c * SR + (i - gi0)) * SC + v);
            }
        }
    };

    // Phase A: the normals of every site this block draws in this sweep.  They depend on
    // (site, sweep, chain) only, so this phase has no barriers and carries most of the
    // arithmetic.
    if (a.update && a.lanes == 4) {
        // One Philox block per (site, chain quadruple).
        for (int c = 0; c < K; ++c)
            for_region(c, [&](int i, int j, int idx) {
                T z[V];
                site_normals<T, V>(a.key, static_cast<uint32_t>(i * Wl + j), sweep, f.stream,
                                   static_cast<uint32_t>(cvo), 4, z);
                Vec<T, V>::st(zs + idx * Cp + cvo, z);
            });
    } else if (a.update) {
        // One Philox block per group of G = 4 / lanes consecutive natural sites (one or two
        // chains, so every thread holds all chains): its four normals go to the group's sites
        // in this row that some colour step of this block draws.
        const int gs = lanes_shift(a.lanes), G = 1 << gs, L = a.lanes;
        const int ngmax = (RC >> gs) + 2;
        const int jl = max(0, gj0), jh = min(Wl, gj0 + RC);
        for (int q = threadIdx.x; q < RR * ngmax; q += kFusedBlock) {
            const int ri = fast_div(q, a.ng_m, a.ng_s), k = q - ri * ngmax;
            const int i = gi0 + ri;
            if (i < 0 || i >= Hl || jl >= jh) continue;
            const int s0 = i * Wl + jl, s1 = i * Wl + jh;
            const int g = (s0 >> gs) + k;
            if ((g << gs) >= s1) continue;
            T n4[4];
            block_normals<T>(a.key, static_cast<uint32_t>(g), sweep, f.stream, 0u, n4);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r >= G) break;
                const int st = (g << gs) + r;
                if (st < s0 || st >= s1) continue;
                const int j = st - i * Wl;
                const int e = K - 1 - D::colour(i, j);
                if (i < t.i0 - e || i >= t.i0 + TR + e || j < t.j0 - e || j >= t.j0 + TC + e) continue;
                T *zp = zs + sm_index<KIND>(i, j, gi0, gj0, SR, SC) * Cp;
                for (int ch = 0; ch < L; ++ch) zp[ch] = n4[r * L + ch];
            }
        }
    }
    __syncthreads();

    // Phase B: colour steps in shared memory.  Neighbour k of a colour-c site sits at a fixed
    // offset from the site (block-uniform per step; for the 4-neighbour lattice the in-row
    // offsets depend on the row's parity); positions outside the lattice hold zeros, so the
    // sum needs no bounds tests.  The owned sites also fold their terms of the two sums of the
    // hyperparameter conditionals here, while their neighbours are in registers: (1 - rho) d x^2
    // + rho sum over lower-colour neighbours of (x - x_j)^2, and e^2 and e, e = y - beta0 - x.
    T accS[V], accR[V], accA[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        accS[v] = 0;
        accR[v] = 0;
        accA[v] = 0;
    }
#pragma unroll 1
    for (int c = 0; c < (a.update ? K : 0); ++c) {
        int off8[8];
        uint32_t lower = 0;
        if (E8) {
            const int ca = c >> 1, cb = c & 1;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int ai = ca + D::di(k), bj = cb + D::dj(k);
                const int cc = 2 * (ai & 1) + (bj & 1);
                off8[k] = ((cc - c) * SR + (ai >> 1)) * SC + (bj >> 1);
                if (cc < c) lower |= 1u << k;
            }
        } else if (c == 1) {
            lower = 0xfu;
        }
        for_region(c, [&, off8](int i, int j, int idx) {
            int off[D::N];
            if (E8) {
#pragma unroll
                for (int k = 0; k < D::N; ++k) off[k] = off8[k];
            } else {
                const int p = (c + i) & 1, o = (1 - 2 * c) * SR * SC;  // other colour's sub-array
                off[0] = o - SC;         // (i - 1, j)
                off[1] = o - 1 + p;      // (i, j - 1)
                off[2] = o + p;          // (i, j + 1)
                off[3] = o + SC;         // (i + 1, j)
            }
            const T *xc = xs + idx * Cp + cvo;
            T nb[D::N][V], s[V];
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
            for (int k = 0; k < D::N; ++k) {
                Vec<T, V>::ld(xc + off[k] * Cp, nb[k]);
#pragma unroll
                for (int v = 0; v < V; ++v) s[v] += nb[k][v];
            }
            int deg = D::N;
            uint32_t valid = (1u << D::N) - 1u;
            if (!interior) {
                const bool up = i > 0, down = i + 1 < Hl, left = j > 0, right = j + 1 < Wl;
                valid = 0;
#pragma unroll
                for (int k = 0; k < D::N; ++k) {
                    const int di = D::di(k), dj = D::dj(k);
                    const bool ok = (di < 0 ? up : (di > 0 ? down : true)) && (dj < 0 ? left : (dj > 0 ? right : true));
                    valid |= ok ? (1u << k) : 0u;
                }
                deg = __popc(valid);
            }
            T z[V];
            Vec<T, V>::ld(zs + idx * Cp + cvo, z);
            const T yv = ys[idx];
            const T d = static_cast<T>(deg);
            T xn[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T P = tau[v] * d + isig[v];
                const T m = (tau[v] * rho * s[v] + (yv - beta[v]) * isig[v]) * FArith<T>::rcp(P);
                xn[v] = m + z[v] * FArith<T>::rsq(P);
            }
            Vec<T, V>::st(xs + idx * Cp + cvo, xn);
            if (i >= t.i0 && i < t.i0 + TR && j >= t.j0 && j < t.j0 + TC) {
                const uint32_t lv = lower & valid;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    T e = 0;
#pragma unroll
                    for (int k = 0; k < D::N; ++k)
                        if ((lv >> k) & 1u) {
                            const T df = xn[v] - nb[k][v];
                            e += df * df;
                        }
                    accS[v] += (static_cast<T>(1) - rho) * d * xn[v] * xn[v] + rho * e;
                    const T r = (yv - beta[v]) - xn[v];
                    accR[v] += r * r;
                    accA[v] += r;
                }
            }
        });
        __syncthreads();
    }

    // Reduce-only mode (no colour steps): fold the owned sites' terms from the staged state.
    if (!a.update) {
        for (int c = 0; c < K; ++c) {
            for_region(c, [&](int i, int j, int idx) {
                if (i < t.i0 || i >= t.i0 + TR || j < t.j0 || j >= t.j0 + TC) return;
                T xn[V];
                Vec<T, V>::ld(xs + idx * Cp + cvo, xn);
                int deg = 0;
                T e[V];
#pragma unroll
                for (int v = 0; v < V; ++v) e[v] = 0;
#pragma unroll
                for (int k = 0; k < D::N; ++k) {
                    const int ii = i + D::di(k), jj = j + D::dj(k);
                    if (ii < 0 || ii >= Hl || jj < 0 || jj >= Wl) continue;
                    ++deg;
                    if (D::colour(ii, jj) >= c) continue;
                    T nbv[V];
                    Vec<T, V>::ld(xs + sm_index<KIND>(ii, jj, gi0, gj0, SR, SC) * Cp + cvo, nbv);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const T df = xn[v] - nbv[v];
                        e[v] += df * df;
                    }
                }
                const T yv = ys[idx];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    accS[v] += (static_cast<T>(1) - rho) * static_cast<T>(deg) * xn[v] * xn[v] + rho * e[v];
                    const T r = (yv - beta[v]) - xn[v];
                    accR[v] += r * r;
                    accA[v] += r;
                }
            });
        }
    }

    // Write-back of the owned sites (rows of the sub-arrays) and the running mean / M2.
    const bool acc = a.update && a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin);
    if (a.update) {
        T inv_k = 0;
        if (acc) inv_k = static_cast<T>(1) / static_cast<T>(a.ctl->acc_count + 1);
        T *XW = static_cast<T *>(xdst) + f.slot0 * Cp + cvo;
        T *MEAN = static_cast<T *>(a.mean) + f.slot0 * Cp + cvo;
        T *M2 = static_cast<T *>(a.m2) + f.slot0 * Cp + cvo;
        const int orow = E8 ? (TR >> 1) : TR;          // owned rows per sub-array
        const int r0 = E8 ? (K >> 1) : K, v0 = K >> 1;  // first owned row / column in a sub-array
        const int rowu = (TC >> 1) << cv_shift;
        const float rcp_rowu = __frcp_rn(static_cast<float>(rowu)), rcp_orow = __frcp_rn(static_cast<float>(orow));
        for (int q = threadIdx.x; q < NS * orow * rowu; q += kFusedBlock) {
            const int rr = div_small(q, rcp_rowu), w = q - rr * rowu;
            const int sa = div_small(rr, rcp_orow), r = rr - sa * orow;
            const int sr = r0 + r, gu = gu0 + sr;
            const int i = E8 ? gi0 + 2 * sr + (sa >> 1) : gi0 + sr;
            if (i >= Hl) continue;
            {
                const int v = v0 + (w >> cv_shift);
                const int pj = E8 ? (sa & 1) : ((sa + i) & 1);
                const int j = gj0 + 2 * v + pj;
                if (j >= Wl) continue;
                const int64_t go = (sa * gsub + static_cast<int64_t>(gu) * f.cols + gv0 + v) * Cp;
                T xn[V];
                Vec<T, V>::ld(xs + ((sa * SR + sr) * SC + v) * Cp + cvo, xn);
                Vec<T, V>::st(XW + go, xn);
                if (acc) {
                    T mu[V], mm[V];
                    Vec<T, V>::ld(MEAN + go, mu);
                    Vec<T, V>::ld(M2 + go, mm);
#pragma unroll
                    for (int q = 0; q < V; ++q) {
                        const T delta = xn[q] - mu[q];
                        mu[q] += delta * inv_k;
                        mm[q] += delta * (xn[q] - mu[q]);
                    }
                    Vec<T, V>::st(MEAN + go, mu);
                    Vec<T, V>::st(M2 + go, mm);
                }
            }
        }
    }

    // Deterministic block reduction in precision T (shuffle tree over lanes sharing a chain
    // vector, then warps in order) into the tile's FP64 partial-sum slot; a tile holds at most a
    // few thousand terms, the sum over tiles is FP64.
    // Reduction scratch [NW][Cp][3] reuses the normals' space (dead after phase B).
    T *red = zs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T sS = accS[v], sR = accR[v], sA = accA[v];
        for (int off = 16; off >= CV; off >>= 1) {
            sS += __shfl_xor_sync(0xffffffffu, sS, off);
            sR += __shfl_xor_sync(0xffffffffu, sR, off);
            sA += __shfl_xor_sync(0xffffffffu, sA, off);
        }
        if (lane < CV) {
            red[(warp * Cp + lane * V + v) * 3] = sS;
            red[(warp * Cp + lane * V + v) * 3 + 1] = sR;
            red[(warp * Cp + lane * V + v) * 3 + 2] = sA;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < Cp * 3; q += kFusedBlock) {
        const int chain = q / 3, k = q - 3 * chain;
        T sum = 0;
        for (int w = 0; w < NW; ++w) sum += red[(w * Cp + chain) * 3 + k];
        reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * Cp + chain)[k] = static_cast<double>(sum);
    }
}

// Fast path: every thread holds all CP chains of a site (CP = 1, 2 or 4, the chain count of the
// layout), so chain strides are compile-time constants; only colour steps (update mode).  Same
// phases and results as lattice_fused_kernel, with the per-site index work cut down:
// field-relative 32-bit offsets, staging indices equal to the shared-memory index, normals
// drawn for every staged site (no per-site region tests), neighbour offsets fixed per colour
// step, lower-colour terms as 0/1 weights, and bounds tests only for sites on the lattice edge.
// Two 512-thread blocks per SM (64 registers) for FP32 with up to two chains per thread; with four
// chains the 128 registers of one block per SM avoid spilling the neighbours' chain vectors.
template <typename T, int KIND, int NT, int CP>
__global__ void __launch_bounds__(NT, (NT == 512 && sizeof(T) == 4 && CP < 4) ? 2 : 1) lattice_fused_fast(const FusedArgs a)
{
    using D = Dirs<KIND>;
    constexpr bool E8 = (KIND == kLat2D8);
    constexpr int K = E8 ? 4 : 2;
    constexpr int NS = E8 ? 4 : 2;
    constexpr int NW = NT / 32;
    constexpr int ND = D::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileXY t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const int Hl = f.dims[0], Wl = f.dims[1];
    const int TR = a.TR, TC = a.TC, RR = TR + 2 * K, RC = TC + 2 * K;
    const int SR = E8 ? (RR >> 1) : RR, SC = RC >> 1, SUB = SR * SC;
    T *xs = reinterpret_cast<T *>(smem_raw);  // [NS * SUB][CP]
    T *zs = xs + NS * SUB * CP;               // [NS * SUB][CP]
    T *ys = zs + NS * SUB * CP;               // [NS * SUB]
    const int gi0 = t.i0 - K, gj0 = t.j0 - K;
    const int gu0 = E8 ? (gi0 >> 1) : gi0, gv0 = gj0 >> 1;
    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + RR <= Hl && gj0 + RC <= Wl;
    const T *Y = static_cast<const T *>(a.y) + f.slot0;
    const int gsub = f.rows * f.cols, gcols = f.cols, grows = f.rows;
    const T rho = static_cast<T>(a.rho);
    const float rcp_sc = __frcp_rn(static_cast<float>(SC)), rcp_sr = __frcp_rn(static_cast<float>(SR));

    // Stage rows of the sub-arrays into shared memory (four loads in flight per thread): the
    // observations (src_y) or the state (src_x, CP chains).  The staged index q is the
    // shared-memory index; positions off the lattice are 0.
    auto stage = [&](const T *src_x, const T *src_y) {
        constexpr int UNR = 4;
        const int total = NS * SUB;
        for (int q0 = threadIdx.x; q0 < total; q0 += UNR * NT) {
            T val[UNR][CP];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int q = q0 + k * NT;
                if (q >= total) continue;
                const int rr = div_small(q, rcp_sc), v = q - rr * SC;
                const int sa = div_small(rr, rcp_sr), r = rr - sa * SR;
                const int gu = gu0 + r, gv = gv0 + v;
                const bool ok = interior || (gu >= 0 && gu < grows && gv >= 0 && gv < gcols);
                const int go = sa * gsub + gu * gcols + gv;
#pragma unroll
                for (int w = 0; w < CP; ++w) val[k][w] = 0;
                if (ok) {
                    if (src_x) Vec<T, CP>::ld(src_x + go * CP, val[k]);
                    else val[k][0] = src_y[go];
                }
            }
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int q = q0 + k * NT;
                if (q >= total) continue;
                if (src_x) Vec<T, CP>::st(xs + q * CP, val[k]);
                else ys[q] = val[k][0];
            }
        }
    };

    // Phase A: normals of every staged site for sweep `sweep` (those outside the drawn regions
    // are unused).
    auto normals = [&](uint32_t sweep) {
        if (CP == 4) {
            for (int q = threadIdx.x; q < NS * SUB; q += NT) {
                const int rr = div_small(q, rcp_sc), v = q - rr * SC;
                const int sa = div_small(rr, rcp_sr), r = rr - sa * SR;
                const int i = E8 ? gi0 + 2 * r + (sa >> 1) : gi0 + r;
                const int j = E8 ? gj0 + 2 * v + (sa & 1) : gj0 + 2 * v + ((sa + i) & 1);
                if (!interior && (i < 0 || i >= Hl || j < 0 || j >= Wl)) continue;
                T z[CP];
                site_normals<T, CP>(a.key, static_cast<uint32_t>(i * Wl + j), sweep, f.stream, 0u, 4, z);
                Vec<T, CP>::st(zs + q * CP, z);
            }
        } else {
            // Groups of G = 4 / CP consecutive natural sites share a Philox block.
            constexpr int GS = (CP == 2) ? 1 : 2, G = 1 << GS;
            const int NG = (RC >> GS) + 2;
            const float rcp_ng = __frcp_rn(static_cast<float>(NG));
            const int jl = max(0, gj0), jh = min(Wl, gj0 + RC);
            for (int q = threadIdx.x; q < RR * NG; q += NT) {
                const int ri = div_small(q, rcp_ng), k = q - ri * NG;
                const int i = gi0 + ri;
                if (i < 0 || i >= Hl || jl >= jh) continue;
                const int s0 = i * Wl + jl, s1 = i * Wl + jh;
                const int g = (s0 >> GS) + k;
                if ((g << GS) >= s1) continue;
                T n4[4];
                block_normals<T>(a.key, static_cast<uint32_t>(g), sweep, f.stream, 0u, n4);
#pragma unroll
                for (int r = 0; r < G; ++r) {
                    const int st = (g << GS) + r;
                    if (st < s0 || st >= s1) continue;
                    const int j = st - i * Wl;
                    T *zp = zs + sm_index<KIND>(i, j, gi0, gj0, SR, SC) * CP;
#pragma unroll
                    for (int ch = 0; ch < CP; ++ch) zp[ch] = n4[r * CP + ch];
                }
            }
        }
    };

    // Before the dependency wait: the observations (never written by a sweep) and, when this is
    // the sweep's only sweep kernel (a.early), the normals of the predicted sweep number, as in
    // lattice_quad.cu (the last block to read the prediction replaces it after the wait; a wrong
    // prediction only costs drawing the normals again).
    stage(nullptr, Y);
    __shared__ long long s_pred;
    __shared__ int s_last;
    long long predicted = -1;
    if (a.early) {
        if (threadIdx.x == 0) {
            s_pred = *reinterpret_cast<volatile const long long *>(&a.ctl->fnext);
            s_last = atomicAdd(&a.ctl->fticket, 1ull) == gridDim.x - 1;
        }
        __syncthreads();
        predicted = s_pred;
        normals(static_cast<uint32_t>(predicted));
    }
    pdl_wait();
    const long long sweep_ll = a.ctl->sweep;
    if (a.early && threadIdx.x == 0 && s_last) {
        a.ctl->fnext = sweep_ll + 1;
        a.ctl->fticket = 0;
        if (sweep_ll != predicted) a.ctl->fmiss += 1;
    }
    pdl_release();
    const uint32_t sweep = static_cast<uint32_t>(sweep_ll);
    if (!a.early || sweep_ll != predicted) normals(sweep);
    const T *X = static_cast<const T *>((sweep_ll & 1) ? a.x_alt : a.x) + f.slot0 * CP;
    T *XW = static_cast<T *>((sweep_ll & 1) ? a.x : a.x_alt) + f.slot0 * CP;
    T tau[CP], isig[CP], beta[CP];
    {
        const T *hyp = static_cast<const T *>(a.hyp) + static_cast<int64_t>(t.field) * CP * kHypStride;
#pragma unroll
        for (int v = 0; v < CP; ++v) {
            tau[v] = hyp[kHypStride * v];
            isig[v] = hyp[kHypStride * v + 1];
            beta[v] = hyp[kHypStride * v + 2];
        }
    }
    stage(X, nullptr);
    __syncthreads();

    // Phase B: colour steps.  An owned site is final after its own colour step: it is written
    // back then (state and, on accumulated sweeps, the running mean / M2), so the stores overlap
    // the remaining steps, and it folds its terms of the hyperparameter sums.
    const bool acc = a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin);
    T inv_k = 0;
    if (acc) inv_k = static_cast<T>(1) / static_cast<T>(a.ctl->acc_count + 1);
    T *MEAN = static_cast<T *>(a.mean) + f.slot0 * CP;
    T *M2 = static_cast<T *>(a.m2) + f.slot0 * CP;
    T accS[CP], accR[CP], accA[CP];
#pragma unroll
    for (int v = 0; v < CP; ++v) {
        accS[v] = 0;
        accR[v] = 0;
        accA[v] = 0;
    }
    // One colour step per colour, the colour a compile-time constant (the lower-colour
    // directions, whose edge terms enter the prior sum, are then known per direction).
    auto colour_step = [&](auto colour) {
        constexpr int c = decltype(colour)::value;
        const int e = K - 1 - c;
        const int lo_i = max(0, t.i0 - e), hi_i = min(Hl, t.i0 + TR + e);
        const int lo_j = max(0, t.j0 - e), hi_j = min(Wl, t.j0 + TC + e);
        // Fixed neighbour offsets (shared-memory index units) and 0/1 weights of the
        // lower-colour directions for this colour.
        int off[ND];
        T wl[ND];
        bool lw[ND];  // lower-colour direction (its weight in wl is 1)
        if (E8) {
            const int ca = c >> 1, cb = c & 1;
#pragma unroll
            for (int k = 0; k < ND; ++k) {
                const int ai = ca + D::di(k), bj = cb + D::dj(k);
                const int cc = 2 * (ai & 1) + (bj & 1);
                off[k] = ((cc - c) * SR + (ai >> 1)) * SC + (bj >> 1);
                wl[k] = cc < c ? static_cast<T>(1) : static_cast<T>(0);
                lw[k] = cc < c;
            }
        } else {
            const int o = (1 - 2 * c) * SR * SC;
            off[0] = o - SC;
            off[1] = o - 1;  // + p, added per row
            off[2] = o;      // + p
            off[3] = o + SC;
#pragma unroll
            for (int k = 0; k < ND; ++k) {
                wl[k] = static_cast<T>(c);
                lw[k] = c != 0;
            }
        }
        int n_rows, n_cols, first_u = 0, first_v = 0;
        if (E8) {
            const int ca = c >> 1, cb = c & 1;
            first_u = (lo_i - gi0 - ca + 1) >> 1;
            first_v = (lo_j - gj0 - cb + 1) >> 1;
            n_rows = ((hi_i - gi0 - ca + 1) >> 1) - first_u;
            n_cols = ((hi_j - gj0 - cb + 1) >> 1) - first_v;
        } else {
            n_rows = hi_i - lo_i;
            n_cols = (hi_j - lo_j + 1) >> 1;
        }
        if (n_rows > 0 && n_cols > 0) {
            const float rcp_nc = __frcp_rn(static_cast<float>(n_cols));
            for (int q = threadIdx.x; q < n_rows * n_cols; q += NT) {
                const int ru = div_small(q, rcp_nc), w = q - ru * n_cols;
                int i, j, idx, sr, sv, dp = 0;
                if (E8) {
                    sr = first_u + ru;
                    sv = first_v + w;
                    i = gi0 + 2 * sr + (c >> 1);
                    j = gj0 + 2 * sv + (c & 1);
                } else {
                    i = lo_i + ru;
                    const int p = (c + i) & 1;
                    sr = i - gi0;
                    sv = ((lo_j - gj0 - p + 1) >> 1) + w;
                    j = gj0 + 2 * sv + p;
                    if (j >= hi_j) continue;
                    dp = p;
                }
                idx = (c * SR + sr) * SC + sv;
                const bool owned = i >= t.i0 && i < t.i0 + TR && j >= t.j0 && j < t.j0 + TC;
                const int go = (c * gsub + (gu0 + sr) * gcols + gv0 + sv) * CP;
                T mu[CP], mm[CP];
                if (owned && acc) {
                    Vec<T, CP>::ld(MEAN + go, mu);
                    Vec<T, CP>::ld(M2 + go, mm);
                }
                T nb[ND][CP], s[CP];
#pragma unroll
                for (int v = 0; v < CP; ++v) s[v] = 0;
#pragma unroll
                for (int k = 0; k < ND; ++k) {
                    const int o = off[k] + ((!E8 && (k == 1 || k == 2)) ? dp : 0);
                    Vec<T, CP>::ld(xs + (idx + o) * CP, nb[k]);
#pragma unroll
                    for (int v = 0; v < CP; ++v) s[v] += nb[k][v];
                }
                T d = static_cast<T>(ND);
                T wv[ND];
#pragma unroll
                for (int k = 0; k < ND; ++k) wv[k] = wl[k];
                if (!interior && (i == 0 || j == 0 || i == Hl - 1 || j == Wl - 1)) {
                    // Edge site: missing neighbours hold zero (the sum is right) but must not
                    // count in the degree or the prior sum.
                    int deg = 0;
#pragma unroll
                    for (int k = 0; k < ND; ++k) {
                        const int ii = i + D::di(k), jj = j + D::dj(k);
                        const bool ok = ii >= 0 && ii < Hl && jj >= 0 && jj < Wl;
                        deg += ok;
                        if (!ok) wv[k] = 0;
                    }
                    d = static_cast<T>(deg);
                }
                T z[CP];
                Vec<T, CP>::ld(zs + idx * CP, z);
                const T yv = ys[idx];
                T xn[CP];
#pragma unroll
                for (int v = 0; v < CP; ++v) {
                    const T P = tau[v] * d + isig[v];
                    const T m = (tau[v] * rho * s[v] + (yv - beta[v]) * isig[v]) * FArith<T>::rcp(P);
                    xn[v] = m + z[v] * FArith<T>::rsq(P);
                }
                Vec<T, CP>::st(xs + idx * CP, xn);
                if (owned) {
                    Vec<T, CP>::st(XW + go, xn);
                    if (acc) {
#pragma unroll
                        for (int v = 0; v < CP; ++v) {
                            const T delta = xn[v] - mu[v];
                            mu[v] += delta * inv_k;
                            mm[v] += delta * (xn[v] - mu[v]);
                        }
                        Vec<T, CP>::st(MEAN + go, mu);
                        Vec<T, CP>::st(M2 + go, mm);
                    }
#pragma unroll
                    for (int v = 0; v < CP; ++v) {
                        T e2 = 0;
#pragma unroll
                        for (int k = 0; k < ND; ++k) {
                            if (lw[k]) {  // the other directions' weights are 0: their terms add +0
                                const T df = xn[v] - nb[k][v];
                                e2 += wv[k] * df * df;
                            }
                        }
                        accS[v] += (static_cast<T>(1) - rho) * d * xn[v] * xn[v] + rho * e2;
                        const T r = (yv - beta[v]) - xn[v];
                        accR[v] += r * r;
                        accA[v] += r;
                    }
                }
            }
        }
        __syncthreads();
    };
    colour_step(std::integral_constant<int, 0>{});
    colour_step(std::integral_constant<int, 1>{});
    if constexpr (K == 4) {
        colour_step(std::integral_constant<int, 2>{});
        colour_step(std::integral_constant<int, 3>{});
    }

    // Block reduction (all lanes hold the same chains): warp shuffle tree, then warps in order.
    T *red = zs;  // [NW][CP][3], the normals are dead
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < CP; ++v) {
        T sS = accS[v], sR = accR[v], sA = accA[v];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            sS += __shfl_xor_sync(0xffffffffu, sS, o);
            sR += __shfl_xor_sync(0xffffffffu, sR, o);
            sA += __shfl_xor_sync(0xffffffffu, sA, o);
        }
        if (lane == 0) {
            red[(warp * CP + v) * 3] = sS;
            red[(warp * CP + v) * 3 + 1] = sR;
            red[(warp * CP + v) * 3 + 2] = sA;
        }
    }
    __syncthreads();
    if (threadIdx.x < CP * 3) {
        const int chain = threadIdx.x / 3, k = threadIdx.x - 3 * chain;
        T sum = 0;
        for (int w = 0; w < NW; ++w) sum += red[(w * CP + chain) * 3 + k];
        reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * CP + chain)[k] = static_cast<double>(sum);
    }
}

template <typename T, int V, int KIND>
cudaError_t launch_t(const FusedArgs &a, size_t smem, cudaStream_t stream)
{
    const bool fast = a.update && a.Cp == V;  // every thread holds all chains
    if (a.threads == 1024) {
        if (fast) return launch_sweep_kernel(lattice_fused_fast<T, KIND, 1024, V>, a.ntiles, 1024, smem, stream, a);
        return launch_sweep_kernel(lattice_fused_kernel<T, V, KIND, 1024>, a.ntiles, 1024, smem, stream, a);
    }
    if (fast) return launch_sweep_kernel(lattice_fused_fast<T, KIND, 512, V>, a.ntiles, 512, smem, stream, a);
    return launch_sweep_kernel(lattice_fused_kernel<T, V, KIND, 512>, a.ntiles, 512, smem, stream, a);
}

template <typename T, int V, int KIND>
cudaError_t prepare_t(size_t smem)
{
    const int b = static_cast<int>(smem);
    cudaError_t e = cudaFuncSetAttribute(lattice_fused_kernel<T, V, KIND, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lattice_fused_kernel<T, V, KIND, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lattice_fused_fast<T, KIND, 512, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lattice_fused_fast<T, KIND, 1024, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

template <int KIND>
cudaError_t dispatch(bool prepare, int precision, int V, const FusedArgs &a, size_t smem, cudaStream_t stream)
{
    if (precision == 0) {
        if (V == 4) return prepare ? prepare_t<float, 4, KIND>(smem) : launch_t<float, 4, KIND>(a, smem, stream);
        if (V == 2) return prepare ? prepare_t<float, 2, KIND>(smem) : launch_t<float, 2, KIND>(a, smem, stream);
        return prepare ? prepare_t<float, 1, KIND>(smem) : launch_t<float, 1, KIND>(a, smem, stream);
    }
    if (V == 2) return prepare ? prepare_t<double, 2, KIND>(smem) : launch_t<double, 2, KIND>(a, smem, stream);
    return prepare ? prepare_t<double, 1, KIND>(smem) : launch_t<double, 1, KIND>(a, smem, stream);
}

}  // namespace

size_t lattice_fused_smem(int precision, int kind, int Cp, int TR, int TC)
{
    const int K = (kind == kLat2D8) ? 4 : 2;
    const size_t S = precision == 0 ? sizeof(float) : sizeof(double);
    return static_cast<size_t>(TR + 2 * K) * (TC + 2 * K) * (2 * Cp + 1) * S;
}

cudaError_t prepare_lattice_fused(int precision, int V, int kind, size_t smem)
{
    FusedArgs dummy{};
    if (kind == kLat2D8) return dispatch<kLat2D8>(true, precision, V, dummy, smem, nullptr);
    return dispatch<kLat2D4>(true, precision, V, dummy, smem, nullptr);
}

cudaError_t launch_lattice_fused(int precision, int V, int kind, const FusedArgs &a, size_t smem, cudaStream_t stream)
{
    if (a.ntiles <= 0) return cudaSuccess;
    if (kind == kLat2D8) return dispatch<kLat2D8>(false, precision, V, a, smem, stream);
    return dispatch<kLat2D4>(false, precision, V, a, smem, stream);
}

}  // namespace gmrf
