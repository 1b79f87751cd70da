// lattice_fused_resident.cu -- the resident form of the fused 2-D lattice sweep (lattice_fused.cu,
// lattice_fused_fast: every thread holding all CP chains of a site) for FP32 samplers of a single
// field whose tiles can all be resident at once: `count` whole sweeps in one cooperative launch,
// each block keeping its staged tile (state, observations, normals) in shared memory from sweep
// to sweep.  Per sweep:
//   * the K colour steps with the arithmetic of lattice_fused_fast (each owned site written to
//     the next sweep's state buffer right after its step, the running mean and M2 updated in
//     global memory on accumulated sweeps; the colour a compile-time constant, so only the
//     lower-colour directions' edge terms are formed);
//   * the block's sums in that kernel's order to its tile partial, then the grid barrier
//     (grid_barrier.cuh); while the other blocks finish, the block draws the normals of its
//     staged sites for the next sweep;
//   * every block draws tau | x and beta0, sigma^2 for every chain (warp 2v + which) from all tile
//     partials, summed in the order of the hyperparameter kernel and drawn by hyper_draw with the
//     batch's precomputed variates, so it holds the values the per-sweep path would have; block 0
//     alone stores them and the traces (with four chains per thread the partials are read from a
//     copy laid out by field, TileResArgs::pm, so a warp's reads are consecutive); meanwhile the
//     other warps stage again, through L2, the ring of staged sites around the tile (its halo),
//     which the neighbouring tiles have just written.
// The results equal the per-sweep path's bit for bit.  The state buffers alternate by sweep
// number as on that path, so one barrier per sweep suffices.
#include <cuda_runtime.h>

#include <type_traits>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "grid_barrier.cuh"
#include "hyper_task.cuh"
#include "lattice_common.cuh"

namespace gmrf {
namespace {

constexpr int kResGpre = 128;  // sweeps whose precomputed variates are staged in shared memory

template <int CP> struct LdCg;
template <> struct LdCg<1> {
    __device__ __forceinline__ static void ld(const float *p, float (&v)[1]) { v[0] = __ldcg(p); }
};
template <> struct LdCg<2> {
    __device__ __forceinline__ static void ld(const float *p, float (&v)[2])
    {
        const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x;
        v[1] = t.y;
    }
};
template <> struct LdCg<4> {
    __device__ __forceinline__ static void ld(const float *p, float (&v)[4])
    {
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
};

template <int KIND, int NT, int CP>
__global__ void __launch_bounds__(NT, (NT == 512 && CP < 4) ? 2 : 1) lattice_fused_resident(const TileResArgs ra)
{
    using T = float;
    using D = Dirs<KIND>;
    constexpr bool E8 = (KIND == kLat2D8);
    constexpr int K = E8 ? 4 : 2;
    constexpr int NS = E8 ? 4 : 2;
    constexpr int NW = NT / 32;
    constexpr int ND = D::N;
    const FusedArgs &a = ra.f;
    const HyperArgs &h = ra.h;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T hs[CP][3];          // tau, 1/sigma^2, beta0 of the current sweep per chain
    __shared__ double dcur[CP][2];   // tau and sigma^2 (FP64) as last drawn, per chain
    __shared__ double gsh[kResGpre][CP][3];
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    SweepCtl *ctl = a.ctl;
    const long long sweep0 = ctl->sweep;
    long long acc_count = ctl->acc_count;
    const long long bbase = ctl->batch_base, bcount = ctl->batch_count;
    const unsigned long long nblk = gridDim.x;

    // Staged index q of the NS sub-arrays -> natural site (i, j).
    auto site_of = [&](int q, int &i, int &j, int &sa, int &r, int &v) {
        const int rr = div_small(q, rcp_sc);
        v = q - rr * SC;
        sa = div_small(rr, rcp_sr);
        r = rr - sa * SR;
        i = E8 ? gi0 + 2 * r + (sa >> 1) : gi0 + r;
        j = E8 ? gj0 + 2 * v + (sa & 1) : gj0 + 2 * v + ((sa + i) & 1);
    };

    // Stage rows of the sub-arrays (four loads in flight per thread), as lattice_fused_fast.
    auto stage = [&](const T *src_x, const T *src_y) {
        constexpr int UNR = 4;
        const int total = NS * SUB;
        for (int q0 = tid; q0 < total; q0 += UNR * NT) {
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

    // Normals of every staged site for sweep `sweep`, as lattice_fused_fast.
    auto normals = [&](uint32_t sweep) {
        if (CP == 4) {
            for (int q = tid; q < NS * SUB; q += NT) {
                int i, j, sa, r, v;
                site_of(q, i, j, sa, r, v);
                if (!interior && (i < 0 || i >= Hl || j < 0 || j >= Wl)) continue;
                T z[CP];
                site_normals<T, CP>(a.key, static_cast<uint32_t>(i * Wl + j), sweep, f.stream, 0u, 4, z);
                Vec<T, CP>::st(zs + q * CP, z);
            }
        } else {
            constexpr int GS = (CP == 2) ? 1 : 2, G = 1 << GS;
            const int NG = (RC >> GS) + 2;
            const float rcp_ng = __frcp_rn(static_cast<float>(NG));
            const int jl = max(0, gj0), jh = min(Wl, gj0 + RC);
            for (int q = tid; q < RR * NG; q += NT) {
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

    stage(nullptr, Y);
    stage(static_cast<const T *>((sweep0 & 1) ? a.x_alt : a.x) + f.slot0 * CP, nullptr);
    if (tid < CP * 3) {
        const int v = tid / 3, k = tid - 3 * v;
        hs[v][k] = static_cast<const T *>(a.hyp)[(static_cast<int64_t>(t.field) * CP + v) * kHypStride + k];
    }
    if (tid < CP) {
        dcur[tid][0] = h.tau[tid];
        dcur[tid][1] = h.sig2[tid];
    }
    if (tid == 0) s_abort = 0;
    for (int q = tid; q < min(ra.count, kResGpre) * CP * 3; q += NT) {
        const int it = q / (CP * 3), rem = q - it * CP * 3, v = rem / 3, k = rem - 3 * v;
        const long long kb = sweep0 + it - bbase;
        gsh[it][v][k] = (h.gpre && kb >= 0 && kb < bcount) ? h.gpre[(kb * h.nfields * h.Cp + v) * 4 + k] : 0.0;
    }
    normals(static_cast<uint32_t>(sweep0));
    T *MEAN = static_cast<T *>(a.mean) + f.slot0 * CP;
    T *M2 = static_cast<T *>(a.m2) + f.slot0 * CP;

    for (int it = 0; it < ra.count; ++it) {
        const long long sw = sweep0 + it;
        __syncthreads();  // staged state (halo), normals and the sweep's parameters
        T tau[CP], isig[CP], beta[CP];
#pragma unroll
        for (int v = 0; v < CP; ++v) {
            tau[v] = hs[v][0];
            isig[v] = hs[v][1];
            beta[v] = hs[v][2];
        }
        T *XW = static_cast<T *>((sw & 1) ? a.x : a.x_alt) + f.slot0 * CP;
        const bool acc = a.acc_enabled && sweep_accumulated(sw, a.burn_in, a.thin);
        T inv_k = 0;
        if (acc) inv_k = static_cast<T>(1) / static_cast<T>(acc_count + 1);
        T accS[CP], accR[CP], accA[CP];
#pragma unroll
        for (int v = 0; v < CP; ++v) {
            accS[v] = 0;
            accR[v] = 0;
            accA[v] = 0;
        }
        // The colour steps of lattice_fused_fast, the colour a compile-time constant.
        auto colour_step = [&](auto colour) {
            constexpr int c = decltype(colour)::value;
            const int e = K - 1 - c;
            const int lo_i = max(0, t.i0 - e), hi_i = min(Hl, t.i0 + TR + e);
            const int lo_j = max(0, t.j0 - e), hi_j = min(Wl, t.j0 + TC + e);
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
                for (int q = tid; q < n_rows * n_cols; q += NT) {
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
        if (acc) ++acc_count;

        // The tile's sums, in lattice_fused_fast's order (its reduction scratch is the normals').
        T *red = zs;
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
        if (tid < CP * 3) {
            const int chain = tid / 3, k = tid - 3 * chain;
            T sum = 0;
            for (int w = 0; w < NW; ++w) sum += red[(w * CP + chain) * 3 + k];
            reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * CP + chain)[k] = static_cast<double>(sum);
            if (CP == 4) ra.pm[(chain * 3 + k) * f.nparts + (t.part - f.part0)] = static_cast<double>(sum);
        }
        __syncthreads();  // the partial and every owned site of the sweep are stored; `red` is free

        // Grid barrier: arrive, draw the next sweep's normals, then wait (bounded).
        if (tid == 0) grid_arrive(ctl);
        if (it + 1 < ra.count) normals(static_cast<uint32_t>(sw + 1));
        if (tid == 0) {
            const unsigned long long target = (static_cast<unsigned long long>(it) + 1) * nblk + ra.extra_arrivals;
            if (grid_wait(ctl, target, ra.wait_ns)) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;

        if (warp >= 2 * CP) {
            // The halo for the next sweep (its state buffer is XW), through L2: the K rows above
            // and below the tile (RC sites each), then the K columns left and right of its rows.
            const int HB = 2 * K * RC, HN = HB + 2 * K * TR;
            const float rcp_rc = __frcp_rn(static_cast<float>(RC));
            for (int q = tid - 64 * CP; q < HN; q += NT - 64 * CP) {
                int i, j;
                if (q < HB) {
                    const int b = div_small(q, rcp_rc);
                    i = gi0 + (b < K ? b : TR + b);
                    j = gj0 + (q - b * RC);
                } else {
                    const int r2 = static_cast<int>(static_cast<unsigned>(q - HB) / (2u * K)), k = q - HB - r2 * (2 * K);
                    i = t.i0 + r2;
                    j = gj0 + (k < K ? k : TC + k);
                }
                if (!interior && (i < 0 || i >= Hl || j < 0 || j >= Wl)) continue;  // stays 0
                const int sa = E8 ? 2 * (i & 1) + (j & 1) : ((i + j) & 1);
                const int r = E8 ? (i - gi0) >> 1 : i - gi0, v = (j - gj0) >> 1;
                T val[CP];
                LdCg<CP>::ld(XW + (sa * gsub + (gu0 + r) * gcols + gv0 + v) * CP, val);
                Vec<T, CP>::st(xs + ((sa * SR + r) * SC + v) * CP, val);
            }
        } else {
            // The conjugate draws at the end of sweep sw: warp 2 v draws tau of chain v, warp
            // 2 v + 1 beta0 and then sigma^2 of chain v.
            const int chain = warp >> 1, which = warp & 1;
            const bool need_sum = which ? (h.draw || h.draw_beta) : h.draw;
            const bool need_a = which && h.draw_beta;
            double S = 0.0, A = 0.0;
            if (need_sum) {
                // four chains per thread: from the copy by field (measured 16.1 -> 14.1 us per
                // sweep of the 512 x 512 image with the intercept; with one or two chains the
                // records' reads measured faster)
                if (CP == 4) {
                    const double *pc = ra.pm + chain * 3 * f.nparts;
                    hyper_sums_by_field(pc + which * f.nparts, pc + 2 * f.nparts, need_a, f.nparts, S, A);
                } else if (h.max_parts >= 256) {
                    hyper_sums<true, true>(h, which, need_a, chain, f.part0, f.nparts, S, A);
                } else {
                    hyper_sums<false, true>(h, which, need_a, chain, f.part0, f.nparts, S, A);
                }
            }
            if (lane == 0) {
                const long long kb = sw - bbase;
                const bool pre = h.gpre && kb >= 0 && kb < bcount;
                double gpv = 0.0, zb = 0.0;
                if (pre) {
                    if (it < kResGpre) {
                        gpv = gsh[it][chain][which];
                        zb = gsh[it][chain][2];
                    } else {
                        const double *gp = h.gpre + (kb * h.nfields * h.Cp + chain) * 4;
                        gpv = gp[which];
                        zb = gp[2];
                    }
                }
                // (the tau draw reads neither sigma^2 nor beta0, which the other warp replaces)
                const double cur = dcur[chain][which], s2old = which ? dcur[chain][1] : 0.0;
                const double b = which ? static_cast<double>(hs[chain][2]) : 0.0;
                double val, bval;
                hyper_draw<float>(h, which, chain, chain, sw, S, A, cur, s2old, b, gpv, zb, pre, 0, f.stream, f.n,
                                  f.rank, val, bval, blockIdx.x == 0);
                if (which == 0) {
                    if (h.draw) hs[chain][0] = static_cast<T>(val);
                } else {
                    if (h.draw_beta) hs[chain][2] = static_cast<T>(bval);
                    if (h.draw) hs[chain][1] = static_cast<T>(1.0 / val);
                }
                dcur[chain][which] = val;
            }
        }
    }

    // The last block to finish advances the counters and clears the barrier for the next launch.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ctl->ticket, 1ull) == nblk - 1) {
            ctl->sweep = sweep0 + ra.count;
            ctl->fnext = sweep0 + ra.count;
            ctl->acc_count = acc_count;
            ctl->ticket = 0;
            ctl->gbar = 0;
            ctl->gabort = 0;
        }
    }
}

#define GMRF_FR_CONFIGS(X) \
    X(kLat2D8, 512, 1) X(kLat2D8, 512, 2) X(kLat2D8, 512, 4) X(kLat2D8, 1024, 1) X(kLat2D8, 1024, 2) \
    X(kLat2D8, 1024, 4) X(kLat2D4, 512, 1) X(kLat2D4, 512, 2) X(kLat2D4, 512, 4) X(kLat2D4, 1024, 1) \
    X(kLat2D4, 1024, 2) X(kLat2D4, 1024, 4)

}  // namespace

cudaError_t lattice_fused_resident_fits(int kind, int threads, int Cp, size_t smem, int ntiles, bool *fits)
{
    *fits = false;
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return e;
#define GMRF_FR_FITS(KD, N, C)                                                                                  \
    if (kind == KD && threads == N && Cp == C) {                                                              \
        e = cudaFuncSetAttribute(lattice_fused_resident<KD, N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 static_cast<int>(smem));                                                     \
        if (e == cudaSuccess)                                                                                 \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lattice_fused_resident<KD, N, C>, N, smem); \
        if (e != cudaSuccess) {                                                                               \
            cudaGetLastError();                                                                               \
            return cudaSuccess; /* the shared memory does not fit: not resident */                            \
        }                                                                                                     \
        *fits = coop != 0 && static_cast<int64_t>(per_sm) * sms >= ntiles;                                   \
        return cudaSuccess;                                                                                   \
    }
    GMRF_FR_CONFIGS(GMRF_FR_FITS)
#undef GMRF_FR_FITS
    return cudaSuccess;
}

cudaError_t launch_lattice_fused_resident(int kind, int threads, int Cp, const TileResArgs &ra, size_t smem,
                                          cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ra.f.ntiles);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define GMRF_FR_LAUNCH(KD, N, C) \
    if (kind == KD && threads == N && Cp == C) return cudaLaunchKernelEx(&cfg, lattice_fused_resident<KD, N, C>, ra);
    GMRF_FR_CONFIGS(GMRF_FR_LAUNCH)
#undef GMRF_FR_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace gmrf
