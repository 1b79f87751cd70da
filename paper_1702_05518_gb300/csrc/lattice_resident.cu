// lattice_resident.cu -- many whole sweeps of a small 2-D lattice field in one launch, one block
// per chain.
//
// A field of a few thousand sites (the 50 x 50 and 64 x 64 images of Sec. 3.1) fills a few SMs at
// most, so the time per sweep of the per-sweep path is the length of its dependency chain: one
// launch per sweep, the partial sums through global memory, and the conjugate draws' FP64
// arithmetic (whose dependent operations are slow on this GPU).  Here one block holds a whole
// chain in shared memory -- state, observations, running mean and M2, each in the colour-split
// layout of the global arrays with a ring of zeros around every sub-array -- and runs `count`
// sweeps of Algorithm 1 back to back:
//   * colour step c: every thread draws its positions of colour class c (the normals of
//     (site, sweep, chain) come from the same counters as on the per-sweep path), then a block
//     barrier; the sites of one class are conditionally independent given the others (Sec. 2.3),
//     so the step needs no other ordering;
//   * the two sums of the conditionals of tau and sigma^2 (and the residual sum of the intercept)
//     are folded in during the steps, as in the fused kernel: (1 - rho) d x^2 + rho times the
//     squared differences to lower-colour neighbours, and e^2 and e with e = y - beta0 - x;
//   * after the last step a shuffle tree per warp, one barrier, and two warps finish the sums in
//     FP64 and draw tau and (beta0, then sigma^2) in parallel (the conditionals of Sec. 3.1, from
//     the batch's precomputed unit-rate variates), with the formulas of the per-sweep path;
//   * a barrier publishes the new values to the next sweep.
// A sweep thus costs K + 1 barriers (K - 1 of the site threads alone) and no launch.  State and accumulators go back to
// global memory at the end of the launch (into the buffer the per-sweep path reads next), and the
// last block to finish advances the sweep and accumulation counters.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "gamma_pre.cuh"
#include "lattice_common.cuh"
#include "resident_draws.cuh"

namespace gmrf {
namespace {

// Threads per block: up to 640 site threads with one position per class (80 registers each), or
// 576 with two or four (96 registers), and the two drawing warps.
constexpr int kResMaxThreads = 704;
template <int NI> constexpr int res_threads() { return NI == 1 ? 704 : 640; }

// Per position of a thread, in shared memory ([colour][k][site thread]): x = shared index |
// natural site << 16; y = degree (bits 0-3), lower-colour in-lattice neighbours (bits 4-11),
// column parity (bit 12), in use (bit 31).
constexpr uint32_t kItemUsed = 1u << 31;

template <typename T, int KIND, int NI>
__global__ void __launch_bounds__(res_threads<NI>(), 1) lattice_resident_kernel(const ResidentArgs a)
{
    using D = Dirs<KIND>;
    constexpr bool E8 = (KIND == kLat2D8);
    constexpr int K = E8 ? 4 : 2;  // colours = sub-arrays
    constexpr int ND = D::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[kResMaxThreads / 32][3];
    __shared__ T hs[3];  // tau, 1/sigma^2, beta0 of the current sweep, precision T

    // Everything up to the first normals depends only on the previous batch's kernel (complete
    // before this launch's predecessor, the batch's normals, let this one start), so the chain is
    // staged while the normals are still being drawn; pdl_wait comes before their first use.
    const HyperArgs &h = a.h;
    const int chain = blockIdx.x, NT = blockDim.x, tid = threadIdx.x;
    const int NTS = NT - 64;  // site threads; the last two warps draw the hyperparameters
    const int lane = tid & 31, warp = tid >> 5, nsw = NTS >> 5;
    const bool drawer = tid >= NTS;
    const int dw = warp - nsw;  // drawing warp: 0 tau, 1 beta0 and sigma^2
    const FieldDev f = a.fields[0];
    const int Hl = f.dims[0], Wl = f.dims[1];
    const int SR = a.SR, SC = a.SC, SUB = SR * SC, cells = K * SUB;
    const int grows = f.rows, gcols = f.cols;
    const int Cp = h.Cp;
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *ys = xs + cells;
    T *ms = ys + cells;
    T *m2s = ms + cells;
    uint2 *meta = reinterpret_cast<uint2 *>(m2s + cells);  // [K][NI][NTS]; 8-byte aligned (4 cells arrays)

    const long long sweep0 = h.ctl->sweep;
    long long acc = h.ctl->acc_count;
    if (tid < 3) hs[tid] = static_cast<const T *>(h.hyp)[static_cast<int64_t>(chain) * kHypStride + tid];
    // The drawing lanes' state lives in shared memory (no thread keeps registers for it).
    __shared__ ResidentDraws<T> drs[2];
    ResidentDraws<T> &dr = drs[drawer ? dw : 0];
    if (drawer && lane == 0) dr.init(h, dw, chain, f);

    // Stage the chain: every cell of every sub-array, the ring and padding as zeros.
    {
        const T *X = static_cast<const T *>((sweep0 & 1) ? a.x_alt : a.x) + f.slot0 * Cp + chain;
        const T *Y = static_cast<const T *>(a.y) + f.slot0;
        const T *MEAN = static_cast<const T *>(a.mean) + f.slot0 * Cp + chain;
        const T *M2 = static_cast<const T *>(a.m2) + f.slot0 * Cp + chain;
        for (int q = tid; q < cells; q += NT) {
            const int s = q / SUB, r = q - s * SUB, u = r / SC, v = r - u * SC;
            T xv = 0, yv = 0, mv = 0, m2v = 0;
            if (u >= 1 && u <= grows && v >= 1 && v <= gcols) {
                const int64_t g = static_cast<int64_t>(s * grows + u - 1) * gcols + (v - 1);
                xv = X[g * Cp];
                yv = Y[g];
                mv = MEAN[g * Cp];
                m2v = M2[g * Cp];
            }
            xs[q] = xv;
            ys[q] = yv;
            ms[q] = mv;
            m2s[q] = m2v;
        }
    }

    // A site thread's positions: NI of every colour class, fixed for the launch.
    if (!drawer) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                const int q = tid + k * NTS;
                int i, j, idx;
                bool ok;
                if (E8) {
                    const int ca = c >> 1, cb = c & 1;
                    const int cols_c = (Wl - cb + 1) >> 1, rows_c = (Hl - ca + 1) >> 1;
                    const int u = cols_c > 0 ? q / cols_c : 0, v = q - u * cols_c;
                    i = 2 * u + ca;
                    j = 2 * v + cb;
                    ok = cols_c > 0 && u < rows_c;
                    idx = (c * SR + u + 1) * SC + v + 1;
                } else {
                    const int u = q / gcols, v = q - u * gcols;
                    i = u;
                    j = 2 * v + ((c + i) & 1);
                    ok = u < Hl && j < Wl;
                    idx = (c * SR + i + 1) * SC + v + 1;
                }
                uint2 m = make_uint2(0u, 0u);
                if (ok) {
                    uint32_t valid = 0, lower = 0;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const int ii = i + D::di(d), jj = j + D::dj(d);
                        if (ii < 0 || ii >= Hl || jj < 0 || jj >= Wl) continue;
                        valid |= 1u << d;
                        if (D::colour(ii, jj) < c) lower |= 1u << d;
                    }
                    m.x = static_cast<uint32_t>(idx) | (static_cast<uint32_t>(i * Wl + j) << 16);
                    m.y = kItemUsed | static_cast<uint32_t>(__popc(valid)) | (lower << 4) |
                          (static_cast<uint32_t>(j & 1) << 12);
                }
                meta[(c * NI + k) * NTS + tid] = m;
            }
        }
    }

    // This sweep's normals of the thread's positions, from the batch buffer that
    // resident_normals_kernel filled (the same counters as the per-sweep path); the next sweep's
    // are loaded one sweep ahead, so their latency hides behind a whole sweep.
    const int64_t zstride = static_cast<int64_t>(a.C) * K * NI * NTS;  // per sweep
    const T *ZB = static_cast<const T *>(a.zbuf) + static_cast<int64_t>(chain) * K * NI * NTS + tid;
    T z[K][NI], zn[K][NI];
    pdl_wait();  // the batch's normals and Gamma variates
    const long long bbase = h.ctl->batch_base, bcount = h.ctl->batch_count;
    __syncthreads();
    if (!drawer) {
#pragma unroll
        for (int c = 0; c < K; ++c)
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                z[c][k] = ZB[(c * NI + k) * NTS];
                zn[c][k] = 0;
            }
    }

    const T rho = static_cast<T>(a.rho);
    const bool acc_on = h.acc_enabled != 0;
    // Position in the accumulation schedule and in the trace ring, advanced sweep by sweep.
    int thin_phase = sweep0 >= h.burn_in ? static_cast<int>((sweep0 - h.burn_in) % h.thin) : 0;
    long long slot = h.trace_cap > 0 ? sweep0 % h.trace_cap : 0;
    for (int t = 0; t < a.count; ++t) {
        const long long sw = sweep0 + t;
        const bool more = t + 1 < a.count;
        if (!drawer && more) {
#pragma unroll
            for (int c = 0; c < K; ++c)
#pragma unroll
                for (int k = 0; k < NI; ++k) zn[c][k] = ZB[(t + 1) * zstride + (c * NI + k) * NTS];
        }
        // Drawing lanes: the record of the last sweep's draws (FP32 state), then what this sweep's
        // draws need that does not depend on its state, while the site threads run the colour steps.
        if (drawer && lane == 0) dr.prep(h, sw, slot, t > 0, bbase, bcount, Cp);
        const T tau = hs[0], isig = hs[1], beta = hs[2];
        const bool acc_now = acc_on && sw >= h.burn_in && thin_phase == 0;
        const T inv_k = acc_now ? static_cast<T>(1) / static_cast<T>(acc + 1) : static_cast<T>(0);
        T accS = 0, accR = 0, accA = 0;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (!drawer) {
                // Neighbour offsets of colour-c cells (8-neighbour: fixed per colour; 4-neighbour:
                // the in-row ones depend on the column parity).
                int off[ND];
                if (E8) {
                    const int ca = c >> 1, cb = c & 1;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const int ai = ca + D::di(d), bj = cb + D::dj(d);
                        const int cc = 2 * (ai & 1) + (bj & 1);
                        off[d] = ((cc - c) * SR + (ai >> 1)) * SC + (bj >> 1);
                    }
                }
#pragma unroll
                for (int k = 0; k < NI; ++k) {
                    const uint2 m = meta[(c * NI + k) * NTS + tid];
                    if (!(m.y & kItemUsed)) continue;
                    const int idx = static_cast<int>(m.x & 0xffffu);
                    if (!E8) {
                        const int p = static_cast<int>((m.y >> 12) & 1u), o = (1 - 2 * c) * SUB;
                        off[0] = o - SC;
                        off[1] = o - 1 + p;
                        off[2] = o + p;
                        off[3] = o + SC;
                    }
                    T nb[ND], s = 0;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        nb[d] = xs[idx + off[d]];
                        s += nb[d];
                    }
                    const T dg = static_cast<T>(m.y & 0xfu);
                    const T yv = ys[idx];
                    const T P = tau * dg + isig;
                    const T mn = (tau * rho * s + (yv - beta) * isig) * FArith<T>::rcp(P);
                    const T xn = mn + z[c][k] * FArith<T>::rsq(P);
                    xs[idx] = xn;
                    const uint32_t lv = (m.y >> 4) & 0xffu;
                    T e = 0;
#pragma unroll
                    for (int d = 0; d < ND; ++d)
                        if ((lv >> d) & 1u) {
                            const T df = xn - nb[d];
                            e += df * df;
                        }
                    accS += (static_cast<T>(1) - rho) * dg * xn * xn + rho * e;
                    const T r = (yv - beta) - xn;
                    accR += r * r;
                    accA += r;
                    // The site's running mean and M2 (Welford) when the sweep is accumulated.
                    if (acc_now) {
                        T mu = ms[idx], mm = m2s[idx];
                        const T delta = xn - mu;
                        mu += delta * inv_k;
                        mm += delta * (xn - mu);
                        ms[idx] = mu;
                        m2s[idx] = mm;
                    }
                }
            }
            // Between colour steps only the site threads meet (named barrier 1), so the drawing
            // lanes' FP64 work delays no step.
            if (c + 1 < K && !drawer) asm volatile("bar.sync 1, %0;" ::"r"(NTS) : "memory");
        }
        // The sums: a shuffle tree per site warp, then over the site warps, in precision T (as a
        // tile's sum in the fused kernel).
        if (!drawer) {
            for (int o = 16; o >= 1; o >>= 1) {
                accS += __shfl_xor_sync(0xffffffffu, accS, o);
                accR += __shfl_xor_sync(0xffffffffu, accR, o);
                accA += __shfl_xor_sync(0xffffffffu, accA, o);
            }
            if (lane == 0) {
                red[warp][0] = accS;
                red[warp][1] = accR;
                red[warp][2] = accA;
            }
        }
        __syncthreads();
        if (drawer) {
            // Warp 0: tau | x.  Warp 1: beta0 | x, sigma^2 (with the intercept), then sigma^2 | x,
            // beta0 (Sec. 3.1).
            T v0 = lane < nsw ? red[lane][dw] : static_cast<T>(0);
            T v1 = (dw == 1 && lane < nsw) ? red[lane][2] : static_cast<T>(0);
            for (int o = 16; o >= 1; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            }
            if (lane == 0) dr.draw(h, v0, v1, beta, hs);
        }
        if (!drawer && more) {
#pragma unroll
            for (int c = 0; c < K; ++c)
#pragma unroll
                for (int k = 0; k < NI; ++k) z[c][k] = zn[c][k];
        }
        if (acc_now) ++acc;
        if (sw >= h.burn_in) thin_phase = (thin_phase + 1 == h.thin) ? 0 : thin_phase + 1;
        if (h.trace_cap > 0) slot = (slot + 1 == h.trace_cap) ? 0 : slot + 1;
        __syncthreads();
    }
    if (drawer && lane == 0 && a.count > 0) dr.finish(h);
    pdl_release();

    // State and accumulators back to global memory; the state into the buffer that holds the
    // state at the start of the next sweep.
    {
        T *X = static_cast<T *>(((sweep0 + a.count) & 1) ? a.x_alt : a.x) + f.slot0 * Cp + chain;
        T *MEAN = static_cast<T *>(a.mean) + f.slot0 * Cp + chain;
        T *M2 = static_cast<T *>(a.m2) + f.slot0 * Cp + chain;
        for (int q = tid; q < cells; q += NT) {
            const int s = q / SUB, r = q - s * SUB, u = r / SC, v = r - u * SC;
            if (u >= 1 && u <= grows && v >= 1 && v <= gcols) {
                const int64_t g = static_cast<int64_t>(s * grows + u - 1) * gcols + (v - 1);
                X[g * Cp] = xs[q];
                MEAN[g * Cp] = ms[q];
                M2[g * Cp] = m2s[q];
            }
        }
    }
    // The last block to finish advances the counters (every block read them at its start).
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&h.ctl->ticket, 1ull) == gridDim.x - 1) {
            h.ctl->sweep = sweep0 + a.count;
            h.ctl->acc_count = acc;
            h.ctl->ticket = 0;
        }
    }
}

// The normals of a batch of `count` sweeps for the resident kernels: lattices in the lattice
// kernel's per-thread order [sweep][chain][colour][k][site thread], graphs by permuted position
// [sweep][chain][position]; one thread per Philox block (a group of G = 4 / lanes
// sites and a quadruple of chains, as in site_normals), whose four normals go to the positions of
// their (site, chain) pairs.  Position q of colour class c belongs to site thread q mod NTS, slot
// q / NTS; the class positions are those of lattice_resident_kernel.  The first gamma_blocks
// blocks instead draw the batch's Gamma variates (gamma_pre.cuh) with 64 threads each, so those
// long FP64 draws spread over as many SMs and run beside the normals.
template <typename T>
__global__ void resident_normals_kernel(const ResNormArgs a)
{
    pdl_wait_then_release();
    if (static_cast<int>(blockIdx.x) < a.gamma_blocks) {
        const long long gbase = a.ctl->sweep;
        const int total = gamma_pre_tasks(a.g);
        if (threadIdx.x < 64)
            for (int q = blockIdx.x * 64 + threadIdx.x; q < total; q += a.gamma_blocks * 64) gamma_pre_task(a.g, q, gbase);
        if (blockIdx.x == 0 && threadIdx.x == 0) gamma_pre_record(a.g, gbase);
        return;
    }
    const int bid = blockIdx.x - a.gamma_blocks, nblk = gridDim.x - a.gamma_blocks;
    const FieldDev f = a.fields[0];
    const int Wl = f.dims[1], n = f.n;
    const bool e8 = f.kind == kLat2D8;
    const int K = e8 ? 4 : 2;
    const long long base = a.ctl->sweep;
    const int gs = lanes_shift(a.lanes), L = a.lanes;
    const int64_t ngroups = (static_cast<int64_t>(n) + (1 << gs) - 1) >> gs;
    const int nquads = a.lanes == 4 ? (a.Cp >> 2) : 1;
    const int64_t per_sweep = ngroups * nquads;
    const int64_t total = per_sweep * a.count;
    T *out = static_cast<T *>(a.out);
    for (int64_t q = bid * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(nblk) * blockDim.x) {
        const int64_t t = q / per_sweep, r0 = q - t * per_sweep;
        const int cq = static_cast<int>(r0 / ngroups);
        const int64_t g = r0 - static_cast<int64_t>(cq) * ngroups;
        T n4[4];
        block_normals<T>(a.key, static_cast<uint32_t>(g), static_cast<uint32_t>(base + t), f.stream,
                         static_cast<uint32_t>(cq), n4);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            // normal r serves site G g + r / lanes and chain 4 cq + r mod lanes
            const int64_t site = (g << gs) + r / L;
            const int chain = cq * 4 + (r & (L - 1));
            if (site >= n || chain >= a.C) continue;
            if (a.perm_inv) {  // graph: by permuted position
                out[(t * a.C + chain) * n + a.perm_inv[f.csr0 + site]] = n4[r];
                continue;
            }
            const int i = static_cast<int>(site / Wl), j = static_cast<int>(site - static_cast<int64_t>(i) * Wl);
            int c, pos;
            if (e8) {
                c = 2 * (i & 1) + (j & 1);
                pos = (i >> 1) * ((Wl - (j & 1) + 1) >> 1) + (j >> 1);
            } else {
                c = (i + j) & 1;
                pos = i * f.cols + (j >> 1);
            }
            const int k = pos / a.NTS, tid = pos - k * a.NTS;
            out[((t * a.C + chain) * K * a.NI + c * a.NI + k) * a.NTS + tid] = n4[r];
        }
    }
}

template <typename T, int KIND>
cudaError_t launch_ni(int NI, int threads, int chains, const ResidentArgs &a, size_t smem, cudaStream_t st)
{
    if (NI == 1) return launch_sweep_kernel(lattice_resident_kernel<T, KIND, 1>, chains, threads, smem, st, a);
    if (NI == 2 || KIND == kLat2D8)  // four positions per class only for the 4-neighbour lattice
        return launch_sweep_kernel(lattice_resident_kernel<T, KIND, 2>, chains, threads, smem, st, a);
    return launch_sweep_kernel(lattice_resident_kernel<T, kLat2D4, 4>, chains, threads, smem, st, a);
}

template <typename T, int KIND>
cudaError_t prepare_ni(int NI, size_t smem)
{
    const int s = static_cast<int>(smem);
    constexpr auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (NI == 1) return cudaFuncSetAttribute(lattice_resident_kernel<T, KIND, 1>, attr, s);
    if (NI == 2 || KIND == kLat2D8) return cudaFuncSetAttribute(lattice_resident_kernel<T, KIND, 2>, attr, s);
    return cudaFuncSetAttribute(lattice_resident_kernel<T, kLat2D4, 4>, attr, s);
}

}  // namespace

cudaError_t prepare_lattice_resident(int precision, int kind, int NI, size_t smem)
{
    const bool e8 = kind == kLat2D8;
    if (precision == 0) return e8 ? prepare_ni<float, kLat2D8>(NI, smem) : prepare_ni<float, kLat2D4>(NI, smem);
    return e8 ? prepare_ni<double, kLat2D8>(NI, smem) : prepare_ni<double, kLat2D4>(NI, smem);
}

cudaError_t launch_resident_normals(int precision, const ResNormArgs &a, int64_t blocks_needed, cudaStream_t stream)
{
    int64_t blocks = (blocks_needed + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    blocks += a.gamma_blocks;
    if (precision == 0)
        return launch_sweep_kernel(resident_normals_kernel<float>, static_cast<int>(blocks), 256, 0, stream, a);
    return launch_sweep_kernel(resident_normals_kernel<double>, static_cast<int>(blocks), 256, 0, stream, a);
}

cudaError_t launch_lattice_resident(int precision, int kind, int NI, int threads, int chains, const ResidentArgs &a,
                                    size_t smem, cudaStream_t stream)
{
    const bool e8 = kind == kLat2D8;
    if (precision == 0)
        return e8 ? launch_ni<float, kLat2D8>(NI, threads, chains, a, smem, stream)
                  : launch_ni<float, kLat2D4>(NI, threads, chains, a, smem, stream);
    return e8 ? launch_ni<double, kLat2D8>(NI, threads, chains, a, smem, stream)
              : launch_ni<double, kLat2D4>(NI, threads, chains, a, smem, stream);
}

}  // namespace gmrf
