// csr_resident.cu -- many whole sweeps of a small graph field in one launch, one thread-block
// cluster per chain.
//
// The graph counterpart of lattice_resident.cu, for a single CSR field with unit weights and
// the Gaussian likelihood (the precinct-sized graphs of Sec. 3.2: a few thousand to ~18,000
// sites).  On the per-sweep path such a field's sweep is k launches of a few thousand sites each
// plus the draws, bound by launch latency.  Here one block holds a chain: its state, running mean
// and M2 in shared memory by permuted position (colour classes contiguous, Sec. 2.3), and runs
// `count` sweeps of Algorithm 1 back to back.  A chain is shared by a cluster of CL blocks (on CL
// SMs): every block keeps the chain's whole state in its shared memory and owns a contiguous share
// of each colour class; after updating its share it stores the new values into the other blocks'
// copies (distributed shared memory) with asynchronous stores that complete on the receiving
// block's mbarrier, and a colour step ends when the other blocks' values have arrived (a
// transaction barrier per step, two alternating), so each block reads all neighbours locally.
// The block sums go to block 0, whose drawing warps draw and store the new parameters into every
// block, with cluster barriers (release / acquire) around that exchange.
// What a sweep reads from L2 is the neighbour lists
// -- re-packed for this kernel as one 16-byte record of eight 16-bit positions per site (a second
// record for sites of degree 9 to 16), so a site's neighbours arrive in one load -- the
// observations and the sweep's normals (produced ahead for the whole batch by
// resident_normals_kernel).  In a colour step a site thread first issues the loads of all its
// positions of the class, then updates them: one L2 round trip per step.  The sums of the
// conjugate draws fold in as on the per-sweep path (lower-colour neighbours: permuted position
// below the class's first), and two drawing warps draw as in lattice_resident.cu.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "mbarrier.cuh"
#include "lattice_common.cuh"
#include "resident_draws.cuh"

namespace gmrf {
namespace {

constexpr int kCsrSiteThreads = 512;
constexpr int kCsrThreads = kCsrSiteThreads + 64;  // and two drawing warps
constexpr int kCsrMaxPos = 8;                       // positions of a class per site thread
constexpr int kCsrMaxColours = 64;

// Entry q (0..7) of a record; in the first record bit 15 of entry 0 is the "more in nbr2" flag.
__device__ __forceinline__ int rec_entry(const uint4 &r, int q)
{
    const uint32_t w = q < 2 ? r.x : (q < 4 ? r.y : (q < 6 ? r.z : r.w));
    return static_cast<int>((q & 1) ? (w >> 16) : (w & 0xffffu));
}
__device__ __forceinline__ int rec_id(const uint4 &r, int q) { return q == 0 ? (rec_entry(r, 0) & 0x7fff) : rec_entry(r, q); }

__global__ void pack_csr_records_kernel(int32_t n, const int32_t *rp, const int32_t *ci, uint4 *nbr, uint4 *nbr2)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int rb = rp[p], deg = rp[p + 1] - rb;
        uint32_t id[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) id[q] = q < deg ? static_cast<uint32_t>(ci[rb + q]) : static_cast<uint32_t>(n);
        if (deg > 8) id[0] |= 0x8000u;
        nbr[p] = make_uint4(id[0] | (id[1] << 16), id[2] | (id[3] << 16), id[4] | (id[5] << 16), id[6] | (id[7] << 16));
        nbr2[p] = make_uint4(id[8] | (id[9] << 16), id[10] | (id[11] << 16), id[12] | (id[13] << 16),
                             id[14] | (id[15] << 16));
    }
}

// Cluster primitives (PTX): this block's rank in its cluster, the address of the same shared
// location in block `rank`, a store there, and the cluster barrier (arrive with release, wait
// with acquire: stores to other blocks before the arrive are visible after the wait).
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t remote_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_remote(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_remote(uint32_t addr, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Transaction barriers of the colour steps in a cluster: a block's new values go to the other
// blocks' copies by asynchronous remote stores that complete on the receiving block's mbarrier
// (complete_tx); the receiver expects the bytes of the other blocks' shares of the class and waits
// for that phase.  No fence on the sending side.
__device__ __forceinline__ void st_async(uint32_t addr, float v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
                 "l"(__double_as_longlong(v)), "r"(bar)
                 : "memory");
}

// MP: positions of a colour class per site thread, 1 or kCsrMaxPos.  With one, the loads of the
// next colour step's position (its neighbour record, observation and normal) are issued before the
// current step's update, so the step does not wait for L2.
template <typename T, int CL, int MP>
__global__ void __launch_bounds__(kCsrThreads, 1) csr_resident_kernel(const ResCsrArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[kCsrThreads / 32][3];
    __shared__ T red_cl[CL > 8 ? CL : 8][3];  // block 0: the blocks' sums
    __shared__ T hs[3];         // tau, 1/sigma^2, beta0 of the current sweep
    __shared__ int coffs[kCsrMaxColours + 1];
    __shared__ int own_lo[kCsrMaxColours], own_hi[kCsrMaxColours], own_off[kCsrMaxColours];
    __shared__ __align__(8) uint64_t sbar[2];  // cluster: the colour steps' barriers, by step parity
    __shared__ int s_gave_up;                  // cluster: a step's wait ran out (no more waits)

    // Everything up to the first normals depends only on the previous batch's kernel (complete
    // before this launch's predecessor, the batch's normals, let this one start), so the chain is
    // staged while the normals are still being drawn; pdl_wait comes before their first use.
    const HyperArgs &h = a.h;
    const uint32_t rank = CL > 1 ? cluster_rank() : 0u;
    const int chain = blockIdx.x / CL, tid = threadIdx.x, NT = blockDim.x, NTS = kCsrSiteThreads;
    const int lane = tid & 31, warp = tid >> 5, nsw = NTS >> 5;
    const bool drawer = tid >= NTS;
    const int dw = warp - nsw;  // drawing warp: 0 tau, 1 beta0 and sigma^2 (block 0 only)
    const FieldDev f = a.fields[0];
    const int n = f.n, K = a.ncolors, Cp = h.Cp;
    T *xs = reinterpret_cast<T *>(smem_raw);  // [n + 1] the whole chain; position n is a zero (pad)
    T *ms = xs + n + 1;                       // the owned positions' mean and M2
    T *m2s = ms + a.own_max;

    const long long sweep0 = h.ctl->sweep;
    long long acc = h.ctl->acc_count;
    if (tid < 3) hs[tid] = static_cast<const T *>(h.hyp)[static_cast<int64_t>(chain) * kHypStride + tid];
    if (tid <= K) coffs[tid] = a.coff[tid];
    __syncthreads();
    if (tid == 0) {  // this block's share of every colour class and its place in ms / m2s
        if (CL > 1) {
            mbar_init(&sbar[0], 1);
            mbar_init(&sbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        s_gave_up = 0;
        int off = 0;
        for (int c = 0; c < K; ++c) {
            const int lo = coffs[c], len = coffs[c + 1] - lo, q = (len + CL - 1) / CL;
            own_lo[c] = lo + min(static_cast<int>(rank) * q, len);
            own_hi[c] = lo + min((static_cast<int>(rank) + 1) * q, len);
            own_off[c] = off;
            off += own_hi[c] - own_lo[c];
        }
    }
    // The drawing lanes' state (block 0) lives in shared memory.
    __shared__ ResidentDraws<T> drs[2];
    ResidentDraws<T> &dr = drs[drawer ? dw : 0];
    const bool draws = drawer && lane == 0 && rank == 0;
    if (draws) dr.init(h, dw, chain, f);
    __syncthreads();
    {
        const T *X = static_cast<const T *>(a.x) + f.slot0 * Cp + chain;
        const T *MEAN = static_cast<const T *>(a.mean) + f.slot0 * Cp + chain;
        const T *M2 = static_cast<const T *>(a.m2) + f.slot0 * Cp + chain;
        for (int p = tid; p < n; p += NT) xs[p] = X[static_cast<int64_t>(p) * Cp];
        if (tid == 0) xs[n] = 0;
        for (int c = 0; c < K; ++c)
            for (int p = own_lo[c] + tid; p < own_hi[c]; p += NT) {
                const int l = own_off[c] + p - own_lo[c];
                ms[l] = MEAN[static_cast<int64_t>(p) * Cp];
                m2s[l] = M2[static_cast<int64_t>(p) * Cp];
            }
    }
    __syncthreads();
    if (CL > 1) cluster_sync();  // every block of the cluster has its copy before any store into it
    pdl_wait();                  // the batch's normals and Gamma variates
    const long long bbase = h.ctl->batch_base, bcount = h.ctl->batch_count;

    const T *Y = static_cast<const T *>(a.y) + f.slot0;
    const T *ZB = static_cast<const T *>(a.zbuf) + static_cast<int64_t>(chain) * n;
    const int64_t zstride = static_cast<int64_t>(a.C) * n;
    const T rho = static_cast<T>(a.rho);
    const bool acc_on = h.acc_enabled != 0;
    int thin_phase = sweep0 >= h.burn_in ? static_cast<int>((sweep0 - h.burn_in) % h.thin) : 0;
    long long slot = h.trace_cap > 0 ? sweep0 % h.trace_cap : 0;
    // MP == 1: the position of the first colour step, loaded ahead.
    uint4 rn = make_uint4(0u, 0u, 0u, 0u);
    T yn = 0, zn = 0;
    if (MP == 1 && !drawer && K > 0 && a.count > 0 && own_lo[0] + tid < own_hi[0]) {
        rn = a.nbr[own_lo[0] + tid];
        yn = Y[own_lo[0] + tid];
        zn = ZB[own_lo[0] + tid];
    }
    // Colour steps of this launch so far (cluster: step g uses barrier g & 1, phase parity
    // (g >> 1) & 1; a block starts step g + 1 only when every other block's values of step g have
    // arrived, i.e. after every block has read its neighbours of step g, so no copy is written
    // while it is still read).
    int g = 0;
    for (int t = 0; t < a.count; ++t) {
        const long long sw = sweep0 + t;
        if (draws) dr.prep(h, sw, slot, t > 0, bbase, bcount, Cp);
        const T tau = hs[0], isig = hs[1], beta = hs[2];
        const bool acc_now = acc_on && sw >= h.burn_in && thin_phase == 0;
        const T inv_k = acc_now ? static_cast<T>(1) / static_cast<T>(acc + 1) : static_cast<T>(0);
        const T *Z = ZB + t * zstride;
        T accS = 0, accR = 0, accA = 0;
        // One position of colour class c (first position lo; ob maps it into ms / m2s).
        auto update = [&](int p, const uint4 &rc, T yv, T zv, int lo, int ob) {
            T nb[8], s = 0;
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int id = rec_id(rc, q);
                nb[q] = xs[id];
                s += nb[q];
                cnt += id != n;
            }
            const bool more = (rc.x & 0x8000u) != 0;
            uint4 r2 = make_uint4(0u, 0u, 0u, 0u);
            if (more) {  // degree 9..16 (rare): the second record
                r2 = a.nbr2[p];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int id = rec_entry(r2, q);
                    s += xs[id];
                    cnt += id != n;
                }
            }
            const T d = static_cast<T>(cnt);
            const T P = tau * d + isig;
            const T mn = (tau * rho * s + (yv - beta) * isig) * FArith<T>::rcp(P);
            const T xn = mn + zv * FArith<T>::rsq(P);
            xs[p] = xn;
#pragma unroll
            for (int r = 1; r < CL; ++r) {  // the other blocks' copies
                const uint32_t dst = (rank + r) % CL;
                st_async(remote_addr(xs + p, dst), xn, remote_addr(&sbar[g & 1], dst));
            }
            T e = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (rec_id(rc, q) < lo) {  // lower colour (the pad n is never below lo)
                    const T df = xn - nb[q];
                    e += df * df;
                }
            }
            if (more) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int id = rec_entry(r2, q);
                    if (id < lo) {
                        const T df = xn - xs[id];
                        e += df * df;
                    }
                }
            }
            accS += (static_cast<T>(1) - rho) * d * xn * xn + rho * e;
            const T r = (yv - beta) - xn;
            accR += r * r;
            accA += r;
            if (acc_now) {
                T mu = ms[ob + p], mm = m2s[ob + p];
                const T delta = xn - mu;
                mu += delta * inv_k;
                mm += delta * (xn - mu);
                ms[ob + p] = mu;
                m2s[ob + p] = mm;
            }
        };
        for (int c = 0; c < K; ++c, ++g) {
            if (CL > 1 && tid == 0 && !s_gave_up) {  // this step's expected bytes: the other blocks' shares
                const int others = (coffs[c + 1] - coffs[c]) - (own_hi[c] - own_lo[c]);
                mbar_arrive_expect(&sbar[g & 1], static_cast<uint32_t>(others) * sizeof(T) + a.extra_bytes);
            }
            if (!drawer) {
                const int lo = coffs[c], a0 = own_lo[c], a1 = own_hi[c], ob = own_off[c] - a0;
                if constexpr (MP == 1) {
                    // this step's position (loaded during the previous step), then the next one's loads
                    const int p = a0 + tid;
                    const uint4 rc = rn;
                    const T yc = yn, zc = zn;
                    int c2 = c + 1, t2 = t;
                    if (c2 == K) {
                        c2 = 0;
                        ++t2;
                    }
                    const int p2 = own_lo[c2] + tid;
                    if (t2 < a.count && p2 < own_hi[c2]) {
                        rn = a.nbr[p2];
                        yn = Y[p2];
                        zn = ZB[t2 * zstride + p2];
                    }
                    if (p < a1) update(p, rc, yc, zc, lo, ob);
                } else {
                    // Loads of all of this thread's positions of the share first (one round trip).
                    uint4 rec[MP];
                    T yv[MP], zv[MP];
#pragma unroll
                    for (int j = 0; j < MP; ++j) {
                        const int p = a0 + tid + j * NTS;
                        if (p < a1) {
                            rec[j] = a.nbr[p];
                            yv[j] = Y[p];
                            zv[j] = Z[p];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < MP; ++j) {
                        const int p = a0 + tid + j * NTS;
                        if (p < a1) update(p, rec[j], yv[j], zv[j], lo, ob);
                    }
                }
            }
            // End of the colour step: the class is final in this block's copy (the other blocks'
            // values have arrived; the site threads' own ones after the named barrier).  With one
            // block, after the last step the barrier of the sums below serves.
            if (CL > 1 && !drawer) {
                if (!s_gave_up && !mbar_try_wait(&sbar[g & 1], (g >> 1) & 1)) {
                    const uint64_t t0 = global_ns();
                    bool ok = false;
                    while (!(ok = mbar_try_wait(&sbar[g & 1], (g >> 1) & 1)) && global_ns() - t0 < a.wait_ns) {
                    }
                    if (!ok) {
                        s_gave_up = 1;
                        atomicAdd(&h.ctl->wait_timeouts, 1ull);
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(NTS) : "memory");
            } else if (CL == 1 && c + 1 < K && !drawer) {
                asm volatile("bar.sync 1, %0;" ::"r"(NTS) : "memory");
            }
        }
        // The sums: a shuffle tree per site warp, over the site warps, then over the blocks
        // (block 0, in rank order), in precision T.
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
        if (warp == nsw) {  // the first drawing warp of every block: this block's sums to block 0
            T b0 = lane < nsw ? red[lane][0] : static_cast<T>(0);
            T b1 = lane < nsw ? red[lane][1] : static_cast<T>(0);
            T b2 = lane < nsw ? red[lane][2] : static_cast<T>(0);
            for (int o = 16; o >= 1; o >>= 1) {
                b0 += __shfl_xor_sync(0xffffffffu, b0, o);
                b1 += __shfl_xor_sync(0xffffffffu, b1, o);
                b2 += __shfl_xor_sync(0xffffffffu, b2, o);
            }
            if (lane == 0) {
                if (CL > 1) {
                    st_remote(remote_addr(&red_cl[rank][0], 0), b0);
                    st_remote(remote_addr(&red_cl[rank][1], 0), b1);
                    st_remote(remote_addr(&red_cl[rank][2], 0), b2);
                } else {
                    red_cl[0][0] = b0;
                    red_cl[0][1] = b1;
                    red_cl[0][2] = b2;
                }
            }
        }
        if (CL > 1) cluster_sync();
        else __syncthreads();
        if (draws) {
            T v0 = 0, v1 = 0;
            for (int r = 0; r < CL; ++r) {
                v0 += red_cl[r][dw];
                if (dw == 1) v1 += red_cl[r][2];
            }
            dr.draw(h, v0, v1, beta, hs);
            for (int r = 1; r < CL; ++r) {  // the new parameters into every block
                if (dw == 0) {
                    st_remote(remote_addr(&hs[0], r), hs[0]);
                } else {
                    st_remote(remote_addr(&hs[1], r), hs[1]);
                    st_remote(remote_addr(&hs[2], r), hs[2]);
                }
            }
        }
        if (acc_now) ++acc;
        if (sw >= h.burn_in) thin_phase = (thin_phase + 1 == h.thin) ? 0 : thin_phase + 1;
        if (h.trace_cap > 0) slot = (slot + 1 == h.trace_cap) ? 0 : slot + 1;
        if (CL > 1) cluster_sync();
        else __syncthreads();
    }
    if (draws && a.count > 0) dr.finish(h);
    pdl_release();

    {
        T *X = static_cast<T *>(a.x) + f.slot0 * Cp + chain;
        T *MEAN = static_cast<T *>(a.mean) + f.slot0 * Cp + chain;
        T *M2 = static_cast<T *>(a.m2) + f.slot0 * Cp + chain;
        for (int c = 0; c < K; ++c)
            for (int p = own_lo[c] + tid; p < own_hi[c]; p += NT) {
                const int l = own_off[c] + p - own_lo[c];
                X[static_cast<int64_t>(p) * Cp] = xs[p];
                MEAN[static_cast<int64_t>(p) * Cp] = ms[l];
                M2[static_cast<int64_t>(p) * Cp] = m2s[l];
            }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&h.ctl->ticket, 1ull) == gridDim.x - 1) {
            h.ctl->sweep = sweep0 + a.count;
            h.ctl->acc_count = acc;
            h.ctl->ticket = 0;
        }
    }
    if (CL > 1) cluster_sync();  // no block leaves while another may still address its memory
}

}  // namespace

int csr_resident_threads() { return kCsrThreads; }
int csr_resident_max_positions() { return kCsrMaxPos * kCsrSiteThreads; }  // per block and class
int csr_resident_site_threads() { return kCsrSiteThreads; }

cudaError_t launch_pack_csr_records(int32_t n, const int32_t *rp, const int32_t *ci, uint4 *nbr, uint4 *nbr2,
                                    cudaStream_t stream)
{
    pack_csr_records_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, rp, ci, nbr, nbr2);
    return cudaGetLastError();
}

namespace {

template <typename T, int CL, int MP>
cudaError_t launch_cl(int chains, const ResCsrArgs &a, size_t smem, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(chains * CL);
    cfg.blockDim = dim3(kCsrThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    int na = 0;
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = CL;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
    if (pdl_enabled()) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, csr_resident_kernel<T, CL, MP>, a);
}

template <typename T, int MP>
cudaError_t prepare_mp(size_t smem)
{
    constexpr auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(csr_resident_kernel<T, 1, MP>, attr, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(csr_resident_kernel<T, 2, MP>, attr, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(csr_resident_kernel<T, 4, MP>, attr, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(csr_resident_kernel<T, 8, MP>, attr, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(csr_resident_kernel<T, 16, MP>, attr, static_cast<int>(smem));
    // clusters of 16 blocks exceed the portable size of 8
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(csr_resident_kernel<T, 16, MP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename T>
cudaError_t prepare_t(size_t smem)
{
    cudaError_t e = prepare_mp<T, 1>(smem);
    return e == cudaSuccess ? prepare_mp<T, kCsrMaxPos>(smem) : e;
}

template <typename T, int MP>
cudaError_t launch_mp(int cl, int chains, const ResCsrArgs &a, size_t smem, cudaStream_t stream)
{
    if (cl == 16) return launch_cl<T, 16, MP>(chains, a, smem, stream);
    if (cl == 8) return launch_cl<T, 8, MP>(chains, a, smem, stream);
    if (cl == 4) return launch_cl<T, 4, MP>(chains, a, smem, stream);
    if (cl == 2) return launch_cl<T, 2, MP>(chains, a, smem, stream);
    return launch_cl<T, 1, MP>(chains, a, smem, stream);
}

template <typename T>
cudaError_t launch_t(int cl, int mp, int chains, const ResCsrArgs &a, size_t smem, cudaStream_t stream)
{
    return mp == 1 ? launch_mp<T, 1>(cl, chains, a, smem, stream) : launch_mp<T, kCsrMaxPos>(cl, chains, a, smem, stream);
}

}  // namespace

cudaError_t prepare_csr_resident(int precision, size_t smem)
{
    return precision == 0 ? prepare_t<float>(smem) : prepare_t<double>(smem);
}

cudaError_t launch_csr_resident(int precision, int cluster, int positions, int chains, const ResCsrArgs &a,
                                size_t smem, cudaStream_t stream)
{
    return precision == 0 ? launch_t<float>(cluster, positions, chains, a, smem, stream)
                          : launch_t<double>(cluster, positions, chains, a, smem, stream);
}

}  // namespace gmrf
