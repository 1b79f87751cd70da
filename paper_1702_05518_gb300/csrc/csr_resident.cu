// csr_resident.cu -- many whole sweeps of a small graph field in one launch, one block per chain.
//
// The graph counterpart of lattice_resident.cu, for a single CSR field with unit weights and
// the Gaussian likelihood (the precinct-sized graphs of Sec. 3.2: a few thousand to ~18,000
// sites).  On the per-sweep path such a field's sweep is k launches of a few thousand sites each
// plus the draws, bound by launch latency.  Here one block holds a chain: its state, running mean
// and M2 in shared memory by permuted position (colour classes contiguous, Sec. 2.3), and runs
// `count` sweeps of Algorithm 1 back to back.  What a sweep reads from L2 is the neighbour lists
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

template <typename T>
__global__ void __launch_bounds__(kCsrThreads, 1) csr_resident_kernel(const ResCsrArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[kCsrThreads / 32][3];
    __shared__ T hs[3];  // tau, 1/sigma^2, beta0 of the current sweep
    __shared__ int coffs[kCsrMaxColours + 1];

    pdl_wait();
    const HyperArgs &h = a.h;
    const int chain = blockIdx.x, tid = threadIdx.x, NT = blockDim.x, NTS = kCsrSiteThreads;
    const int lane = tid & 31, warp = tid >> 5, nsw = NTS >> 5;
    const bool drawer = tid >= NTS;
    const int dw = warp - nsw;  // drawing warp: 0 tau, 1 beta0 and sigma^2
    const FieldDev f = a.fields[0];
    const int n = f.n, K = a.ncolors, Cp = h.Cp;
    T *xs = reinterpret_cast<T *>(smem_raw);  // [n + 1]: position n is a zero (the records' pad)
    T *ms = xs + n + 1;
    T *m2s = ms + n;

    const long long sweep0 = h.ctl->sweep;
    long long acc = h.ctl->acc_count;
    const long long bbase = h.ctl->batch_base, bcount = h.ctl->batch_count;
    if (tid < 3) hs[tid] = static_cast<const T *>(h.hyp)[static_cast<int64_t>(chain) * kHypStride + tid];
    if (tid <= K) coffs[tid] = a.coff[tid];
    // The drawing lanes' state lives in shared memory (no thread keeps registers for it).
    __shared__ ResidentDraws<T> drs[2];
    ResidentDraws<T> &dr = drs[drawer ? dw : 0];
    if (drawer && lane == 0) dr.init(h, dw, chain, f);
    {
        const T *X = static_cast<const T *>(a.x) + f.slot0 * Cp + chain;
        const T *MEAN = static_cast<const T *>(a.mean) + f.slot0 * Cp + chain;
        const T *M2 = static_cast<const T *>(a.m2) + f.slot0 * Cp + chain;
        for (int p = tid; p < n; p += NT) {
            xs[p] = X[static_cast<int64_t>(p) * Cp];
            ms[p] = MEAN[static_cast<int64_t>(p) * Cp];
            m2s[p] = M2[static_cast<int64_t>(p) * Cp];
        }
        if (tid == 0) xs[n] = 0;
    }
    __syncthreads();

    const T *Y = static_cast<const T *>(a.y) + f.slot0;
    const T *ZB = static_cast<const T *>(a.zbuf) + static_cast<int64_t>(chain) * n;
    const int64_t zstride = static_cast<int64_t>(a.C) * n;
    const T rho = static_cast<T>(a.rho);
    const bool acc_on = h.acc_enabled != 0;
    int thin_phase = sweep0 >= h.burn_in ? static_cast<int>((sweep0 - h.burn_in) % h.thin) : 0;
    long long slot = h.trace_cap > 0 ? sweep0 % h.trace_cap : 0;
    for (int t = 0; t < a.count; ++t) {
        const long long sw = sweep0 + t;
        if (drawer && lane == 0) dr.prep(h, sw, slot, t > 0, bbase, bcount, Cp);
        const T tau = hs[0], isig = hs[1], beta = hs[2];
        const bool acc_now = acc_on && sw >= h.burn_in && thin_phase == 0;
        const T inv_k = acc_now ? static_cast<T>(1) / static_cast<T>(acc + 1) : static_cast<T>(0);
        const T *Z = ZB + t * zstride;
        T accS = 0, accR = 0, accA = 0;
        for (int c = 0; c < K; ++c) {
            if (!drawer) {
                const int lo = coffs[c], hi = coffs[c + 1];
                // Loads of all of this thread's positions of the class first (one round trip).
                uint4 rec[kCsrMaxPos];
                T yv[kCsrMaxPos], zv[kCsrMaxPos];
#pragma unroll
                for (int j = 0; j < kCsrMaxPos; ++j) {
                    const int p = lo + tid + j * NTS;
                    if (p < hi) {
                        rec[j] = a.nbr[p];
                        yv[j] = Y[p];
                        zv[j] = Z[p];
                    }
                }
#pragma unroll
                for (int j = 0; j < kCsrMaxPos; ++j) {
                    const int p = lo + tid + j * NTS;
                    if (p >= hi) continue;
                    T nb[8], s = 0;
                    int cnt = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int id = rec_id(rec[j], q);
                        nb[q] = xs[id];
                        s += nb[q];
                        cnt += id != n;
                    }
                    const bool more = (rec[j].x & 0x8000u) != 0;
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
                    const T mn = (tau * rho * s + (yv[j] - beta) * isig) * FArith<T>::rcp(P);
                    const T xn = mn + zv[j] * FArith<T>::rsq(P);
                    xs[p] = xn;
                    T e = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (rec_id(rec[j], q) < lo) {  // lower colour (the pad n is never below lo)
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
                    const T r = (yv[j] - beta) - xn;
                    accR += r * r;
                    accA += r;
                    if (acc_now) {
                        T mu = ms[p], mm = m2s[p];
                        const T delta = xn - mu;
                        mu += delta * inv_k;
                        mm += delta * (xn - mu);
                        ms[p] = mu;
                        m2s[p] = mm;
                    }
                }
                if (c + 1 < K) asm volatile("bar.sync 1, %0;" ::"r"(NTS) : "memory");
            }
        }
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
            T v0 = lane < nsw ? red[lane][dw] : static_cast<T>(0);
            T v1 = (dw == 1 && lane < nsw) ? red[lane][2] : static_cast<T>(0);
            for (int o = 16; o >= 1; o >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            }
            if (lane == 0) dr.draw(h, v0, v1, beta, hs);
        }
        if (acc_now) ++acc;
        if (sw >= h.burn_in) thin_phase = (thin_phase + 1 == h.thin) ? 0 : thin_phase + 1;
        if (h.trace_cap > 0) slot = (slot + 1 == h.trace_cap) ? 0 : slot + 1;
        __syncthreads();
    }
    if (drawer && lane == 0 && a.count > 0) dr.finish(h);
    pdl_release();

    {
        T *X = static_cast<T *>(a.x) + f.slot0 * Cp + chain;
        T *MEAN = static_cast<T *>(a.mean) + f.slot0 * Cp + chain;
        T *M2 = static_cast<T *>(a.m2) + f.slot0 * Cp + chain;
        for (int p = tid; p < n; p += NT) {
            X[static_cast<int64_t>(p) * Cp] = xs[p];
            MEAN[static_cast<int64_t>(p) * Cp] = ms[p];
            M2[static_cast<int64_t>(p) * Cp] = m2s[p];
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
}

}  // namespace

int csr_resident_threads() { return kCsrThreads; }
int csr_resident_max_positions() { return kCsrMaxPos * kCsrSiteThreads; }

cudaError_t launch_pack_csr_records(int32_t n, const int32_t *rp, const int32_t *ci, uint4 *nbr, uint4 *nbr2,
                                    cudaStream_t stream)
{
    pack_csr_records_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, rp, ci, nbr, nbr2);
    return cudaGetLastError();
}

cudaError_t prepare_csr_resident(int precision, size_t smem)
{
    constexpr auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (precision == 0) return cudaFuncSetAttribute(csr_resident_kernel<float>, attr, static_cast<int>(smem));
    return cudaFuncSetAttribute(csr_resident_kernel<double>, attr, static_cast<int>(smem));
}

cudaError_t launch_csr_resident(int precision, int chains, const ResCsrArgs &a, size_t smem, cudaStream_t stream)
{
    if (precision == 0) return launch_sweep_kernel(csr_resident_kernel<float>, chains, kCsrThreads, smem, stream, a);
    return launch_sweep_kernel(csr_resident_kernel<double>, chains, kCsrThreads, smem, stream, a);
}

}  // namespace gmrf
