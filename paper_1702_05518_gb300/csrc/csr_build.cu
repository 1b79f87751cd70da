// csr_build.cu -- graph colouring and the colour-permuted layout of CSR fields.
//
// Colouring (Sec. 2.3: any proper colouring works; it is computed once before the MCMC run) by
// Jones-Plassmann: in each round every uncoloured vertex whose (priority, index) exceeds that
// of each uncoloured neighbour is selected; the selected set is independent, so its vertices
// then take, without conflict, the smallest colour absent among their coloured neighbours.  A
// vertex is selected exactly when all neighbours of higher priority are coloured and none of
// lower priority is, so the result equals first-fit greedy colouring in decreasing (priority,
// index) order, and with priority decreasing in the index it is the paper's greedy colouring.
// Selection and assignment are separate launches, so a round reads only the colours of the
// previous rounds and the result is independent of scheduling.
//
// Layout (Sec. 3.1: chromatic sampling needs only the list of sites of each colour): a stable
// counting sort by colour gives perm (position -> site), perm_inv and the colour offsets; the
// permuted CSR keeps each row's entry order with columns renamed to positions.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {
namespace {

constexpr int kScanBlock = 1024;

__global__ void jp_priorities_kernel(int32_t n, uint2 key, uint32_t *prio)
{
    for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x)
        prio[v] = philox4x32_10(make_uint4(static_cast<uint32_t>(v), 0u, 0u, kTagPrio << 24), key).x;
}

// Largest-degree-first priorities: min(degree, 255) in the top 8 bits, the top 24 bits of the
// random priority below (vertices of larger degree are coloured first; equal degrees in the
// random order, then by index).
__global__ void jp_priorities_ldf_kernel(int32_t n, uint2 key, const int32_t *rp, uint32_t *prio)
{
    for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t w = philox4x32_10(make_uint4(static_cast<uint32_t>(v), 0u, 0u, kTagPrio << 24), key).x;
        const int32_t d = min(rp[v + 1] - rp[v], 255);
        prio[v] = (static_cast<uint32_t>(d) << 24) | (w >> 8);
    }
}

__global__ void fill_kernel(int32_t *p, int64_t n, int32_t value)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = value;
}

__device__ __forceinline__ bool beats(uint32_t pu, int32_t u, uint32_t pv, int32_t v)
{
    return pu > pv || (pu == pv && u > v);
}

// Round, phase 1: mark the uncoloured local maxima of (priority, index).
__global__ void jp_select_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const uint32_t *prio,
                                 const int32_t *colors, uint8_t *selected)
{
    for (int64_t vv = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; vv < n;
         vv += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = static_cast<int32_t>(vv);
        uint8_t sel = 0;
        if (colors[v] < 0) {
            sel = 1;
            const uint32_t pv = prio[v];
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
                const int32_t u = ci[e];
                if (colors[u] < 0 && beats(prio[u], u, pv, v)) {
                    sel = 0;
                    break;
                }
            }
        }
        selected[v] = sel;
    }
}

// Round, phase 2: each selected vertex takes the smallest colour absent among its coloured
// neighbours (searched 64 colours at a time) and counts itself as coloured.
__global__ void jp_assign_kernel(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *colors,
                                 const uint8_t *selected, unsigned long long *ncolored, int32_t *maxcolor)
{
    int local = 0;
    int32_t localmax = -1;
    for (int64_t vv = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; vv < n;
         vv += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = static_cast<int32_t>(vv);
        if (!selected[v]) continue;
        int32_t chosen = -1;
        for (int32_t base = 0; chosen < 0; base += 64) {
            unsigned long long used = 0;
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
                const int32_t cu = colors[ci[e]] - base;
                if (cu >= 0 && cu < 64) used |= 1ull << cu;
            }
            if (~used) chosen = base + __ffsll(static_cast<long long>(~used)) - 1;
        }
        colors[v] = chosen;
        ++local;
        localmax = max(localmax, chosen);
    }
    if (local) atomicAdd(ncolored, static_cast<unsigned long long>(local));
    if (localmax >= 0) atomicMax(maxcolor, localmax);
}

// The layout visits the vertices in the sequence order[0..n) (natural order when order is
// null): element i of the sequence is vertex order[i].

// Per block of kScanBlock elements of the sequence: count of each colour (colour-major
// [c][block]).
__global__ void block_colour_counts_kernel(int32_t n, int32_t ncolors, const int32_t *colors, const int32_t *order,
                                           int32_t *counts, int32_t nblocks)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(kScanBlock) + threadIdx.x;
    const int32_t cv = i < n ? colors[order ? order[i] : i] : -1;
    for (int32_t c = 0; c < ncolors; ++c) {
        const int cnt = __syncthreads_count(cv == c);
        if (threadIdx.x == 0) counts[static_cast<int64_t>(c) * nblocks + blockIdx.x] = cnt;
    }
}

// Exclusive scan of the colour-major counts: base[c][b] = offset of colour c + sum over earlier
// blocks; coff[c] = first position of colour c, coff[ncolors] = n.  One thread per colour, then
// a serial prefix over colours (ncolors is small).
__global__ void colour_bases_kernel(int32_t ncolors, int32_t nblocks, const int32_t *counts, int32_t *bases,
                                    int32_t *coff)
{
    __shared__ int32_t totals[1024];
    for (int32_t c = threadIdx.x; c < ncolors; c += blockDim.x) {
        int32_t acc = 0;
        for (int32_t b = 0; b < nblocks; ++b) {
            bases[static_cast<int64_t>(c) * nblocks + b] = acc;
            acc += counts[static_cast<int64_t>(c) * nblocks + b];
        }
        if (c < 1024) totals[c] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t off = 0;
        for (int32_t c = 0; c < ncolors; ++c) {
            coff[c] = off;
            off += totals[c];
        }
        coff[ncolors] = off;
    }
    __syncthreads();
    for (int32_t c = threadIdx.x; c < ncolors; c += blockDim.x)
        for (int32_t b = 0; b < nblocks; ++b) bases[static_cast<int64_t>(c) * nblocks + b] += coff[c];
}

// Stable scatter: position of the sequence's element i (vertex v) = base[colour][block] + rank
// of i among the block's elements of its colour (warp ballots, then warps in order), so each
// colour class keeps the sequence order.
__global__ void colour_scatter_kernel(int32_t n, int32_t ncolors, const int32_t *colors, const int32_t *order,
                                      const int32_t *bases, int32_t nblocks, int32_t *perm, int32_t *perm_inv)
{
    __shared__ int32_t wcount[kScanBlock / 32];
    const int64_t i = blockIdx.x * static_cast<int64_t>(kScanBlock) + threadIdx.x;
    const int64_t v = i < n ? (order ? order[i] : i) : -1;
    const int32_t cv = i < n ? colors[v] : -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int32_t c = 0; c < ncolors; ++c) {
        const unsigned mask = __ballot_sync(0xffffffffu, cv == c);
        if (lane == 0) wcount[warp] = __popc(mask);
        __syncthreads();
        if (cv == c) {
            int32_t before = 0;
            for (int w = 0; w < warp; ++w) before += wcount[w];
            const int32_t rank = before + __popc(mask & ((1u << lane) - 1u));
            const int32_t pos = bases[static_cast<int64_t>(c) * nblocks + blockIdx.x] + rank;
            perm[pos] = static_cast<int32_t>(v);
            perm_inv[v] = pos;
        }
        __syncthreads();
    }
}

// Row lengths of the permuted graph and, per row, the degree d = sum_j w_ij.
template <typename T>
__global__ void permuted_rows_kernel(int32_t n, const int32_t *rp, const double *w, const int32_t *perm,
                                     int32_t *len, T *deg)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = perm[p];
        len[p] = rp[v + 1] - rp[v];
        double d = 0.0;
        if (w) {
            for (int32_t e = rp[v]; e < rp[v + 1]; ++e) d += w[e];
        } else {
            d = static_cast<double>(rp[v + 1] - rp[v]);
        }
        deg[p] = static_cast<T>(d);
    }
}

// In-place exclusive scan of len[0..n) into out[0..n] (out[n] = total), single block.
__global__ void exclusive_scan_kernel(int32_t n, const int32_t *len, int32_t *out)
{
    __shared__ int32_t part[kScanBlock];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int32_t val = i < n ? len[i] : 0;
        part[threadIdx.x] = val;
        __syncthreads();
        for (int off = 1; off < kScanBlock; off <<= 1) {
            const int32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) out[i] = carry + part[threadIdx.x] - val;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry += part[kScanBlock - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

template <typename T>
__global__ void permuted_fill_kernel(int32_t n, const int32_t *rp, const int32_t *ci, const double *w,
                                     const int32_t *perm, const int32_t *perm_inv, const int32_t *rp_out,
                                     int32_t *ci_out, T *w_out)
{
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = perm[p];
        int32_t o = rp_out[p];
        for (int32_t e = rp[v]; e < rp[v + 1]; ++e, ++o) {
            ci_out[o] = perm_inv[ci[e]];
            if (w_out) w_out[o] = static_cast<T>(w[e]);
        }
    }
}

int grid_of(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return static_cast<int>(g);
}

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

}  // namespace

size_t jp_scratch_bytes(int32_t n)
{
    return align256(sizeof(uint32_t) * static_cast<size_t>(n > 0 ? n : 1)) +
           align256(static_cast<size_t>(n > 0 ? n : 1)) + align256(sizeof(unsigned long long) * 2);
}

cudaError_t jp_color(int32_t n, const int32_t *rp, const int32_t *ci, const uint32_t *prio_in, uint64_t seed,
                     int32_t *colors, void *scratch, int32_t *num_colors_host, cudaStream_t stream, bool ldf)
{
    char *sp = static_cast<char *>(scratch);
    uint32_t *prio = reinterpret_cast<uint32_t *>(sp);
    sp += align256(sizeof(uint32_t) * static_cast<size_t>(n > 0 ? n : 1));
    uint8_t *selected = reinterpret_cast<uint8_t *>(sp);
    sp += align256(static_cast<size_t>(n > 0 ? n : 1));
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(sp);
    int32_t *maxcolor = reinterpret_cast<int32_t *>(counters + 1);
    cudaError_t err;
    if (n == 0) {
        *num_colors_host = 0;
        return cudaSuccess;
    }
    if (prio_in) {
        err = cudaMemcpyAsync(prio, prio_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, stream);
        if (err != cudaSuccess) return err;
    } else if (ldf) {
        jp_priorities_ldf_kernel<<<grid_of(n, 256), 256, 0, stream>>>(n, philox_key(seed), rp, prio);
    } else {
        jp_priorities_kernel<<<grid_of(n, 256), 256, 0, stream>>>(n, philox_key(seed), prio);
    }
    fill_kernel<<<grid_of(n, 256), 256, 0, stream>>>(colors, n, -1);
    if ((err = cudaMemsetAsync(counters, 0, sizeof(unsigned long long), stream)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(maxcolor, 0xff, sizeof(int32_t), stream)) != cudaSuccess) return err;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // Rounds in batches of 8 between host checks; every round colours at least the vertex of
    // globally largest (priority, index) among the uncoloured, so at most n rounds are needed.
    unsigned long long done = 0;
    int64_t rounds = 0;
    while (done < static_cast<unsigned long long>(n)) {
        for (int r = 0; r < 8; ++r) {
            jp_select_kernel<<<grid_of(n, 256), 256, 0, stream>>>(n, rp, ci, prio, colors, selected);
            jp_assign_kernel<<<grid_of(n, 256), 256, 0, stream>>>(n, rp, ci, colors, selected, counters, maxcolor);
        }
        rounds += 8;
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = cudaMemcpyAsync(&done, counters, sizeof(done), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
            return err;
        if ((err = cudaStreamSynchronize(stream)) != cudaSuccess) return err;
        if (rounds > static_cast<int64_t>(n) + 8) return cudaErrorUnknown;  // cannot happen
    }
    int32_t mx = -1;
    if ((err = cudaMemcpyAsync(&mx, maxcolor, sizeof(mx), cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return err;
    if ((err = cudaStreamSynchronize(stream)) != cudaSuccess) return err;
    *num_colors_host = mx + 1;
    return cudaSuccess;
}

size_t layout_scratch_bytes(int32_t n, int32_t ncolors)
{
    const int64_t nblocks = (static_cast<int64_t>(n) + kScanBlock - 1) / kScanBlock;
    const size_t nb = static_cast<size_t>(nblocks > 0 ? nblocks : 1);
    return 2 * align256(sizeof(int32_t) * nb * static_cast<size_t>(ncolors > 0 ? ncolors : 1)) +
           align256(sizeof(int32_t) * static_cast<size_t>(n > 0 ? n : 1));
}

cudaError_t csr_layout(int precision, int32_t n, int32_t ncolors, const int32_t *rp, const int32_t *ci,
                       const double *w, const int32_t *colors, const int32_t *order, void *scratch, int32_t *perm,
                       int32_t *perm_inv, int32_t *coff, int32_t *rp_out, int32_t *ci_out, void *w_out,
                       void *deg_out, cudaStream_t stream)
{
    const int32_t nblocks = static_cast<int32_t>((static_cast<int64_t>(n) + kScanBlock - 1) / kScanBlock);
    const size_t nb = static_cast<size_t>(nblocks > 0 ? nblocks : 1);
    char *sp = static_cast<char *>(scratch);
    int32_t *counts = reinterpret_cast<int32_t *>(sp);
    sp += align256(sizeof(int32_t) * nb * static_cast<size_t>(ncolors > 0 ? ncolors : 1));
    int32_t *bases = reinterpret_cast<int32_t *>(sp);
    sp += align256(sizeof(int32_t) * nb * static_cast<size_t>(ncolors > 0 ? ncolors : 1));
    int32_t *len = reinterpret_cast<int32_t *>(sp);
    if (n == 0) {
        cudaError_t err = cudaMemsetAsync(coff, 0, sizeof(int32_t) * (ncolors + 1), stream);
        if (err != cudaSuccess) return err;
        return cudaMemsetAsync(rp_out, 0, sizeof(int32_t), stream);
    }
    block_colour_counts_kernel<<<nblocks, kScanBlock, 0, stream>>>(n, ncolors, colors, order, counts, nblocks);
    colour_bases_kernel<<<1, 1024, 0, stream>>>(ncolors, nblocks, counts, bases, coff);
    colour_scatter_kernel<<<nblocks, kScanBlock, 0, stream>>>(n, ncolors, colors, order, bases, nblocks, perm,
                                                              perm_inv);
    if (precision == 0) {
        permuted_rows_kernel<float><<<grid_of(n, 256), 256, 0, stream>>>(n, rp, w, perm, len, static_cast<float *>(deg_out));
    } else {
        permuted_rows_kernel<double><<<grid_of(n, 256), 256, 0, stream>>>(n, rp, w, perm, len, static_cast<double *>(deg_out));
    }
    exclusive_scan_kernel<<<1, kScanBlock, 0, stream>>>(n, len, rp_out);
    if (precision == 0) {
        permuted_fill_kernel<float><<<grid_of(n, 256), 256, 0, stream>>>(n, rp, ci, w, perm, perm_inv, rp_out, ci_out,
                                                                          static_cast<float *>(w_out));
    } else {
        permuted_fill_kernel<double><<<grid_of(n, 256), 256, 0, stream>>>(n, rp, ci, w, perm, perm_inv, rp_out, ci_out,
                                                                           static_cast<double *>(w_out));
    }
    return cudaGetLastError();
}

}  // namespace gmrf
