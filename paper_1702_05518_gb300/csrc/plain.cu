// plain.cu -- the plain FP64 chromatic sweep: the reference point the fused, colour-split,
// batched path is measured against.  It is Algorithm 1 written the direct way for one field:
// the state stays in natural site order ([chain][site]), each colour step is one launch over
// all n sites in which the sites of other colours return at once, the two sums of the
// hyperparameter conditionals (Sec. 3.1) are a separate pass with FP64 atomics, and the draws a
// third launch.  Same counters and formulas as the fused path, so the two agree to rounding.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {
namespace {

// Neighbours of natural site `site` of a lattice; returns their count.
__device__ __forceinline__ int lattice_neighbours(int kind, const int32_t *dims, int64_t site, int64_t (&nb)[8])
{
    int cnt = 0;
    if (kind == kLat3D6) {
        const int64_t L = dims[0], H = dims[1], W = dims[2];
        const int64_t j = site % W, i = (site / W) % H, l = site / (W * H);
        if (l > 0) nb[cnt++] = site - H * W;
        if (i > 0) nb[cnt++] = site - W;
        if (j > 0) nb[cnt++] = site - 1;
        if (j + 1 < W) nb[cnt++] = site + 1;
        if (i + 1 < H) nb[cnt++] = site + W;
        if (l + 1 < L) nb[cnt++] = site + H * W;
        return cnt;
    }
    const int64_t H = dims[0], W = dims[1];
    const int64_t i = site / W, j = site % W;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
            if (di == 0 && dj == 0) continue;
            if (kind == kLat2D4 && di != 0 && dj != 0) continue;
            const int64_t ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
            nb[cnt++] = ii * W + jj;
        }
    return cnt;
}

__device__ __forceinline__ int lattice_colour(int kind, const int32_t *dims, int64_t site)
{
    if (kind == kLat3D6) {
        const int64_t W = dims[2], H = dims[1];
        return static_cast<int>(((site % W) + ((site / W) % H) + site / (W * H)) & 1);
    }
    const int64_t W = dims[1];
    const int64_t i = site / W, j = site % W;
    if (kind == kLat2D8) return static_cast<int>(2 * (i & 1) + (j & 1));
    return static_cast<int>((i + j) & 1);
}

__global__ void plain_colour_kernel(const PlainArgs a, int colour)
{
    const long long sweep = a.ctl->sweep;
    const int64_t total = static_cast<int64_t>(a.n) * a.C;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int chain = static_cast<int>(q / a.n);
        const int64_t i = q - static_cast<int64_t>(chain) * a.n;
        const int col = a.rp ? a.colors[i] : lattice_colour(a.kind, a.dims, i);
        if (col != colour) continue;
        const double *xc = a.x + static_cast<int64_t>(chain) * a.n;
        double s = 0.0, d = 0.0;
        if (a.rp) {
            for (int32_t e = a.rp[i]; e < a.rp[i + 1]; ++e) {
                const double wv = a.w ? a.w[e] : 1.0;
                s += wv * xc[a.ci[e]];
                d += wv;
            }
        } else {
            int64_t nb[8];
            const int cnt = lattice_neighbours(a.kind, a.dims, i, nb);
            for (int k = 0; k < cnt; ++k) s += xc[nb[k]];
            d = cnt;
        }
        const double tau = a.tau[chain], isig = 1.0 / a.sig2[chain];
        const double P = tau * d + isig;
        const double m = (tau * a.rho * s + a.y[i] * isig) / P;
        double z[1];
        site_normals<double, 1>(a.key, static_cast<uint32_t>(i), static_cast<uint32_t>(sweep), a.stream_id,
                                static_cast<uint32_t>(chain), a.lanes, z);
        a.x[static_cast<int64_t>(chain) * a.n + i] = m + z[0] / sqrt(P);
    }
}

// x'(D - rho W)x over undirected edges (each taken at its endpoint of larger index) and
// ||y - x||^2, accumulated into red[chain] with FP64 atomics.
__global__ void plain_reduce_kernel(const PlainArgs a)
{
    const int64_t total = static_cast<int64_t>(a.n) * a.C;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int chain = static_cast<int>(q / a.n);
        const int64_t i = q - static_cast<int64_t>(chain) * a.n;
        const double *xc = a.x + static_cast<int64_t>(chain) * a.n;
        const double xi = xc[i];
        double S = 0.0, d = 0.0;
        if (a.rp) {
            for (int32_t e = a.rp[i]; e < a.rp[i + 1]; ++e) {
                const double wv = a.w ? a.w[e] : 1.0;
                d += wv;
                if (a.ci[e] < i) {
                    const double df = xi - xc[a.ci[e]];
                    S += wv * df * df;
                }
            }
        } else {
            int64_t nb[8];
            const int cnt = lattice_neighbours(a.kind, a.dims, i, nb);
            for (int k = 0; k < cnt; ++k)
                if (nb[k] < i) {
                    const double df = xi - xc[nb[k]];
                    S += df * df;
                }
            d = cnt;
        }
        S = a.rho * S + (1.0 - a.rho) * d * xi * xi;
        const double r = a.y[i] - xi;
        atomicAdd(&a.red[chain * 2], S);
        atomicAdd(&a.red[chain * 2 + 1], r * r);
    }
}

__global__ void plain_hyper_kernel(const PlainArgs a)
{
    const long long sweep = a.ctl->sweep;
    for (int c = threadIdx.x; c < a.C; c += blockDim.x) {
        double tau = a.tau[c], sig2 = a.sig2[c];
        if (a.draw) {
            int fb1 = 0, fb2 = 0;
            tau = gamma_mt(a.a_tau + 0.5 * a.rank, a.b_tau + 0.5 * a.red[c * 2], a.key, static_cast<uint32_t>(sweep),
                           a.stream_id, (kTagTau << 24) | static_cast<uint32_t>(c), fb1);
            sig2 = 1.0 / gamma_mt(a.a_sig + 0.5 * a.n, a.b_sig + 0.5 * a.red[c * 2 + 1], a.key,
                                  static_cast<uint32_t>(sweep), a.stream_id, (kTagSig << 24) | static_cast<uint32_t>(c),
                                  fb2);
            if (fb1 + fb2)
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->fallbacks),
                          static_cast<unsigned long long>(fb1 + fb2));
            a.tau[c] = tau;
            a.sig2[c] = sig2;
        }
        a.red[c * 2] = 0.0;
        a.red[c * 2 + 1] = 0.0;
        if (a.trace_cap > 0) {
            a.trace_tau[static_cast<int64_t>(c) * a.trace_cap + sweep % a.trace_cap] = tau;
            a.trace_sig[static_cast<int64_t>(c) * a.trace_cap + sweep % a.trace_cap] = sig2;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) a.ctl->sweep = sweep + 1;
}

}  // namespace

cudaError_t launch_plain_sweep(const PlainArgs &a, cudaStream_t stream, int64_t *launches)
{
    const int64_t total = static_cast<int64_t>(a.n) * a.C;
    int64_t g = (total + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    for (int c = 0; c < a.ncolors; ++c) plain_colour_kernel<<<static_cast<int>(g), 256, 0, stream>>>(a, c);
    if (a.draw) plain_reduce_kernel<<<static_cast<int>(g), 256, 0, stream>>>(a);
    plain_hyper_kernel<<<1, 64, 0, stream>>>(a);
    if (launches) *launches = a.ncolors + (a.draw ? 2 : 1);
    return cudaGetLastError();
}

}  // namespace gmrf
