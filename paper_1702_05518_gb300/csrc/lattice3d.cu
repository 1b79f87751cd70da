// lattice3d.cu -- the colour step of 3-D 6-neighbour lattices under the parity colouring
// (Algorithm 1, steps 2-3, with the full conditionals of Sec. 3.1) for FP32 samplers of 4 or 8
// chains.  One thread updates every chain of a site:
//     s_i = sum of the six neighbours (all of the other colour),
//     P_i = tau d_i + 1/sigma^2,  m_i = (tau rho s_i + (y_i - beta0)/sigma^2) / P_i,
//     x_i = m_i + z_i / sqrt(P_i),
// so the site's index arithmetic, boundary mask and neighbour addresses serve all its chains,
// and its Philox blocks (counter (site, sweep, stream, g) for chains 4g .. 4g + 3) give exactly
// the normals of its chains: the per-update work is the random numbers, the loads and the
// update itself.  The state is HBM-resident (a 256^3 lattice with 8 chains holds 537 MB), so the
// kernel is built to stream it: one pass over the other colour's state and this colour's
// observations, one write of this colour's state.
//
// Layout (colour-split, chains innermost): the colour-c sites of sub-array row r = l*H + i are
// columns h = 0 .. cols-1 at j = 2h + p, p = (c + l + i) & 1; their neighbours are columns
// h - 1 + p and h + p of the other colour's row r and column h of its rows r -+ 1 and r -+ H.
//
// Work: block k of a field's nt blocks takes the sub-array rows k, k + nt, k + 2 nt, ...; a
// launch is one wave, so at any time all blocks work on a band of about nt rows, and each row
// of the other colour, which six sites of three rows and two planes read, comes from DRAM once.
// Colour 1 walks the rows from the end, so each colour step starts on the rows the previous
// step wrote last, which are still in L2.  A warp whose sites are all interior (six
// neighbours) takes a path without boundary masks, with m_i = a s_i + b (y_i - beta0) and
// a = tau rho / P, b = (1/sigma^2) / P, 1/sqrt(P) computed once per thread for d = 6; other
// warps compute them per site by the same operations, so a site's result does not depend on
// the path its warp took.
//
// Sums for the conjugate draws, per chain: colour 1 adds rho sum_k (x_i - x_k)^2 over its
// neighbours (all of lower colour, final by then), both colours add (1 - rho) d_i x_i^2 (proper
// prior only), (y_i - beta0 - x_i)^2 and, with the intercept, y_i - beta0 - x_i.  Summed over a
// sweep that is x'(D - rho W)x with every edge counted once.  Thread and block partial sums are
// FP32 (a few hundred sites per thread at most), the block's sums are stored in FP64 and summed
// over blocks in FP64 by the draw kernel, each in a fixed order.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {
namespace {

constexpr int k3Block = 256;

__device__ __forceinline__ void ld4(const float *p, float *v)
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}

__device__ __forceinline__ void st4(float *p, const float *v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Per chain parameters of the launch, in shared memory: tau, tau rho, 1/sigma^2, beta0, and the
// interior coefficients (d = 6) tau rho / P, (1/sigma^2) / P, 1/sqrt(P).
template <int NC>
struct alignas(16) Params3 {
    float tau[NC], tr[NC], isig[NC], beta[NC];
    float ca[NC], cb[NC], crs[NC];
};

// Per-thread partial sums.
template <int NC>
struct Acc3 {
    float S[NC], R[NC], A[NC];
};

struct Site3 {
    const float *xo;   // the other colour's slot of this site's column in row r
    float *xs, *ms, *qs;
    int64_t noff[6];   // neighbour offsets from xo (floats)
    uint32_t valid;    // neighbours present (bit k: noff[k])
    uint32_t site;     // natural site index
    float y, d;
};

// Update chain groups G0 .. G0 + GN - 1 (four chains each) of one site.
template <int NC, int G0, int GN, bool ODD, bool ICPT, bool PCAR, bool INTERIOR>
__device__ __forceinline__ void site_groups(const StepArgs &a, const Params3<NC> &pp, Acc3<NC> &ac, const Site3 &st,
                                            uint32_t sweep, uint32_t stream, bool update, bool acc, float inv_k,
                                            float rho, float om)
{
    constexpr int M = 4 * GN;
    float nb[6][M];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (INTERIOR || ((st.valid >> k) & 1u)) {
#pragma unroll
            for (int g = 0; g < GN; ++g) ld4(st.xo + st.noff[k] + 4 * (G0 + g), &nb[k][4 * g]);
        } else {
#pragma unroll
            for (int v = 0; v < M; ++v) nb[k][v] = 0.0f;
        }
    }
    float x[M];
    if (update) {
        float z[M];
#pragma unroll
        for (int g = 0; g < GN; ++g) {
            const uint4 w = philox4x32_10(make_uint4(st.site, sweep, stream, (kTagX << 24) | (G0 + g)), a.key);
            box_muller_f32(w.x, w.y, z[4 * g], z[4 * g + 1]);
            box_muller_f32(w.z, w.w, z[4 * g + 2], z[4 * g + 3]);
        }
#pragma unroll
        for (int u = 0; u < M; ++u) {
            const int v = 4 * G0 + u;
            float s = nb[0][u];
#pragma unroll
            for (int k = 1; k < 6; ++k) s += nb[k][u];
            float ca, cb, crs;
            if (INTERIOR) {
                ca = pp.ca[v];
                cb = pp.cb[v];
                crs = pp.crs[v];
            } else {
                const float P = fmaf(pp.tau[v], st.d, pp.isig[v]);
                const float rP = rcp_approx(P);
                ca = pp.tr[v] * rP;
                cb = pp.isig[v] * rP;
                crs = rsqrt_approx(P);
            }
            const float yb = ICPT ? st.y - pp.beta[v] : st.y;
            x[u] = fmaf(z[u], crs, fmaf(ca, s, yb * cb));
        }
#pragma unroll
        for (int g = 0; g < GN; ++g) st4(st.xs + 4 * (G0 + g), &x[4 * g]);
    } else {
#pragma unroll
        for (int g = 0; g < GN; ++g) ld4(st.xs + 4 * (G0 + g), &x[4 * g]);
    }
#pragma unroll
    for (int u = 0; u < M; ++u) {
        const int v = 4 * G0 + u;
        float sv = 0.0f;
        if (ODD) {
            float ev = 0.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (INTERIOR || ((st.valid >> k) & 1u)) {
                    const float df = x[u] - nb[k][u];
                    ev = fmaf(df, df, ev);
                }
            }
            sv = PCAR ? rho * ev : ev;
        }
        if (PCAR) sv = fmaf(om * st.d * x[u], x[u], sv);
        if (ODD || PCAR) ac.S[v] += sv;
        const float res = (ICPT ? st.y - pp.beta[v] : st.y) - x[u];
        ac.R[v] = fmaf(res, res, ac.R[v]);
        if (ICPT) ac.A[v] += res;
    }
    if (acc) {
#pragma unroll
        for (int g = 0; g < GN; ++g) {
            float mu[4], mm[4];
            ld4(st.ms + 4 * (G0 + g), mu);
            ld4(st.qs + 4 * (G0 + g), mm);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float xv = x[4 * g + u];
                const float delta = xv - mu[u];
                mu[u] = fmaf(delta, inv_k, mu[u]);
                mm[u] = fmaf(delta, xv - mu[u], mm[u]);
            }
            st4(st.ms + 4 * (G0 + g), mu);
            st4(st.qs + 4 * (G0 + g), mm);
        }
    }
}

// NG: groups of four chains (Cp = 4 NG); ODD: the launch updates colour 1 (whose neighbours are
// all of lower colour); ICPT: the model has the intercept; PCAR: rho < 1.
template <int NG, bool ODD, bool ICPT, bool PCAR>
__global__ void __launch_bounds__(k3Block, 2) lattice3d_kernel(const StepArgs a)
{
    constexpr int NC = 4 * NG;
    __shared__ Params3<NC> pp;
    __shared__ float red[k3Block / 32][NC][3];
    pdl_wait_then_release();
    const Tile t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const long long sweep_ll = a.ctl->sweep;
    const uint32_t sweep = static_cast<uint32_t>(sweep_ll);
    const float rho = static_cast<float>(a.rho);
    const float om = 1.0f - rho;
    if (threadIdx.x < NC) {
        const int v = threadIdx.x;
        const float *hyp = static_cast<const float *>(a.hyp) + (static_cast<int64_t>(t.field) * NC + v) * kHypStride;
        pp.tau[v] = hyp[0];
        pp.tr[v] = PCAR ? hyp[0] * rho : hyp[0];
        pp.isig[v] = hyp[1];
        pp.beta[v] = ICPT ? hyp[2] : 0.0f;
        // the operations of the boundary path at d = 6
        const float P = fmaf(pp.tau[v], 6.0f, pp.isig[v]);
        const float rP = rcp_approx(P);
        pp.ca[v] = pp.tr[v] * rP;
        pp.cb[v] = pp.isig[v] * rP;
        pp.crs[v] = rsqrt_approx(P);
    }
    __syncthreads();
    Acc3<NC> ac;
#pragma unroll
    for (int v = 0; v < NC; ++v) {
        ac.S[v] = 0.0f;
        ac.R[v] = 0.0f;
        ac.A[v] = 0.0f;
    }
    const bool update = a.update != 0;
    bool acc = false;
    float inv_k = 0.0f;
    if (update && a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin)) {
        acc = true;
        inv_k = 1.0f / static_cast<float>(a.ctl->acc_count + 1);
    }

    const int L = f.dims[0], H = f.dims[1], W = f.dims[2];
    const int cols = f.cols;
    constexpr int c = ODD ? 1 : 0;
    const int64_t sub = static_cast<int64_t>(f.rows) * cols;
    const float *XO = static_cast<const float *>(a.x) + (f.slot0 + (1 - c) * sub) * NC;
    float *XS = static_cast<float *>(a.x) + (f.slot0 + c * sub) * NC;
    float *MS = static_cast<float *>(a.mean) + (f.slot0 + c * sub) * NC;
    float *QS = static_cast<float *>(a.m2) + (f.slot0 + c * sub) * NC;
    const float *YS = static_cast<const float *>(a.y) + f.slot0 + c * sub;
    const int64_t off_row = static_cast<int64_t>(cols) * NC;
    const int64_t off_plane = static_cast<int64_t>(H) * cols * NC;
    const int stride = t.stride > 1 ? t.stride : 1;
    const int nelem = t.count * cols;

    for (int q = threadIdx.x; q < nelem; q += k3Block) {
        const int e = ODD ? nelem - 1 - q : q;
        const int m = fast_div(e, f.cols_m, f.cols_s);
        const int h = e - m * cols;
        const int r = t.start + m * stride;
        const int l = fast_div(r, f.h_m, f.h_s);
        const int i = r - l * H;
        const int p = (c + l + i) & 1;
        const int j = 2 * h + p;
        const bool ok = j < W;
        const uint32_t valid = (j > 0 ? 1u : 0u) | (j + 1 < W ? 2u : 0u) | (i > 0 ? 4u : 0u) |
                               (i + 1 < H ? 8u : 0u) | (l > 0 ? 16u : 0u) | (l + 1 < L ? 32u : 0u);
        const bool interior = __all_sync(__activemask(), valid == 63u || !ok);
        if (!ok)
            continue;
        Site3 st;
        const int64_t rb = static_cast<int64_t>(r) * cols + h;
        st.xo = XO + rb * NC;
        st.xs = XS + rb * NC;
        st.ms = MS + rb * NC;
        st.qs = QS + rb * NC;
        st.noff[0] = static_cast<int64_t>(p - 1) * NC;
        st.noff[1] = static_cast<int64_t>(p) * NC;
        st.noff[2] = -off_row;
        st.noff[3] = off_row;
        st.noff[4] = -off_plane;
        st.noff[5] = off_plane;
        st.valid = valid;
        st.site = static_cast<uint32_t>(r) * static_cast<uint32_t>(W) + static_cast<uint32_t>(j);
        st.y = YS[rb];
        st.d = static_cast<float>(__popc(valid));
        if (interior)
            site_groups<NC, 0, NG, ODD, ICPT, PCAR, true>(a, pp, ac, st, sweep, f.stream, update, acc, inv_k, rho, om);
        else
            site_groups<NC, 0, NG, ODD, ICPT, PCAR, false>(a, pp, ac, st, sweep, f.stream, update, acc, inv_k, rho, om);
    }

    // Block sums per chain: a shuffle tree over the warp's lanes, then the warps in order.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NC; ++v) {
        float sS = ac.S[v], sR = ac.R[v], sA = ac.A[v];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            if (ODD || PCAR) sS += __shfl_xor_sync(0xffffffffu, sS, off);
            sR += __shfl_xor_sync(0xffffffffu, sR, off);
            if (ICPT) sA += __shfl_xor_sync(0xffffffffu, sA, off);
        }
        if (lane == 0) {
            red[warp][v][0] = sS;
            red[warp][v][1] = sR;
            red[warp][v][2] = sA;
        }
    }
    __syncthreads();
    if (threadIdx.x < NC * 3) {
        const int chain = threadIdx.x / 3, k = threadIdx.x - 3 * chain;
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < k3Block / 32; ++w) s += red[w][chain][k];
        double *dst = reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * NC + chain);
        dst[k] = static_cast<double>(s);
    }
}

template <int NG, bool ICPT, bool PCAR>
cudaError_t launch_v(bool odd, const StepArgs &a, cudaStream_t stream)
{
    if (odd)
        return launch_sweep_kernel(lattice3d_kernel<NG, true, ICPT, PCAR>, dim3(a.ntiles), dim3(k3Block), 0, stream, a);
    return launch_sweep_kernel(lattice3d_kernel<NG, false, ICPT, PCAR>, dim3(a.ntiles), dim3(k3Block), 0, stream, a);
}

template <int NG>
cudaError_t launch_model3d(bool odd, bool icpt, bool pcar, const StepArgs &a, cudaStream_t stream)
{
    if (icpt) return pcar ? launch_v<NG, true, true>(odd, a, stream) : launch_v<NG, true, false>(odd, a, stream);
    return pcar ? launch_v<NG, false, true>(odd, a, stream) : launch_v<NG, false, false>(odd, a, stream);
}

template <int NG>
cudaError_t occupancy(int *blocks)
{
    // the colour-1 kernel with the intercept and the proper prior holds the most registers
    int b0 = 0, b1 = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, lattice3d_kernel<NG, true, true, true>, k3Block, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, lattice3d_kernel<NG, false, false, false>, k3Block, 0);
    *blocks = b0 < b1 ? b0 : b1;
    if (*blocks < 1) *blocks = 1;
    return e;
}

}  // namespace

cudaError_t launch_lattice3d(int chains_padded, const StepArgs &a, cudaStream_t stream)
{
    if (a.ntiles <= 0) return cudaSuccess;
    const bool odd = a.colour == 1, icpt = a.intercept != 0, pcar = a.rho != 1.0;
    if (chains_padded == 8) return launch_model3d<2>(odd, icpt, pcar, a, stream);
    return launch_model3d<1>(odd, icpt, pcar, a, stream);
}

cudaError_t lattice3d_blocks_per_sm(int chains_padded, int *blocks)
{
    if (chains_padded == 8) return occupancy<2>(blocks);
    return occupancy<1>(blocks);
}

}  // namespace gmrf
