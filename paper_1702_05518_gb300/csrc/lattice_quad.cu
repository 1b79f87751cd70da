// lattice_quad.cu -- one launch per sweep for single-chain 8-neighbour lattices in single
// precision, with a fixed thread-to-site map.
//
// The 2 x 2 colouring c = 2 (i & 1) + (j & 1) of the 8-neighbour lattice puts one site of each
// colour in every aligned 2 x 2 block of sites (a "quad").  In the colour-split layout quad
// (u, v) is slot (u, v) of all four sub-arrays.  A block owns a TR x TC tile of sites, stages
// the tile plus a halo of 4 sites (2 quads) into shared memory, and every thread keeps the same
// quads through the whole sweep: it stages them, draws their four normals into registers, draws
// its colour-c site of each quad at colour step c (Algorithm 1; step c covers the tile grown by
// 3 - c sites, so the owned sites end exact, as in lattice_fused.cu), and writes back the owned
// ones.  Consecutive threads hold consecutive quads of a row, so every shared-memory access of
// a warp is to consecutive words, and the eight neighbour offsets of each colour are constants.
//
// Normals (the layout of include/gmrf.h with one chain: a Philox block serves 4 consecutive
// sites of a row, site s taking normal s mod 4).  With the row length W a multiple of 4 and the
// staged origin at a column multiple of 4, the two quads of a lane pair (v even, v + 1) cover
// the four columns of one Philox block in each of their two rows.  The even lane draws the block
// of the upper row and the odd lane that of the lower row; each passes the other the two words
// it needs (one shuffle pair) and both run two Box-Muller pairs: four normals per quad and one
// Philox block per quad, with no shared-memory traffic.
//
// Overlap with the previous sweep's hyperparameter draw: the kernel is launched as a
// programmatic dependent of that draw, so it may start while the draw runs.  Before waiting on
// it, it stages the observations (constant) and draws the normals for the predicted sweep number
// (the previous sweep kernel's number + 1); after the wait it reads the real number and draws
// the normals again in the rare case the prediction was wrong (a reset, or stages launched
// one by one), so the results never depend on the prediction.
#include <cuda_runtime.h>

#include "gmrf_device.cuh"
#include "gmrf_internal.h"
#include "hyper_task.cuh"
#include "grid_barrier.cuh"

namespace gmrf {
namespace {

// Direction k of the 8-neighbour stencil: (di, dj) row by row.
__host__ __device__ constexpr int qdi(int k) { return k < 3 ? -1 : (k < 5 ? 0 : 1); }
__host__ __device__ constexpr int qdj(int k) { return k < 3 ? k - 1 : (k == 3 ? -1 : (k == 4 ? 1 : k - 6)); }
// Colour-(a, b) site, direction k: sub-array of the neighbour and its quad offset (floor halves).
__host__ __device__ constexpr int qsub(int a, int b, int k) { return 2 * ((a + qdi(k)) & 1) + ((b + qdj(k)) & 1); }
__host__ __device__ constexpr int qdu(int a, int k) { return (a + qdi(k)) >= 0 ? (a + qdi(k)) / 2 : -1; }
__host__ __device__ constexpr int qdv(int b, int k) { return (b + qdj(k)) >= 0 ? (b + qdj(k)) / 2 : -1; }

struct QuadCtx {
    float tau, isig, beta, rho;
    float accS, accR, accA;
    // Write-back of the owned sites, issued right after their colour step: the state buffer of
    // the next sweep and, in accumulated sweeps, the running mean and M2 (Welford, from the
    // shared-memory copies ms, m2s).
    float *XW, *MEAN, *M2;
    float *ms, *m2s;
    int gsub, gcols, gu0, gv0;
    bool acc;
    float inv_k;
};

// Colour step C for the thread's quads.  RES (the resident kernel): the running moments stay in
// shared memory (ms, m2s) instead of going to global memory.
template <int C, int QCS, int NQ, int NT, bool RES = false>
__device__ __forceinline__ void quad_colour_step(float *xs, const float *ys, int SUB, const float (&z)[NQ][4],
                                                 int gi0, int gj0, int Hl, int Wl, int lo_i, int hi_i, int lo_j,
                                                 int hi_j, int own_i0, int own_i1, int own_j0, int own_j1,
                                                 bool interior, int nquads, QuadCtx &cx)
{
    constexpr int A = C >> 1, B = C & 1;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int q = threadIdx.x + k * NT;
        if (q >= nquads) break;
        const int u = q / QCS, v = q % QCS;
        const int i = gi0 + 2 * u + A, j = gj0 + 2 * v + B;
        if (i < lo_i || i >= hi_i || j < lo_j || j >= hi_j) continue;
        const int base = u * QCS + v;
        float nb[8];
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            nb[d] = xs[qsub(A, B, d) * SUB + base + qdu(A, d) * QCS + qdv(B, d)];
            s += nb[d];
        }
        float deg = 8.0f;
        uint32_t valid = 0xffu;
        if (!interior && (i == 0 || j == 0 || i == Hl - 1 || j == Wl - 1)) {
            valid = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int ii = i + qdi(d), jj = j + qdj(d);
                valid |= (ii >= 0 && ii < Hl && jj >= 0 && jj < Wl) ? (1u << d) : 0u;
            }
            deg = static_cast<float>(__popc(valid));
        }
        const float yb = ys[C * SUB + base] - cx.beta;
        const float P = cx.tau * deg + cx.isig;
        const float m = (cx.tau * cx.rho * s + yb * cx.isig) * rcp_approx(P);
        const float x = m + z[k][C] * rsqrt_approx(P);
        xs[C * SUB + base] = x;
        if (i >= own_i0 && i < own_i1 && j >= own_j0 && j < own_j1) {
            float e2 = 0.0f;
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                if (qsub(A, B, d) < C) {  // neighbour of lower colour: final before this step
                    const float df = x - nb[d];
                    e2 += ((valid >> d) & 1u) ? df * df : 0.0f;
                }
            }
            cx.accS += (1.0f - cx.rho) * deg * x * x + cx.rho * e2;
            const float r = yb - x;
            cx.accR += r * r;
            cx.accA += r;
            // The site is final for this sweep: its stores leave now and drain under the later
            // steps (all blocks storing at the end of the kernel would queue behind each other).
            const int go = C * cx.gsub + (cx.gu0 + u) * cx.gcols + cx.gv0 + v;
            cx.XW[go] = x;
            if (cx.acc) {
                const float mu = cx.ms[C * SUB + base], mm = cx.m2s[C * SUB + base];
                const float delta = x - mu;
                const float m1 = mu + delta * cx.inv_k;
                const float m2 = mm + delta * (x - m1);
                if (RES) {
                    cx.ms[C * SUB + base] = m1;
                    cx.m2s[C * SUB + base] = m2;
                } else {
                    cx.MEAN[go] = m1;
                    cx.M2[go] = m2;
                }
            }
        }
    }
}

// Whether site s (sub-array s = 2a + b) of staged quad (u, v) is owned by the tile and on the
// lattice.
__device__ __forceinline__ bool quad_owned_site(int u, int v, int s, int QR, int TC, int gu0, int gv0, int Hl, int Wl)
{
    if (u < 2 || u >= QR - 2 || v < 2 || v >= 2 + TC / 2) return false;
    return 2 * (gu0 + u) + (s >> 1) < Hl && 2 * (gv0 + v) + (s & 1) < Wl;
}

// Normals of the thread's quads for sweep `sweep` (z[k][c]: the colour-c site of quad k).  Every
// lane of the warp takes part (the lane pairs exchange words), whether or not its quads exist.
template <int QCS, int NT, int NQ>
__device__ __forceinline__ void quad_normals(float (&z)[NQ][4], uint2 key, uint32_t sweep, uint32_t stream,
                                             uint32_t blocks_per_row, int gu0, int gv0)
{
    const bool odd = threadIdx.x & 1;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int q = threadIdx.x + k * NT;  // the partner lane holds q ^ 1 (NT even, QCS even)
        const int u = q / QCS, v = q % QCS;
        const int row = 2 * (gu0 + u) + (odd ? 1 : 0);
        const int grp = (gv0 + (v & ~1)) >> 1;  // column group: natural columns 4 grp .. 4 grp + 3
        const uint32_t blk = static_cast<uint32_t>(row) * blocks_per_row + static_cast<uint32_t>(grp);
        const uint4 w = philox4x32_10(make_uint4(blk, sweep, stream, kTagX << 24), key);
        // even lane: keeps (w0, w1) of the upper row, gets (w0, w1) of the lower row;
        // odd lane: keeps (w2, w3) of the lower row, gets (w2, w3) of the upper row.
        const uint32_t p0 = __shfl_xor_sync(0xffffffffu, odd ? w.x : w.z, 1);
        const uint32_t p1 = __shfl_xor_sync(0xffffffffu, odd ? w.y : w.w, 1);
        float c0, s0, c1, s1;
        box_muller_f32(odd ? w.z : w.x, odd ? w.w : w.y, c0, s0);  // own row
        box_muller_f32(p0, p1, c1, s1);                          // partner's row
        // colour c = 2a + b: row a (0 upper, 1 lower), column b within the lane's two columns
        z[k][0] = odd ? c1 : c0;
        z[k][1] = odd ? s1 : s0;
        z[k][2] = odd ? c0 : c1;
        z[k][3] = odd ? s0 : s1;
    }
}

template <int QCS, int NT, int NQ>
__global__ void __launch_bounds__(NT, 1) lattice_quad_kernel(const FusedArgs a)
{
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileXY t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const int Hl = f.dims[0], Wl = f.dims[1];
    const int TR = a.TR, TC = a.TC;
    const int QR = TR / 2 + 4;         // staged quad rows
    const int SUB = QR * QCS;          // slots per staged sub-array
    const int nquads = SUB;
    float *xs = reinterpret_cast<float *>(smem_raw);  // [4][QR][QCS]
    float *ys = xs + 4 * SUB;                         // [4][QR][QCS]
    float *ms = ys + 4 * SUB;                         // [4][QR][QCS] running mean of owned sites
    float *m2s = ms + 4 * SUB;                        // [4][QR][QCS] running M2 of owned sites
    const int gi0 = t.i0 - 4, gj0 = t.j0 - 4;        // staged origin (site units, even / multiple of 4)
    const int gu0 = gi0 >> 1, gv0 = gj0 >> 1;         // in quads
    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + 2 * QR <= Hl && gj0 + 2 * QCS <= Wl;
    const float *Y = static_cast<const float *>(a.y) + f.slot0;
    const int gsub = f.rows * f.cols, gcols = f.cols;

    // Before the wait: observations (never written by a sweep) and the normals of the predicted
    // sweep.
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int q = threadIdx.x + k * NT;
        if (q >= nquads) break;
        const int u = q / QCS, v = q % QCS;
        const int gu = gu0 + u, gv = gv0 + v;
        const int go = gu * gcols + gv;
        float yv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = 2 * gu + (s >> 1), j = 2 * gv + (s & 1);
            const bool ok = interior || (gu >= 0 && gv >= 0 && i < Hl && j < Wl);
            yv[s] = ok ? Y[s * gsub + go] : 0.0f;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) ys[s * SUB + q] = yv[s];
    }
    // The prediction: thread 0 reads it and counts the block; the last block to read it
    // replaces it (after the wait) with this sweep's number + 1.
    __shared__ long long s_pred;
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        s_pred = *reinterpret_cast<volatile const long long *>(&a.ctl->fnext);
        s_last = atomicAdd(&a.ctl->fticket, 1ull) == gridDim.x - 1;
    }
    __syncthreads();
    const long long predicted = s_pred;
    float z[NQ][4];
    quad_normals<QCS, NT, NQ>(z, a.key, static_cast<uint32_t>(predicted), f.stream, static_cast<uint32_t>(Wl) >> 2, gu0,
                              gv0);

    pdl_wait();
    const long long sweep_ll = a.ctl->sweep;
    if (threadIdx.x == 0 && s_last) {  // the next launch's prediction, before it may start
        a.ctl->fnext = sweep_ll + 1;
        a.ctl->fticket = 0;
        if (sweep_ll != predicted) a.ctl->fmiss += 1;
    }
    pdl_release();
    if (sweep_ll != predicted)
        quad_normals<QCS, NT, NQ>(z, a.key, static_cast<uint32_t>(sweep_ll), f.stream, static_cast<uint32_t>(Wl) >> 2,
                                  gu0, gv0);
    const float *X = static_cast<const float *>((sweep_ll & 1) ? a.x_alt : a.x) + f.slot0;
    float *XW = static_cast<float *>((sweep_ll & 1) ? a.x : a.x_alt) + f.slot0;
    QuadCtx cx;
    {
        const float *hyp = static_cast<const float *>(a.hyp) + static_cast<int64_t>(t.field) * kHypStride;
        cx.tau = hyp[0];
        cx.isig = hyp[1];
        cx.beta = hyp[2];
        cx.rho = static_cast<float>(a.rho);
        cx.accS = 0.0f;
        cx.accR = 0.0f;
        cx.accA = 0.0f;
    }

    // The running moments of accumulated sweeps: asynchronous copies (cp.async) of the thread's
    // owned sites into shared memory now, waited for (by this thread only, which alone reads
    // them) at the write-back, so their latency runs under the colour steps.
    const bool acc = a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin);
    const float inv_k = acc ? 1.0f / static_cast<float>(a.ctl->acc_count + 1) : 0.0f;
    float *MEAN = static_cast<float *>(a.mean) + f.slot0;
    float *M2 = static_cast<float *>(a.m2) + f.slot0;
    if (acc) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int q = threadIdx.x + k * NT;
            const int u = q / QCS, v = q % QCS;
            const int go = (gu0 + u) * gcols + gv0 + v;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!(q < nquads && quad_owned_site(u, v, s, QR, TC, gu0, gv0, Hl, Wl))) continue;
                const uint32_t dm = static_cast<uint32_t>(__cvta_generic_to_shared(ms + s * SUB + q));
                const uint32_t d2 = static_cast<uint32_t>(__cvta_generic_to_shared(m2s + s * SUB + q));
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dm), "l"(MEAN + s * gsub + go) : "memory");
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d2), "l"(M2 + s * gsub + go) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // Stage the state of the thread's quads: slot (u, v) of the four sub-arrays; sites off the
    // lattice are 0.
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int q = threadIdx.x + k * NT;
        if (q >= nquads) break;
        const int u = q / QCS, v = q % QCS;
        const int gu = gu0 + u, gv = gv0 + v;
        const int go = gu * gcols + gv;
        float xv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = 2 * gu + (s >> 1), j = 2 * gv + (s & 1);
            const bool ok = interior || (gu >= 0 && gv >= 0 && i < Hl && j < Wl);
            xv[s] = ok ? X[s * gsub + go] : 0.0f;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) xs[s * SUB + q] = xv[s];
    }
    cx.XW = XW;
    cx.MEAN = MEAN;
    cx.M2 = M2;
    cx.ms = ms;
    cx.m2s = m2s;
    cx.gsub = gsub;
    cx.gcols = gcols;
    cx.gu0 = gu0;
    cx.gv0 = gv0;
    cx.acc = acc;
    cx.inv_k = inv_k;
    if (acc) asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's copies of the moments
    __syncthreads();

    // Colour steps 0..3; step c covers the tile grown by 3 - c sites (clipped to the lattice);
    // each step writes back its owned sites.
    const int own_i0 = t.i0, own_i1 = min(Hl, t.i0 + TR), own_j0 = t.j0, own_j1 = min(Wl, t.j0 + TC);
#define GMRF_QUAD_STEP(C)                                                                                        \
    quad_colour_step<C, QCS, NQ, NT>(xs, ys, SUB, z, gi0, gj0, Hl, Wl, max(0, t.i0 - (3 - C)),                \
                                     min(Hl, t.i0 + TR + (3 - C)), max(0, t.j0 - (3 - C)),                     \
                                     min(Wl, t.j0 + TC + (3 - C)), own_i0, own_i1, own_j0, own_j1, interior, \
                                     nquads, cx);                                                              \
    __syncthreads();
    GMRF_QUAD_STEP(0)
    GMRF_QUAD_STEP(1)
    GMRF_QUAD_STEP(2)
    GMRF_QUAD_STEP(3)
#undef GMRF_QUAD_STEP

    // Block reduction: warp shuffle tree, then the warps' sums in order (the last colour step
    // ended with a barrier, so the observations are dead).
    float *red = ys;  // [NW][3], the observations are dead
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float sS = cx.accS, sR = cx.accR, sA = cx.accA;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        sS += __shfl_xor_sync(0xffffffffu, sS, o);
        sR += __shfl_xor_sync(0xffffffffu, sR, o);
        sA += __shfl_xor_sync(0xffffffffu, sA, o);
    }
    if (lane == 0) {
        red[warp * 3] = sS;
        red[warp * 3 + 1] = sR;
        red[warp * 3 + 2] = sA;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float sum = 0.0f;
        for (int w = 0; w < NW; ++w) sum += red[w * 3 + threadIdx.x];
        reinterpret_cast<double *>(a.partials + t.part)[threadIdx.x] = static_cast<double>(sum);
    }
}

constexpr int kQuadResGpre = 128;

// The resident form of the quad sweep: `count` whole sweeps of the single field in one
// cooperative launch (every block resident at once), the tile of each block kept in shared
// memory from sweep to sweep.  Per sweep:
//   * the four colour steps as in lattice_quad_kernel (the owned sites go to the next sweep's
//     state buffer right after their step; the running moments of accumulated sweeps stay in
//     shared memory until the end of the launch);
//   * the block's sums (as in lattice_quad_kernel) to its tile partial, then a grid barrier: one
//     arrival per block on a counter in the sweep control block; while the other blocks finish,
//     the threads draw their normals of the next sweep;
//   * every block then draws tau | x (warp 0) and beta0, sigma^2 (warp 1) from all the tile
//     partials, summed in the order of the hyperparameter kernel and drawn by hyper_draw with the
//     batch's precomputed variates, so each block holds the values the per-sweep path would have;
//     block 0 alone stores them and the traces;
//   * the halo (the two quad rows and columns around the tile), which the neighbouring tiles
//     have just written, is staged again from global memory through L2.
// The state buffers alternate by sweep number as on the per-sweep path, so a block that writes
// sweep t + 1's state never overwrites what a slower block may still read for sweep t.  A wait at
// the barrier gives up after `wait_ns`: the block counts it in ctl->wait_timeouts and sets
// ctl->gabort, at which every block leaves its sweep loop.
template <int QCS, int NT, int NQ>
__global__ void __launch_bounds__(NT, 1) lattice_quad_resident_kernel(const TileResArgs ra)
{
    constexpr int NW = NT / 32;
    const FusedArgs &a = ra.f;
    const HyperArgs &h = ra.h;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[NW][3];
    __shared__ float hs[3];        // tau, 1/sigma^2, beta0 of the current sweep (FP32 copies)
    __shared__ double dcur[2];     // tau and sigma^2 (FP64) as last drawn
    __shared__ int s_abort;
    // the precomputed variates of the launch's first kQuadResGpre sweeps: tau's and 1/sigma^2's
    // unit-rate Gamma variates and the intercept's normal
    __shared__ double gsh[kQuadResGpre][3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TileXY t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const int Hl = f.dims[0], Wl = f.dims[1];
    const int TR = a.TR, TC = a.TC;
    const int QR = TR / 2 + 4;
    const int SUB = QR * QCS;
    const int nquads = SUB;
    float *xs = reinterpret_cast<float *>(smem_raw);
    float *ys = xs + 4 * SUB;
    float *ms = ys + 4 * SUB;
    float *m2s = ms + 4 * SUB;
    const int gi0 = t.i0 - 4, gj0 = t.j0 - 4;
    const int gu0 = gi0 >> 1, gv0 = gj0 >> 1;
    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + 2 * QR <= Hl && gj0 + 2 * QCS <= Wl;
    const int gsub = f.rows * f.cols, gcols = f.cols;
    SweepCtl *ctl = a.ctl;
    const long long sweep0 = ctl->sweep;
    long long acc_count = ctl->acc_count;
    const long long bbase = ctl->batch_base, bcount = ctl->batch_count;
    const float *Y = static_cast<const float *>(a.y) + f.slot0;
    const float *X0 = static_cast<const float *>((sweep0 & 1) ? a.x_alt : a.x) + f.slot0;
    float *MEAN = static_cast<float *>(a.mean) + f.slot0;
    float *M2 = static_cast<float *>(a.m2) + f.slot0;

    // Stage the observations, the state and (owned sites) the running moments once.
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int q = tid + k * NT;
        if (q >= nquads) break;
        const int u = q / QCS, v = q % QCS;
        const int gu = gu0 + u, gv = gv0 + v;
        const int go = gu * gcols + gv;
        float yv[4], xv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = 2 * gu + (s >> 1), j = 2 * gv + (s & 1);
            const bool ok = interior || (gu >= 0 && gv >= 0 && i < Hl && j < Wl);
            yv[s] = ok ? Y[s * gsub + go] : 0.0f;
            xv[s] = ok ? X0[s * gsub + go] : 0.0f;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            ys[s * SUB + q] = yv[s];
            xs[s * SUB + q] = xv[s];
            if (a.acc_enabled && quad_owned_site(u, v, s, QR, TC, gu0, gv0, Hl, Wl)) {
                ms[s * SUB + q] = MEAN[s * gsub + go];
                m2s[s * SUB + q] = M2[s * gsub + go];
            }
        }
    }
    if (tid < 3) hs[tid] = static_cast<const float *>(a.hyp)[static_cast<int64_t>(t.field) * kHypStride + tid];
    for (int q = tid; q < 3 * min(ra.count, kQuadResGpre); q += NT) {
        const long long kb = sweep0 + q / 3 - bbase;
        gsh[q / 3][q % 3] = (h.gpre && kb >= 0 && kb < bcount) ? h.gpre[kb * h.nfields * h.Cp * 4 + q % 3] : 0.0;
    }
    if (tid == 0) {
        dcur[0] = h.tau[0];
        dcur[1] = h.sig2[0];
        s_abort = 0;
    }
    float z[NQ][4];
    quad_normals<QCS, NT, NQ>(z, a.key, static_cast<uint32_t>(sweep0), f.stream, static_cast<uint32_t>(Wl) >> 2, gu0,
                              gv0);
    const int own_i0 = t.i0, own_i1 = min(Hl, t.i0 + TR), own_j0 = t.j0, own_j1 = min(Wl, t.j0 + TC);
    const unsigned long long nblk = gridDim.x;

    for (int it = 0; it < ra.count; ++it) {
        const long long sw = sweep0 + it;
        __syncthreads();  // the staged state (halo) and the sweep's parameters
        QuadCtx cx;
        cx.tau = hs[0];
        cx.isig = hs[1];
        cx.beta = hs[2];
        cx.rho = static_cast<float>(a.rho);
        cx.accS = 0.0f;
        cx.accR = 0.0f;
        cx.accA = 0.0f;
        float *XW = static_cast<float *>((sw & 1) ? a.x : a.x_alt) + f.slot0;
        cx.XW = XW;
        cx.MEAN = MEAN;
        cx.M2 = M2;
        cx.ms = ms;
        cx.m2s = m2s;
        cx.gsub = gsub;
        cx.gcols = gcols;
        cx.gu0 = gu0;
        cx.gv0 = gv0;
        cx.acc = a.acc_enabled && sweep_accumulated(sw, a.burn_in, a.thin);
        cx.inv_k = cx.acc ? 1.0f / static_cast<float>(acc_count + 1) : 0.0f;
#define GMRF_QUAD_STEP(C)                                                                                        \
    quad_colour_step<C, QCS, NQ, NT, true>(xs, ys, SUB, z, gi0, gj0, Hl, Wl, max(0, t.i0 - (3 - C)),          \
                                           min(Hl, t.i0 + TR + (3 - C)), max(0, t.j0 - (3 - C)),               \
                                           min(Wl, t.j0 + TC + (3 - C)), own_i0, own_i1, own_j0, own_j1,       \
                                           interior, nquads, cx);                                               \
    __syncthreads();
        GMRF_QUAD_STEP(0)
        GMRF_QUAD_STEP(1)
        GMRF_QUAD_STEP(2)
        GMRF_QUAD_STEP(3)
#undef GMRF_QUAD_STEP
        if (cx.acc) ++acc_count;

        // The tile's sums, in the order of lattice_quad_kernel.
        float sS = cx.accS, sR = cx.accR, sA = cx.accA;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            sS += __shfl_xor_sync(0xffffffffu, sS, o);
            sR += __shfl_xor_sync(0xffffffffu, sR, o);
            sA += __shfl_xor_sync(0xffffffffu, sA, o);
        }
        if (lane == 0) {
            red[warp][0] = sS;
            red[warp][1] = sR;
            red[warp][2] = sA;
        }
        __syncthreads();
        if (tid < 3) {
            float sum = 0.0f;
            for (int w = 0; w < NW; ++w) sum += red[w][tid];
            reinterpret_cast<double *>(a.partials + t.part)[tid] = static_cast<double>(sum);
        }
        __syncthreads();  // the partial and every owned site of the sweep are stored

        // Grid barrier: arrive, draw the next sweep's normals, then wait (bounded).
        if (tid == 0) grid_arrive(ctl);  // release: this block's stores, ordered before by the barrier above
        if (it + 1 < ra.count)
            quad_normals<QCS, NT, NQ>(z, a.key, static_cast<uint32_t>(sw + 1), f.stream, static_cast<uint32_t>(Wl) >> 2,
                                      gu0, gv0);
        if (tid == 0) {
            const unsigned long long target = (static_cast<unsigned long long>(it) + 1) * nblk + ra.extra_arrivals;
            if (grid_wait(ctl, target, ra.wait_ns)) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;

        // The halo of the next sweep (its state buffer is XW), through L2, by the threads of the
        // warps that do not draw (one halo quad each: the two quad rows above and below the tile,
        // then the two quad columns on each side), while warps 0 and 1 draw.
        if (warp >= 2) {
            const int nhalo = 4 * QCS + 4 * (QR - 4);
            for (int hq = tid - 64; hq < nhalo; hq += NT - 64) {
                int u, v;
                if (hq < 4 * QCS) {
                    const int r = hq / QCS;
                    u = r < 2 ? r : QR - 4 + r;
                    v = hq - r * QCS;
                } else {
                    const int r = hq - 4 * QCS, c = r & 3;
                    u = 2 + (r >> 2);
                    v = c < 2 ? c : QCS - 4 + c;
                }
                const int q = u * QCS + v;
                const int gu = gu0 + u, gv = gv0 + v;
                const int go = gu * gcols + gv;
                float hv[4];
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int i = 2 * gu + (s >> 1), j = 2 * gv + (s & 1);
                    const bool ok = interior || (gu >= 0 && gv >= 0 && i < Hl && j < Wl);
                    hv[s] = ok ? __ldcg(XW + s * gsub + go) : 0.0f;
                }
#pragma unroll
                for (int s = 0; s < 4; ++s) xs[s * SUB + q] = hv[s];
            }
        }

        // The conjugate draws at the end of sweep sw (warp 0: tau; warp 1: beta0, then sigma^2).
        if (warp < 2) {
            const int which = warp;
            const bool need_sum = which ? (h.draw || h.draw_beta) : h.draw;
            const bool need_a = which && h.draw_beta;
            double S = 0.0, A = 0.0;
            if (need_sum) hyper_sums<false, true>(h, which, need_a, 0, f.part0, f.nparts, S, A);
            if (lane == 0) {
                const long long kb = sw - bbase;
                const bool pre = h.gpre && kb >= 0 && kb < bcount;
                double gpv = 0.0, zb = 0.0;
                if (pre) {
                    const double *gp = it < kQuadResGpre ? gsh[it] : h.gpre + kb * h.nfields * h.Cp * 4;
                    gpv = gp[which];
                    zb = gp[2];
                }
                // (warp 0's draw reads neither sigma^2 nor beta0, which warp 1 replaces meanwhile)
                const double cur = dcur[which], s2old = which ? dcur[1] : 0.0;
                const double b = which ? static_cast<double>(hs[2]) : 0.0;
                double val, bval;
                hyper_draw<float>(h, which, 0, 0, sw, S, A, cur, s2old, b, gpv, zb, pre, 0, f.stream, f.n, f.rank, val,
                                  bval, blockIdx.x == 0);
                if (which == 0) {
                    if (h.draw) hs[0] = static_cast<float>(val);
                } else {
                    if (h.draw_beta) hs[2] = static_cast<float>(bval);
                    if (h.draw) hs[1] = static_cast<float>(1.0 / val);
                }
                dcur[which] = val;
            }
        }
    }

    // The running moments of the owned sites back to global memory.
    if (a.acc_enabled) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int q = tid + k * NT;
            if (q >= nquads) break;
            const int u = q / QCS, v = q % QCS;
            const int go = (gu0 + u) * gcols + gv0 + v;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!quad_owned_site(u, v, s, QR, TC, gu0, gv0, Hl, Wl)) continue;
                MEAN[s * gsub + go] = ms[s * SUB + q];
                M2[s * gsub + go] = m2s[s * SUB + q];
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

}  // namespace

// Configurations: (quad columns per staged row, threads, quads per thread).
// (state, observations, running mean and M2: four sub-arrays each)
size_t lattice_quad_smem(int qcs, int TR) { return static_cast<size_t>(16) * (TR / 2 + 4) * qcs * sizeof(float); }

cudaError_t prepare_lattice_quad(int qcs, int nt, int nq, size_t smem)
{
#define GMRF_QUAD_CFG(Q, N, M)                                                                                   \
    if (qcs == Q && nt == N && nq == M)                                                                       \
        return cudaFuncSetAttribute(lattice_quad_kernel<Q, N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    static_cast<int>(smem));
    GMRF_QUAD_CFG(64, 768, 3)
    GMRF_QUAD_CFG(64, 1024, 2)
    GMRF_QUAD_CFG(32, 1024, 2)
    GMRF_QUAD_CFG(32, 512, 2)
    GMRF_QUAD_CFG(68, 704, 3)
#undef GMRF_QUAD_CFG
    return cudaErrorInvalidValue;
}

cudaError_t launch_lattice_quad(int qcs, int nt, int nq, const FusedArgs &a, size_t smem, cudaStream_t stream)
{
#define GMRF_QUAD_CFG(Q, N, M)                                                          \
    if (qcs == Q && nt == N && nq == M) {                                              \
        return launch_sweep_kernel(lattice_quad_kernel<Q, N, M>, a.ntiles, N, smem, stream, a); \
    }
    GMRF_QUAD_CFG(64, 768, 3)
    GMRF_QUAD_CFG(64, 1024, 2)
    GMRF_QUAD_CFG(32, 1024, 2)
    GMRF_QUAD_CFG(32, 512, 2)
    GMRF_QUAD_CFG(68, 704, 3)
#undef GMRF_QUAD_CFG
    return cudaErrorInvalidValue;
}

// The resident form: whether every tile's block can be resident at once (one wave), and the
// cooperative launch of `ra.count` sweeps.
cudaError_t lattice_quad_resident_fits(int qcs, int nt, int nq, size_t smem, int ntiles, bool *fits)
{
    *fits = false;
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return e;
#define GMRF_QUAD_CFG(Q, N, M)                                                                                   \
    if (qcs == Q && nt == N && nq == M) {                                                                     \
        e = cudaFuncSetAttribute(lattice_quad_resident_kernel<Q, N, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 static_cast<int>(smem));                                                     \
        if (e == cudaSuccess)                                                                                 \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lattice_quad_resident_kernel<Q, N, M>, N, smem); \
        if (e != cudaSuccess) return e;                                                                       \
        *fits = coop != 0 && static_cast<int64_t>(per_sm) * sms >= ntiles;                                   \
        return cudaSuccess;                                                                                   \
    }
    GMRF_QUAD_CFG(64, 768, 3)
    GMRF_QUAD_CFG(64, 1024, 2)
    GMRF_QUAD_CFG(32, 1024, 2)
    GMRF_QUAD_CFG(32, 512, 2)
    GMRF_QUAD_CFG(68, 704, 3)
#undef GMRF_QUAD_CFG
    return cudaSuccess;
}

cudaError_t launch_lattice_quad_resident(int qcs, int nt, int nq, const TileResArgs &ra, size_t smem,
                                         cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ra.f.ntiles);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define GMRF_QUAD_CFG(Q, N, M) \
    if (qcs == Q && nt == N && nq == M) return cudaLaunchKernelEx(&cfg, lattice_quad_resident_kernel<Q, N, M>, ra);
    GMRF_QUAD_CFG(64, 768, 3)
    GMRF_QUAD_CFG(64, 1024, 2)
    GMRF_QUAD_CFG(32, 1024, 2)
    GMRF_QUAD_CFG(32, 512, 2)
    GMRF_QUAD_CFG(68, 704, 3)
#undef GMRF_QUAD_CFG
    return cudaErrorInvalidValue;
}

}  // namespace gmrf
