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

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {
namespace {

template <typename T> struct FArith;
template <> struct FArith<float> {
    __device__ __forceinline__ static float rcp(float x) { return __frcp_rn(x); }
    __device__ __forceinline__ static float rsq(float x) { return rsqrtf(x); }
};
template <> struct FArith<double> {
    __device__ __forceinline__ static double rcp(double x) { return 1.0 / x; }
    __device__ __forceinline__ static double rsq(double x) { return 1.0 / sqrt(x); }
};

// Neighbour directions in a fixed order (the summation order of s_i): 8-neighbour lattice all
// (di, dj) != (0, 0) row by row; 4-neighbour lattice the four axis steps.
template <int KIND> struct Dirs;
template <> struct Dirs<kLat2D8> {
    static constexpr int N = 8;
    __device__ __forceinline__ static int di(int k) { return (k < 3) ? -1 : (k < 5 ? 0 : 1); }
    __device__ __forceinline__ static int dj(int k) { return (k < 3) ? k - 1 : (k == 3 ? -1 : (k == 4 ? 1 : k - 6)); }
    __device__ __forceinline__ static int colour(int i, int j) { return 2 * (i & 1) + (j & 1); }
};
template <> struct Dirs<kLat2D4> {
    static constexpr int N = 4;
    __device__ __forceinline__ static int di(int k) { return k == 0 ? -1 : (k == 3 ? 1 : 0); }
    __device__ __forceinline__ static int dj(int k) { return k == 1 ? -1 : (k == 2 ? 1 : 0); }
    __device__ __forceinline__ static int colour(int i, int j) { return (i + j) & 1; }
};

// Slot of site (i, j) relative to the field's first slot (32-bit: fields hold < 2^31 slots).
template <int KIND>
__device__ __forceinline__ int slot_rel(const FieldDev &f, int i, int j)
{
    if (KIND == kLat2D8) return ((2 * (i & 1) + (j & 1)) * f.rows + (i >> 1)) * f.cols + (j >> 1);
    return (((i + j) & 1) * f.rows + i) * f.cols + (j >> 1);
}

// Invariant-divisor constants for a divisor known only on the device (computed once per loop).
__device__ __forceinline__ void device_magic(uint32_t d, uint32_t &m, int &s)
{
    s = (d <= 1) ? 0 : 32 - __clz(d - 1);
    m = static_cast<uint32_t>((static_cast<unsigned long long>(1) << 32) *
                              ((static_cast<unsigned long long>(1) << s) - d) / d + 1);
}

constexpr int kFusedBlock = 512;

template <typename T, int V, int KIND>
__global__ void __launch_bounds__(kFusedBlock) lattice_fused_kernel(const FusedArgs a)
{
    using D = Dirs<KIND>;
    constexpr int K = (KIND == kLat2D8) ? 4 : 2;  // colours = halo width
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileXY t = a.tiles[blockIdx.x];
    const FieldDev f = a.fields[t.field];
    const int Hl = f.dims[0], Wl = f.dims[1];
    const int TR = a.TR, TC = a.TC, RR = TR + 2 * K, RC = TC + 2 * K;
    const int Cp = a.Cp, CV = Cp / V, cv_shift = __ffs(CV) - 1;
    const int cvo = (threadIdx.x & (CV - 1)) * V;  // chain offset of this thread (fixed)
    T *xs = reinterpret_cast<T *>(smem_raw);       // [RR * RC][Cp] state
    T *zs = xs + RR * RC * Cp;                     // [RR * RC][Cp] this sweep's normals
    T *ys = zs + RR * RC * Cp;                     // [RR * RC] observations
    const int gi0 = t.i0 - K, gj0 = t.j0 - K;
    // Ping-pong state: sweep t reads buffer t & 1 and writes the other, so no block can see a
    // neighbour's new values while staging its halo.
    const long long sweep_ll = a.ctl->sweep;
    const void *xsrc = (sweep_ll & 1) ? a.x_alt : a.x;
    void *xdst = (sweep_ll & 1) ? a.x : a.x_alt;
    const T *X = static_cast<const T *>(xsrc) + f.slot0 * Cp + cvo;
    const T *Y = static_cast<const T *>(a.y) + f.slot0;
    const uint32_t sweep = static_cast<uint32_t>(sweep_ll);
    const T rho = static_cast<T>(a.rho);

    // Chain parameters of this thread's chain vector.
    T tau[V], isig[V];
    const T *hyp = static_cast<const T *>(a.hyp);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int64_t hc = (static_cast<int64_t>(t.field) * Cp + cvo + v) * 2;
        tau[v] = hyp[hc];
        isig[v] = hyp[hc + 1];
    }

    // Stage x (all chains) and y of the tile and its halo.
    for (int q = threadIdx.x; q < RR * RC * CV; q += kFusedBlock) {
        const int p = q >> cv_shift;
        const int ri = fast_div(p, a.rc_m, a.rc_s), rj = p - ri * RC;
        const int gi = gi0 + ri, gj = gj0 + rj;
        T v[V];
        if (gi >= 0 && gi < Hl && gj >= 0 && gj < Wl) {
            const int slot = slot_rel<KIND>(f, gi, gj);
            Vec<T, V>::ld(X + slot * Cp, v);
            if (cvo == 0) ys[p] = Y[slot];
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = 0;
            if (cvo == 0) ys[p] = 0;
        }
        Vec<T, V>::st(xs + p * Cp + cvo, v);
    }

    // Phase A: the normals of every site this block draws in this sweep (colour c within
    // k - 1 - c rings of the tile).  They depend on (site, sweep, chain) only, so this phase has
    // no barriers and carries most of the arithmetic.
    if (a.update) {
        for (int q = threadIdx.x; q < RR * RC * CV; q += kFusedBlock) {
            const int p = q >> cv_shift;
            const int ri = fast_div(p, a.rc_m, a.rc_s), rj = p - ri * RC;
            const int i = gi0 + ri, j = gj0 + rj;
            if (i < 0 || i >= Hl || j < 0 || j >= Wl) continue;
            const int c = D::colour(i, j);
            const int e = K - 1 - c;
            if (i < t.i0 - e || i >= t.i0 + TR + e || j < t.j0 - e || j >= t.j0 + TC + e) continue;
            T z[V];
            site_normals<T, V>(a.key, static_cast<uint32_t>(i * Wl + j), sweep, f.stream, static_cast<uint32_t>(cvo), z);
            Vec<T, V>::st(zs + p * Cp + cvo, z);
        }
    }
    __syncthreads();

    // Colour steps in shared memory (skipped in reduce-only mode).
#pragma unroll 1
    for (int c = 0; c < (a.update ? K : 0); ++c) {
        const int e = K - 1 - c;
        const int lo_i = max(0, t.i0 - e), hi_i = min(Hl, t.i0 + TR + e);
        const int lo_j = max(0, t.j0 - e), hi_j = min(Wl, t.j0 + TC + e);
        int fi, ni, ncols;
        if (KIND == kLat2D8) {
            fi = lo_i + (((c >> 1) - lo_i) & 1);
            ni = hi_i > fi ? (hi_i - fi + 1) >> 1 : 0;
            const int fj = lo_j + (((c & 1) - lo_j) & 1);
            ncols = hi_j > fj ? (hi_j - fj + 1) >> 1 : 0;
        } else {
            fi = lo_i;
            ni = hi_i - lo_i;
            ncols = (hi_j - lo_j + 1) >> 1;
        }
        const int nq = ni * ncols * CV;
        uint32_t nc_m;
        int nc_s;
        device_magic(static_cast<uint32_t>(ncols > 0 ? ncols : 1), nc_m, nc_s);
        for (int q = threadIdx.x; q < nq; q += kFusedBlock) {
            const int p = q >> cv_shift;
            const int u = fast_div(p, nc_m, nc_s), w = p - u * ncols;
            int i, j;
            if (KIND == kLat2D8) {
                i = fi + 2 * u;
                j = lo_j + (((c & 1) - lo_j) & 1) + 2 * w;
            } else {
                i = fi + u;
                j = lo_j + ((c + i - lo_j) & 1) + 2 * w;
                if (j >= hi_j) continue;
            }
            const int ri = i - gi0, rj = j - gj0;
            const T *xc = xs + (ri * RC + rj) * Cp + cvo;
            // Staged positions outside the lattice hold zeros, so the neighbour sum needs no
            // bounds tests; the degree follows from how many of the rows i-1..i+1 and columns
            // j-1..j+1 exist.
            T s[V];
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] = 0;
#pragma unroll
            for (int k = 0; k < D::N; ++k) {
                T nb[V];
                Vec<T, V>::ld(xc + (D::di(k) * RC + D::dj(k)) * Cp, nb);
#pragma unroll
                for (int v = 0; v < V; ++v) s[v] += nb[v];
            }
            const int vr = (i > 0) + (i + 1 < Hl), vc = (j > 0) + (j + 1 < Wl);
            const int deg = (KIND == kLat2D8) ? (vr + 1) * (vc + 1) - 1 : vr + vc;
            T z[V];
            Vec<T, V>::ld(zs + (ri * RC + rj) * Cp + cvo, z);
            const T yv = ys[ri * RC + rj];
            const T d = static_cast<T>(deg);
            T xn[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T P = tau[v] * d + isig[v];
                const T m = (tau[v] * rho * s[v] + yv * isig[v]) * FArith<T>::rcp(P);
                xn[v] = m + z[v] * FArith<T>::rsq(P);
            }
            Vec<T, V>::st(xs + (ri * RC + rj) * Cp + cvo, xn);
        }
        __syncthreads();
    }

    // Owned sites: write back, reduce, accumulate.
    const bool acc = a.update && a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin);
    T inv_k = 0;
    if (acc) inv_k = static_cast<T>(1) / static_cast<T>(a.ctl->acc_count + 1);
    T *XW = static_cast<T *>(xdst) + f.slot0 * Cp + cvo;
    T *MEAN = static_cast<T *>(a.mean) + f.slot0 * Cp + cvo;
    T *M2 = static_cast<T *>(a.m2) + f.slot0 * Cp + cvo;
    T accS[V], accR[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        accS[v] = 0;
        accR[v] = 0;
    }
    const int oq = TR * TC * CV;
    for (int q = threadIdx.x; q < oq; q += kFusedBlock) {
        const int p = q >> cv_shift;
        const int oi = fast_div(p, a.tc_m, a.tc_s), oj = p - oi * TC;
        const int i = t.i0 + oi, j = t.j0 + oj;
        if (i >= Hl || j >= Wl) continue;
        const int ri = oi + K, rj = oj + K;
        const T *xc = xs + (ri * RC + rj) * Cp + cvo;
        T xn[V];
        Vec<T, V>::ld(xc, xn);
        const int c = D::colour(i, j);
        const bool up = i > 0, down = i + 1 < Hl, left = j > 0, right = j + 1 < Wl;
        T e[V];
#pragma unroll
        for (int v = 0; v < V; ++v) e[v] = 0;
#pragma unroll
        for (int k = 0; k < D::N; ++k) {
            const int di = D::di(k), dj = D::dj(k);
            const bool ok = (di < 0 ? up : (di > 0 ? down : true)) && (dj < 0 ? left : (dj > 0 ? right : true));
            if (ok && D::colour(i + di, j + dj) < c) {
                T nb[V];
                Vec<T, V>::ld(xc + (di * RC + dj) * Cp, nb);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const T df = xn[v] - nb[v];
                    e[v] += df * df;
                }
            }
        }
        const int vr = up + down, vc = left + right;
        const int deg = (KIND == kLat2D8) ? (vr + 1) * (vc + 1) - 1 : vr + vc;
        const T yv = ys[ri * RC + rj];
        const T d = static_cast<T>(deg);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            accS[v] += (static_cast<T>(1) - rho) * d * xn[v] * xn[v] + rho * e[v];
            const T r = yv - xn[v];
            accR[v] += r * r;
        }
        const int so = slot_rel<KIND>(f, i, j) * Cp;
        if (a.update) Vec<T, V>::st(XW + so, xn);
        if (acc) {
            T mu[V], mm[V];
            Vec<T, V>::ld(MEAN + so, mu);
            Vec<T, V>::ld(M2 + so, mm);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T delta = xn[v] - mu[v];
                mu[v] += delta * inv_k;
                mm[v] += delta * (xn[v] - mu[v]);
            }
            Vec<T, V>::st(MEAN + so, mu);
            Vec<T, V>::st(M2 + so, mm);
        }
    }

    // Deterministic block reduction in precision T (shuffle tree over lanes sharing a chain
    // vector, then warps in order) into the tile's FP64 partial-sum slot; a tile holds at most a
    // few thousand terms, the sum over tiles is FP64.
    __shared__ T red[kFusedBlock / 32][kMaxChains][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T sS = accS[v], sR = accR[v];
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
    for (int q = threadIdx.x; q < Cp * 2; q += kFusedBlock) {
        const int chain = q >> 1, k = q & 1;
        T sum = 0;
        for (int w = 0; w < kFusedBlock / 32; ++w) sum += red[w][chain][k];
        reinterpret_cast<double *>(a.partials + static_cast<int64_t>(t.part) * Cp + chain)[k] = static_cast<double>(sum);
    }
}

template <typename T, int V, int KIND>
cudaError_t launch_t(const FusedArgs &a, size_t smem, cudaStream_t stream)
{
    lattice_fused_kernel<T, V, KIND><<<a.ntiles, kFusedBlock, smem, stream>>>(a);
    return cudaGetLastError();
}

template <typename T, int V, int KIND>
cudaError_t prepare_t(size_t smem)
{
    return cudaFuncSetAttribute(lattice_fused_kernel<T, V, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
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
