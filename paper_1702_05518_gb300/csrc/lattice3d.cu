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
// Chain values travel in pairs: two chains' FP32 values in one 64-bit register, and the per-chain
// arithmetic (the two Box-Muller pairs of a Philox block, neighbour sums, the update, the sums
// for the draws, the running moments) uses the packed two-lane FP32 instructions
// (add/sub/mul/fma .rn.f32x2), one instruction per pair with each lane rounded as the scalar
// operation would be.
//
// Layout (colour-split, chains innermost): the colour-c sites of sub-array row r = l*H + i are
// columns h = 0 .. cols-1 at j = 2h + p, p = (c + l + i) & 1; their neighbours are columns
// h - 1 + p and h + p of the other colour's row r and column h of its rows r -+ 1 and r -+ H.
//
// Work: block k of a field's nt blocks takes the sub-array rows k, k + nt, k + 2 nt, ...; a
// launch is one wave, so at any time all blocks work on a band of about nt rows, and each row
// of the other colour, which six sites of three rows and two planes read, comes from DRAM once.
// Colour 1 walks the rows from the end, so each colour step starts on the rows the previous
// step wrote last, which are still in L2.  In accumulating sweeps a site's running mean and M2
// (read after its draw) are prefetched into L2 when its neighbours are loaded.  A thread's loads
// of its next site's neighbours are in flight while it computes: in colour 0 they are issued once the current site's neighbour sums
// are taken, before its draw; colour 1 keeps a site's neighbour values for its edge sums, so it
// issues them after those and then draws the next site's normals while they arrive.
// Every site takes m_i = a s_i + b (y_i - beta0) and x_i = m_i + c z_i with a = tau rho / P,
// b = (1/sigma^2) / P, c = 1/sqrt(P), computed once per launch for each degree d = 0 .. 6 (a
// row's first and last sites are boundary sites, so at 256^3 half the warps hold one); a warp
// whose sites all have six neighbours takes a path without boundary masks, one whose sites all
// have their four off-row neighbours (at 256^3 nearly every other warp) tests only the two in-row
// ones, and a site's result does not depend on the path its warp took.
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

// Two FP32 values (low half: the even chain) in one 64-bit register.
using f2 = unsigned long long;

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a * b + c, rounded once per lane
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Four chain values (two pairs) at p, 16-byte aligned.
__device__ __forceinline__ void ld2x2(const float *p, f2 &a, f2 &b)
{
    const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
    a = t.x;
    b = t.y;
}
__device__ __forceinline__ void st2x2(float *p, f2 a, f2 b) { *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(a, b); }

__device__ __forceinline__ f2 splat(float v) { return pk(v, v); }
__device__ __forceinline__ f2 lanes_f(uint32_t a, uint32_t b) { return pk(static_cast<float>(a), static_cast<float>(b)); }

// The two Box-Muller pairs of one Philox block, (w.x, w.y) in the low lanes and (w.z, w.w) in
// the high lanes, with the operations of box_muller_f32 lane by lane (so the normals are those of
// the scalar routine, bit for bit): -2 ln u from the base-2 logarithm for u < 3/4 and from the
// atanh series in v = 1 - u above, r = that times its reciprocal square root, and the angle
// reduced on the word to a quadrant and a Taylor-series sine and cosine.  Returns the normals of
// chains (0, 1) and (2, 3) of the block as pairs.
__device__ __forceinline__ void box_muller_block_f32x2(uint4 w, f2 &z01, f2 &z23)
{
    const f2 k32 = splat(0x1p-32f), k33 = splat(0x1p-33f);
    const f2 ua = fma2(lanes_f(w.x, w.z), k32, k33);
    float ua0, ua1;
    upk(ua, ua0, ua1);
    const f2 l1 = mul2(pk(lg2_approx(ua0), lg2_approx(ua1)), splat(-1.3862943611198906f));
    const f2 v = fma2(lanes_f(~w.x, ~w.z), k32, k33);
    float d0, d1;
    upk(sub2(splat(2.0f), v), d0, d1);
    const f2 t = mul2(v, pk(rcp_approx(d0), rcp_approx(d1)));
    const f2 t2 = mul2(t, t);
    const f2 p = fma2(fma2(fma2(fma2(splat(1.0f / 9.0f), t2, splat(1.0f / 7.0f)), t2, splat(1.0f / 5.0f)), t2,
                           splat(1.0f / 3.0f)),
                      t2, splat(1.0f));
    const f2 l2 = mul2(mul2(splat(4.0f), t), p);
    float l1a, l1b, l2a, l2b;
    upk(l1, l1a, l1b);
    upk(l2, l2a, l2b);
    const float q0 = w.x >= 0xC0000000u ? l2a : l1a, q1 = w.z >= 0xC0000000u ? l2b : l1b;
    const f2 q2 = pk(q0, q1);
    const f2 r = mul2(q2, pk(rsqrt_approx(q0), rsqrt_approx(q1)));
    const uint32_t s0 = w.y + 0x20000000u, s1 = w.w + 0x20000000u;
    const f2 dd = add2(sub2(pk(__uint_as_float(0x3F800000u | ((s0 >> 7) & 0x7FFFFFu)),
                               __uint_as_float(0x3F800000u | ((s1 >> 7) & 0x7FFFFFu))),
                            splat(1.5f)),
                       splat(0x1p-24f));
    const f2 dsq = mul2(dd, dd);
    const f2 ps = fma2(fma2(fma2(fma2(splat(1.6044118478735982e-4f), dsq, splat(-4.6817541353186881e-3f)), dsq,
                                 splat(7.9692626246167046e-2f)),
                            dsq, splat(-6.4596409750624625e-1f)),
                       dsq, splat(1.5707963267948966f));
    float sn[2], cs[2];
    upk(mul2(dd, ps), sn[0], sn[1]);
    upk(fma2(fma2(fma2(fma2(splat(9.1926027483942659e-4f), dsq, splat(-2.0863480763352961e-2f)), dsq,
                       splat(2.5366950790104802e-1f)),
                  dsq, splat(-1.2337005501361697f)),
             dsq, splat(1.0f)),
        cs[0], cs[1]);
    const uint32_t quad[2] = {s0 >> 30, s1 >> 30};
    float cq[2], sq[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        cq[h] = (quad[h] & 1u) ? -sn[h] : cs[h];
        sq[h] = (quad[h] & 1u) ? cs[h] : sn[h];
        if (quad[h] & 2u) {
            cq[h] = -cq[h];
            sq[h] = -sq[h];
        }
    }
    // each pair's radius times its (cos, sin): the chains' order, with no transposition
    float r0, r1;
    upk(r, r0, r1);
    z01 = mul2(splat(r0), pk(cq[0], sq[0]));
    z23 = mul2(splat(r1), pk(cq[1], sq[1]));
}

// Per chain parameters of the launch, in shared memory: tau, tau rho, 1/sigma^2, beta0, and for
// every degree d = 0 .. 6 the coefficients tau rho / P, (1/sigma^2) / P, 1/sqrt(P) with
// P = tau d + 1/sigma^2 (a boundary site reads those of its degree instead of computing them).
template <int NC>
struct alignas(16) Params3 {
    float tau[NC], tr[NC], isig[NC], beta[NC];
    float ca[7][NC], cb[7][NC], crs[7][NC];
};

template <int NC>
__device__ __forceinline__ f2 pair_of(const float (&v)[NC], int u)
{
    return *reinterpret_cast<const f2 *>(&v[2 * u]);
}

// Per-thread partial sums, by chain pair.
template <int NP>
struct Acc3 {
    f2 S[NP], R[NP], A[NP];
};

struct Site3 {
    int64_t rb;           // slot of the site in its colour's sub-array (and of its column in the
                          // other colour's)
    uint32_t valid;       // neighbours present: bit k for j - 1, j + 1, i - 1, i + 1, l - 1, l + 1
    uint32_t site;        // natural site index
    float y, d;           // observation, degree
    int dg;               // degree
    int p;                // column parity of the site's row
    bool ok;              // a site of the lattice
    int mode;             // kMaskNone: every site of the warp has six neighbours; kMaskRow: every
                          // site of the warp has its four off-row neighbours; kMaskAll: neither
};

// Offsets of the six neighbours' chain vectors from the other colour's slot rb (in floats).
struct NbrOff {
    int64_t row, plane;
};

// The neighbours' values of a site (zeros for missing ones); XO: the other colour's sub-array.
// Which neighbours a warp's sites must test before use (see Site3::mode).
constexpr int kMaskAll = 0, kMaskRow = 1, kMaskNone = 2;
__host__ __device__ constexpr bool always_present(int mode, int k) { return mode == kMaskNone || (mode == kMaskRow && k >= 2); }

template <int NG, int MODE>
__device__ __forceinline__ void load_neighbours(const float *XO, const NbrOff &no, const Site3 &st, f2 (&nb)[6][2 * NG])
{
    constexpr int NC = 4 * NG;
    const float *xo = XO + st.rb * NC;
    const float *nbp[6] = {xo + (st.p - 1) * NC, xo + st.p * NC, xo - no.row, xo + no.row, xo - no.plane, xo + no.plane};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (always_present(MODE, k) || ((st.valid >> k) & 1u)) {
#pragma unroll
            for (int g = 0; g < NG; ++g) ld2x2(nbp[k] + 4 * g, nb[k][2 * g], nb[k][2 * g + 1]);
        } else {
#pragma unroll
            for (int u = 0; u < 2 * NG; ++u) nb[k][u] = 0ull;
        }
    }
}

// The neighbour sums of a site, per chain pair.
template <int NG>
__device__ __forceinline__ void sum_neighbours(const f2 (&nb)[6][2 * NG], f2 (&s)[2 * NG])
{
#pragma unroll
    for (int u = 0; u < 2 * NG; ++u) {
        s[u] = add2(nb[0][u], nb[1][u]);
#pragma unroll
        for (int k = 2; k < 6; ++k) s[u] = add2(s[u], nb[k][u]);
    }
}

// Draw the NC = 4 NG chains of one site from its neighbour sums s and add its terms to the sums
// (colour 1's edge terms from the neighbour values nb).
template <int NG>
__device__ __forceinline__ void draw_normals(const StepArgs &a, const Site3 &st, uint32_t sweep, uint32_t stream,
                                             f2 (&z)[2 * NG])
{
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const uint4 w = philox4x32_10_rk(make_uint4(st.site, sweep, stream, (kTagX << 24) | g), a.rk);
        box_muller_block_f32x2(w, z[2 * g], z[2 * g + 1]);
    }
}

template <int NG, bool ODD, bool ICPT, bool PCAR, int MODE>
__device__ __forceinline__ void site_update(const StepArgs &a, const Params3<4 * NG> &pp, Acc3<2 * NG> &ac,
                                            const Site3 &st, const f2 (&s)[2 * NG], const f2 (&nb)[6][2 * NG],
                                            const f2 (&z)[2 * NG], float *XS, float *MS, float *QS, bool update,
                                            bool acc, f2 invk2, f2 rho2, float om)
{
    constexpr int NC = 4 * NG, NP = 2 * NG;
    float *xs = XS + st.rb * NC;
    const f2 yy = pk(st.y, st.y);
    f2 x[NP];
    if (update) {
        const int dg = MODE == kMaskNone ? 6 : st.dg;
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const f2 ca = pair_of<NC>(pp.ca[dg], u), cb = pair_of<NC>(pp.cb[dg], u), crs = pair_of<NC>(pp.crs[dg], u);
            const f2 yb = ICPT ? sub2(yy, pair_of<NC>(pp.beta, u)) : yy;
            x[u] = fma2(z[u], crs, fma2(ca, s[u], mul2(yb, cb)));
        }
#pragma unroll
        for (int g = 0; g < NG; ++g) st2x2(xs + 4 * g, x[2 * g], x[2 * g + 1]);
    } else {
#pragma unroll
        for (int g = 0; g < NG; ++g) ld2x2(xs + 4 * g, x[2 * g], x[2 * g + 1]);
    }
    const f2 omd2 = pk(om * st.d, om * st.d);
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        f2 sv = 0ull;
        if (ODD) {
            f2 ev = 0ull;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (always_present(MODE, k) || ((st.valid >> k) & 1u)) {
                    const f2 df = sub2(x[u], nb[k][u]);
                    ev = fma2(df, df, ev);
                }
            }
            sv = PCAR ? mul2(rho2, ev) : ev;
        }
        if (PCAR) sv = fma2(mul2(omd2, x[u]), x[u], sv);
        if (ODD || PCAR) ac.S[u] = add2(ac.S[u], sv);
        const f2 res = sub2(ICPT ? sub2(yy, pair_of<NC>(pp.beta, u)) : yy, x[u]);
        ac.R[u] = fma2(res, res, ac.R[u]);
        if (ICPT) ac.A[u] = add2(ac.A[u], res);
    }
    if (acc) {
        float *ms = MS + st.rb * NC, *qs = QS + st.rb * NC;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            f2 mu[2], mm[2];
            ld2x2(ms + 4 * g, mu[0], mu[1]);
            ld2x2(qs + 4 * g, mm[0], mm[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const f2 xv = x[2 * g + h];
                const f2 delta = sub2(xv, mu[h]);
                mu[h] = fma2(delta, invk2, mu[h]);
                mm[h] = fma2(delta, sub2(xv, mu[h]), mm[h]);
            }
            st2x2(ms + 4 * g, mu[0], mu[1]);
            st2x2(qs + 4 * g, mm[0], mm[1]);
        }
    }
}

// NG: groups of four chains (Cp = 4 NG); ODD: the launch updates colour 1 (whose neighbours are
// all of lower colour); ICPT: the model has the intercept; PCAR: rho < 1.
template <int NG, bool ODD, bool ICPT, bool PCAR>
__global__ void __launch_bounds__(k3Block, 2) lattice3d_kernel(const StepArgs a)
{
    constexpr int NC = 4 * NG, NP = 2 * NG;
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
    }
    __syncthreads();
    if (threadIdx.x < 7 * NC) {
        const int d = threadIdx.x / NC, v = threadIdx.x - d * NC;
        const float P = fmaf(pp.tau[v], static_cast<float>(d), pp.isig[v]);
        const float rP = rcp_approx(P);
        pp.ca[d][v] = pp.tr[v] * rP;
        pp.cb[d][v] = pp.isig[v] * rP;
        pp.crs[d][v] = rsqrt_approx(P);
    }
    __syncthreads();
    Acc3<NP> ac;
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        ac.S[u] = 0ull;
        ac.R[u] = 0ull;
        ac.A[u] = 0ull;
    }
    const bool update = a.update != 0;
    bool acc = false;
    float inv_k = 0.0f;
    if (update && a.acc_enabled && sweep_accumulated(sweep_ll, a.burn_in, a.thin)) {
        acc = true;
        inv_k = 1.0f / static_cast<float>(a.ctl->acc_count + 1);
    }
    const f2 invk2 = pk(inv_k, inv_k), rho2 = pk(rho, rho);

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

    const NbrOff no{off_row, off_plane};
    // Site of element q (in processing order) and its masks; its observation load is issued here.
    auto site_at = [&](int q, Site3 &st) {
        const int e = ODD ? nelem - 1 - q : q;
        const int m = fast_div(e, f.cols_m, f.cols_s);
        const int h = e - m * cols;
        const int r = t.start + m * stride;
        const int l = fast_div(r, f.h_m, f.h_s);
        const int i = r - l * H;
        st.p = (c + l + i) & 1;
        const int j = 2 * h + st.p;
        st.ok = j < W;
        // 0 < j < W - 1 and the same for i, l (unsigned comparisons; false for extents below 3)
        const bool jin = static_cast<unsigned>(j - 1) < static_cast<unsigned>(W - 2);
        const bool rin = static_cast<unsigned>(i - 1) < static_cast<unsigned>(H - 2) &&
                         static_cast<unsigned>(l - 1) < static_cast<unsigned>(L - 2);
        const unsigned act = __activemask();
        st.mode = __all_sync(act, (jin && rin) || !st.ok) ? kMaskNone
                                                          : (__all_sync(act, rin || !st.ok) ? kMaskRow : kMaskAll);
        if (st.mode == kMaskNone)
            st.valid = 63u;
        else if (st.mode == kMaskRow)
            st.valid = 60u | (j > 0 ? 1u : 0u) | (j + 1 < W ? 2u : 0u);
        else
            st.valid = (j > 0 ? 1u : 0u) | (j + 1 < W ? 2u : 0u) | (i > 0 ? 4u : 0u) | (i + 1 < H ? 8u : 0u) |
                       (l > 0 ? 16u : 0u) | (l + 1 < L ? 32u : 0u);
        st.rb = static_cast<int64_t>(r) * cols + h;
        st.site = static_cast<uint32_t>(r) * static_cast<uint32_t>(W) + static_cast<uint32_t>(j);
        st.y = st.ok ? YS[st.rb] : 0.0f;
        st.dg = __popc(st.valid);
        st.d = static_cast<float>(st.dg);
    };
    auto start_loads = [&](const Site3 &st, f2 (&nb)[6][NP]) {
        if (st.ok && acc) {
            // the site's running moments, read after its draw: on their way to L2 from now
            asm volatile("prefetch.global.L2 [%0];" ::"l"(MS + st.rb * NC));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(QS + st.rb * NC));
        }
        if (st.ok) {
            if (st.mode == kMaskNone) load_neighbours<NG, kMaskNone>(XO, no, st, nb);
            else if (st.mode == kMaskRow) load_neighbours<NG, kMaskRow>(XO, no, st, nb);
            else load_neighbours<NG, kMaskAll>(XO, no, st, nb);
        }
    };
    f2 nb[6][NP];
    auto update_site = [&](const Site3 &st, const f2 (&s)[NP], const f2 (&z)[NP]) {
        if (st.mode == kMaskNone)
            site_update<NG, ODD, ICPT, PCAR, kMaskNone>(a, pp, ac, st, s, nb, z, XS, MS, QS, update, acc, invk2, rho2, om);
        else if (st.mode == kMaskRow)
            site_update<NG, ODD, ICPT, PCAR, kMaskRow>(a, pp, ac, st, s, nb, z, XS, MS, QS, update, acc, invk2, rho2, om);
        else
            site_update<NG, ODD, ICPT, PCAR, kMaskAll>(a, pp, ac, st, s, nb, z, XS, MS, QS, update, acc, invk2, rho2, om);
    };
    if (!ODD) {
        // Colour 0: a site's neighbour sums are taken first (freeing `nb`), then the loads of the
        // thread's next site are issued, then the site is drawn and updated while they arrive.
        Site3 cur;
        int q = threadIdx.x;
        if (q < nelem) {
            site_at(q, cur);
            start_loads(cur, nb);
        }
        for (; q < nelem; q += k3Block) {
            f2 s[NP], z[NP];
            if (cur.ok) sum_neighbours<NG>(nb, s);
            Site3 nxt;
            nxt.ok = false;
            if (q + k3Block < nelem) {
                site_at(q + k3Block, nxt);
                start_loads(nxt, nb);
            }
            if (cur.ok) {
                if (update) draw_normals<NG>(a, cur, sweep, f.stream, z);
                update_site(cur, s, z);
            }
            cur = nxt;
        }
    } else {
        // Colour 1 keeps a site's neighbour values until its edge sums: after those, the loads of
        // the thread's next site are issued and that site's normals drawn while they arrive.
        Site3 cur;
        f2 z[NP];
        int q = threadIdx.x;
        if (q < nelem) {
            site_at(q, cur);
            start_loads(cur, nb);
            if (cur.ok && update) draw_normals<NG>(a, cur, sweep, f.stream, z);
        }
        for (; q < nelem; q += k3Block) {
            if (cur.ok) {
                f2 s[NP];
                sum_neighbours<NG>(nb, s);
                update_site(cur, s, z);
            }
            Site3 nxt;
            nxt.ok = false;
            if (q + k3Block < nelem) {
                site_at(q + k3Block, nxt);
                start_loads(nxt, nb);
                if (nxt.ok && update) draw_normals<NG>(a, nxt, sweep, f.stream, z);
            }
            cur = nxt;
        }
    }

    // Block sums per chain: a shuffle tree over the warp's lanes, then the warps in order.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int u = 0; u < NP; ++u) {
        float sS[2], sR[2], sA[2];
        upk(ac.S[u], sS[0], sS[1]);
        upk(ac.R[u], sR[0], sR[1]);
        upk(ac.A[u], sA[0], sA[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                if (ODD || PCAR) sS[h] += __shfl_xor_sync(0xffffffffu, sS[h], off);
                sR[h] += __shfl_xor_sync(0xffffffffu, sR[h], off);
                if (ICPT) sA[h] += __shfl_xor_sync(0xffffffffu, sA[h], off);
            }
            if (lane == 0) {
                red[warp][2 * u + h][0] = sS[h];
                red[warp][2 * u + h][1] = sR[h];
                red[warp][2 * u + h][2] = sA[h];
            }
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

// The normals of one colour step alone: for each of `sites` sites, the NG Philox blocks and
// packed Box-Muller pairs of the kernel above (same counters, same arithmetic), summed per
// thread and written once per thread, so the launch moves no state: its time is the random
// numbers' share of a colour step.
template <int NG>
__global__ void __launch_bounds__(k3Block, 2) normals_only_kernel(const StepArgs a, int64_t sites, uint32_t sweep,
                                                                  unsigned long long *out)
{
    constexpr int NP = 2 * NG;
    f2 acc[NP];
#pragma unroll
    for (int u = 0; u < NP; ++u) acc[u] = 0ull;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(k3Block) + threadIdx.x; i < sites;
         i += static_cast<int64_t>(gridDim.x) * k3Block) {
        Site3 st;
        st.site = static_cast<uint32_t>(i);
        f2 z[NP];
        draw_normals<NG>(a, st, sweep, 0u, z);
#pragma unroll
        for (int u = 0; u < NP; ++u) acc[u] = add2(acc[u], z[u]);
    }
    f2 t = acc[0];
#pragma unroll
    for (int u = 1; u < NP; ++u) t = add2(t, acc[u]);
    out[blockIdx.x * static_cast<int64_t>(k3Block) + threadIdx.x] = t;
}

}  // namespace

int normals_only_threads(int chains_padded)
{
    int bps = 1, nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        lattice3d_blocks_per_sm(chains_padded, &bps) != cudaSuccess)
        return 0;
    return nsm * bps * k3Block;
}

cudaError_t time_normals_only(uint64_t seed, int64_t sites, int chains_padded, int reps, unsigned long long *out,
                              cudaStream_t stream, double *us_per_launch)
{
    StepArgs a{};
    a.key = philox_key(seed);
    philox_round_keys(a.key, a.rk);
    const int grid = normals_only_threads(chains_padded) / k3Block;
    if (grid < 1) return cudaErrorInvalidConfiguration;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto launch = [&](uint32_t sweep) {
        if (chains_padded == 8) normals_only_kernel<2><<<grid, k3Block, 0, stream>>>(a, sites, sweep, out);
        else normals_only_kernel<1><<<grid, k3Block, 0, stream>>>(a, sites, sweep, out);
        return cudaGetLastError();
    };
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch(static_cast<uint32_t>(r));
    if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch(static_cast<uint32_t>(r + 3));
    if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) *us_per_launch = 1e3 * ms / reps;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

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
