// gmrf_device.cuh -- device-side building blocks of libgmrf: the counter-based generators
// (Philox4x32-10, Box-Muller normals, Marsaglia-Tsang Gamma variates), the field/tile
// descriptors shared by host and device code, and small vector load/store helpers.
//
// The generators follow their published definitions (Salmon et al., SC'11 for Philox;
// Box-Muller; Marsaglia & Tsang, ACM TOMS 2000 for Gamma) with the counter assignment stated
// in include/gmrf.h, so every draw is a pure function of (seed, counter).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gmrf {

constexpr uint32_t kTagX = 0, kTagTau = 1, kTagSig = 2, kTagPrio = 3, kTagTauExtra = 5,
                   kTagSigExtra = 6, kTagBeta = 7, kTagBetaExtra = 8;
// Per (field, chain) parameter copies read by the sweep kernels, in the state precision:
// tau, 1/sigma^2, beta0 (0 without the intercept), and one pad.
constexpr int kHypStride = 4;
constexpr int kMaxChains = 64;
constexpr int kBlock = 256;            // threads per block of the colour-step kernels
constexpr int kMaxGammaAttempts = 64;  // bounded rejection loop

enum FieldKind : int32_t { kLat2D4 = 0, kLat2D8 = 1, kLat3D6 = 2, kCsr = 3 };

// Per-field descriptor, device-resident.  "Slots" index the colour-split layout: a lattice of
// colour count k keeps k sub-arrays of rows x cols slots each (padded; invalid slots are never
// read); a CSR field keeps its n sites permuted so each colour class is contiguous.
struct FieldDev {
    int32_t kind;
    int32_t ncolors;
    int32_t n;          // sites
    int32_t rows;       // lattice: sub-array rows; CSR: 0
    int32_t cols;       // lattice: sub-array columns (padded); CSR: 0
    int32_t dims[3];    // 2-D: H, W; 3-D: L, H, W; CSR: n
    uint32_t stream;    // Philox counter word 2
    int32_t rank;       // n - components (intrinsic prior) or n (proper prior)
    int64_t slot0;      // first slot of this field in the concatenated state arrays
    int64_t nslots;     // slots of this field
    int64_t csr0;       // CSR: first index into the per-site CSR arrays (perm, deg)
    int64_t rp0;        // CSR: first index into the row-pointer array (n + 1 entries)
    int64_t nnz0;       // CSR: first index into col_idx / weights
    int64_t coff0;      // CSR: first index into the colour-offset array (ncolors + 1 entries)
    int32_t part0;      // first partial-sum slot (tiles of all colours of this field)
    int32_t nparts;     // partial-sum slots of this field
    uint32_t cols_m;    // lattice: invariant-divisor multiplier and shift of cols (fast_div)
    int32_t cols_s;
    uint32_t h_m;       // 3-D lattice: the same for H
    int32_t h_s;
};

// Division by an invariant divisor d >= 1 for 0 <= n < 2^31 (Granlund & Montgomery, PLDI'94,
// round-up variant): s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, q = (mulhi(n, m) + n) >> s.
__host__ __device__ __forceinline__ void fast_div_magic(uint32_t d, uint32_t &m, int32_t &s)
{
    s = 0;
    while ((uint64_t(1) << s) < d) ++s;
    m = static_cast<uint32_t>((uint64_t(1) << 32) * ((uint64_t(1) << s) - d) / d + 1);
}
__device__ __forceinline__ int fast_div(int n, uint32_t m, int s)
{
    return static_cast<int>((__umulhi(static_cast<uint32_t>(n), m) + static_cast<uint32_t>(n)) >> s);
}

// A unit of work of one colour step: a range of sub-array rows (lattice) or of permuted
// positions (CSR) of one field's colour class.  With stride > 1 (the 3-D kernel of
// lattice3d.cu) the tile's rows are start, start + stride, ... (count of them).
struct Tile {
    int32_t field;
    int32_t colour;
    int32_t start;
    int32_t count;
    int32_t part;       // partial-sum slot
    int32_t stride;     // 0 or 1: contiguous rows
    int32_t pad[2];
};

// Device-resident sweep control, read by every kernel of a sweep and advanced by the last.
// Per tile and chain: the sums behind the conjugate draws, FP64.
//   S = the tile's part of x'(D - rho W)x,  R = sum (y - beta0 - x)^2,  A = sum (y - beta0 - x)
// (beta0 = 0 without the intercept).
struct alignas(16) Part3 {
    double S, R, A, pad;
};

struct SweepCtl {
    long long sweep;       // number of the sweep in progress
    long long extra;       // gmrf_hyper_update calls so far
    long long fallbacks;   // Gamma draws that hit the attempt limit
    long long acc_count;   // sweeps accumulated into the running mean / M2
    unsigned long long ticket;  // blocks of the current hyper launch that have finished
    long long batch_base;  // first sweep of the current batch of precomputed Gamma variates
    long long batch_count; // sweeps in that batch
    long long fnext;       // the sweep number a sweep kernel that starts early predicts (the
                           // last such kernel's sweep + 1); checked against `sweep` before use
    unsigned long long fticket;  // blocks of that kernel that have read fnext
    long long fmiss;       // launches whose prediction was wrong (their normals were redrawn)
    unsigned long long wait_timeouts;  // bounded device waits that gave up (results invalid)
    unsigned long long pad0;
    // The resident quad kernel's grid barrier (16-byte aligned, read as one vector): arrivals
    // (0 between launches), and a flag set when a block gave up waiting (the others stop too).
    unsigned long long gbar;
    unsigned long long gabort;
};
static_assert(offsetof(SweepCtl, gbar) % 16 == 0, "the grid barrier's two words are read as one 16-byte vector");

// Whether sweep number `sweep` is accumulated (burn-in, then every thin-th sweep).
__host__ __device__ __forceinline__ bool sweep_accumulated(long long sweep, long long burn_in, int thin)
{
    return sweep >= burn_in && (sweep - burn_in) % thin == 0;
}

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product gives both halves of each multiplication
        const uint64_t p0 = static_cast<uint64_t>(c.x) * 0xD2511F53u;
        const uint64_t p1 = static_cast<uint64_t>(c.z) * 0xCD9E8D57u;
        const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
        const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The same with the ten round keys given: rk[2r], rk[2r + 1] = the key after r Weyl increments
// (philox_round_keys).  Kept in a kernel's parameters, they are read from constant memory by the
// XOR that uses them, so no round spends instructions on the key schedule.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(c.x) * 0xD2511F53u;
        const uint64_t p1 = static_cast<uint64_t>(c.z) * 0xCD9E8D57u;
        const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
        const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

__host__ __device__ __forceinline__ void philox_round_keys(uint2 k, uint32_t (&rk)[20])
{
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k.x;
        rk[2 * r + 1] = k.y;
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
}

__host__ __device__ __forceinline__ uint2 philox_key(uint64_t seed)
{
    return make_uint2(static_cast<uint32_t>(seed & 0xffffffffu), static_cast<uint32_t>(seed >> 32));
}

// Programmatic dependent launch: a sweep kernel launched with programmatic stream serialization
// may be scheduled before its predecessor in the stream has finished.  It waits here, before
// it reads anything a predecessor wrote, and then lets its own successor be scheduled (which in
// turn waits for this grid to finish).  Without that launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_then_release()
{
    pdl_wait();
    pdl_release();
}

// ------------------------------------------------------------------------------------------
// Uniforms u = (w + 1/2) 2^-32 and Box-Muller normals (r = sqrt(-2 ln u_a), angle 2 pi u_b).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double u01_f64(uint32_t w) { return (static_cast<double>(w) + 0.5) * 0x1p-32; }

__device__ __forceinline__ float u01_f32(uint32_t w)
{
    return fmaf(static_cast<float>(w), 0x1p-32f, 0x1p-33f);
}

// Hardware approximations (PTX .approx, flush-to-zero): reciprocal and reciprocal square root
// within 1 ulp, base-2 logarithm within 2^-22 absolute.  Every argument here is a normal float.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// -2 ln u in single precision with small relative error for every word, without branches:
// for u < 3/4 from the base-2 logarithm of u itself (|ln u| > 0.28, so its absolute error is a
// relative error below 1e-6); for u >= 3/4, with v = 1 - u formed from the complemented word,
// ln(1 - v) = -2 atanh(t), t = v / (2 - v) <= 1/7, by the atanh series
// t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9) (truncation below 4e-10 relative), so radii near zero
// keep their precision.
__device__ __forceinline__ float neg2log_u_f32(uint32_t w)
{
    const float l1 = lg2_approx(u01_f32(w)) * -1.3862943611198906f;  // -2 ln 2 log2(u)
    const float v = u01_f32(~w);
    const float t = v * rcp_approx(2.0f - v);
    const float t2 = t * t;
    const float p = fmaf(fmaf(fmaf(fmaf(1.0f / 9.0f, t2, 1.0f / 7.0f), t2, 1.0f / 5.0f), t2, 1.0f / 3.0f), t2, 1.0f);
    const float l2 = 4.0f * t * p;
    return w >= 0xC0000000u ? l2 : l1;
}

// sin and cos of the angle pi d / 2, |d| <= 1/2 (a quarter turn centred at 0), by their Taylor
// series in d: coefficients (-1)^j (pi/2)^k / k!, to d^9 for the sine and d^8 for the cosine;
// the truncation error is below 3e-8 on the interval.
__device__ __forceinline__ void sincos_quarter_turn(float d, float &s, float &c)
{
    const float d2 = d * d;
    const float ps = fmaf(fmaf(fmaf(fmaf(1.6044118478735982e-4f, d2, -4.6817541353186881e-3f), d2,
                                    7.9692626246167046e-2f), d2, -6.4596409750624625e-1f), d2, 1.5707963267948966f);
    s = d * ps;
    c = fmaf(fmaf(fmaf(fmaf(9.1926027483942659e-4f, d2, -2.0863480763352961e-2f), d2, 2.5366950790104802e-1f), d2,
                   -1.2337005501361697f), d2, 1.0f);
}

// Box-Muller pair in single precision: r = sqrt(-2 ln u_a), angle 2 pi u_b.  The angle is reduced
// exactly on the word: adding 2^29 shifts u_b by 1/8 turn, the top two bits of the sum give the
// quadrant q and the next 23 bits (bucket midpoint, error below 1e-7 rad) the offset d in
// [-1/2, 1/2), so that 2 pi u_b = q pi/2 + pi d/2; (cos, sin) of pi d/2 is then turned by q
// quarter turns.
__device__ __forceinline__ void box_muller_f32(uint32_t wa, uint32_t wb, float &zc, float &zs)
{
    const float q2 = neg2log_u_f32(wa);  // > 0 for every word
    const float r = q2 * rsqrt_approx(q2);
    const uint32_t ws = wb + 0x20000000u;
    const uint32_t quad = ws >> 30;
    const float d = __uint_as_float(0x3F800000u | ((ws >> 7) & 0x7FFFFFu)) - 1.5f + 0x1p-24f;
    float s, c;
    sincos_quarter_turn(d, s, c);
    float cq = (quad & 1u) ? -s : c;
    float sq = (quad & 1u) ? c : s;
    if (quad & 2u) {
        cq = -cq;
        sq = -sq;
    }
    zc = r * cq;
    zs = r * sq;
}

__device__ __forceinline__ void box_muller_f64(uint32_t wa, uint32_t wb, double &zc, double &zs)
{
    const double r = sqrt(-2.0 * log(u01_f64(wa)));
    double s, c;
    sincospi(2.0 * u01_f64(wb), &s, &c);
    zc = r * c;
    zs = r * s;
}

template <typename T> struct Prec;
template <> struct Prec<float> {
    __device__ __forceinline__ static void bm(uint32_t a, uint32_t b, float &c, float &s) { box_muller_f32(a, b, c, s); }
};
template <> struct Prec<double> {
    __device__ __forceinline__ static void bm(uint32_t a, uint32_t b, double &c, double &s) { box_muller_f64(a, b, c, s); }
};

// Normal layout: a Philox block gives four normals n0, n1 (cos, sin of Box-Muller(w0, w1)) and
// n2, n3 (of (w2, w3)).  With `lanes` = min(4, chains rounded up to a power of two) it serves
// G = 4 / lanes consecutive sites and `lanes` chains: block counter (site / G, sweep, stream,
// (kTagX << 24) | chain / 4), normal n[(site mod G) * lanes + chain mod lanes].
__device__ __forceinline__ int lanes_shift(int lanes) { return lanes == 4 ? 0 : (lanes == 2 ? 1 : 2); }

// The V normals that update chains chain0 .. chain0+V-1 of `site` at `sweep` (chain0 a multiple
// of V; V = 4 implies lanes = 4, V = 1 any lanes, V = 2 lanes 2 or 4).
template <typename T, int V>
__device__ __forceinline__ void site_normals(uint2 key, uint32_t site, uint32_t sweep, uint32_t stream,
                                             uint32_t chain0, int lanes, T (&z)[V])
{
    const int gs = lanes_shift(lanes);
    const uint32_t first = ((site & ((1u << gs) - 1u)) * static_cast<uint32_t>(lanes)) +
                           (chain0 & static_cast<uint32_t>(lanes - 1));
    const uint4 w = philox4x32_10(make_uint4(site >> gs, sweep, stream, (kTagX << 24) | (chain0 >> 2)), key);
    if constexpr (V == 4) {
        Prec<T>::bm(w.x, w.y, z[0], z[1]);
        Prec<T>::bm(w.z, w.w, z[2], z[3]);
    } else if constexpr (V == 2) {
        if ((first & 2u) == 0) Prec<T>::bm(w.x, w.y, z[0], z[1]);
        else Prec<T>::bm(w.z, w.w, z[0], z[1]);
    } else {
        T c, s;
        if ((first & 2u) == 0) Prec<T>::bm(w.x, w.y, c, s);
        else Prec<T>::bm(w.z, w.w, c, s);
        z[0] = (first & 1u) ? s : c;
    }
}

// All four normals of block `grp` (chains 0 .. 3 of the quadruple chain_quad).
template <typename T>
__device__ __forceinline__ void block_normals(uint2 key, uint32_t grp, uint32_t sweep, uint32_t stream,
                                              uint32_t chain_quad, T (&n)[4])
{
    const uint4 w = philox4x32_10(make_uint4(grp, sweep, stream, (kTagX << 24) | chain_quad), key);
    Prec<T>::bm(w.x, w.y, n[0], n[1]);
    Prec<T>::bm(w.z, w.w, n[2], n[3]);
}

// ------------------------------------------------------------------------------------------
// Gamma(shape, rate) by Marsaglia & Tsang (2000), FP64.  The accept/reject loop depends on the
// shape only; the rate divides the accepted variate at the end, so gamma_mt(a, rate) ==
// gamma_mt(a, 1) / rate exactly (same operations in the same order).  Attempt k uses the block at counter
// (k, word1, stream, tag_chain): z = Box-Muller cos of (w0, w1), acceptance uniform w2, boost
// uniform w3 (shape < 1: Gamma(a) = Gamma(a + 1) U^(1/a)).  At most kMaxGammaAttempts
// attempts; if all reject (probability < 1e-100 here) the draw is d / rate and *fell_back = 1.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double gamma_mt(double shape, double rate, uint2 key, uint32_t word1,
                                           uint32_t stream, uint32_t tag_chain, int &fell_back)
{
    const bool boost = shape < 1.0;
    const double a = boost ? shape + 1.0 : shape;
    const double d = a - 1.0 / 3.0;
    const double c = 1.0 / sqrt(9.0 * d);
    fell_back = 0;
    for (uint32_t k = 0; k < static_cast<uint32_t>(kMaxGammaAttempts); ++k) {
        const uint4 w = philox4x32_10(make_uint4(k, word1, stream, tag_chain), key);
        double z, unused;
        box_muller_f64(w.x, w.y, z, unused);
        double v = 1.0 + c * z;
        if (v <= 0.0)
            continue;
        v = v * v * v;
        const double u = u01_f64(w.z);
        if (log(u) < 0.5 * z * z + d - d * v + d * log(v)) {
            double g = d * v;
            if (boost)
                g *= pow(u01_f64(w.w), 1.0 / shape);
            return g / rate;
        }
    }
    fell_back = 1;
    return d / rate;
}

// ------------------------------------------------------------------------------------------
// Vector loads/stores of V consecutive chain values.
// ------------------------------------------------------------------------------------------
template <typename T, int V> struct Vec;
template <> struct Vec<float, 1> {
    __device__ __forceinline__ static void ld(const float *p, float (&v)[1]) { v[0] = *p; }
    __device__ __forceinline__ static void st(float *p, const float (&v)[1]) { *p = v[0]; }
};
template <> struct Vec<float, 2> {
    __device__ __forceinline__ static void ld(const float *p, float (&v)[2]) { float2 t = *reinterpret_cast<const float2 *>(p); v[0] = t.x; v[1] = t.y; }
    __device__ __forceinline__ static void st(float *p, const float (&v)[2]) { *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]); }
};
template <> struct Vec<float, 4> {
    __device__ __forceinline__ static void ld(const float *p, float (&v)[4]) { float4 t = *reinterpret_cast<const float4 *>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    __device__ __forceinline__ static void st(float *p, const float (&v)[4]) { *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct Vec<double, 1> {
    __device__ __forceinline__ static void ld(const double *p, double (&v)[1]) { v[0] = *p; }
    __device__ __forceinline__ static void st(double *p, const double (&v)[1]) { *p = v[0]; }
};
template <> struct Vec<double, 2> {
    __device__ __forceinline__ static void ld(const double *p, double (&v)[2]) { double2 t = *reinterpret_cast<const double2 *>(p); v[0] = t.x; v[1] = t.y; }
    __device__ __forceinline__ static void st(double *p, const double (&v)[2]) { *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]); }
};

// Natural site index <-> slot of the colour-split lattice layouts.
//   2-D 4-neighbour and 3-D 6-neighbour: colour c = parity of the coordinate sum; sub-array
//   row = (l*H + i), column h = j / 2 (the colour-c sites of a row are j = 2h + ((c+l+i) & 1)).
//   2-D 8-neighbour: colour c = 2 (i & 1) + (j & 1); sub-array (i / 2, j / 2).
__device__ __forceinline__ int64_t lattice_slot_of_site(const FieldDev &f, int64_t site)
{
    if (f.kind == kLat2D8) {
        const int64_t W = f.dims[1];
        const int64_t i = site / W, j = site - i * W;
        const int64_t c = 2 * (i & 1) + (j & 1);
        return (c * f.rows + (i >> 1)) * f.cols + (j >> 1);
    }
    const int64_t W = (f.kind == kLat3D6) ? f.dims[2] : f.dims[1];
    const int64_t r = site / W, j = site - r * W;  // r = l*H + i
    int64_t par = r + j;
    if (f.kind == kLat3D6) {
        const int64_t H = f.dims[1];
        const int64_t l = r / H, i = r - l * H;
        par = l + i + j;
    }
    const int64_t c = par & 1;
    return (c * f.rows + r) * f.cols + (j >> 1);
}

}  // namespace gmrf
