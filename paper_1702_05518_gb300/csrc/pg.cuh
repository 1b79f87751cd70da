// pg.cuh -- Polya-Gamma variates on the device, for binomial data with the logistic link
// (Sec. 3.2; Polson, Scott & Windle, JASA 2013).
//
// PG(b, c) for an integer b >= 0 is the sum of b independent PG(1, c) = J*(1, z) / 4 variates,
// z = |c| / 2.  Each J*(1, z) is drawn by Devroye's alternating-series method: propose from the
// envelope exp(-z^2 x / 2) a_0(x), a mixture of an exponential tail on (t, inf) (weight
// p / (p + q)) and an inverse Gaussian IG(1/z, 1) truncated to (0, t), t = 0.64, and accept when
// V a_0(X) falls below a partial sum a_0 - a_1 + a_2 - ... of the J*(1, 0) density.
//
// Arithmetic in precision P: FP64 for FP64 samplers (the accept/reject decisions are then taken
// in the oracle's precision and the chains stay coupled with it draw for draw), FP32 for FP32
// samplers (the same algorithm; its decisions see single-precision rounding, which the state
// already carries, and FP64 special functions are slow on this GPU).  Random numbers: draw k of (site, sweep, chain) reads uniforms
// u = (w + 1/2) 2^-32 in order from the words of the Philox blocks at counters
// (site, sweep, stream, 0xA << 28 | chain << 22 | k << 10 | j), j = 0, 1, ...; a normal takes two
// (Box-Muller cosine).  A draw that would need more than 1024 blocks (never observed) returns
// the mean tanh(z) / z of J*(1, z) and counts a fallback.
#pragma once

#include "gmrf_device.cuh"

namespace gmrf {

struct PgStream {
    uint2 key;
    uint4 ctr;     // word 3 holds the tag, chain and draw; the block index is or-ed in
    uint4 w;
    int idx;       // next word of w; 4 = fetch the next block
    int blk;
    bool out;      // ran past the last block
};

__device__ __forceinline__ void pg_stream_init(PgStream &s, uint2 key, uint32_t site, uint32_t sweep,
                                               uint32_t stream, uint32_t chain, uint32_t k)
{
    s.key = key;
    s.ctr = make_uint4(site, sweep, stream, (0xAu << 28) | (chain << 22) | (k << 10));
    s.idx = 4;
    s.blk = 0;
    s.out = false;
}

template <typename P> __device__ __forceinline__ P pg_u01(uint32_t w);
template <> __device__ __forceinline__ double pg_u01<double>(uint32_t w) { return u01_f64(w); }
template <> __device__ __forceinline__ float pg_u01<float>(uint32_t w) { return u01_f32(w); }

template <typename P>
__device__ __forceinline__ P pg_uniform(PgStream &s)
{
    if (s.idx == 4) {
        if (s.blk >= 1024) {
            s.out = true;
            return static_cast<P>(0.5);
        }
        s.w = philox4x32_10(make_uint4(s.ctr.x, s.ctr.y, s.ctr.z, s.ctr.w | static_cast<uint32_t>(s.blk)), s.key);
        ++s.blk;
        s.idx = 0;
    }
    const uint32_t v = s.idx == 0 ? s.w.x : (s.idx == 1 ? s.w.y : (s.idx == 2 ? s.w.z : s.w.w));
    ++s.idx;
    return pg_u01<P>(v);
}

constexpr double kPgT = 0.64;
constexpr double kPi = 3.14159265358979323846;

// Term n of the J*(1, 0) density series: small-x form for x <= t, large-x form above.
template <typename P>
__device__ __forceinline__ P pg_term(int n, P x)
{
    const P t = static_cast<P>(kPgT), pi = static_cast<P>(kPi);
    const P h = static_cast<P>(n) + static_cast<P>(0.5);
    if (x <= t) {
        const P r = static_cast<P>(2) / (pi * x);
        return pi * h * r * sqrt(r) * exp(static_cast<P>(-2) * h * h / x);
    }
    return pi * h * exp(-h * h * pi * pi * x / static_cast<P>(2));
}

template <typename P>
__device__ __forceinline__ P pg_norm_cdf(P x) { return static_cast<P>(0.5) * erfc(-x / sqrt(static_cast<P>(2))); }

// Weight of the exponential piece of the envelope, p / (p + q):
//   p = pi / (2K) exp(-K t), K = pi^2/8 + z^2/2;
//   q = 2 exp(-z) F_IG(t; 1/z, 1) = 2 exp(-z) [Phi((tz - 1)/sqrt t) + exp(2z) Phi(-(tz + 1)/sqrt t)],
//   q = 4 Phi(-1/sqrt t) at z = 0; the inverse-Gaussian piece is dropped for z > 40 (weight < 1e-17).
template <typename P>
__device__ __forceinline__ P pg_exp_weight(P z)
{
    const P t = static_cast<P>(kPgT), pi = static_cast<P>(kPi), one = static_cast<P>(1);
    if (z > static_cast<P>(40)) return one;
    const P K = pi * pi / static_cast<P>(8) + static_cast<P>(0.5) * z * z;
    const P p = pi / (static_cast<P>(2) * K) * exp(-K * t);
    const P rt = sqrt(t);
    const P q = z == static_cast<P>(0) ? static_cast<P>(4) * pg_norm_cdf<P>(-one / rt)
                                       : static_cast<P>(2) * exp(-z) * (pg_norm_cdf<P>((t * z - one) / rt) +
                                                                         exp(static_cast<P>(2) * z) *
                                                                             pg_norm_cdf<P>(-(t * z + one) / rt));
    return p / (p + q);
}

// IG(1/z, 1) truncated to (0, t).
template <typename P>
__device__ __forceinline__ P pg_trunc_ig(P z, PgStream &s)
{
    const P t = static_cast<P>(kPgT), one = static_cast<P>(1), half = static_cast<P>(0.5);
    if (z == static_cast<P>(0) || one / z > t) {
        // 1/X from a truncated chi-square-like tail (rejection on two exponentials), then the
        // exp(-z^2 X / 2) tilt by rejection.
        while (true) {
            P e1, e2;
            do {
                e1 = -log(pg_uniform<P>(s));
                e2 = -log(pg_uniform<P>(s));
                if (s.out) return t / static_cast<P>(2);
            } while (e1 * e1 > static_cast<P>(2) * e2 / t);
            const P a = one + t * e1;
            const P x = t / (a * a);
            const P keep = exp(-half * z * z * x);
            if (pg_uniform<P>(s) <= keep || s.out) return x;
        }
    }
    const P mu = one / z;
    while (true) {
        const P ua = pg_uniform<P>(s);  // the two uniforms of a normal, in this order
        const P ub = pg_uniform<P>(s);
        const P g = sqrt(static_cast<P>(-2) * log(ua)) * cos(static_cast<P>(2 * kPi) * ub);
        const P y = g * g;
        P x = mu + half * mu * mu * y - half * mu * sqrt(static_cast<P>(4) * mu * y + (mu * y) * (mu * y));
        if (pg_uniform<P>(s) > mu / (mu + x)) x = mu * mu / x;
        if (x <= t || s.out) return x;
    }
}

// J*(1, z); negative when the stream ran out.
template <typename P>
__device__ __forceinline__ P pg_jstar(P z, P wexp, PgStream &s)
{
    const P t = static_cast<P>(kPgT), pi = static_cast<P>(kPi);
    const P K = pi * pi / static_cast<P>(8) + static_cast<P>(0.5) * z * z;
    while (true) {
        const P U = pg_uniform<P>(s), V = pg_uniform<P>(s);
        const P x = U < wexp ? t - log(pg_uniform<P>(s)) / K : pg_trunc_ig<P>(z, s);
        if (s.out) return static_cast<P>(-1);
        P S = pg_term<P>(0, x);
        const P Y = V * S;
        for (int n = 1; n < 1000; ++n) {
            if (n & 1) {
                S -= pg_term<P>(n, x);
                if (Y <= S) return x;
            } else {
                S += pg_term<P>(n, x);
                if (Y > S) break;
            }
        }
    }
}

}  // namespace gmrf
