// pg.cuh -- Polya-Gamma variates on the device, for binomial data with the logistic link
// (Sec. 3.2; Polson, Scott & Windle, JASA 2013).
//
// PG(b, c) for an integer b >= 0 is the sum of b independent PG(1, c) = J*(1, z) / 4 variates,
// z = |c| / 2.  Each J*(1, z) is drawn by Devroye's alternating-series method: propose from the
// envelope exp(-z^2 x / 2) a_0(x), a mixture of an exponential tail on (t, inf) (weight
// p / (p + q)) and an inverse Gaussian IG(1/z, 1) truncated to (0, t), t = 0.64, and accept when
// V a_0(X) falls below a partial sum a_0 - a_1 + a_2 - ... of the J*(1, 0) density.
//
// Arithmetic is FP64 throughout (the accept/reject decisions must be taken in the same
// precision as the oracle's).  Random numbers: draw k of (site, sweep, chain) reads uniforms
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

__device__ __forceinline__ double pg_uniform(PgStream &s)
{
    if (s.idx == 4) {
        if (s.blk >= 1024) {
            s.out = true;
            return 0.5;
        }
        s.w = philox4x32_10(make_uint4(s.ctr.x, s.ctr.y, s.ctr.z, s.ctr.w | static_cast<uint32_t>(s.blk)), s.key);
        ++s.blk;
        s.idx = 0;
    }
    const uint32_t v = s.idx == 0 ? s.w.x : (s.idx == 1 ? s.w.y : (s.idx == 2 ? s.w.z : s.w.w));
    ++s.idx;
    return u01_f64(v);
}

constexpr double kPgT = 0.64;
constexpr double kPi = 3.14159265358979323846;

// Term n of the J*(1, 0) density series: small-x form for x <= t, large-x form above.
__device__ __forceinline__ double pg_term(int n, double x)
{
    const double h = n + 0.5;
    if (x <= kPgT) {
        const double r = 2.0 / (kPi * x);
        return kPi * h * r * sqrt(r) * exp(-2.0 * h * h / x);
    }
    return kPi * h * exp(-h * h * kPi * kPi * x / 2.0);
}

__device__ __forceinline__ double pg_norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

// Weight of the exponential piece of the envelope, p / (p + q):
//   p = pi / (2K) exp(-K t), K = pi^2/8 + z^2/2;
//   q = 2 exp(-z) F_IG(t; 1/z, 1) = 2 exp(-z) [Phi((tz - 1)/sqrt t) + exp(2z) Phi(-(tz + 1)/sqrt t)],
//   q = 4 Phi(-1/sqrt t) at z = 0; the inverse-Gaussian piece is dropped for z > 40 (weight < 1e-17).
__device__ __forceinline__ double pg_exp_weight(double z)
{
    if (z > 40.0) return 1.0;
    const double K = kPi * kPi / 8.0 + 0.5 * z * z;
    const double p = kPi / (2.0 * K) * exp(-K * kPgT);
    const double rt = sqrt(kPgT);
    const double q = z == 0.0 ? 4.0 * pg_norm_cdf(-1.0 / rt)
                              : 2.0 * exp(-z) * (pg_norm_cdf((kPgT * z - 1.0) / rt) +
                                                 exp(2.0 * z) * pg_norm_cdf(-(kPgT * z + 1.0) / rt));
    return p / (p + q);
}

// IG(1/z, 1) truncated to (0, t).
__device__ __forceinline__ double pg_trunc_ig(double z, PgStream &s)
{
    if (z == 0.0 || 1.0 / z > kPgT) {
        // 1/X from a truncated chi-square-like tail (rejection on two exponentials), then the
        // exp(-z^2 X / 2) tilt by rejection.
        while (true) {
            double e1, e2;
            do {
                e1 = -log(pg_uniform(s));
                e2 = -log(pg_uniform(s));
                if (s.out) return kPgT / 2.0;
            } while (e1 * e1 > 2.0 * e2 / kPgT);
            const double a = 1.0 + kPgT * e1;
            const double x = kPgT / (a * a);
            const double keep = exp(-0.5 * z * z * x);
            if (pg_uniform(s) <= keep || s.out) return x;
        }
    }
    const double mu = 1.0 / z;
    while (true) {
        const double ua = pg_uniform(s);  // the two uniforms of a normal, in this order
        const double ub = pg_uniform(s);
        const double g = sqrt(-2.0 * log(ua)) * cos(2.0 * kPi * ub);
        const double y = g * g;
        double x = mu + 0.5 * mu * mu * y - 0.5 * mu * sqrt(4.0 * mu * y + (mu * y) * (mu * y));
        if (pg_uniform(s) > mu / (mu + x)) x = mu * mu / x;
        if (x <= kPgT || s.out) return x;
    }
}

// J*(1, z); negative when the stream ran out.
__device__ __forceinline__ double pg_jstar(double z, double wexp, PgStream &s)
{
    const double K = kPi * kPi / 8.0 + 0.5 * z * z;
    while (true) {
        const double U = pg_uniform(s), V = pg_uniform(s);
        const double x = U < wexp ? kPgT - log(pg_uniform(s)) / K : pg_trunc_ig(z, s);
        if (s.out) return -1.0;
        double S = pg_term(0, x);
        const double Y = V * S;
        for (int n = 1; n < 1000; ++n) {
            if (n & 1) {
                S -= pg_term(n, x);
                if (Y <= S) return x;
            } else {
                S += pg_term(n, x);
                if (Y > S) break;
            }
        }
    }
}

// PG(b, c) for the (site, sweep, chain) counters; *fallbacks counts exhausted streams.
__device__ __forceinline__ double pg_draw(int b, double c, uint2 key, uint32_t site, uint32_t sweep, uint32_t stream,
                                          uint32_t chain, int &fallbacks)
{
    const double z = 0.5 * fabs(c);
    const double wexp = b > 0 ? pg_exp_weight(z) : 0.0;
    double sum = 0.0;
    for (int k = 0; k < b; ++k) {
        PgStream s;
        pg_stream_init(s, key, site, sweep, stream, chain, static_cast<uint32_t>(k));
        double j = pg_jstar(z, wexp, s);
        if (j < 0.0) {
            ++fallbacks;
            j = z > 0.0 ? tanh(z) / z : 1.0;
        }
        sum += 0.25 * j;
    }
    return sum;
}

}  // namespace gmrf
