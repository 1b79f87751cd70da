// hyper_task.cuh -- the conjugate draws of one (field, chain) pair after a sweep (Sec. 3.1), as a
// warp-level device function shared by the hyperparameter kernel and the quad kernel's tail.
#pragma once

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {

// Task 2p draws tau of (field, chain) pair p, task 2p + 1 the intercept (when present) and then
// 1/sigma^2 of pair p (given x, tau is conditionally independent of beta0 and sigma^2,
// Sec. 3.1).  A warp sums what it needs over the field's tile partials in a fixed order (lane
// strides, then a shuffle tree), and lane 0 draws from the full conditionals, refreshes the
// precision-T copies the colour kernels read, and records the traces.  FP64 arithmetic has a
// long dependent-operation latency on this GPU, so everything a draw needs is loaded before
// the sums, and tasks run in parallel warps.  Once every task of a launch has run,
// hyper_advance moves the counters on.
//
// Binomial model (Sec. 3.2): task 2p + 1 draws beta0 from its normal conditional given the sums
// of psi_i and kappa_i - psi_i x_i that the partials then hold; there is no sigma^2.
//
// Intercept: the partials hold R = sum e_i^2 and A = sum e_i with e_i = y_i - b - x_i, b the
// copy of beta0 the sweep used.  beta0 | x, sigma^2 ~ N(1'(y - x)/n, sigma^2/n) is drawn as
// b + delta, delta = A/n + sqrt(sigma^2/n) z, and the sigma^2 draw takes
// sum (e_i - delta)^2 = R - 2 delta A + n delta^2 (exact algebra; delta is small next to e).
//
// Gamma draws: G = Marsaglia-Tsang variate at rate 1 (precomputed for the batch, or drawn here);
// tau = G / rate, sigma^2 = rate / G (the reciprocal of the precision draw G / rate).

// The draw of one task given its sums, by one thread (see hyper_task): `cur` is the current value
// of the parameter drawn (tau, or sigma^2), `s2old` the current sigma^2, `b` the beta0 copy the
// sweep used, gpv and zb the precomputed Gamma variate and normal when `pre`.  With `rec`, writes
// the FP64 values, the precision-T copies and the traces (without it the caller only takes the
// results: the blocks of the resident quad kernel that draw redundantly); returns the parameter's
// new value (tau or sigma^2) in val and, for task 1, beta0 in bval.
template <typename T>
__device__ __forceinline__ void hyper_draw(const HyperArgs &a, int which, int chain, int64_t hc, long long sweep,
                                           double S, double A, double cur, double s2old, double b, double gpv,
                                           double zb, bool pre, long long extra, uint32_t fstream, int32_t fn,
                                           int32_t frank, double &val_out, double &bval_out, bool rec = true)
{
    T *hyp = static_cast<T *>(a.hyp);
    const uint32_t word1 = static_cast<uint32_t>(a.end_of_sweep ? sweep : extra);
    double val = cur, bval = 0.0;
    if (which && a.draw_beta) {
        if (!pre) {
            const uint32_t tag = a.end_of_sweep ? kTagBeta : kTagBetaExtra;
            const uint4 w = philox4x32_10(
                make_uint4(0u, word1, fstream, (tag << 24) | static_cast<uint32_t>(chain)), a.key);
            double unused;
            box_muller_f64(w.x, w.y, zb, unused);
        }
        if (a.binomial) {
            // beta0 | x, psi ~ N(mean, 1/Pb), Pb = 1/v0 + sum psi_i,
            // mean = (mu0/v0 + sum (kappa_i - psi_i x_i)) / Pb  (S and A hold the two sums).
            const double Pb = 1.0 / a.beta0_var + S;
            bval = (a.beta0_mean / a.beta0_var + A) / Pb + zb / sqrt(Pb);
        } else {
            const double delta = A / fn + sqrt(s2old / fn) * zb;
            bval = b + delta;
            S = S - 2.0 * delta * A + fn * (delta * delta);
        }
        if (rec) {
            a.beta[hc] = bval;
            hyp[hc * kHypStride + 2] = static_cast<T>(bval);
        }
    } else if (which && a.trace_beta) {
        bval = a.beta[hc];
    }
    if (a.draw && !(which && a.binomial)) {
        const double rate = which ? a.b_sig + 0.5 * S : a.b_tau + 0.5 * S;
        double G = gpv;
        if (!pre) {
            const uint32_t tag =
                which ? (a.end_of_sweep ? kTagSig : kTagSigExtra) : (a.end_of_sweep ? kTagTau : kTagTauExtra);
            const double shape = which ? a.a_sig + 0.5 * fn : a.a_tau + 0.5 * frank;
            int fb = 0;
            G = gamma_mt(shape, 1.0, a.key, word1, fstream, (tag << 24) | static_cast<uint32_t>(chain), fb);
            if (fb) atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->fallbacks), 1ull);
        }
        if (which) {
            // The sweep kernels use 1/sigma^2 recomputed from sigma^2, so a run resumed
            // from a fetched sigma^2 continues bit for bit.
            val = rate / G;
            if (rec) {
                a.sig2[hc] = val;
                hyp[hc * kHypStride + 1] = static_cast<T>(1.0 / val);
            }
        } else {
            val = G / rate;
            if (rec) {
                a.tau[hc] = val;
                hyp[hc * kHypStride] = static_cast<T>(val);
            }
        }
    }
    if (rec && a.end_of_sweep && a.trace_cap > 0) {
        const int64_t slot = hc * a.trace_cap + (sweep % a.trace_cap);
        (which ? a.trace_sig : a.trace_tau)[slot] = val;
        if (which && a.trace_beta) a.trace_beta[slot] = bval;
    }
    val_out = val;
    bval_out = bval;
}

// The values task `which` needs of one tile partial: S (which 0) or R, and A when need_a.  CG:
// loaded through L2 only, field by field.
template <bool CG>
__device__ __forceinline__ void part_values(const Part3 *p, int which, bool need_a, double &v, double &va)
{
    if constexpr (CG) {
        v = __ldcg(which ? &p->R : &p->S);
        va = need_a ? __ldcg(&p->A) : 0.0;
    } else {
        const Part3 q = *p;
        v = which ? q.R : q.S;
        va = need_a ? q.A : 0.0;
    }
}

// The sums of task `which` over the field's tile partials, by all 32 lanes of the calling warp,
// in a fixed order: lane l adds partials l, l + 32, l + 64, ... in that order, then a shuffle
// tree.  S: the S (which 0) or R (which 1) sums; A: the intercept's sums when need_a.  BATCH
// (fields of 256 or more tiles): eight loads are issued before their additions, so a warp waits
// for one L2 round trip per 256 partials, not per 32 (the sums are the same); for fewer partials
// one load at a time measured faster (the draws of the 512 x 512 image: 15.3 against 15.9 us per
// sweep with eight predicated loads in flight).  CG: the partials are loaded through L2 only (the
// resident quad kernel reads partials that other blocks of the same launch rewrite every sweep).
template <bool BATCH, bool CG>
__device__ __forceinline__ void hyper_sums(const HyperArgs &a, int which, bool need_a, int chain, int32_t part0,
                                           int32_t nparts, double &S, double &A)
{
    const int lane = threadIdx.x & 31;
    const Part3 *P = a.partials + static_cast<int64_t>(part0) * a.Cp + chain;
    constexpr int U = 8;
    int k = lane;
    if constexpr (BATCH) {
        for (; k + 32 * (U - 1) < nparts; k += 32 * U) {
            double vs[U], va[U];
#pragma unroll
            for (int j = 0; j < U; ++j)
                part_values<CG>(P + static_cast<int64_t>(k + 32 * j) * a.Cp, which, need_a, vs[j], va[j]);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                S += vs[j];
                if (need_a) A += va[j];
            }
        }
    }
    for (; k < nparts; k += 32) {
        double v, va;
        part_values<CG>(P + static_cast<int64_t>(k) * a.Cp, which, need_a, v, va);
        S += v;
        if (need_a) A += va;
    }
    for (int off = 16; off >= 1; off >>= 1) S += __shfl_xor_sync(0xffffffffu, S, off);
    if (need_a)
        for (int off = 16; off >= 1; off >>= 1) A += __shfl_xor_sync(0xffffffffu, A, off);
}

// The sums of hyper_sums<*, true> from a copy of the partials laid out by field: sv[k] is the
// S (which 0) or R (which 1) value of partial k and av[k] its A value, so a warp's loads cover
// consecutive doubles (the partial records put 32 lanes' loads in 32 sectors).  Each lane issues
// up to eight loads through L2 before adding them, in the order of hyper_sums (lane l: partials
// l, l + 32, ...; the same shuffle tree), so the sums are bit for bit those of hyper_sums.
__device__ __forceinline__ void hyper_sums_by_field(const double *sv, const double *av, bool need_a,
                                                    int32_t nparts, double &S, double &A)
{
    const int lane = threadIdx.x & 31;
    constexpr int U = 8;
    for (int k0 = lane; k0 < nparts; k0 += 32 * U) {
        double vs[U], va[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int k = k0 + 32 * j;
            vs[j] = k < nparts ? __ldcg(sv + k) : 0.0;
            va[j] = (need_a && k < nparts) ? __ldcg(av + k) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (k0 + 32 * j < nparts) {
                S += vs[j];
                if (need_a) A += va[j];
            }
        }
    }
    for (int off = 16; off >= 1; off >>= 1) S += __shfl_xor_sync(0xffffffffu, S, off);
    if (need_a)
        for (int off = 16; off >= 1; off >>= 1) A += __shfl_xor_sync(0xffffffffu, A, off);
}

// One task, run by all 32 lanes of the calling warp; `sweep` is the sweep being finished.
template <typename T, bool BATCH>
__device__ __forceinline__ void hyper_task(const HyperArgs &a, int task, long long sweep)
{
    const int lane = threadIdx.x & 31;
    const int pidx = task >> 1, which = task & 1;  // which: 0 tau, 1 beta0 and sigma^2
    const int fi = pidx / a.Cp, chain = pidx - fi * a.Cp;
    const int64_t hc = static_cast<int64_t>(fi) * a.Cp + chain;
    const int32_t part0 = a.fields[fi].part0, nparts = a.fields[fi].nparts;
    // Loads of lane 0 first, so their latency overlaps the partial sums.
    T *hyp = static_cast<T *>(a.hyp);
    double cur = 0.0, s2old = 0.0, b = 0.0, gpv = 0.0, zb = 0.0;
    long long extra = 0, kb = -1, bcount = 0;
    uint32_t fstream = 0;
    int32_t fn = 0, frank = 0;
    if (lane == 0) {
        cur = which ? a.sig2[hc] : a.tau[hc];
        s2old = a.sig2[hc];
        b = static_cast<double>(hyp[hc * kHypStride + 2]);
        extra = a.ctl->extra;
        kb = sweep - a.ctl->batch_base;
        bcount = a.ctl->batch_count;
        fstream = a.fields[fi].stream;
        fn = a.fields[fi].n;
        frank = a.fields[fi].rank;
    }
    const bool pre = a.end_of_sweep && a.gpre && kb >= 0 && kb < bcount;
    if (lane == 0 && pre) {
        const double *gp = a.gpre + (kb * a.nfields * a.Cp + pidx) * 4;
        gpv = gp[which];
        zb = gp[2];
    }
    const bool need_sum = which ? (a.draw || a.draw_beta) : a.draw;
    const bool need_a = which && a.draw_beta;
    double S = 0.0, A = 0.0;
    if (need_sum) hyper_sums<BATCH, false>(a, which, need_a, chain, part0, nparts, S, A);
    if (lane == 0) {
        double val, bval;
        hyper_draw<T>(a, which, chain, hc, sweep, S, A, cur, s2old, b, gpv, zb, pre, extra, fstream, fn, frank, val,
                      bval);
    }
}

// The counters after every task of a launch has read them (one thread): the sweep number and
// the accumulation count at the end of a sweep, the extra-draw count otherwise.
__device__ __forceinline__ void hyper_advance(const HyperArgs &a, long long sweep)
{
    if (a.end_of_sweep) {
        if (a.acc_enabled && sweep_accumulated(sweep, a.burn_in, a.thin)) a.ctl->acc_count += 1;
        a.ctl->sweep = sweep + 1;
    } else {
        a.ctl->extra += 1;
    }
}

}  // namespace gmrf
