// resident_draws.cuh -- the conjugate draws of the resident kernels (Sec. 3.1), run by lane 0 of
// the two drawing warps of a block that holds one chain: warp 0 draws tau | x, warp 1 beta0 | x,
// sigma^2 (with the intercept) and then sigma^2 | x, beta0.  The formulas, variates and counters
// are those of hyper_draw.
//
// prep() runs while the site threads sweep: it takes the sweep's unit-rate Gamma variate (from
// the batch precomputed by gamma_pre_kernel, else drawn here) and the intercept's normal and
// scale, which depend on no state of this sweep.  draw() runs between the barrier after the
// block's sums and the barrier that ends the sweep, and publishes the next sweep's copies in the
// state precision T to shared memory.  FP32 state: draw() computes those copies in single
// precision from the block's single-precision sums (a few short-latency operations), and the
// stored and traced values are the same numbers widened to FP64 (sigma^2 as the FP64 reciprocal
// of the 1/sigma^2 used), written by record() in the next sweep's shadow, so a run resumed from
// fetched values continues bit for bit.  FP64 state: draw() runs the FP64 formulas and records.
#pragma once

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {

template <typename T>
struct ResidentDraws {
    static constexpr bool kSplit = sizeof(T) == 4;
    int dw;                       // 0: tau; 1: beta0, sigma^2
    int chain;
    int64_t hc;                   // (field 0, chain)
    uint32_t stream;
    int32_t rank;
    double fn;
    T *hyp;                       // the precision-T copies in global memory
    double tau_d, sig2_d, beta_d; // current values (FP64)
    double G, dz;                 // this sweep's unit-rate Gamma variate and intercept term
    float Gf, dzf, b_tau_f, b_sig_f, fn_f, inv_n_f;
    float tau_f, isig_f, beta_f;  // kSplit: the last sweep's draws
    long long slot_used;          // trace slot of the sweep being drawn

    __device__ __forceinline__ void init(const HyperArgs &h, int dw_, int chain_, const FieldDev &f)
    {
        dw = dw_;
        chain = chain_;
        hc = chain_;
        stream = f.stream;
        rank = f.rank;
        fn = static_cast<double>(f.n);
        hyp = static_cast<T *>(h.hyp) + hc * kHypStride;
        tau_d = h.tau[hc];
        sig2_d = h.sig2[hc];
        beta_d = h.beta[hc];
        G = dz = 0.0;
        Gf = dzf = 0.0f;
        b_tau_f = static_cast<float>(h.b_tau);
        b_sig_f = static_cast<float>(h.b_sig);
        fn_f = static_cast<float>(f.n);
        inv_n_f = static_cast<float>(1.0 / f.n);
        tau_f = isig_f = beta_f = 0.0f;
        slot_used = 0;
    }

    // kSplit: store and trace the last sweep's draws.
    __device__ __forceinline__ void record(const HyperArgs &h)
    {
        if (dw == 0) {
            if (h.draw) {
                tau_d = static_cast<double>(tau_f);
                h.tau[hc] = tau_d;
                hyp[0] = static_cast<T>(tau_f);
            }
            if (h.trace_cap > 0) h.trace_tau[hc * h.trace_cap + slot_used] = tau_d;
        } else {
            if (h.draw_beta) {
                beta_d = static_cast<double>(beta_f);
                h.beta[hc] = beta_d;
                hyp[2] = static_cast<T>(beta_f);
            }
            if (h.draw) {
                sig2_d = 1.0 / static_cast<double>(isig_f);
                h.sig2[hc] = sig2_d;
                hyp[1] = static_cast<T>(isig_f);
            }
            if (h.trace_cap > 0) {
                h.trace_sig[hc * h.trace_cap + slot_used] = sig2_d;
                if (h.trace_beta) h.trace_beta[hc * h.trace_cap + slot_used] = beta_d;
            }
        }
    }

    // The state-independent part of sweep `sw` (after the record of the previous sweep when
    // kSplit and `after_first`); `slot` is the sweep's trace slot.
    __device__ __forceinline__ void prep(const HyperArgs &h, long long sw, long long slot, bool after_first,
                                         long long bbase, long long bcount, int Cp)
    {
        if (kSplit && after_first) record(h);
        const uint32_t sweep = static_cast<uint32_t>(sw);
        const long long kb = sw - bbase;
        const bool pre = h.gpre != nullptr && kb >= 0 && kb < bcount;
        const double *gp = pre ? h.gpre + (kb * h.nfields * Cp + chain) * 4 : nullptr;
        G = 0.0;
        dz = 0.0;
        if (h.draw) {
            if (pre) {
                G = gp[dw];
            } else {
                const uint32_t tag = dw ? kTagSig : kTagTau;
                const double shape = dw ? h.a_sig + 0.5 * fn : h.a_tau + 0.5 * rank;
                int fb = 0;
                G = gamma_mt(shape, 1.0, h.key, sweep, stream, (tag << 24) | static_cast<uint32_t>(chain), fb);
                if (fb) atomicAdd(reinterpret_cast<unsigned long long *>(&h.ctl->fallbacks), 1ull);
            }
        }
        if (dw == 1 && h.draw_beta) {
            double zb = 0.0;
            if (pre) {
                zb = gp[2];
            } else {
                const uint4 w =
                    philox4x32_10(make_uint4(0u, sweep, stream, (kTagBeta << 24) | static_cast<uint32_t>(chain)), h.key);
                double unused;
                box_muller_f64(w.x, w.y, zb, unused);
            }
            dz = sqrt(sig2_d / fn) * zb;
        }
        Gf = static_cast<float>(G);
        dzf = static_cast<float>(dz);
        slot_used = slot;
    }

    // The draws from the block's sums: warp 0 v0 = S; warp 1 v0 = R, v1 = A.  `beta` is the beta0
    // copy the sweep used; the next sweep's copies go to hs[0..2].
    __device__ __forceinline__ void draw(const HyperArgs &h, T v0, T v1, T beta, T *hs)
    {
        if constexpr (kSplit) {
            if (dw == 0) {
                if (h.draw) {
                    tau_f = Gf / (b_tau_f + 0.5f * v0);
                    hs[0] = tau_f;
                }
            } else {
                float R = v0;
                if (h.draw_beta) {
                    const float delta = v1 * inv_n_f + dzf;
                    beta_f = beta + delta;
                    hs[2] = beta_f;
                    R = R - 2.0f * delta * v1 + fn_f * (delta * delta);
                }
                if (h.draw) {
                    isig_f = Gf / (b_sig_f + 0.5f * R);
                    hs[1] = isig_f;
                }
            }
        } else {
            const double S = static_cast<double>(v0), A = static_cast<double>(v1);
            if (dw == 0) {
                if (h.draw) {
                    tau_d = G / (h.b_tau + 0.5 * S);
                    hs[0] = static_cast<T>(tau_d);
                    h.tau[hc] = tau_d;
                    hyp[0] = static_cast<T>(tau_d);
                }
                if (h.trace_cap > 0) h.trace_tau[hc * h.trace_cap + slot_used] = tau_d;
            } else {
                double R = S;
                if (h.draw_beta) {
                    const double delta = A / fn + dz;
                    beta_d = static_cast<double>(beta) + delta;
                    R = R - 2.0 * delta * A + fn * (delta * delta);
                    hs[2] = static_cast<T>(beta_d);
                    h.beta[hc] = beta_d;
                    hyp[2] = static_cast<T>(beta_d);
                }
                if (h.draw) {
                    sig2_d = (h.b_sig + 0.5 * R) / G;
                    const double prec = 1.0 / sig2_d;  // from sigma^2, as the per-sweep path
                    hs[1] = static_cast<T>(prec);
                    h.sig2[hc] = sig2_d;
                    hyp[1] = static_cast<T>(prec);
                }
                if (h.trace_cap > 0) {
                    h.trace_sig[hc * h.trace_cap + slot_used] = sig2_d;
                    if (h.trace_beta) h.trace_beta[hc * h.trace_cap + slot_used] = beta_d;
                }
            }
        }
    }

    // After the last sweep of a launch.
    __device__ __forceinline__ void finish(const HyperArgs &h)
    {
        if (kSplit) record(h);
    }
};

}  // namespace gmrf
