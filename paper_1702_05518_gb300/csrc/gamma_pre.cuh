// gamma_pre.cuh -- the unit-rate Gamma variates (Marsaglia-Tsang) of tau and 1/sigma^2 and the
// intercept's standard normals for a batch of sweeps (Sec. 3.1 conditionals), one task per
// thread; shared by gamma_pre_kernel and the resident normals kernel, which draws them in blocks
// of its own while its other blocks draw the batch's site normals.
#pragma once

#include "gmrf_device.cuh"
#include "gmrf_internal.h"

namespace gmrf {

// Tasks of a batch: 4 per (sweep, field, chain); task q: which = q & 3 (0: tau's variate, 1:
// 1/sigma^2's, 2: the intercept's normal, 3: unused), pair (q >> 2) mod F Cp, sweep base + (q >> 2)
// / F Cp.  The variates do not depend on the state, so a batch runs in parallel and the
// per-sweep draw reduces to a division by the rate (and a shift for the intercept).
__device__ __forceinline__ int gamma_pre_tasks(const GammaPreArgs &a) { return a.count * a.nfields * a.Cp * 4; }

__device__ __forceinline__ void gamma_pre_task(const GammaPreArgs &a, int q, long long base)
{
    const int npairs = a.nfields * a.Cp;
    const int which = q & 3, pidx = (q >> 2) % npairs, k = (q >> 2) / npairs;
    if (which == 3) return;
    const int fi = pidx / a.Cp, chain = pidx - fi * a.Cp;
    const FieldDev &f = a.fields[fi];
    const uint32_t word1 = static_cast<uint32_t>(base + k);
    if (which == 2) {
        double zb = 0.0, unused;
        if (a.intercept) {
            const uint4 w =
                philox4x32_10(make_uint4(0u, word1, f.stream, (kTagBeta << 24) | static_cast<uint32_t>(chain)), a.key);
            box_muller_f64(w.x, w.y, zb, unused);
        }
        a.gpre[q] = zb;
        return;
    }
    const double shape = which ? a.a_sig + 0.5 * f.n : a.a_tau + 0.5 * f.rank;
    const uint32_t tag = which ? kTagSig : kTagTau;
    int fb = 0;
    a.gpre[q] = gamma_mt(shape, 1.0, a.key, word1, f.stream, (tag << 24) | static_cast<uint32_t>(chain), fb);
    if (fb) atomicAdd(reinterpret_cast<unsigned long long *>(&a.ctl->fallbacks), 1ull);
}

// Records the batch in the control block (one thread, after reading `base` = ctl->sweep).
__device__ __forceinline__ void gamma_pre_record(const GammaPreArgs &a, long long base)
{
    a.ctl->batch_base = base;
    a.ctl->batch_count = a.count;
}

}  // namespace gmrf
