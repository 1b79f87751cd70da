// grid_barrier.cuh -- the grid barrier of the resident tile kernels (lattice_quad.cu,
// lattice_fused_resident.cu): every block of a cooperative launch (all resident at once) arrives
// once per sweep on a counter in the sweep control block and waits, with a bounded wait, until
// all blocks of that sweep have arrived.  A wait that runs out counts itself in
// ctl->wait_timeouts and sets ctl->gabort, at which every other waiting block stops waiting too;
// the caller then leaves its sweep loop (the results are invalid and the host reports
// GMRF_E_TIMEOUT).  The counter is cleared by the last block of the launch.
#pragma once

#include <cstdint>

#include "gmrf_device.cuh"
#include "mbarrier.cuh"

namespace gmrf {

// The barrier's arrival count and abort flag in one load (ctl->gbar, ctl->gabort; 16-byte aligned).
__device__ __forceinline__ void ld_barrier(const unsigned long long *p, unsigned long long &arrivals,
                                           unsigned long long &abort)
{
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(arrivals), "=l"(abort) : "l"(p) : "memory");
}

// One arrival (one thread of the block, after a block barrier that orders the block's stores).
__device__ __forceinline__ void grid_arrive(SweepCtl *ctl)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&ctl->gbar) : "memory");
}

// Wait (one thread) until `target` arrivals, for at most wait_ns; true if the block must stop.
__device__ __forceinline__ bool grid_wait(SweepCtl *ctl, unsigned long long target, uint64_t wait_ns)
{
    bool stop = false;
    unsigned long long arrived, aborted;
    ld_barrier(&ctl->gbar, arrived, aborted);
    const uint64_t t0 = global_ns();
    for (uint32_t spin = 1; arrived < target; ++spin) {
        if (aborted != 0) {
            stop = true;
            break;
        }
        if ((spin & 15u) == 0 && global_ns() - t0 >= wait_ns) {
            atomicAdd(&ctl->wait_timeouts, 1ull);
            atomicExch(&ctl->gabort, 1ull);
            stop = true;
            break;
        }
        ld_barrier(&ctl->gbar, arrived, aborted);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");  // acquire: the stores before every arrival
    return stop;
}

}  // namespace gmrf
