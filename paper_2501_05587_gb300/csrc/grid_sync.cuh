// Grid-wide barrier for cooperative launches (every CTA of the grid resident at once),
// shared by the one-launch fit (fused_fit.cu) and K-means++ seeding (seeding.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_common.cuh"

namespace popcorn {
namespace gsync {

// Grid-wide barrier of the cooperative launch (all CTAs resident).  After the CTA's own
// barrier, thread 0 arrives with an acquire-release add on a monotonic arrival count: the
// add's release covers the CTA's writes (ordered before it by the CTA barrier), and each add
// acquires the previous one, so the adds form one chain.  The barrier's target is the next
// multiple of the grid size above this CTA's arrival; the last to arrive passes at once, the
// others wait with acquire loads, bounded, until the count reaches the target (a CTA already
// arriving at the next barrier only raises it further).  No reset and no generation word:
// one round trip to L2 fewer than a count reset by the last arrival plus a generation flag.
// False when the wait ran out or another CTA gave up, in which case the whole CTA leaves.
// bar: a word zero before the launch (at most 2^31 / gridDim.x barriers a launch).
// (Measured on the blobs workload, one counter beats a two-level counter tree and per-CTA
// release flags polled with acquire loads: the cost is round trips to L2, not contention.)
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ inline bool grid_barrier(unsigned* bar, int* err, unsigned long long limit_ns = tc::kWaitLimitNs) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = err;
        const unsigned arrival = atom_add_acq_rel(bar, 1u);
        const unsigned target = (arrival / gridDim.x + 1u) * gridDim.x;
        int ok = 1;
        if (arrival + 1u != target) {
            const unsigned long long t0 = tc::globaltimer();
            unsigned spins = 0;
            while ((int)(ld_acquire(bar) - target) < 0) {
                if ((++spins & 63u) == 0u) {
                    if (*verr || tc::globaltimer() - t0 > limit_ns) {
                        if (!*verr) atomicExch(err, 1);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace gsync
}  // namespace popcorn
