// Grid-wide barrier for cooperative launches (every CTA of the grid resident at once),
// shared by the one-launch fit (fused_fit.cu) and K-means++ seeding (seeding.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_common.cuh"

namespace popcorn {
namespace gsync {

// Grid-wide barrier of the cooperative launch (all CTAs resident).  After the CTA's own
// barrier, thread 0 arrives with an acquire-release add on the arrival count (its release
// covers the CTA's writes, ordered before it by the CTA barrier); the last to arrive resets
// the count and publishes the next generation with a release store, the others wait for it
// with acquire loads, bounded.  False when the wait ran out or another CTA gave up, in which
// case the whole CTA leaves.  bar: two words in one 128-byte line, zero before the launch.
// (Measured on the blobs workload, this single counter beats a two-level counter tree and
// per-CTA release flags polled with acquire loads: the cost is round trips to L2, not
// contention.)
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

__device__ inline bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* verr = err;
        const unsigned g = ld_acquire(bar + 1);
        int ok = 1;
        if (atom_add_acq_rel(bar, 1u) == gridDim.x - 1) {
            st_relaxed(bar, 0u);
            st_release(bar + 1, g + 1);
        } else {
            const unsigned long long t0 = tc::globaltimer();
            unsigned spins = 0;
            while (ld_acquire(bar + 1) == g) {
                if ((++spins & 63u) == 0u) {
                    if (*verr || tc::globaltimer() - t0 > tc::kWaitLimitNs) {
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
