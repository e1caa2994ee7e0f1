// Building blocks of the K-streaming reductions (iterate.cu, reduce_sym.cu) and the
// pass finalization they share.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "popcorn_internal.cuh"

namespace popcorn {
namespace stream {

__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// hi + lo += x without rounding loss (Knuth's TwoSum; FP32 pipe only).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += e;
}

// Cluster whose warp total lane `lane` holds after butterfly<KB>.
template <int KB>
__device__ __forceinline__ int bfly_cluster(int lane) {
    int c = 0;
#pragma unroll
    for (int w = KB >> 1, off = 16; w >= 1; w >>= 1, off >>= 1)
        if (lane & off) c += w;
    return c;
}

// Reduce-scatter of KB per-lane partials over the warp: each level halves
// the values a lane carries (one half goes to the partner, the other half is
// kept), then the remaining levels all-reduce the single value left.
template <int KB>
__device__ __forceinline__ float butterfly(const float (&acc)[KB], int lane) {
    float v[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) v[t] = acc[t];
    int off = 16;
#pragma unroll
    for (int cnt = KB; cnt > 1; cnt >>= 1, off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int t = 0; t < cnt / 2; ++t) {
            const float send = up ? v[t] : v[t + cnt / 2];
            const float keep = up ? v[t + cnt / 2] : v[t];
            v[t] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
#pragma unroll
    for (; off > 0; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
    return v[0];
}

// Last block of a pass's reduction, all its threads (a multiple of 32): sum the
// per-block FP64 partials of sum_{i in L_c} S_ic, then ||c_c||^2 =
// (1/m_c^2) sum_{i in L_c} S_ic (Eq. 13/14), 1/m_c, and
// J = trace K - sum_c (1/m_c) sum_{i in L_c} S_ic.  Warp w takes clusters
// w, w + nw, ...; its lanes split the blocks and a butterfly adds them, so the
// partials are read 32 at a time rather than one after another.  Every order
// is fixed: the result is deterministic.
__device__ inline void finalize_pass(const double* zpart, int nblocks, int k, const int32_t* counts, double* zsum,
                                     double* cnorm, double* invm, LoopState* st, double* J_hist, int eval_only) {
    __shared__ double jpart[32];
    const int32_t* m = counts + (size_t)(st->iter & 1) * k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double jw = 0.0;
    for (int c = warp; c < k; c += nw) {
        double t = 0.0;
        for (int b = lane; b < nblocks; b += 32) t += __ldcg(zpart + (size_t)b * k + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const double mc = (double)__ldcg(m + c);
        const double inv = mc > 0 ? 1.0 / mc : 0.0;
        if (lane == 0) {
            zsum[c] = t;
            invm[c] = inv;
            cnorm[c] = t * inv * inv;
        }
        jw += t * inv;
    }
    if (lane == 0 && warp < 32) jpart[warp] = jw;
    __syncthreads();
    if (threadIdx.x == 0) {
        double J = st->trace;
        for (int w = 0; w < nw && w < 32; ++w) J -= jpart[w];
        if (eval_only) {
            st->J_eval = J;
        } else {
            J_hist[st->iter] = J;
            st->J_last = J;
        }
        st->reduce_ticket = 0u;
    }
}

}  // namespace stream
}  // namespace popcorn
