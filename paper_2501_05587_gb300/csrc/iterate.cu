// Per-pass kernels of Kernel K-means (Alg. 2, lines 6-15).
//
// reduce_kernel  -- streams K once per pass.  For every row i and cluster c it
//                   forms the segment sums S_ic = sum_{j in L_c} K_ij, i.e.
//                   (K V^T)_ic * |L_c| (the paper's SpMM, Alg. 2 line 7).  It
//                   also accumulates, in FP64, sum_{i in L_c} S_{i,c} -- the
//                   entries of z (Eq. 14) grouped by cluster, which is the
//                   paper's SpMV V z (Alg. 2 lines 8-9) -- and its last block
//                   turns them into ||c_c||^2 and the objective J.
// assign_kernel  -- D_ic = K_ii - 2 S_ic/|L_c| + ||c_c||^2 (Alg. 2 line 10),
//                   the row argmin (lines 11-13), new labels, the cluster
//                   sizes of the new labels (warp-aggregated atomics) and the
//                   loop-control decision of the pass.
//
// V is never built: a label byte per column is all the K-stream needs.  E and
// D are never stored (E only on request for tests).
#include "popcorn_internal.cuh"
#include "stream_common.cuh"

#include <cuda/std/limits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace popcorn {
namespace {

using namespace stream;

// 16 bytes of a K row: 4 FP32 or 8 FP16 / BF16 elements, and their labels.
template <typename TK> struct KVec;
template <> struct KVec<float> {
    static constexpr int N = 4;
    using Lab = uint32_t;
    __device__ static void unpack(const float4& r, float (&o)[4]) {
        o[0] = r.x; o[1] = r.y; o[2] = r.z; o[3] = r.w;
    }
    __device__ static uint32_t label(const Lab& L, int e) { return (L >> (8 * e)) & 0xffu; }
};
template <> struct KVec<__half> {
    static constexpr int N = 8;
    using Lab = uint2;
    __device__ static void unpack(const float4& r, float (&o)[8]) {
        const uint32_t w[4] = {__float_as_uint(r.x), __float_as_uint(r.y), __float_as_uint(r.z), __float_as_uint(r.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[t]));
            o[2 * t] = f.x;
            o[2 * t + 1] = f.y;
        }
    }
    __device__ static uint32_t label(const Lab& L, int e) { return ((e < 4 ? L.x : L.y) >> (8 * (e & 3))) & 0xffu; }
};
template <> struct KVec<__nv_bfloat16> {
    static constexpr int N = 8;
    using Lab = uint2;
    __device__ static void unpack(const float4& r, float (&o)[8]) {
        const uint32_t w[4] = {__float_as_uint(r.x), __float_as_uint(r.y), __float_as_uint(r.z), __float_as_uint(r.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[t]));
            o[2 * t] = f.x;
            o[2 * t + 1] = f.y;
        }
    }
    __device__ static uint32_t label(const Lab& L, int e) { return ((e < 4 ? L.x : L.y) >> (8 * (e & 3))) & 0xffu; }
};

__device__ __forceinline__ float kval(float v) { return v; }
__device__ __forceinline__ float kval(__half v) { return __half2float(v); }
__device__ __forceinline__ float kval(__nv_bfloat16 v) { return __bfloat162float(v); }

template <int UNR, bool LAB_SMEM, typename LabT = uint32_t>
__device__ __forceinline__ void load_batch(const float4* row4, const LabT* lab4, int q, int q1,
                                           float4 (&v)[UNR], LabT (&L)[UNR]) {
#pragma unroll
    for (int t = 0; t < UNR; ++t) {
        const int qq = q + 32 * t;
        if (qq < q1) {
            v[t] = ld_stream(row4 + qq);
            L[t] = LAB_SMEM ? lab4[qq] : __ldg(lab4 + qq);
        } else {
            v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            L[t] = LabT{};
        }
    }
}

struct ReduceArgs {
    const void* K;        // TK elements, row pitch ldk elements (16-byte aligned rows)
    int64_t ldk;
    int n, k, nseg, seglen;
    const uint8_t* lab8;
    float* Spart;
    double* zpart;
    double* zsum;
    double* cnorm;
    double* invm;
    const int32_t* counts;
    LoopState* st;
    double* J_hist;
    int eval_only;
};

// Per-lane partial sums live in lane-private shared-memory columns acc[c][lane]
// (bank = lane: a conflict-free scatter for any k).  At the end of a unit the
// warp reduces them: for k <= KB each lane pulls its k partials into
// registers and a butterfly reduce-scatter leaves one cluster total per lane
// group; for larger k (KB == 0) lane c walks row c in rotated order.  UNR
// float4 per lane per batch; the next batch -- across unit boundaries too --
// is in flight while the current one is scattered.
template <int KB, int UNR, bool LAB_SMEM, typename TK>
__global__ void __launch_bounds__(kReduceMaxWarps * 32, 2) reduce_kernel(ReduceArgs a) {
    using V = KVec<TK>;
    using LabT = typename V::Lab;
    constexpr int NV = V::N;
    LoopState* st = a.st;
    if (a.eval_only) {
        // J(final labels) is already known when the last pass changed nothing
        if (st->iter > 0 && st->last_changed == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) st->J_eval = st->J_last;
            return;
        }
    } else if (st->done) {
        return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, k = a.k, nseg = a.nseg;
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nlab = LAB_SMEM ? ((n + 15) & ~15) : 0;
    uint8_t* slab = smem;
    float* sacc = reinterpret_cast<float*>(smem + nlab);
    const int nacc = W * k * 32;
    float* zhi = sacc + nacc;                 // per-warp float-float z partials
    float* zlo = zhi + W * k;

    if (LAB_SMEM) {
        const uint4* src = reinterpret_cast<const uint4*>(a.lab8);
        uint4* dst = reinterpret_cast<uint4*>(slab);
        for (int t = threadIdx.x; t < nlab / 16; t += blockDim.x) dst[t] = src[t];
    }
    for (int t = threadIdx.x; t < nacc; t += blockDim.x) sacc[t] = 0.f;
    for (int t = threadIdx.x; t < 2 * W * k; t += blockDim.x) zhi[t] = 0.f;
    __syncthreads();

    const uint8_t* labs = LAB_SMEM ? slab : a.lab8;
    const LabT* lab4 = reinterpret_cast<const LabT*>(labs);
    const TK* Kb = static_cast<const TK*>(a.K);
    float* accw = sacc + (size_t)warp * k * 32;   // this warp's [k][32] block
    float* accl = accw + lane;
    float* zwh = zhi + (size_t)warp * k;
    float* zwl = zlo + (size_t)warp * k;

    auto scatter = [&](uint32_t l, float x) { accl[l * 32] += x; };

    // unit indices fit in 32 bits: n < 2^31 / nseg is checked on the host
    const int units = n * nseg;
    const int GW = (int)gridDim.x * W;
    int u = (int)blockIdx.x * W + warp;
    if (u < units) {
        auto geom = [&](int uu, int& ii, int& ss, int& cc1, int& qqb, int& qq1, const float4*& r4) {
            ii = uu / nseg;
            ss = uu - ii * nseg;
            const int c0 = ss * a.seglen;
            cc1 = min(n, c0 + a.seglen);
            qqb = c0 / NV;
            qq1 = cc1 / NV;
            r4 = reinterpret_cast<const float4*>(Kb + (int64_t)ii * a.ldk);
        };
        int i, s, c1, qb, q1;
        const float4* row4;
        geom(u, i, s, c1, qb, q1, row4);
        float4 v[UNR];
        LabT L[UNR];
        load_batch<UNR, LAB_SMEM, LabT>(row4, lab4, qb + lane, q1, v, L);
        while (true) {
            const bool last = qb + 32 * UNR >= q1;
            const int un = last ? u + GW : u;
            int in_ = i, sn = s, c1n = c1, qbn = qb + 32 * UNR, q1n = q1;
            const float4* row4n = row4;
            float4 vn[UNR];
            LabT Ln[UNR];
            if (last && un < units) geom(un, in_, sn, c1n, qbn, q1n, row4n);
            if (!last || un < units) load_batch<UNR, LAB_SMEM, LabT>(row4n, lab4, qbn + lane, q1n, vn, Ln);
#pragma unroll
            for (int t = 0; t < UNR; ++t) {
                float e[NV];
                V::unpack(v[t], e);
#pragma unroll
                for (int x = 0; x < NV; ++x) scatter(V::label(L[t], x), e[x]);
            }
            if (last) {
                {   // ragged tail of the row (n not a multiple of the vector width)
                    const int j = q1 * NV + lane;
                    if (j < c1) scatter(labs[j], kval(Kb[(int64_t)i * a.ldk + j]));
                }
                const int li = labs[i];
                // layout [s][c][i] (i fastest): cluster c of this unit at out[c * n]
                float* out = a.Spart + (size_t)s * k * n + i;
                __syncwarp();
                if constexpr (KB > 0) {
                    float part[KB];
#pragma unroll
                    for (int c = 0; c < KB; ++c) {
                        part[c] = c < k ? accl[c * 32] : 0.f;
                        if (c < k) accl[c * 32] = 0.f;
                    }
                    const float tot = butterfly<KB>(part, lane);
                    const int c = bfly_cluster<KB>(lane);
                    if ((lane & (32 / KB - 1)) == 0 && c < k) {
                        out[(size_t)c * n] = tot;
                        if (c == li) ff_add(zwh[c], zwl[c], tot);
                    }
                } else {
                    for (int cb = 0; cb < k; cb += 32) {
                        const int c = cb + lane;
                        if (c < k) {
                            // lane c walks row c of the warp block in rotated order: conflict-free
                            float tot = 0.f;
                            float* row = accw + (size_t)c * 32;
#pragma unroll 8
                            for (int j = 0; j < 32; ++j) {
                                const int idx = (j + lane) & 31;
                                tot += row[idx];
                                row[idx] = 0.f;
                            }
                            out[(size_t)c * n] = tot;
                            if (c == li) ff_add(zwh[c], zwl[c], tot);
                        }
                    }
                }
                __syncwarp();
                if (un >= units) break;
                u = un;
                i = in_;
                s = sn;
                c1 = c1n;
                q1 = q1n;
                row4 = row4n;
            }
            qb = qbn;
#pragma unroll
            for (int t = 0; t < UNR; ++t) {
                v[t] = vn[t];
                L[t] = Ln[t];
            }
        }
    }
    __syncthreads();

    // block partial of sum_{i in L_c} S_ic, fixed warp order
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < W; ++w) t += (double)zhi[(size_t)w * k + c] + (double)zlo[(size_t)w * k + c];
        a.zpart[(size_t)blockIdx.x * k + c] = t;
    }
    __threadfence();
    __syncthreads();
    __shared__ int am_last;
    if (threadIdx.x == 0) am_last = (atomicAdd(&st->reduce_ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();

    finalize_pass(a.zpart, (int)gridDim.x, k, a.counts, a.zsum, a.cnorm, a.invm, st, a.J_hist, a.eval_only);
}

struct AssignArgs {
    int n, k, nseg;
    const float* Spart;
    const float* kdiag;
    const double* cnorm;
    const double* invm;
    int32_t* counts;
    int32_t* lab32;
    uint8_t* lab8;
    LoopState* st;
    int32_t* changed_hist;
    float* E_out;
};

// One block of the distance/argmin pass: rows [block * blockDim, ...), and
// the pass's loop control when this is the last of nblocks blocks to finish.
__device__ __forceinline__ void assign_body(const AssignArgs& a, int block, int nblocks) {
    LoopState* st = a.st;
    if (st->done) return;
    __shared__ int hist[kMaxClusters];
    __shared__ float cn32[kMaxClusters], im32[kMaxClusters];   // ||c||^2 and 1/|L_c| in FP32
    __shared__ int am_last;
    const int n = a.n, k = a.k;
    const int it = st->iter;
    const int32_t* m = a.counts + (size_t)(it & 1) * k;
    int32_t* mnext = a.counts + (size_t)((it + 1) & 1) * k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        hist[c] = 0;
        cn32[c] = (float)a.cnorm[c];
        im32[c] = (float)a.invm[c];
    }
    __syncthreads();

    const int i = block * blockDim.x + threadIdx.x;
    int newl = 0, changed = 0;
    if (i < n) {
        const int li = a.lab32[i];
        const double kd = (double)a.kdiag[i];
        double best = cuda::std::numeric_limits<double>::infinity();
        int bi = li;
        const float* Si = a.Spart + i;               // [s][c][i]: consecutive threads, consecutive rows
        const size_t cs = (size_t)n, ss = (size_t)k * n;
        // The argmin in FP32, screened: GB300 runs FP64 at a small fraction of the FP32 rate,
        // and a pass has n k distances.  Each FP32 distance is within
        //   B = 16 u (|K_ii| + max_c ||c||^2 + max_c |E_ic|),  u = 2^-24,
        // of the FP64 one (from the roundings of 1/|L_c|, ||c||^2, the sum, the product and
        // the multiply-add: under 8.2 u (|E| + ||c||^2 + |K_ii|)).  Where the FP32 best beats
        // every other cluster by more than 2 B, the FP64 argmin is the same cluster; otherwise
        // (near-ties, and every row when E is requested) the row is decided in FP64 below.
        bool decided = false;
        if (!a.E_out) {
            const float kd32 = a.kdiag[i];
            float b1 = cuda::std::numeric_limits<float>::infinity(), b2 = b1, emax = 0.f, cmax = 0.f;
            int c1 = li;
            for (int c0 = 0; c0 < k; c0 += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = c0 + u < k ? Si[(size_t)(c0 + u) * cs] : 0.f;
                float hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    hi[u] = lo[u] = 0.f;
                    ff_add(hi[u], lo[u], v[u]);
                }
                for (int s = 1; s < a.nseg; ++s) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = c0 + u < k ? Si[s * ss + (size_t)(c0 + u) * cs] : 0.f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) ff_add(hi[u], lo[u], v[u]);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int c = c0 + u;
                    if (c >= k) break;
                    if (m[c] == 0) continue;
                    const float E = (hi[u] + lo[u]) * im32[c];
                    const float D = fmaf(-2.f, E, kd32 + cn32[c]);
                    emax = fmaxf(emax, fabsf(E));
                    cmax = fmaxf(cmax, fabsf(cn32[c]));
                    if (D < b1) {
                        b2 = b1;
                        b1 = D;
                        c1 = c;
                    } else if (D < b2) {
                        b2 = D;
                    }
                }
            }
            const float B = 16.f * 0x1p-24f * (fabsf(kd32) + cmax + emax);
            if (b2 - b1 > 2.f * B) {
                bi = c1;
                decided = true;
            }
        }
        // 8 clusters at a time: their segment sums are loaded before any is used, so a thread
        // keeps 8 loads in flight instead of one (the same additions in the same order)
        for (int c0 = 0; c0 < k && !decided; c0 += 8) {
            float hi[8], lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) hi[u] = lo[u] = 0.f;
            for (int s = 0; s < a.nseg; ++s) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = c0 + u < k ? Si[s * ss + (size_t)(c0 + u) * cs] : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) ff_add(hi[u], lo[u], v[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + u;
                if (c >= k) break;
                const int mc = m[c];
                const double E = ((double)hi[u] + (double)lo[u]) * a.invm[c];   // (K V^T)_ic
                if (a.E_out) a.E_out[(int64_t)i * k + c] = (float)E;
                if (mc == 0) continue;
                const double D = fma(-2.0, E, kd + a.cnorm[c]);
                if (D < best) {
                    best = D;
                    bi = c;
                }
            }
        }
        newl = bi;
        changed = (bi != li);
        a.lab32[i] = bi;
        a.lab8[i] = (uint8_t)bi;
    }
    // cluster sizes of the new labels: one shared atomic per distinct label in the warp
    const unsigned act = __ballot_sync(0xffffffffu, i < n);
    if (i < n) {
        const unsigned peers = __match_any_sync(act, newl);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[newl], __popc(peers));
    }
    const int block_changed = __syncthreads_count(changed);
    for (int c = threadIdx.x; c < k; c += blockDim.x)
        if (hist[c]) atomicAdd(mnext + c, hist[c]);
    if (threadIdx.x == 0 && block_changed) atomicAdd(&st->changed_acc, (unsigned)block_changed);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(&st->assign_ticket, 1u) == (unsigned)nblocks - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();

    // last block: the counts of this pass are consumed; clear them for pass it + 2
    int32_t* mcur = a.counts + (size_t)(it & 1) * k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) mcur[c] = 0;
    if (threadIdx.x == 0) {
        const int ch = (int)atomicExch(&st->changed_acc, 0u);
        a.changed_hist[it] = ch;
        st->last_changed = ch;
        st->iter = it + 1;
        int done = (it + 1 >= st->max_iter);
        if (st->check_conv) {
            if (ch == 0) {
                done = 1;
                st->converged = 1;
            }
            if (st->tol > 0.0 && it >= 1 && st->J_prev - st->J_last <= st->tol * fabs(st->J_last)) done = 1;
        }
        st->J_prev = st->J_last;
        st->done = done;
        st->assign_ticket = 0u;
    }
}

__global__ void __launch_bounds__(kAssignThreads) assign_kernel(AssignArgs a) {
    grid_dependency_wait();   // S, z and the loop state come from the pass's reduction
    assign_body(a, blockIdx.x, gridDim.x);
}


// sum_{i in L_c} S_ic for the recompute path and batched mode, from Spart[s][c][i]: a
// block takes kZReduceRows consecutive rows and sums each cluster's rows in a fixed order
// (deterministic), then the last block finalizes the pass.
struct ZArgs {
    int n, k, nseg;
    const float* Spart;
    const uint8_t* lab8;
    double* zpart;
    double* zsum;
    double* cnorm;
    double* invm;
    const int32_t* counts;
    LoopState* st;
    double* J_hist;
    int eval_only;
};

__device__ __forceinline__ void zreduce_body(const ZArgs& a, int block, int nblocks) {
    LoopState* st = a.st;
    if (pass_skip(st, a.eval_only)) {
        if (a.eval_only && block == 0 && threadIdx.x == 0) st->J_eval = st->J_last;
        return;
    }
    // The block's rows, stably sorted by label in shared memory, so that each cluster's FP64
    // sum touches only its own rows (GB300 runs FP64 at a small fraction of the FP32 rate; a
    // walk of all rows for every cluster issued k x 1024 predicated FP64 adds).  Stable rank
    // of a row: its rank among the earlier rows of its warp with its label (warp match), plus
    // the rows with that label in earlier warps and in earlier clusters.
    constexpr int NW = kZReduceRows / 32;
    __shared__ double val_s[kZReduceRows];                 // values in sorted order
    __shared__ unsigned short cnt_s[NW][kMaxClusters];     // per warp and cluster: count, then offset
    __shared__ int cstart[kMaxClusters + 1];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = block * kZReduceRows + threadIdx.x;
    for (int e = threadIdx.x; e < NW * a.k; e += kZReduceRows) cnt_s[e / a.k][e % a.k] = 0;
    int l = -1;
    double v = 0.0;
    if (i < a.n) {
        l = a.lab8[i];
        const float* Si = a.Spart + (size_t)l * a.n + i;
        float hi = 0.f, lo = 0.f;
        for (int s = 0; s < a.nseg; ++s) ff_add(hi, lo, Si[(size_t)s * a.k * a.n]);
        v = (double)hi + (double)lo;
    }
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    const int wrank = __popc(peers & ((1u << lane) - 1u));
    if (l >= 0 && wrank == 0) cnt_s[warp][l] = (unsigned short)__popc(peers);
    __syncthreads();
    // per cluster: its total, then (after the scan over clusters) each warp's starting offset
    for (int c = threadIdx.x; c < a.k; c += kZReduceRows) {
        int t = 0;
        for (int w = 0; w < NW; ++w) t += cnt_s[w][c];
        cstart[c + 1] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cstart[0] = 0;
        for (int c = 0; c < a.k; ++c) cstart[c + 1] += cstart[c];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < a.k; c += kZReduceRows) {
        int o = cstart[c];
        for (int w = 0; w < NW; ++w) {
            const int m = cnt_s[w][c];
            cnt_s[w][c] = (unsigned short)o;
            o += m;
        }
    }
    __syncthreads();
    if (l >= 0) val_s[cnt_s[warp][l] + wrank] = v;
    __syncthreads();
    // warp w: clusters w, w + 32, ...; lanes stride the cluster's sorted rows, a butterfly adds
    // the lanes' sums (a fixed order)
    for (int c = warp; c < a.k; c += NW) {
        double t = 0.0;
        for (int r = cstart[c] + lane; r < cstart[c + 1]; r += 32) t += val_s[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) a.zpart[(size_t)block * a.k + c] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(&st->reduce_ticket, 1u) == (unsigned)nblocks - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    finalize_pass(a.zpart, nblocks, a.k, a.counts, a.zsum, a.cnorm, a.invm, st, a.J_hist, a.eval_only);
}

__global__ void __launch_bounds__(kZReduceRows) zreduce_kernel(ZArgs a) { zreduce_body(a, blockIdx.x, gridDim.x); }

__device__ __forceinline__ void init_state_fn(LoopState* st, int max_iter, int check_conv, double tol) {
    st->iter = 0;
    st->done = (max_iter <= 0);
    st->converged = 0;
    st->max_iter = max_iter;
    st->check_conv = check_conv;
    st->last_changed = -1;
    st->reduce_ticket = 0u;
    st->assign_ticket = 0u;
    st->changed_acc = 0u;
    st->bad_label = 0;
    st->wait_err = 0;
    st->tol = tol;
    st->trace = 0.0;
    st->J_last = 0.0;
    st->J_prev = 0.0;
    st->J_eval = 0.0;
}

__global__ void init_state_kernel(LoopState* st, int max_iter, int check_conv, double tol) {
    init_state_fn(st, max_iter, check_conv, tol);
}

// sum of diag(K) in FP64; one block, fixed reduction order
__device__ __forceinline__ void trace_body(const float* __restrict__ kdiag, int n, LoopState* st) {
    __shared__ double part[1024];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += (double)kdiag[i];
    part[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) st->trace = part[0];
}

__global__ void __launch_bounds__(1024) trace_kernel(const float* __restrict__ kdiag, int n, LoopState* st) {
    trace_body(kdiag, n, st);
}

__device__ __forceinline__ void init_labels_body(const int32_t* __restrict__ in, int n, int k, int32_t* lab32,
                                                 uint8_t* lab8, int nlab, int32_t* counts, LoopState* st, int block) {
    __shared__ int hist[kMaxClusters];
    for (int c = threadIdx.x; c < k; c += blockDim.x) hist[c] = 0;
    __syncthreads();
    const int i = block * blockDim.x + threadIdx.x;
    if (i < n) {
        int l = in[i];
        if (l < 0 || l >= k) {
            atomicExch(&st->bad_label, 1);
            l = 0;
        }
        lab32[i] = l;
        lab8[i] = (uint8_t)l;
        atomicAdd(&hist[l], 1);
    } else if (i < nlab) {
        lab8[i] = 0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x)
        if (hist[c]) atomicAdd(counts + c, hist[c]);
}

__global__ void __launch_bounds__(256) init_labels_kernel(const int32_t* __restrict__ in, int n, int k,
                                                          int32_t* lab32, uint8_t* lab8, int nlab,
                                                          int32_t* counts, LoopState* st) {
    init_labels_body(in, n, k, lab32, lab8, nlab, counts, st, blockIdx.x);
}

}  // namespace

namespace {

using ReduceFn = void (*)(ReduceArgs);

// 16-byte loads per lane per batch: 4 for FP32 K, 2 for half types (8 elements each)
template <typename TK>
ReduceFn reduce_fn_t(int variant, bool lab_smem) {
    constexpr int U = sizeof(TK) == 4 ? 4 : 2;
    switch (variant) {
        case kReduceBfly4: return lab_smem ? reduce_kernel<4, U, true, TK> : reduce_kernel<4, U, false, TK>;
        case kReduceBfly8: return lab_smem ? reduce_kernel<8, U, true, TK> : reduce_kernel<8, U, false, TK>;
        default: return lab_smem ? reduce_kernel<0, U, true, TK> : reduce_kernel<0, U, false, TK>;
    }
}

ReduceFn reduce_fn(int variant, bool lab_smem, int k_storage = POPCORN_K_FP32) {
    if (k_storage == POPCORN_K_FP16) return reduce_fn_t<__half>(variant, lab_smem);
    if (k_storage == POPCORN_K_BF16) return reduce_fn_t<__nv_bfloat16>(variant, lab_smem);
    return reduce_fn_t<float>(variant, lab_smem);
}

}  // namespace

ReducePlan plan_reduce(int n, int k, int num_sms, int smem_budget, int k_storage) {
    ReducePlan p{};
    p.k_storage = k_storage;
    p.variant = k <= 4 ? kReduceBfly4 : (k <= 8 ? kReduceBfly8 : kReduceRotated);
    const size_t nlab = ((size_t)n + 15) & ~(size_t)15;
    const size_t per_warp = (size_t)k * 32 * sizeof(float) + 2 * (size_t)k * sizeof(float);
    p.labels_in_smem = nlab + per_warp * 4 <= (size_t)smem_budget;
    const size_t base = p.labels_in_smem ? nlab : 0;
    int w = (int)(((size_t)smem_budget - base) / per_warp);
    if (w > kReduceMaxWarps) w = kReduceMaxWarps;
    if (w < 1) w = 1;
    p.warps = w;
    p.smem = base + per_warp * w;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reduce_fn(p.variant, p.labels_in_smem, k_storage), 32 * w,
                                                  p.smem);
    cudaGetLastError();
    if (per_sm < 1) per_sm = 1;
    p.grid = num_sms * per_sm;
    // split rows into segments so that each warp gets ~16 units (row, segment);
    // the next unit's loads overlap the current unit's reduction
    const long long warps_total = (long long)p.grid * w;
    long long nseg = (16 * warps_total + n - 1) / n;
    if (nseg < 1) nseg = 1;
    long long seglen = (n + nseg - 1) / nseg;
    seglen = (seglen + 127) / 128 * 128;
    if (seglen < 1024) seglen = 1024;
    p.seglen = (int)seglen;
    p.nseg = (int)((n + seglen - 1) / seglen);
    if ((long long)n * p.nseg >= (1LL << 31)) p.grid = 0;   // unit indices would overflow: caller rejects
    return p;
}

cudaError_t launch_init_state(LoopState* st, int max_iter, int check_conv, double tol, cudaStream_t s) {
    init_state_kernel<<<1, 1, 0, s>>>(st, max_iter, check_conv, tol);
    return cudaGetLastError();
}

cudaError_t launch_trace(const float* kdiag, int n, LoopState* st, cudaStream_t s) {
    trace_kernel<<<1, 1024, 0, s>>>(kdiag, n, st);
    return cudaGetLastError();
}

cudaError_t launch_init_labels(const int32_t* in, int n, int k, int32_t* lab32, uint8_t* lab8,
                               int32_t* counts, LoopState* st, cudaStream_t s) {
    const int nlab = (n + 15) & ~15;
    init_labels_kernel<<<(nlab + 255) / 256, 256, 0, s>>>(in, n, k, lab32, lab8, nlab, counts, st);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const PassBuffers& b, const ReducePlan& plan, int eval_only, cudaStream_t s) {
    ReduceArgs a;
    a.K = b.K;
    a.ldk = b.ldk;
    a.n = b.n;
    a.k = b.k;
    a.nseg = plan.nseg;
    a.seglen = plan.seglen;
    a.lab8 = b.lab8;
    a.Spart = b.Spart;
    a.zpart = b.zpart;
    a.zsum = b.zsum;
    a.cnorm = b.cnorm;
    a.invm = b.invm;
    a.counts = b.counts;
    a.st = b.st;
    a.J_hist = b.J_hist;
    a.eval_only = eval_only;
    reduce_fn(plan.variant, plan.labels_in_smem, plan.k_storage)<<<plan.grid, plan.warps * 32, plan.smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_zreduce(const PassBuffers& b, int nseg, int eval, cudaStream_t s) {
    ZArgs a;
    a.n = b.n;
    a.k = b.k;
    a.nseg = nseg;
    a.Spart = b.Spart;
    a.lab8 = b.lab8;
    a.zpart = b.zpart;
    a.zsum = b.zsum;
    a.cnorm = b.cnorm;
    a.invm = b.invm;
    a.counts = b.counts;
    a.st = b.st;
    a.J_hist = b.J_hist;
    a.eval_only = eval;
    zreduce_kernel<<<(b.n + kZReduceRows - 1) / kZReduceRows, kZReduceRows, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_assign_nseg(const PassBuffers& b, int nseg, cudaStream_t s) {
    ReducePlan p{};
    p.nseg = nseg;
    return launch_assign(b, p, s);
}

cudaError_t launch_assign(const PassBuffers& b, const ReducePlan& plan, cudaStream_t s) {
    AssignArgs a;
    a.n = b.n;
    a.k = b.k;
    a.nseg = plan.nseg;
    a.Spart = b.Spart;
    a.kdiag = b.kdiag;
    a.cnorm = b.cnorm;
    a.invm = b.invm;
    a.counts = b.counts;
    a.lab32 = b.lab32;
    a.lab8 = b.lab8;
    a.st = b.st;
    a.changed_hist = b.changed_hist;
    a.E_out = b.E_out;
    return launch_pdl(assign_kernel, dim3((b.n + kAssignThreads - 1) / kAssignThreads), dim3(kAssignThreads), 0, s, a);
}

// Opt the reduction kernels into the largest dynamic shared memory the device
// allows next to their static shared memory; *usable receives that size.
cudaError_t configure_reduce_smem(int optin, int* usable) {
    size_t st = 0;
    for (int ks = 0; ks < 3; ++ks)
        for (int v = 0; v < 3; ++v)
            for (int l = 0; l < 2; ++l) {
                cudaFuncAttributes fa;
                cudaError_t e = cudaFuncGetAttributes(&fa, reduce_fn(v, l != 0, ks));
                if (e != cudaSuccess) return e;
                if (fa.sharedSizeBytes > st) st = fa.sharedSizeBytes;
            }
    const int bytes = optin - (int)((st + 127) / 128 * 128);
    for (int ks = 0; ks < 3; ++ks)
        for (int v = 0; v < 3; ++v)
            for (int l = 0; l < 2; ++l) {
                cudaError_t e = cudaFuncSetAttribute(reduce_fn(v, l != 0, ks), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     bytes);
                if (e != cudaSuccess) return e;
            }
    *usable = bytes;
    return cudaSuccess;
}

namespace {

// ------------------------------------------------------------------ batched mode

// Instance holding flattened index x of a prefix field (fields ascend with t).
template <class F>
__device__ __forceinline__ int find_inst(const BatchInst* I, int count, long long x, F field) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (field(I[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void batched_init_kernel(const BatchInst* I, int count, int max_iter, int check_conv, double tol) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) {
        init_state_fn(I[t].st, max_iter, check_conv, tol);
        for (int c = 0; c < 2 * I[t].k; ++c) I[t].counts[c] = 0;
    }
}

__global__ void __launch_bounds__(kBatchLabelThreads) batched_labels_kernel(const BatchInst* I, int count) {
    const int t = find_inst(I, count, blockIdx.x, [](const BatchInst& x) { return (long long)x.lblock0; });
    const BatchInst& b = I[t];
    init_labels_body(b.init_labels, b.n, b.k, b.lab32, b.lab8, (b.n + 15) & ~15, b.counts, b.st,
                     blockIdx.x - b.lblock0);
}

__global__ void __launch_bounds__(kBatchLabelThreads) batched_copy_labels_kernel(const BatchInst* I, int count) {
    const int t = find_inst(I, count, blockIdx.x, [](const BatchInst& x) { return (long long)x.lblock0; });
    const BatchInst& b = I[t];
    const int i = (blockIdx.x - b.lblock0) * blockDim.x + threadIdx.x;
    if (i < b.n) b.labels_out[i] = b.lab32[i];
}

__global__ void __launch_bounds__(1024) batched_trace_kernel(const BatchInst* I) {
    const BatchInst& b = I[blockIdx.x];
    trace_body(b.kdiag, b.n, b.st);
}

__global__ void __launch_bounds__(kZReduceRows) batched_zreduce_kernel(const BatchInst* I, int count, int eval) {
    const int t = find_inst(I, count, blockIdx.x, [](const BatchInst& x) { return (long long)x.zblock0; });
    const BatchInst& b = I[t];
    ZArgs a;
    a.n = b.n;
    a.k = b.k;
    a.nseg = b.nseg;
    a.Spart = b.Spart;
    a.lab8 = b.lab8;
    a.zpart = b.zpart;
    a.zsum = b.zsum;
    a.cnorm = b.cnorm;
    a.invm = b.invm;
    a.counts = b.counts;
    a.st = b.st;
    a.J_hist = b.J_hist;
    a.eval_only = eval;
    zreduce_body(a, blockIdx.x - b.zblock0, (b.n + kZReduceRows - 1) / kZReduceRows);
}

__global__ void __launch_bounds__(kAssignThreads) batched_assign_kernel(const BatchInst* I, int count) {
    const int t = find_inst(I, count, blockIdx.x, [](const BatchInst& x) { return (long long)x.ablock0; });
    const BatchInst& b = I[t];
    AssignArgs a;
    a.n = b.n;
    a.k = b.k;
    a.nseg = b.nseg;
    a.Spart = b.Spart;
    a.kdiag = b.kdiag;
    a.cnorm = b.cnorm;
    a.invm = b.invm;
    a.counts = b.counts;
    a.lab32 = b.lab32;
    a.lab8 = b.lab8;
    a.st = b.st;
    a.changed_hist = b.changed_hist;
    a.E_out = nullptr;
    assign_body(a, blockIdx.x - b.ablock0, (b.n + kAssignThreads - 1) / kAssignThreads);
}

// K stream over the units (instance, row, segment) of every instance still
// running: lane-private shared-memory cluster columns as in reduce_kernel,
// labels read through L1, the next batch in flight while the current one is
// scattered (across unit boundaries too), and per unit a butterfly reduction
// for k <= 8 or the rotated walk for larger k.  z and J come from the batched
// z kernel that follows.
// U float4 a lane a batch: 4 with two blocks an SM (64 registers); 8 with one block an SM,
// which keeps twice the bytes in flight where the per-warp cluster columns (kmax x 128 bytes)
// leave room for only 16 warps an SM.
template <int U>
__global__ void __launch_bounds__(kReduceMaxWarps * 32, U == 4 ? 2 : 1)
    batched_reduce_kernel(const BatchInst* I, int count, int units, int kmax, int eval) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* accw = reinterpret_cast<float*>(smem) + (size_t)warp * kmax * 32;
    float* accl = accw + lane;
    for (int t = lane; t < kmax * 32; t += 32) accw[t] = 0.f;
    __syncwarp();
    const int GW = (int)gridDim.x * W;

    // next unit at or after u that belongs to an instance still running
    struct Geo {
        const BatchInst* b;
        int u, i, sg, c1, qb, q1;
        const float4* row4;
        const uint32_t* lab4;
    };
    auto geom = [&](int u, Geo& g) -> bool {
        for (; u < units; u += GW) {
            const int t = find_inst(I, count, u, [](const BatchInst& x) { return (long long)x.unit0; });
            const BatchInst* b = I + t;
            if (pass_skip(b->st, eval)) continue;
            const int lu = u - b->unit0;
            g.b = b;
            g.u = u;
            g.i = lu / b->nseg;
            g.sg = lu - g.i * b->nseg;
            const int c0 = g.sg * b->seglen;
            g.c1 = min(b->n, c0 + b->seglen);
            g.qb = c0 >> 2;
            g.q1 = g.c1 >> 2;
            g.row4 = reinterpret_cast<const float4*>(b->K + (int64_t)g.i * b->ldk);
            g.lab4 = reinterpret_cast<const uint32_t*>(b->lab8);
            return true;
        }
        return false;
    };
    Geo cur;
    if (!geom((int)blockIdx.x * W + warp, cur)) return;
    float4 v[U];
    uint32_t L[U];
    load_batch<U, false>(cur.row4, cur.lab4, cur.qb + lane, cur.q1, v, L);
    while (true) {
        const bool last = cur.qb + 32 * U >= cur.q1;
        Geo nxt = cur;
        bool more = true;
        if (last) {
            more = geom(cur.u + GW, nxt);
        } else {
            nxt.qb = cur.qb + 32 * U;
        }
        float4 vn[U];
        uint32_t Ln[U];
        if (more) load_batch<U, false>(nxt.row4, nxt.lab4, nxt.qb + lane, nxt.q1, vn, Ln);
#pragma unroll
        for (int x = 0; x < U; ++x) {
            accl[(L[x] & 0xffu) * 32] += v[x].x;
            accl[((L[x] >> 8) & 0xffu) * 32] += v[x].y;
            accl[((L[x] >> 16) & 0xffu) * 32] += v[x].z;
            accl[(L[x] >> 24) * 32] += v[x].w;
        }
        if (last) {
            const BatchInst& b = *cur.b;
            {
                const int j = (cur.q1 << 2) + lane;
                if (j < cur.c1) accl[(int)b.lab8[j] * 32] += b.K[(int64_t)cur.i * b.ldk + j];
            }
            __syncwarp();
            float* out = b.Spart + (size_t)cur.sg * b.k * b.n + cur.i;   // [s][c][i]
            if (b.k <= 8) {
                float part[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    part[c] = c < b.k ? accl[c * 32] : 0.f;
                    if (c < b.k) accl[c * 32] = 0.f;
                }
                const float tot = butterfly<8>(part, lane);
                const int c = bfly_cluster<8>(lane);
                if ((lane & 3) == 0 && c < b.k) out[(size_t)c * b.n] = tot;
            } else {
                for (int cb = 0; cb < b.k; cb += 32) {
                    const int c = cb + lane;
                    if (c < b.k) {
                        float tot = 0.f;
                        float* rowp = accw + (size_t)c * 32;
#pragma unroll 8
                        for (int j = 0; j < 32; ++j) {
                            const int idx = (j + lane) & 31;
                            tot += rowp[idx];
                            rowp[idx] = 0.f;
                        }
                        out[(size_t)c * b.n] = tot;
                    }
                }
            }
            __syncwarp();
            if (!more) break;
            cur = nxt;
        } else {
            cur.qb = nxt.qb;
        }
#pragma unroll
        for (int x = 0; x < U; ++x) {
            v[x] = vn[x];
            L[x] = Ln[x];
        }
    }
}

}  // namespace

void plan_batched_reduce(BatchPlan* bp, int num_sms, int smem_budget, int warps, int per_sm_req) {
    const size_t per_warp = (size_t)bp->kmax * 32 * sizeof(float);
    int w = (int)((size_t)smem_budget / per_warp);
    if (w > kReduceMaxWarps) w = kReduceMaxWarps;
    if (warps > 0 && warps < w) w = warps;
    if (w < 1) w = 1;
    bp->warps = w;
    bp->smem = per_warp * w;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_reduce_kernel<4>, 32 * w, bp->smem);
    cudaGetLastError();
    if (per_sm_req > 0 && per_sm_req < per_sm) per_sm = per_sm_req;
    if (per_sm < 1) per_sm = 1;
    bp->per_sm = per_sm;
    bp->grid = num_sms * per_sm;
}

cudaError_t launch_batched_reduce(const BatchInst* dI, const BatchPlan& bp, int eval, cudaStream_t s) {
    if (bp.per_sm == 1)
        batched_reduce_kernel<8><<<bp.grid, bp.warps * 32, bp.smem, s>>>(dI, bp.count, bp.units, bp.kmax, eval);
    else
        batched_reduce_kernel<4><<<bp.grid, bp.warps * 32, bp.smem, s>>>(dI, bp.count, bp.units, bp.kmax, eval);
    return cudaGetLastError();
}

cudaError_t configure_batched(int smem_optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, batched_reduce_kernel<4>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batched_reduce_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin_minus_static(smem_optin, fa.sharedSizeBytes));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batched_reduce_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin_minus_static(smem_optin, fa.sharedSizeBytes));
}

cudaError_t launch_batched_init(const BatchInst* dI, const BatchPlan& bp, int max_iter, int check_conv, double tol,
                                cudaStream_t s) {
    batched_init_kernel<<<(bp.count + 127) / 128, 128, 0, s>>>(dI, bp.count, max_iter, check_conv, tol);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batched_labels_kernel<<<bp.lblocks, kBatchLabelThreads, 0, s>>>(dI, bp.count);
    return cudaGetLastError();
}

cudaError_t launch_batched_trace(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s) {
    batched_trace_kernel<<<bp.count, 1024, 0, s>>>(dI);
    return cudaGetLastError();
}

cudaError_t launch_batched_finish(const BatchInst* dI, const BatchPlan& bp, int eval, cudaStream_t s) {
    batched_zreduce_kernel<<<bp.zblocks, kZReduceRows, 0, s>>>(dI, bp.count, eval);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || eval) return e;
    batched_assign_kernel<<<bp.ablocks, kAssignThreads, 0, s>>>(dI, bp.count);
    return cudaGetLastError();
}

cudaError_t launch_batched_pass(const BatchInst* dI, const BatchPlan& bp, int eval, cudaStream_t s) {
    if (bp.per_sm == 1)
        batched_reduce_kernel<8><<<bp.grid, bp.warps * 32, bp.smem, s>>>(dI, bp.count, bp.units, bp.kmax, eval);
    else
        batched_reduce_kernel<4><<<bp.grid, bp.warps * 32, bp.smem, s>>>(dI, bp.count, bp.units, bp.kmax, eval);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_batched_finish(dI, bp, eval, s);
}

cudaError_t launch_batched_copy_labels(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s) {
    batched_copy_labels_kernel<<<bp.lblocks, kBatchLabelThreads, 0, s>>>(dI, bp.count);
    return cudaGetLastError();
}

}  // namespace popcorn
