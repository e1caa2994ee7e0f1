// Whole fits in one kernel, for a stored FP32 K that sits in L2.
//
// When K is small (n of a few thousand: 16 MB at n = 2,000) a pass of Alg. 2 is a few
// microseconds of work, and three dependent launches a pass (stream, z, argmin) cost more
// than the work.  fit_fused_kernel runs every pass of a fit, and the final objective, in
// one cooperative launch of one CTA per SM; the CTAs exchange data twice a pass:
//
//   row sums    CTA b owns rows [b n / G, (b + 1) n / G) (their rows of K copied to shared
//               memory once a fit when they fit).  A warp takes one row at a time: lane l
//               reads the float4 chunks l, l + 32, ... and adds each element to its own bin
//               of the column's cluster (bins[c][l]: bank l, no conflicts); at the row's end
//               lane c adds the 32 bins of cluster c in a rotated order.  S_ic =
//               sum_{j in L_c} K_ij (the SpMM of Alg. 2 line 7) for the CTA's rows stays in
//               shared memory; the CTA's FP64 partials of sum_{i in L_c} S_ic (z, Eq. 14)
//               go to its slot.
//   exchange A  every CTA reads all partials and adds them in the same fixed order:
//               ||c_c||^2, 1/|L_c| and J, identical in every CTA; CTA 0 records them.
//   argmin      D_ic = K_ii - 2 E_ic + ||c_c||^2 in FP64 for the CTA's rows (ties to the
//               lowest index, empty clusters skipped), new labels; the histogram of the
//               CTA's new labels and its change count go to its slot.
//   exchange B  every CTA reads all labels, sums the histograms (the next pass's counts)
//               and the change counts, and takes the same loop decision.
//
// An exchange is a grid barrier (one arrival counter, acquire-release) after which the CTAs
// read the slots from L2.  The pass semantics (stopping
// rules, J history, change history, E report, the final objective pass) are those of the
// launched passes (iterate.cu).  Every wait is bounded: after kWaitLimitNs a CTA raises the
// launch's error word and leaves, so a stuck exchange ends as POPCORN_ERR_TIMEOUT, not as a
// hang.
#include "popcorn_internal.cuh"
#include "stream_common.cuh"
#include "grid_sync.cuh"
#include "tc_common.cuh"

#include <cuda/std/limits>

namespace popcorn {
namespace {

constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;

struct FusedArgs {
    const float* K;            // n x ldk FP32, full square
    int64_t ldk;
    const float* kdiag;
    int n, k;
    int32_t* lab32;
    uint8_t* lab8;             // n rounded up to 16, zero padded
    int32_t* counts;           // [2][k]: counts[0] = those of the initial labels, counts[1] = 0
    double* zpart;             // [gridDim.x][k]
    double* zsum;              // [k] \  the last pass's values, as the pass
    double* cnorm;             // [k]  | kernels leave them
    double* invm;              // [k] /
    unsigned* xchg;            // fused_xchg_words: barrier words (one 128-byte line), histograms [G][k],
                               // change counts [G]; zero before the launch
    LoopState* st;
    double* J_hist;
    int32_t* changed_hist;
    float* E_out;              // optional n x k
    int rows_max;              // ceil(n / gridDim.x)
    int cache_k;               // 1: the CTA's rows of K are copied to shared memory once a fit
    // Test hook for the error path (0 in every ordinary launch): CTA 0 leaves before its first
    // grid barrier, so the others' bounded waits there run out after wait_ns.
    int stall;
    unsigned long long wait_ns;
};

// Dynamic shared memory, in order: per-warp bins [kFusedWarps][k][32] floats, the row
// sums of the CTA's rows [rows_max][k] floats, then cnorm and 1/|L_c| ([k] doubles each),
// the next labels' histogram and the current counts ([k] ints each), the CTA's diag K
// [rows_max] floats, the labels of
// all points (n rounded up to 16) and, when cache_k, the CTA's rows of K [rows_max][ldk].
struct FusedLayout {
    size_t bins, S, cn, iv, hist, m, kd, lab, Kc, bytes;
};
__host__ __device__ inline FusedLayout fused_layout(int n, int k, int rows_max, int64_t ldk, int cache_k) {
    FusedLayout L;
    L.bins = 0;
    L.S = L.bins + (size_t)kFusedWarps * k * 32 * 4;
    L.cn = (L.S + (size_t)rows_max * k * 4 + 15) & ~(size_t)15;
    L.iv = L.cn + (size_t)k * 8;
    L.hist = L.iv + (size_t)k * 8;
    L.m = L.hist + (size_t)k * 4;
    L.kd = (L.m + (size_t)k * 4 + 15) & ~(size_t)15;
    L.lab = (L.kd + (size_t)rows_max * 4 + 15) & ~(size_t)15;
    L.Kc = L.lab + (((size_t)n + 15) & ~(size_t)15);
    L.bytes = L.Kc + (cache_k ? (size_t)rows_max * (size_t)ldk * 4 : 0);
    return L;
}

// A float4 of K: from the CTA's copy in shared memory, or from L2.
template <bool CACHED>
__device__ __forceinline__ float4 kload4(const float4* p) {
    if constexpr (CACHED) return *p;
    else return __ldcg(p);
}
template <bool CACHED>
__device__ __forceinline__ float kload(const float* p) {
    if constexpr (CACHED) return *p;
    else return __ldcg(p);
}

// S_ic of rows [lo, hi) into S[(i - lo) k + c], from the labels in lab_s; rows of K from
// Kc (the CTA's copy, row i at Kc + (i - lo) ldk) or from global memory.
template <bool CACHED>
__device__ void row_sums(const FusedArgs& a, int lo, int hi, const uint8_t* __restrict__ lab_s, float* bins,
                         float* S, const float* Kc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = a.n, k = a.k;
    float* b = bins + (size_t)warp * k * 32;
    const bool vec = (a.ldk & 3) == 0 && ((uintptr_t)a.K & 15) == 0;
    const int n4 = vec ? n >> 2 : 0;
    for (int i = lo + warp; i < hi; i += kFusedWarps) {
        for (int c = 0; c < k; ++c) b[c * 32 + lane] = 0.f;
        const float* row = CACHED ? Kc + (int64_t)(i - lo) * a.ldk : a.K + (int64_t)i * a.ldk;
        const float4* row4 = reinterpret_cast<const float4*>(row);
        int q = lane;
        // eight chunks in flight a lane, then their adds
        for (; q + 7 * 32 < n4; q += 8 * 32) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = kload4<CACHED>(row4 + q + 32 * u);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uchar4 l4 = *reinterpret_cast<const uchar4*>(lab_s + 4 * (q + 32 * u));
                b[l4.x * 32 + lane] += v[u].x;
                b[l4.y * 32 + lane] += v[u].y;
                b[l4.z * 32 + lane] += v[u].z;
                b[l4.w * 32 + lane] += v[u].w;
            }
        }
        for (; q < n4; q += 32) {
            const float4 v = kload4<CACHED>(row4 + q);
            const uchar4 l4 = *reinterpret_cast<const uchar4*>(lab_s + 4 * q);
            b[l4.x * 32 + lane] += v.x;
            b[l4.y * 32 + lane] += v.y;
            b[l4.z * 32 + lane] += v.z;
            b[l4.w * 32 + lane] += v.w;
        }
        for (int j = 4 * n4 + lane; j < n; j += 32) b[lab_s[j] * 32 + lane] += kload<CACHED>(row + j);
        __syncwarp();
        // lane c: the 32 bins of cluster c, lane (c + t) mod 32 at step t (32 distinct banks)
        if (lane < k) {
            float t = 0.f;
#pragma unroll 8
            for (int s = 0; s < 32; ++s) t += b[lane * 32 + ((s + lane) & 31)];
            S[(size_t)(i - lo) * k + lane] = t;
        }
        __syncwarp();
    }
}

// The CTA's FP64 partials of sum_{i in L_c} S_ic over its rows, in row order.
__device__ void z_partials(const FusedArgs& a, int lo, int hi, const uint8_t* __restrict__ lab_s,
                           const float* __restrict__ S) {
    const int k = a.k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        double t = 0.0;
        for (int i = lo; i < hi; ++i)
            if ((int)lab_s[i] == c) t += (double)S[(size_t)(i - lo) * k + c];
        a.zpart[(size_t)blockIdx.x * k + c] = t;
    }
}

// After barrier 1, in every CTA: sum_{i in L_c} S_ic from the partials (warp w takes
// clusters w, w + 16, ...; lanes split the CTAs, a butterfly adds them: the same order in
// every CTA), ||c_c||^2 = (1/m_c^2) sum (Eq. 13/14), 1/m_c, and
// J = trace K - sum_c (1/m_c) sum_{i in L_c} S_ic.  CTA 0 also stores them where the pass
// kernels would.  Returns J.
__device__ double finalize(const FusedArgs& a, const int* __restrict__ m, double trace, double* cn_s,
                           double* iv_s) {
    __shared__ double jpart[kFusedWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = a.k, G = gridDim.x;
    double jw = 0.0;
    for (int c = warp; c < k; c += kFusedWarps) {
        double t = 0.0;
        for (int b = lane; b < G; b += 32) t += __ldcg(a.zpart + (size_t)b * k + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const double mc = (double)m[c];
        const double inv = mc > 0 ? 1.0 / mc : 0.0;
        if (lane == 0) {
            cn_s[c] = t * inv * inv;
            iv_s[c] = inv;
            if (blockIdx.x == 0) {
                a.zsum[c] = t;
                a.invm[c] = inv;
                a.cnorm[c] = t * inv * inv;
            }
        }
        jw += t * inv;
    }
    if (lane == 0) jpart[warp] = jw;
    __syncthreads();
    double J = trace;
    for (int w = 0; w < kFusedWarps; ++w) J -= jpart[w];
    __syncthreads();   // jpart is reused by the next call
    return J;
}

// Distances and argmin for rows [lo, hi) (thread t: row lo + t), new labels, and into the
// CTA's slot the histogram of its new labels and its number of changed labels.
__device__ void assign_rows(const FusedArgs& a, int lo, int hi, const float* __restrict__ S,
                            const double* __restrict__ cn_s, const double* __restrict__ iv_s,
                            const int* __restrict__ m, int* hist, const uint8_t* __restrict__ lab_s,
                            const float* __restrict__ kd_s, int* hslot, int* cslot) {
    const int k = a.k;
    for (int c = threadIdx.x; c < k; c += blockDim.x) hist[c] = 0;
    __syncthreads();
    int changed = 0;
    for (int i0 = lo; i0 < hi; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        int newl = 0;
        const bool own = i < hi;
        if (own) {
            const int li = lab_s[i];
            const double kd = (double)kd_s[i - lo];
            double best = cuda::std::numeric_limits<double>::infinity();
            int bi = li;
            for (int c = 0; c < k; ++c) {
                const double E = (double)S[(size_t)(i - lo) * k + c] * iv_s[c];   // (K V^T)_ic
                if (a.E_out) a.E_out[(int64_t)i * k + c] = (float)E;
                if (m[c] == 0) continue;
                const double D = fma(-2.0, E, kd + cn_s[c]);
                if (D < best) {
                    best = D;
                    bi = c;
                }
            }
            newl = bi;
            changed += bi != li;
            a.lab32[i] = bi;
            a.lab8[i] = (uint8_t)bi;
        }
        const unsigned act = __ballot_sync(0xffffffffu, own);
        if (own) {
            const unsigned peers = __match_any_sync(act, newl);
            if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[newl], __popc(peers));
        }
    }
    const int block_changed = __syncthreads_count(changed);
    for (int c = threadIdx.x; c < k; c += blockDim.x) hslot[(size_t)blockIdx.x * k + c] = hist[c];
    if (threadIdx.x == 0) cslot[blockIdx.x] = block_changed;
}

// After exchange B: m_c = the sum of every CTA's histogram, and the total change count
// (integers: exact in any order).
__device__ int gather_counts(const int* hslot, const int* cslot, int k, int* m) {
    __shared__ int ch_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
    for (int c = warp; c < k + 1; c += kFusedWarps) {
        int t = 0;
        for (int b = lane; b < G; b += 32) t += c < k ? __ldcg(hslot + (size_t)b * k + c) : __ldcg(cslot + b);
        t = __reduce_add_sync(0xffffffffu, t);
        if (lane == 0) {
            if (c < k) m[c] = t;
            else ch_s = t;
        }
    }
    __syncthreads();
    return ch_s;
}

template <bool CACHED>
__device__ void fit_body(const FusedArgs& a, unsigned char* smem) {
    const FusedLayout L = fused_layout(a.n, a.k, a.rows_max, a.ldk, CACHED ? 1 : 0);
    float* bins = reinterpret_cast<float*>(smem + L.bins);
    float* S = reinterpret_cast<float*>(smem + L.S);
    double* cn_s = reinterpret_cast<double*>(smem + L.cn);
    double* iv_s = reinterpret_cast<double*>(smem + L.iv);
    int* hist = reinterpret_cast<int*>(smem + L.hist);
    int* m_s = reinterpret_cast<int*>(smem + L.m);
    float* kd_s = reinterpret_cast<float*>(smem + L.kd);
    uint8_t* lab_s = smem + L.lab;
    float* Kc = reinterpret_cast<float*>(smem + L.Kc);
    LoopState* st = a.st;
    int* err = &st->wait_err;
    const int n = a.n, k = a.k, G = gridDim.x;
    unsigned* bar = a.xchg;   // the grid barrier's arrival count
    int* hslot = reinterpret_cast<int*>(a.xchg + 32);
    int* cslot = hslot + (size_t)G * k;
    const int lo = (int)((int64_t)blockIdx.x * n / G), hi = (int)((int64_t)(blockIdx.x + 1) * n / G);
    const int max_iter = st->max_iter, check = st->check_conv;
    const double tol = st->tol, trace = st->trace;
    const int nl16 = (n + 15) >> 4;
    // once a fit: the CTA's diag K, (when they fit) its rows of K, the initial counts
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) kd_s[i - lo] = a.kdiag[i];
    for (int c = threadIdx.x; c < k; c += blockDim.x) m_s[c] = a.counts[c];
    if constexpr (CACHED) {
        const int64_t q4 = (int64_t)(hi - lo) * a.ldk / 4;
        const float4* src = reinterpret_cast<const float4*>(a.K + (int64_t)lo * a.ldk);
        for (int64_t q = threadIdx.x; q < q4; q += blockDim.x) reinterpret_cast<float4*>(Kc)[q] = __ldcg(src + q);
    }
    auto load_labels = [&]() {
        for (int q = threadIdx.x; q < nl16; q += blockDim.x)
            reinterpret_cast<uint4*>(lab_s)[q] = __ldcg(reinterpret_cast<const uint4*>(a.lab8) + q);
    };
    // S, the CTA's z partials and exchange A; then in every CTA ||c||^2, 1/|L_c| and J
    auto reduce = [&](double* J) -> bool {
        row_sums<CACHED>(a, lo, hi, lab_s, bins, S, Kc);
        __syncthreads();
        z_partials(a, lo, hi, lab_s, S);
        if (!gsync::grid_barrier(bar, err, a.wait_ns)) return false;
        *J = finalize(a, m_s, trace, cn_s, iv_s);
        return true;
    };
    load_labels();
    __syncthreads();

    int it = 0, last_changed = -1;
    double J_last = 0.0, J_prev = 0.0;
    bool done = max_iter <= 0;
    if (a.stall && blockIdx.x == 0) return;   // the test hook: this CTA never arrives
    while (!done) {
        double J;
        if (!reduce(&J)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.J_hist[it] = J;
            st->J_last = J;
        }
        assign_rows(a, lo, hi, S, cn_s, iv_s, m_s, hist, lab_s, kd_s, hslot, cslot);
        if (!gsync::grid_barrier(bar, err, a.wait_ns)) return;
        // exchange B: the next pass's labels (loaded whether or not there is one), its counts
        // and this pass's change count; then the loop decision, taken alike in every CTA
        // (iterate.cu's assign pass)
        load_labels();
        const int ch = gather_counts(hslot, cslot, k, m_s);
        J_last = J;
        done = it + 1 >= max_iter;
        bool conv = false;
        if (check) {
            if (ch == 0) {
                done = true;
                conv = true;
            }
            if (tol > 0.0 && it >= 1 && J_prev - J_last <= tol * fabs(J_last)) done = true;
        }
        J_prev = J_last;
        last_changed = ch;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.changed_hist[it] = ch;
            st->last_changed = ch;
            st->iter = it + 1;
            st->done = done ? 1 : 0;
            if (conv) st->converged = 1;
            st->J_prev = J_prev;
        }
        ++it;
    }
    // J(labels_out): the last pass's J when it changed nothing, else one more reduction (the
    // final labels and their counts are already here)
    if (it > 0 && last_changed == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->J_eval = J_last;
        return;
    }
    double J;
    if (!reduce(&J)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->J_eval = J;
}

__global__ void __launch_bounds__(kFusedThreads, 1) fit_fused_kernel(FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (a.cache_k)
        fit_body<true>(a, smem);
    else
        fit_body<false>(a, smem);
}

}  // namespace

// The CTA's rows of K are kept in shared memory when they fit (n up to ~2,700 on 152 SMs).
size_t fused_fit_smem(int n, int k, int num_sms, int64_t ldk, int cache_k) {
    const int rows_max = (n + num_sms - 1) / num_sms;
    return fused_layout(n, k, rows_max, ldk, cache_k).bytes;
}

// dynamic shared memory the kernel may use next to its static shared memory
int fused_dynamic_limit(int smem_optin) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fit_fused_kernel) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return optin_minus_static(smem_optin, fa.sharedSizeBytes);
}

bool fused_fit_applies(int n, int k, int num_sms, int smem_optin) {
    if (n < 2 || n > kFusedMaxN || k < 1 || k > kFusedMaxK || num_sms < 1) return false;
    return fused_fit_smem(n, k, num_sms, 0, 0) <= (size_t)fused_dynamic_limit(smem_optin);
}

cudaError_t configure_fused_fit(int smem_optin) {
    return cudaFuncSetAttribute(fit_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                fused_dynamic_limit(smem_optin));
}

size_t fused_xchg_words(int num_sms, int k) { return 32 + (size_t)num_sms * (k + 1); }

cudaError_t launch_fused_fit(const PassBuffers& b, double* zpart, unsigned* xchg, int num_sms, int smem_optin,
                             cudaStream_t s, int stall_ms) {
    FusedArgs a;
    a.stall = stall_ms > 0 ? 1 : 0;
    a.wait_ns = stall_ms > 0 ? (unsigned long long)stall_ms * 1000000ull : tc::kWaitLimitNs;
    a.K = static_cast<const float*>(b.K);
    a.ldk = b.ldk;
    a.kdiag = b.kdiag;
    a.n = b.n;
    a.k = b.k;
    a.lab32 = b.lab32;
    a.lab8 = b.lab8;
    a.counts = b.counts;
    a.zpart = zpart;
    a.zsum = b.zsum;
    a.cnorm = b.cnorm;
    a.invm = b.invm;
    a.xchg = xchg;
    a.st = b.st;
    a.J_hist = b.J_hist;
    a.changed_hist = b.changed_hist;
    a.E_out = b.E_out;
    a.rows_max = (b.n + num_sms - 1) / num_sms;
    const bool vec = (b.ldk & 3) == 0 && ((uintptr_t)b.K & 15) == 0;
    a.cache_k = vec && fused_fit_smem(b.n, b.k, num_sms, b.ldk, 1) <= (size_t)fused_dynamic_limit(smem_optin);
    cudaError_t e = cudaMemsetAsync(xchg, 0, fused_xchg_words(num_sms, b.k) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    // one CTA per SM, all resident at once (the CTAs wait on one another at grid barriers)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)num_sms);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = fused_fit_smem(b.n, b.k, num_sms, b.ldk, a.cache_k);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fit_fused_kernel, a);
}

}  // namespace popcorn
