// K-means++ seeding (Sec. 2.1) in the feature space of the kernel, on the GPU.
//
// The paper names K-means++ as the initialization that samples each next initial centroid
// from a weighted distribution favouring points far from those already chosen; the weight of
// the cited method is the squared distance to the nearest chosen point, here in the feature
// space Kernel K-means clusters in:
//   D(i) = min over chosen c of ||phi(p_i) - phi(p_c)||^2 = min_c (K_ii - 2 K_ic + K_cc).
// K is never formed: every step evaluates kappa(p_i, p_c) for all i from the points, in FP64
// (the sampling decision compares running sums of D against a fraction of their total, so it
// is taken in FP64).  The caller supplies the k uniform draws u.  The first point is
// floor(u_0 n); point t >= 1 is the first i, in index order, at which the running sum of D
// exceeds u_t sum_i D(i) (floor(u_t n) if that sum is 0).  Each point's label is the index of
// its nearest chosen point (the lowest on ties): the initial labels for popcorn_fit.
//
// kmeanspp_kernel: one cooperative launch, one CTA of 512 threads per SM.  CTA b owns the
// points [b n / G, (b + 1) n / G) and keeps their D, labels and K_ii in shared memory.  A step:
// the CTA's sum of D (its threads' contiguous chunks, each summed in order, then the chunk
// sums in order) -> grid barrier -> every CTA adds the G sums in order and locates the CTA
// whose range holds the target; that CTA finds the point and publishes it -> grid barrier ->
// every warp evaluates kappa against the new point for its rows (lanes split the coordinates,
// a butterfly adds them) and lowers D.  All orders are fixed: runs are bit-identical.  Every
// wait is bounded (grid_sync.cuh).
#include <cmath>

#include "grid_sync.cuh"
#include "popcorn_internal.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

constexpr int kSeedThreads = 512;
constexpr int kSeedWarps = kSeedThreads / 32;

struct SeedArgs {
    const float* P;
    int64_t ldp;
    int n, d, k;
    int kind, degree;
    double gamma, coef0, neg_gamma_over_sigma2;   // kappa in FP64
    const double* u;           // k draws in [0, 1)
    int32_t* labels;           // n
    int32_t* centers;          // k
    double* part;              // [G] the CTAs' sums of D
    int* chosen;               // the point chosen in the running step
    unsigned* bar;             // grid barrier words
    int* err;
    int rows_max;              // ceil(n / G)
};

// Dynamic shared memory: the center's coordinates [d], then per owned row D, K_ii (doubles)
// and the label (int), then the threads' chunk sums and their prefix [kSeedThreads] and the
// CTAs' sums [G] (doubles).
struct SeedLayout {
    size_t cs, D, kii, lab, tsum, tpre, part, bytes;
};
__host__ __device__ inline SeedLayout seed_layout(int d, int rows_max, int G) {
    SeedLayout L;
    L.cs = 0;
    L.D = L.cs + (size_t)d * 8;
    L.kii = L.D + (size_t)rows_max * 8;
    L.tsum = L.kii + (size_t)rows_max * 8;
    L.tpre = L.tsum + (size_t)kSeedThreads * 8;
    L.part = L.tpre + (size_t)kSeedThreads * 8;
    L.lab = L.part + (size_t)G * 8;
    L.bytes = L.lab + (size_t)rows_max * 4;
    return L;
}

// kappa from the inner product (linear, polynomial) or the squared distance (Gaussian), FP64;
// the polynomial power by repeated multiplication
__device__ __forceinline__ double kappa_of(const SeedArgs& a, double s) {
    if (a.kind == POPCORN_GAUSSIAN) return exp(a.neg_gamma_over_sigma2 * s);
    if (a.kind == POPCORN_POLYNOMIAL) {
        const double base = fma(a.gamma, s, a.coef0);
        double v = base;
        for (int e = 1; e < a.degree; ++e) v *= base;
        return v;
    }
    return s;
}

// The warp's FP64 inner product (or squared distance, Gaussian) of point i with the center
// in shared memory: lane l takes coordinates l, l + 32, ... in order, then a butterfly.
__device__ __forceinline__ double warp_pair(const SeedArgs& a, int i, const double* __restrict__ cs, int lane) {
    const float* p = a.P + (int64_t)i * a.ldp;
    double s = 0.0;
    if (a.kind == POPCORN_GAUSSIAN) {
        for (int l = lane; l < a.d; l += 32) {
            const double t = (double)__ldg(p + l) - cs[l];
            s = fma(t, t, s);
        }
    } else {
        for (int l = lane; l < a.d; l += 32) s = fma((double)__ldg(p + l), cs[l], s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void __launch_bounds__(kSeedThreads, 1) kmeanspp_kernel(SeedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int G = gridDim.x, n = a.n, k = a.k;
    const SeedLayout L = seed_layout(a.d, a.rows_max, G);
    double* cs = reinterpret_cast<double*>(smem + L.cs);
    double* D = reinterpret_cast<double*>(smem + L.D);
    double* kii = reinterpret_cast<double*>(smem + L.kii);
    double* tsum = reinterpret_cast<double*>(smem + L.tsum);
    double* tpre = reinterpret_cast<double*>(smem + L.tpre);
    double* part_s = reinterpret_cast<double*>(smem + L.part);
    int* lab = reinterpret_cast<int*>(smem + L.lab);
    __shared__ double kcc_s, tgt_s;
    __shared__ int bstar_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lo = (int)((int64_t)blockIdx.x * n / G), hi = (int)((int64_t)(blockIdx.x + 1) * n / G);
    const int rows = hi - lo;
    const int ch = (rows + kSeedThreads - 1) / kSeedThreads;   // rows a thread sums, in order
    const int r0 = min(rows, ch * (int)threadIdx.x), r1 = min(rows, r0 + ch);

    // K_ii of the owned points (the Gaussian's is 1)
    for (int i = lo + warp; i < hi; i += kSeedWarps) {
        double v = 1.0;
        if (a.kind != POPCORN_GAUSSIAN) {
            const float* p = a.P + (int64_t)i * a.ldp;
            double s = 0.0;
            for (int l = lane; l < a.d; l += 32) {
                const double x = (double)__ldg(p + l);
                s = fma(x, x, s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            v = kappa_of(a, s);
        }
        if (lane == 0) kii[i - lo] = v;
    }

    // point c joins the chosen set as number t: D and the labels of the owned points
    auto add_center = [&](int t, int c) {
        const float* pc = a.P + (int64_t)c * a.ldp;
        for (int l = threadIdx.x; l < a.d; l += blockDim.x) cs[l] = (double)__ldg(pc + l);
        __syncthreads();
        if (warp == 0) {
            double s = 0.0;
            if (a.kind != POPCORN_GAUSSIAN) {
                for (int l = lane; l < a.d; l += 32) s = fma(cs[l], cs[l], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            }
            if (lane == 0) kcc_s = a.kind == POPCORN_GAUSSIAN ? 1.0 : kappa_of(a, s);
        }
        __syncthreads();
        const double kcc = kcc_s;
        for (int i = lo + warp; i < hi; i += kSeedWarps) {
            const double kic = kappa_of(a, warp_pair(a, i, cs, lane));
            const double dc = fmax(kii[i - lo] - 2.0 * kic + kcc, 0.0);
            if (lane == 0 && (t == 0 || dc < D[i - lo])) {
                D[i - lo] = dc;
                lab[i - lo] = t;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.centers[t] = c;
        __syncthreads();
    };

    __syncthreads();
    add_center(0, min((int)floor(a.u[0] * n), n - 1));
    for (int t = 1; t < k; ++t) {
        // the CTA's sum of D: each thread's chunk in order, then the chunk sums in order
        double s = 0.0;
        for (int r = r0; r < r1; ++r) s += D[r];
        tsum[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double run = 0.0;
            for (int j = 0; j < kSeedThreads; ++j) {
                tpre[j] = run;
                run += tsum[j];
            }
            a.part[blockIdx.x] = run;
        }
        if (!gsync::grid_barrier(a.bar, a.err)) return;
        for (int b = threadIdx.x; b < G; b += blockDim.x) part_s[b] = __ldcg(a.part + b);
        __syncthreads();
        // every CTA: the total in CTA order, the target, and the CTA whose range holds it
        if (threadIdx.x == 0) {
            double W = 0.0;
            for (int b = 0; b < G; ++b) W += part_s[b];
            int bstar = -1;
            double before = 0.0;
            if (W > 0.0) {
                const double target = a.u[t] * W;
                double run = 0.0;
                int lastpos = -1;
                for (int b = 0; b < G && bstar < 0; ++b) {
                    if (part_s[b] > 0.0) lastpos = b;
                    if (run + part_s[b] > target) {
                        bstar = b;
                        before = run;
                    }
                    run += part_s[b];
                }
                if (bstar < 0) {   // u_t W rounded up to W: the last CTA with a positive sum
                    bstar = lastpos;
                    before = 0.0;
                    for (int b = 0; b < bstar; ++b) before += part_s[b];
                }
                tgt_s = target - before;   // the target inside CTA bstar's range
            }
            bstar_s = bstar;
        }
        __syncthreads();
        const int bstar = bstar_s;
        if (bstar == (int)blockIdx.x) {
            // the thread whose chunk holds the target walks it in order; the last point with
            // a positive D of the CTA if rounding leaves the target past the end
            const double tgt = tgt_s;
            const double lo_run = tpre[threadIdx.x];
            if (r0 < r1 && lo_run + tsum[threadIdx.x] > tgt && lo_run <= tgt) {
                double run = lo_run;
                int c = -1, lastpos = r0;
                for (int r = r0; r < r1; ++r) {
                    if (D[r] > 0.0) lastpos = r;
                    run += D[r];
                    if (run > tgt) {
                        c = r;
                        break;
                    }
                }
                *a.chosen = lo + (c >= 0 ? c : lastpos);   // rounding at the chunk's end
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double total = 0.0;
                for (int j = 0; j < kSeedThreads; ++j) total += tsum[j];
                if (!(total > tgt)) {
                    int c = rows - 1;
                    while (c > 0 && !(D[c] > 0.0)) --c;
                    *a.chosen = lo + c;
                }
            }
        }
        if (!gsync::grid_barrier(a.bar, a.err)) return;
        const int c = bstar >= 0 ? __ldcg(a.chosen) : min((int)floor(a.u[t] * n), n - 1);
        add_center(t, c);
    }
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) a.labels[i] = lab[i - lo];
}

}  // namespace

size_t kmeanspp_smem(int n, int d, int num_sms) {
    return seed_layout(d, (n + num_sms - 1) / num_sms, num_sms).bytes;
}

int kmeanspp_dynamic_limit(int smem_optin) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kmeanspp_kernel) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return optin_minus_static(smem_optin, fa.sharedSizeBytes);
}

cudaError_t configure_kmeanspp(int smem_optin) {
    return cudaFuncSetAttribute(kmeanspp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kmeanspp_dynamic_limit(smem_optin));
}

bool kmeanspp_fits(int n, int d, int num_sms, int smem_optin) {
    return kmeanspp_smem(n, d, num_sms) <= (size_t)kmeanspp_dynamic_limit(smem_optin);
}

cudaError_t launch_kmeanspp(const float* P, int n, int d, int64_t ldp, int k, const popcorn_kernel& kern,
                            const double* u, int32_t* labels, int32_t* centers, double* part, int* chosen,
                            unsigned* bar, int* err, int num_sms, cudaStream_t s) {
    SeedArgs a;
    a.P = P;
    a.ldp = ldp;
    a.n = n;
    a.d = d;
    a.k = k;
    a.kind = kern.kind;
    a.degree = kern.degree;
    a.gamma = kern.gamma;
    a.coef0 = kern.coef0;
    a.neg_gamma_over_sigma2 = kern.kind == POPCORN_GAUSSIAN ? -kern.gamma / (kern.sigma * kern.sigma) : 0.0;
    a.u = u;
    a.labels = labels;
    a.centers = centers;
    a.part = part;
    a.chosen = chosen;
    a.bar = bar;
    a.err = err;
    a.rows_max = (n + num_sms - 1) / num_sms;
    cudaError_t e = cudaMemsetAsync(bar, 0, 32 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)num_sms);
    cfg.blockDim = dim3(kSeedThreads);
    cfg.dynamicSmemBytes = kmeanspp_smem(n, d, num_sms);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kmeanspp_kernel, a);
}

}  // namespace popcorn
