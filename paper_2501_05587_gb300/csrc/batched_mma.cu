// Batched mode with K stored in FP16 or BF16: the K stream on the tensor cores.
//
// Each instance's pass needs S_ic = sum_{j in L_c} K_ij for its rows (the paper's SpMM,
// Alg. 2 line 7).  Per 128-row block I of an instance, S over the block's rows is
// sum_J K_IJ V_J^T, with V_J the one-hot label rows of column block J (Eq. 8 without its
// 1 / |L_c| scale): an MMA chain of M = 128 rows, N = k rounded up to 16, reduction over
// the instance's n columns.  A half entry times 1 or 0 is exact and the tensor cores add in
// FP32, so S is the cluster sums of the rounded K up to the order of the FP32 additions.
// The instances are small (n up to a few thousand), so the square is read whole: no slots,
// no fold, S written once a row.
//
// After the build, batched_pack_half_kernel rounds each instance's FP32 square into tiles
// of the 128-byte-swizzled half layout (kPackedSw128H: two boxes of 128 rows x 64 columns,
// entries past n zero), tile (I, J) at Kh + (I T + J) 32 KB: the K-major A operand of the
// MMAs as it lies in memory.  Per pass batched_onehot_kernel writes every block's one-hot
// operand, and batched_mma_kernel (persistent, one CTA an SM) takes the units (instance,
// row block) in the caller's order: warp 0 bulk-copies each tile of the unit's block row
// with V_J into a ring of stages, warp 1 issues 8 MMAs a tile into a TMEM accumulator
// (double-buffered across units), warps 2-5 read it (a lane a row) and store each row's k
// sums.  An instance that has stopped is skipped by every role alike (its loop state does
// not change during the launch).  Every wait is bounded; one that runs out sets *err, every
// role leaves, the CTA waits for its own copies and MMAs and frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "half_common.cuh"
#include "popcorn_internal.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

constexpr int kB = 128;
constexpr int kTileBytes = 32768;
constexpr int kMmaThreads = 192;
constexpr int kPackThreads = 256;
constexpr int kMaxStages = 6;

// the instance holding flattened index x of a prefix field that ascends with the instance
template <class F>
__device__ __forceinline__ int inst_of(const BatchInst* I, int count, long long x, F field) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (field(I[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

using hstore::pack2;
using hstore::round_trip;

// One tile of one instance's square, a 64-column box at a time: the FP32 rows (row-major,
// ldk) into shared memory, then each 32-bit word of the box (row (w >> 5), columns
// 64 box + 8 (((w >> 2) & 7) ^ (row & 7)) + 2 (w & 3) + {0, 1}), zeros past n.
template <typename TH>
__global__ void __launch_bounds__(kPackThreads) batched_pack_half_kernel(const BatchInst* I, int count) {
    __shared__ float half_tile[kB][65];   // 128 rows x 64 columns (+1 against bank conflicts)
    const long long g = blockIdx.x;
    const int t = inst_of(I, count, g, [](const BatchInst& x) { return x.htile0; });
    const BatchInst& b = I[t];
    const int lt = (int)(g - b.htile0);
    const int bi = lt / b.T, bj = lt - bi * b.T;
    const int rows = b.n - bi * kB, cols = b.n - bj * kB;
    const float* src = b.K + (int64_t)bi * kB * b.ldk + (int64_t)bj * kB;
    uint32_t* dst = reinterpret_cast<uint32_t*>(b.Kh + (size_t)lt * kTileBytes);
    for (int box = 0; box < 2; ++box) {
        if (box) __syncthreads();   // the previous box is written out
        // 2048 float4 a box, 8 a thread, all loads issued before the first store
        float4 x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int q = threadIdx.x + kPackThreads * e;   // float4 q: row q >> 4, columns 4 (q & 15) + 0..3
            const int r = q >> 4, c = 64 * box + 4 * (q & 15);
            // ldk is a multiple of 4 and the rows start 16-byte aligned; a float4 past n is read
            // only where its first column is below n (the row padding up to ldk is allocated)
            x[e] = (r < rows && c < cols) ? __ldg(reinterpret_cast<const float4*>(src + (int64_t)r * b.ldk + c))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int q = threadIdx.x + kPackThreads * e;
            const int r = q >> 4, c = 4 * (q & 15), c0 = 64 * box + c;
            half_tile[r][c] = x[e].x;
            half_tile[r][c + 1] = c0 + 1 < cols ? x[e].y : 0.f;
            half_tile[r][c + 2] = c0 + 2 < cols ? x[e].z : 0.f;
            half_tile[r][c + 3] = c0 + 3 < cols ? x[e].w : 0.f;
        }
        __syncthreads();
        if (bi == bj && threadIdx.x < rows && (threadIdx.x >> 6) == box)
            b.kdiag[bi * kB + threadIdx.x] = round_trip<TH>(half_tile[threadIdx.x][threadIdx.x & 63]);
        for (int w = threadIdx.x; w < 4096; w += kPackThreads) {
            const int r = w >> 5;
            const int c = 8 * (((w >> 2) & 7) ^ (r & 7)) + 2 * (w & 3);
            dst[4096 * box + w] = pack2<TH>(half_tile[r][c], half_tile[r][c + 1]);
        }
    }
}

// One 128-block's one-hot operand: V[c][i] = 1 if point 128 X + i has label c (0 past n),
// N rows of 128 entries, K-major in the 128-byte swizzle (16-byte chunk q = (box, c, ch)
// holds points 64 box + 8 (ch ^ (c mod 8)) + 0..7).
template <typename TH>
__global__ void __launch_bounds__(kB) batched_onehot_kernel(const BatchInst* I, int count, int eval) {
    const int t = inst_of(I, count, blockIdx.x, [](const BatchInst& x) { return (long long)x.vblock0; });
    const BatchInst& b = I[t];
    if (pass_skip(b.st, eval)) return;
    __shared__ uint8_t lab[kB];
    const int X = blockIdx.x - b.vblock0, N = b.N;
    const int i = X * kB + threadIdx.x;
    lab[threadIdx.x] = (i < b.n && (int)b.lab8[i] < b.k) ? b.lab8[i] : (uint8_t)0xFF;
    __syncthreads();
    const uint32_t one = std::is_same<TH, __half>::value ? 0x3C00u : 0x3F80u;
    uint4* dst = reinterpret_cast<uint4*>(b.V + (size_t)X * N * kB * 2);
    for (int q = threadIdx.x; q < N * 16; q += kB) {
        const int box = q / (N * 8), c = (q >> 3) % N, ch = q & 7;
        const int i0 = 64 * box + 8 * (ch ^ (c & 7));
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            w[e] = (lab[i0 + 2 * e] == c ? one : 0u) | ((lab[i0 + 2 * e + 1] == c ? one : 0u) << 16);
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// kind::f16 instruction descriptor, FP32 accumulate, A and B both FP16 or both BF16, both
// K-major; N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_half_kmajor(bool bf16, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(kB >> 4) << 24);
}

struct BatchedMmaArgs {
    const BatchInst* I;
    const int2* units;         // (instance, row block), in processing order
    int nunits;
    int stages, stage_bytes, off_bars;
    uint32_t tmem_cols;
    int* err;
    int eval;
    unsigned long long wait_ns;
    // Test hook for the error path (0 in every ordinary launch): CTA 0 never issues the
    // copies of its tile number stall_block - 1, so the waits for it run out after wait_ns.
    int stall_block;
};

template <bool BF16>
__global__ void __launch_bounds__(kMmaThreads, 1) batched_mma_kernel(BatchedMmaArgs a) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment: the swizzle pattern follows address bits 4-9
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = tc::smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.stages;
    const uint32_t bars = sbase + (uint32_t)a.off_bars;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (S + s); };
    auto accf_bar = [&](int b) { return bars + 8u * (2 * S + b); };
    auto acce_bar = [&](int b) { return bars + 8u * (2 * S + 2 + b); };
    const uint32_t down_bar = bars + 8u * (2 * S + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + a.off_bars + 8 * (2 * S + 5));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_bars + 8 * (2 * S + 5) + 4);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full_bar(s), 1);
            tc::mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(accf_bar(b), 1);
            tc::mbar_init(acce_bar(b), 4);
        }
        tc::mbar_init(down_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // whole warp
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32((const void*)tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int G = (int)gridDim.x;
    const uint32_t half_cols = a.tmem_cols / 2;   // accumulator buffer b at column b * half_cols

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: the tiles of the unit's block row with their V_J
            const uint64_t stream_once = tc::l2_evict_first();   // each tile is read once a pass
            const long long skip = blockIdx.x == 0 ? (long long)a.stall_block - 1 : -1;
            long long t = 0;
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < a.nunits && ok; u += G) {
                const int2 w = a.units[u];
                const BatchInst& b = a.I[w.x];
                if (pass_skip(b.st, a.eval)) continue;
                const uint32_t vbytes = (uint32_t)b.N * kB * 2;
                for (int J = 0; J < b.T; ++J) {
                    if (t >= S && !tc::mbar_wait_for(empty_bar(s), ph ^ 1u, abort_flag, a.err, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (t != skip) {   // the test hook: this tile never arrives
                        tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)kTileBytes + vbytes);
                        const uint32_t dst = sbase + (uint32_t)s * (uint32_t)a.stage_bytes;
                        tc::bulk_load_1d_hint(dst, b.Kh + ((size_t)w.y * b.T + J) * kTileBytes,
                                              (uint32_t)kTileBytes, full_bar(s), stream_once);
                        tc::bulk_load_1d(dst + kTileBytes, b.V + (size_t)J * vbytes, vbytes, full_bar(s));
                    }
                    ++t;
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (*abort_flag) {
                // leaving early: let this thread's copies land before the CTA's memory goes
                for (long long t2 = t > S ? t - S : 0; t2 < t; ++t2) {
                    if (t2 == skip) continue;   // nothing was issued for it
                    const uint32_t bar = full_bar((int)(t2 % S)), par = (uint32_t)(t2 / S) & 1u;
                    const unsigned long long t0 = tc::globaltimer();
                    while (!tc::mbar_try_wait(bar, par) && tc::globaltimer() - t0 < a.wait_ns) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: row sums of the unit's block row into buffer lt & 1
            int s = 0;
            uint32_t ph = 0;
            int lt = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < a.nunits && ok; u += G) {
                const int2 w = a.units[u];
                const BatchInst& b = a.I[w.x];
                if (pass_skip(b.st, a.eval)) continue;
                const int buf = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                ++lt;
                if (!tc::mbar_wait_for(acce_bar(buf), (use & 1u) ^ 1u, abort_flag, a.err, a.wait_ns)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const int N = b.N;
                const uint32_t idesc = idesc_half_kmajor(BF16, N);
                const uint32_t d = tmem + (uint32_t)buf * half_cols;
                for (int J = 0; J < b.T; ++J) {
                    if (!tc::mbar_wait_for(full_bar(s), ph, abort_flag, a.err, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t st = sbase + (uint32_t)s * (uint32_t)a.stage_bytes;
                    const uint32_t v = st + kTileBytes;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        tc::mma_bf16(d, tc::sw128_desc(st + (kk >> 2) * 16384 + (kk & 3) * 32),
                                     tc::sw128_desc(v + (kk >> 2) * (N * 128) + (kk & 3) * 32), idesc,
                                     (J | kk) ? 1u : 0u);
                    tc::mma_commit(empty_bar(s));   // the stage is free once these MMAs have read it
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                tc::mma_commit(accf_bar(buf));   // this block row's sums are complete
            }
            // every MMA this thread issued completes before TMEM is released
            tc::mma_commit(down_bar);
            const unsigned long long t0 = tc::globaltimer();
            while (!tc::mbar_try_wait(down_bar, 0) && tc::globaltimer() - t0 < a.wait_ns) {
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lanes 32 (warp % 4) + lane = rows
        const int q = warp & 3;
        int lt = 0;
        for (int u = blockIdx.x; u < a.nunits; u += G) {
            const int2 w = a.units[u];
            const BatchInst& b = a.I[w.x];
            if (pass_skip(b.st, a.eval)) continue;
            const int buf = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            ++lt;
            const bool ok = tc::mbar_wait_for(accf_bar(buf), use & 1u, abort_flag, a.err, a.wait_ns);
            // all epilogue threads agree before touching TMEM
            if (!tc::named_bar_all(1, 128, ok && !*abort_flag)) break;
            tc::tc_fence_after();
            const int n = b.n, k = b.k;
            const int row = w.y * kB + 32 * q + lane;
            float* out = b.Spart + row;   // [c][i], one segment
            for (int c0 = 0; c0 < b.N; c0 += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * half_cols + (uint32_t)c0));
                tc::tmem_ld_wait();
                if (row < n) {
#pragma unroll
                    for (int x = 0; x < 16; ++x)
                        if (c0 + x < k) out[(size_t)(c0 + x) * n] = __uint_as_float(r[x]);
                }
            }
            // the buffer is read: hand it back to the MMA issuer
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acce_bar(buf));
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
    }
}

int batched_mma_bars_bytes(int stages) { return 8 * (2 * stages + 5) + 8; }

}  // namespace

bool plan_batched_mma(BatchPlan* bp, int num_sms, int smem_optin) {
    if (bp->Nmax < 16 || bp->Nmax > 256 || bp->Nmax % 16) return false;
    const int stage_bytes = kTileBytes + bp->Nmax * kB * 2;
    for (int S = kMaxStages; S >= 2; --S) {
        const int bytes = S * stage_bytes + batched_mma_bars_bytes(S) + 1024;   // + 1024-byte alignment slack
        if (bytes > smem_optin) continue;
        bp->mstages = S;
        bp->msmem = (size_t)bytes;
        bp->mgrid = bp->nunits < num_sms ? bp->nunits : num_sms;
        return true;
    }
    return false;
}

cudaError_t configure_batched_mma(int smem_optin) {
    void (*fs[2])(BatchedMmaArgs) = {batched_mma_kernel<false>, batched_mma_kernel<true>};
    for (auto f : fs) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_batched_pack_half(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s) {
    if (bp.htiles <= 0 || bp.htiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (bp.half == POPCORN_K_BF16)
        batched_pack_half_kernel<__nv_bfloat16><<<(unsigned)bp.htiles, kPackThreads, 0, s>>>(dI, bp.count);
    else
        batched_pack_half_kernel<__half><<<(unsigned)bp.htiles, kPackThreads, 0, s>>>(dI, bp.count);
    return cudaGetLastError();
}

cudaError_t launch_batched_mma_stream(const BatchInst* dI, const int2* units, const BatchPlan& bp, int* err, int eval,
                                      cudaStream_t s, int stall_ms) {
    const bool bf16 = bp.half == POPCORN_K_BF16;
    if (!bf16 && bp.half != POPCORN_K_FP16) return cudaErrorInvalidValue;
    if (bf16)
        batched_onehot_kernel<__nv_bfloat16><<<(unsigned)bp.vblocks, kB, 0, s>>>(dI, bp.count, eval);
    else
        batched_onehot_kernel<__half><<<(unsigned)bp.vblocks, kB, 0, s>>>(dI, bp.count, eval);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    BatchedMmaArgs a;
    a.I = dI;
    a.units = units;
    a.nunits = bp.nunits;
    a.stages = bp.mstages;
    a.stage_bytes = kTileBytes + bp.Nmax * kB * 2;
    a.off_bars = bp.mstages * a.stage_bytes;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * bp.Nmax)) cols <<= 1;
    a.tmem_cols = cols;
    a.err = err;
    a.eval = eval;
    a.stall_block = stall_ms > 0 ? 1 : 0;
    a.wait_ns = stall_ms > 0 ? (unsigned long long)stall_ms * 1000000ull : tc::kWaitLimitNs;
    if (bf16)
        batched_mma_kernel<true><<<bp.mgrid, kMmaThreads, bp.msmem, s>>>(a);
    else
        batched_mma_kernel<false><<<bp.mgrid, kMmaThreads, bp.msmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace popcorn
