// Tensor-core (tcgen05) build of the kernel matrix K = kappa(P P^T).
//
// Sec. 3.2 forms B = P P^T with GEMM or SYRK and then applies the kernel
// function elementwise (Gaussian through Eq. 12 from B and the row norms).
// Here one persistent kernel walks the upper-triangle 128 x 128 tiles of B:
//
//   warp 0  (one lane)  TMA loads of 128 x 64 BF16 operand tiles into a
//                       4-stage shared-memory ring (128-byte swizzle);
//   warp 1  (one lane)  tcgen05.mma kind::f16 (BF16 x BF16 -> FP32) into one
//                       of two 128-column TMEM accumulators;
//   warps 2-5           epilogue: tcgen05.ld the accumulator, apply kappa
//                       with FP32 row norms, stage the tile and its transpose
//                       in shared memory and TMA-store both into K.
//
// Double-buffered TMEM lets the MMAs of tile t+1 run under the epilogue of
// tile t.  Precision modes:
//   BF16    A = B = bf16(P);  norms of the rounded rows, so the Gaussian
//           distance r_i + r_j - 2 B_ij is the distance of the rounded points.
//   BF16X3  A = [hi | hi | lo], B = [hi | lo | hi] with hi = bf16(p),
//           lo = bf16(p - hi): one GEMM of depth 3d gives
//           hi.hi + hi.lo + lo.hi, which recovers ~16 significant bits of
//           the cross term that the Gaussian's cancellation needs.
//
// Every mbarrier wait is bounded (about 2 s by %globaltimer).  A wait that
// runs out sets *err, raises a shared abort flag that ends every role's loop,
// waits (bounded again) for the CTA's own TMA copies and MMAs in flight,
// frees TMEM and returns; the host reports POPCORN_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "popcorn_internal.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

using namespace tc;

__device__ __forceinline__ void epi_bar() { named_bar<128>(1); }   // the 4 epilogue warps
constexpr uint32_t kIdesc = idesc_bf16(128, 128);

constexpr int BM = 128, BN = 128, BK = 64;   // tile rows, tile cols, bf16 depth per stage
constexpr int STAGES = 4;
constexpr int TILE_BYTES = BM * BK * 2;      // 16 KB per operand tile
constexpr int STG_BYTES = 128 * 32 * 4;      // one 128 x 32 FP32 staging chunk
constexpr int NTHREADS = 192;                // 6 warps

// shared-memory layout (offsets from a 1024-aligned base)
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + STAGES * TILE_BYTES;
constexpr int OFF_SD = OFF_B + STAGES * TILE_BYTES;   // 2 direct staging chunks (128B swizzle)
constexpr int OFF_ST = OFF_SD + 2 * STG_BYTES;         // 2 transposed staging chunks (no swizzle)
constexpr int OFF_RJ = OFF_ST + 2 * STG_BYTES;         // 128 column norms
constexpr int OFF_BAR = OFF_RJ + 128 * 4;
constexpr int NBAR = 2 * STAGES + 4 + 1;
constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
constexpr int SMEM_BYTES = OFF_MISC + 16 + 1024;       // + slack for 1024 alignment

struct TcArgs {
    int n, T, nkb;            // rows, tile rows, 64-deep k-blocks
    long long tiles;          // T (T + 1) / 2
    KernParams kp;
    const float* norms;       // row norms of the represented rows (Gaussian)
    float* kdiag;
    int* err;
};

__device__ __forceinline__ void tri_coords(long long t, int T, int* bi, int* bj) {
    // t enumerates the upper triangle row by row: row b starts at off(b) = b*T - b*(b-1)/2.
    // An FP32 estimate of the quadratic's root, then exact integer correction (no FP64:
    // GB300 runs FP64 at a small fraction of the FP32 rate).
    const float Tf = (float)T;
    const float disc = fmaxf((2.f * Tf + 1.f) * (2.f * Tf + 1.f) - 8.f * (float)t, 0.f);
    int b = (int)(((2.f * Tf + 1.f) - sqrtf(disc)) * 0.5f);
    if (b < 0) b = 0;
    if (b > T - 1) b = T - 1;
    auto off = [&](long long r) { return r * (long long)T - r * (r - 1) / 2; };
    while (b > 0 && off(b) > t) --b;
    while (b < T - 1 && off(b + 1) <= t) ++b;
    *bi = b;
    *bj = b + (int)(t - off(b));
}

__device__ __forceinline__ float kappa(float b, float ri, float rj, const KernParams& kp) {
    if (kp.kind == POPCORN_LINEAR) return b;
    if (kp.kind == POPCORN_POLYNOMIAL) {
        const float base = fmaf(kp.gamma, b, kp.coef0);
        float r = base;
        for (int e = 1; e < kp.degree; ++e) r *= base;
        return r;
    }
    const float d2 = fmaxf(fmaf(-2.f, b, ri + rj), 0.f);
    return expf(kp.neg_gamma_over_sigma2 * d2);
}

__global__ void __launch_bounds__(NTHREADS, 1)
    kbuild_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                     const __grid_constant__ CUtensorMap map_kd, const __grid_constant__ CUtensorMap map_kt,
                     TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + OFF_BAR;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    const uint32_t down_bar = bar0 + 8u * (2 * STAGES + 4);
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(smem + OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + OFF_MISC + 4);
    float* rj_s = reinterpret_cast<float*>(smem + OFF_RJ);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 4);
        }
        mbar_init(down_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // whole warp: allocate 256 TMEM columns (two 128-column accumulators)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const long long G = gridDim.x;
    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_parity[STAGES];
            bool issued[STAGES];
            for (int s = 0; s < STAGES; ++s) issued[s] = false;
            bool ok = true;
            for (long long t = blockIdx.x; t < a.tiles && ok; t += G) {
                int bi, bj;
                tri_coords(t, a.T, &bi, &bj);
                for (int kb = 0; kb < a.nkb; ++kb) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(full_bar(stage), 2 * TILE_BYTES);
                    tma_load_2d(sbase + OFF_A + stage * TILE_BYTES, &map_a, kb * BK, bi * BM, full_bar(stage));
                    tma_load_2d(sbase + OFF_B + stage * TILE_BYTES, &map_b, kb * BK, bj * BN, full_bar(stage));
                    issued[stage] = true;
                    issued_parity[stage] = phase;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // aborted: let this CTA's own copies land before shared memory goes away
                for (int s = 0; s < STAGES; ++s)
                    if (issued[s]) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try_wait(full_bar(s), issued_parity[s]) && globaltimer() - t0 < kWaitLimitNs) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int lt = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < a.tiles && ok; t += G, ++lt) {
                const int ab = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!mbar_wait(acce_bar(ab), (use & 1u) ^ 1u, abort_flag, a.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(ab * BN);
                for (int kb = 0; kb < a.nkb; ++kb) {
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sbase + OFF_A + stage * TILE_BYTES;
                    const uint32_t sb = sbase + OFF_B + stage * TILE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        // 16 bf16 = 32 bytes further along K inside the 128-byte swizzled row
                        mma_bf16(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), kIdesc, (kb | kk) ? 1u : 0u);
                    }
                    mma_commit(empty_bar(stage));   // stage free once these MMAs have read it
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(accf_bar(ab));           // accumulator ready for the epilogue
            }
            // all MMAs issued by this thread complete before TMEM is released
            mma_commit(down_bar);
            const unsigned long long t0 = globaltimer();
            while (!mbar_try_wait(down_bar, 0) && globaltimer() - t0 < kWaitLimitNs) {
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lanes 32 * (warp % 4) ----------------
        const int q = warp & 3;
        const int et = threadIdx.x - 64;          // 0..127 within the epilogue group
        int lt = 0;
        int chunk_ctr = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < a.tiles; t += G, ++lt) {
            int bi, bj;
            tri_coords(t, a.T, &bi, &bj);
            const int ab = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            // column norms of this tile's J block
            if (a.kp.kind == POPCORN_GAUSSIAN) {
                const int j = bj * BN + et;
                epi_bar();   // previous tile finished reading rj_s
                rj_s[et] = j < a.n ? a.norms[j] : 0.f;
            }
            if (!mbar_wait(accf_bar(ab), use & 1u, abort_flag, a.err)) ok = false;
            // all epilogue threads agree (one barrier, one AND) before touching TMEM or staging
            if (!named_bar_all(1, 128, ok && !*abort_flag)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int row_local = 32 * q + lane;
            const int row = bi * BM + row_local;
            const float ri = (a.kp.kind == POPCORN_GAUSSIAN && row < a.n) ? a.norms[row] : 0.f;
            const bool diag = (bi == bj);
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * BN + 32 * c), v);
                if (c == BN / 32 - 1) {
                    // accumulator fully read: hand it back to the MMA warp
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce_bar(ab));
                }
#pragma unroll
                for (int x = 0; x < 32; ++x) {
                    v[x] = kappa(v[x], ri, rj_s[32 * c + x], a.kp);
                    if (diag && 32 * c + x == row_local) {
                        if (a.kp.kind == POPCORN_GAUSSIAN) v[x] = 1.f;
                        if (row < a.n) a.kdiag[row] = v[x];
                    }
                }
                const int sbuf = chunk_ctr & 1;
                ++chunk_ctr;
                // the store that used this staging buffer two chunks ago has read it
                if (et == 0) bulk_wait_read<1>();
                epi_bar();
                float* sd = reinterpret_cast<float*>(smem + OFF_SD + sbuf * STG_BYTES);
                float* st = reinterpret_cast<float*>(smem + OFF_ST + sbuf * STG_BYTES);
                // direct chunk: row row_local, 8 x 16-byte pieces, piece j at j ^ (row % 8)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float4 w = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    *reinterpret_cast<float4*>(sd + row_local * 32 + ((j ^ (row_local & 7)) * 4)) = w;
                }
                if (!diag) {
#pragma unroll
                    for (int x = 0; x < 32; ++x) st[x * 128 + row_local] = v[x];
                }
                fence_proxy_async();
                epi_bar();
                if (et == 0) {
                    tma_store_2d(&map_kd, bj * BN + 32 * c, bi * BM, smem_u32(sd));
                    if (!diag) tma_store_2d(&map_kt, bi * BM, bj * BN + 32 * c, smem_u32(st));
                    bulk_commit();
                }
            }
        }
        if (et == 0) bulk_wait_all();
        (void)ok;
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

// FP32 rows -> BF16 operand rows (and hi/lo split), zero padding, FP32 norms of
// the represented rows.  One warp per row.
__global__ void __launch_bounds__(256) prep_operands_kernel(const float* __restrict__ P, int n, int d, int64_t ldp,
                                                            int dpad, int x3, __nv_bfloat16* __restrict__ A,
                                                            __nv_bfloat16* __restrict__ B, float* __restrict__ norms) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int64_t lda = (int64_t)(x3 ? 3 : 1) * dpad;
    __nv_bfloat16* ar = A + (int64_t)warp * lda;
    __nv_bfloat16* br = B ? B + (int64_t)warp * lda : nullptr;
    float nrm = 0.f;
    for (int l = lane; l < dpad; l += 32) {
        const float p = l < d ? P[(int64_t)warp * ldp + l] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(p);
        const float hf = __bfloat162float(hi);
        if (!x3) {
            ar[l] = hi;
            nrm = fmaf(hf, hf, nrm);
        } else {
            const __nv_bfloat16 lo = __float2bfloat16_rn(p - hf);
            const float rep = hf + __bfloat162float(lo);
            ar[l] = hi;
            ar[dpad + l] = hi;
            ar[2 * dpad + l] = lo;
            br[l] = hi;
            br[dpad + l] = lo;
            br[2 * dpad + l] = hi;
            nrm = fmaf(rep, rep, nrm);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) norms[warp] = nrm;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

bool make_tensor_map_2d(CUtensorMap* m, CUtensorMapDataType dt, void* base, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


size_t kbuild_tc_workspace(int n, int d, int precision) {
    const size_t dpad = ((size_t)d + BK - 1) / BK * BK;
    const size_t lda = (precision == POPCORN_BF16X3 ? 3 : 1) * dpad;
    const size_t ops = (precision == POPCORN_BF16X3 ? 2 : 1) * (size_t)n * lda * 2;
    return ((ops + 255) & ~(size_t)255) + (size_t)n * 4 + 256;
}

cudaError_t configure_kbuild_tc() {
    encode_fn();
    return cudaFuncSetAttribute(kbuild_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t launch_kbuild_tc(const float* P, int n, int d, int64_t ldp, KernParams kp, int precision, float* K,
                             int64_t ldk, float* kdiag, void* workspace, int* err, int num_sms, cudaStream_t s,
                             int* launches) {
    const int dpad = (d + BK - 1) / BK * BK;
    const int x3 = precision == POPCORN_BF16X3 ? 1 : 0;
    const int64_t lda = (int64_t)(x3 ? 3 : 1) * dpad;
    __nv_bfloat16* A = static_cast<__nv_bfloat16*>(workspace);
    const size_t abytes = (size_t)n * lda * 2;
    __nv_bfloat16* B = x3 ? A + (size_t)n * lda : nullptr;
    const size_t ops = (x3 ? 2 : 1) * abytes;
    float* norms = reinterpret_cast<float*>(static_cast<char*>(workspace) + ((ops + 255) & ~(size_t)255));

    prep_operands_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(P, n, d, ldp, dpad, x3, A, B, norms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;

    CUtensorMap ma, mb, mkd, mkt;
    if (!make_tensor_map_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, A, (uint64_t)lda, (uint64_t)n, (uint64_t)lda * 2, BK, BM,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tensor_map_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, x3 ? B : A, (uint64_t)lda, (uint64_t)n, (uint64_t)lda * 2,
                  BK, BN, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tensor_map_2d(&mkd, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, K, (uint64_t)n, (uint64_t)n, (uint64_t)ldk * 4, 32, BM,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tensor_map_2d(&mkt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, K, (uint64_t)n, (uint64_t)n, (uint64_t)ldk * 4, BM, 32,
                  CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorInvalidValue;

    TcArgs a;
    a.n = n;
    a.T = (n + BM - 1) / BM;
    a.nkb = (int)(lda / BK);
    a.tiles = (long long)a.T * (a.T + 1) / 2;
    a.kp = kp;
    a.norms = norms;
    a.kdiag = kdiag;
    a.err = err;
    const int grid = (int)(a.tiles < num_sms ? a.tiles : num_sms);
    kbuild_tc_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(ma, mb, mkd, mkt, a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace popcorn
