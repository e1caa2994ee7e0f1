// Tensor-core (tcgen05) build of the kernel matrix K = kappa(P P^T).
//
// Sec. 3.2 forms B = P P^T with GEMM or SYRK and then applies the kernel
// function elementwise (Gaussian through Eq. 12 from B and the row norms).
// Here one persistent kernel walks the tiles (p, j) of the upper triangle,
// where a tile is a pair of 128-row blocks (2p, 2p + 1) against one
// 128-column block j >= 2p:
//
//   warp 0  (one lane)  TMA loads, per 64-deep k-block, of the 256 rows of the
//                       row pair and the 128 rows of the column block (128-byte
//                       swizzle) into a ring of stages;
//   warp 1  (one lane)  tcgen05.mma kind::f16 (BF16 x BF16 -> FP32, M = N = 128)
//                       into the two 128-column TMEM accumulators of the tile
//                       (double-buffered: 512 columns);
//   warps 2-5           epilogue: tcgen05.ld the accumulators, apply kappa with
//                       FP32 row norms, stage each 128 x 32 chunk and its
//                       transpose in shared memory and TMA-store both into K --
//                       or, for the block-packed upper triangle the symmetric
//                       pass reads, bulk-copy the swizzled chunk alone to its
//                       place in the packed tile (each value stored once).
//
// Why row pairs: an SM takes in about 36 bytes per clock from L2 whichever path
// it uses (TMA, bulk copy, cp.async or vector loads), and a 128 x 128 tile moves
// 32 KB per k-block for 4 MMAs -- three times what that allows at the MMA rate.
// Sharing each column block between two row blocks cuts the bytes per MMA by a
// quarter; block (2p + 1, 2p), below the diagonal, is computed and not stored.
//
// Precision modes (operand matrix W, one row per point):
//   BF16    W = bf16(P);  norms of the rounded rows, so the Gaussian distance
//           r_i + r_j - 2 B_ij is the distance of the rounded points.
//   BF16X3  W = [hi | lo] with hi = bf16(p), lo = bf16(p - hi); each stage
//           holds the hi and lo parts of both operands once and the MMAs form
//           hi.hi + hi.lo + lo.hi (~16 significant bits of the cross term that
//           the Gaussian's cancellation needs) -- 2 d loaded instead of the 3 d
//           a [hi|hi|lo] x [hi|lo|hi] GEMM would stream.
//
// Every mbarrier wait is bounded (about 2 s by %globaltimer).  A wait that
// runs out sets *err, raises a shared abort flag that ends every role's loop,
// waits (bounded again) for the CTA's own TMA copies and MMAs in flight,
// frees TMEM and returns; the host reports POPCORN_ERR_TIMEOUT.
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "popcorn_internal.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

using namespace tc;

__device__ __forceinline__ void epi_bar() { named_bar<128>(1); }   // the 4 epilogue warps
constexpr uint32_t kIdesc = idesc_bf16(128, 128);

constexpr int BM = 128, BK = 64;             // block rows / columns, bf16 depth per k-block
constexpr int ROWS_BYTES = 2 * BM * BK * 2;  // 32 KB: 256 rows of one part (hi or lo)
constexpr int COLS_BYTES = BM * BK * 2;      // 16 KB: 128 rows of one part
constexpr int STG_BYTES = 128 * 32 * 4;      // one 128 x 32 FP32 staging chunk
constexpr int NTHREADS = 192;                // 6 warps
constexpr int MAX_STAGES = 4;
constexpr int RING_BYTES = 192 * 1024;       // operand ring
constexpr uint32_t kTmemCols = 512;          // 2 buffers x 2 row blocks x 128 columns

struct TcArgs {
    int n, T, T2, nkb;        // rows, 128-blocks, row pairs, 64-deep k-blocks per part
    int dpad;                 // elements per part (W row = [hi | lo] for BF16X3)
    int x3;                   // 1: BF16X3 (three products per k-step)
    int stages, stage_bytes;  // ring: 48 KB (BF16) or 96 KB (BF16X3) stages
    int nstg;                 // staging buffers per kind (2, or 1 when the ring needs the room)
    int off_sd, off_st, off_rj, off_bar, off_misc;
    long long tiles;          // sum_p (T - 2 p)
    float* Kp;                // block-packed K (tile (I, J), I <= J, at its row-by-row triangle index
                              // times 16384 floats, four 128 x 32 boxes; FP16 / BF16: times 32 KB,
                              // two 128 x 64 boxes), or null
    int full;                 // 1: every tile of the square (the GEMM form), each stored once; 0: the
                              // tiles on and above the diagonal (the SYRK form), stored with their
                              // transposes unless K is packed
    int sw4;                  // packed layout kPackedSw4 (element c of row r at c ^ (r mod 32)): the
                              // kernel's SW4 instance; else kPackedSw16 (the 128-byte swizzle)
    KernParams kp;
    const float* norms;       // row norms of the represented rows (Gaussian)
    float* kdiag;
    int* err;
};

// tile t -> (row pair p, column block j): row pair p holds tiles j = 2p .. T-1 and
// starts at off(p) = p T - p (p - 1); a binary search over p (no floating point).
// The full schedule (every column block, the GEMM form) has row pair p at p T.
__device__ __forceinline__ void pair_coords(long long t, int T, int T2, int full, int* p, int* j) {
    if (full) {
        *p = (int)(t / T);
        *j = (int)(t % T);
        return;
    }
    int lo = 0, hi = T2 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long off = (long long)mid * T - (long long)mid * (mid - 1);
        if (off <= t) lo = mid;
        else hi = mid - 1;
    }
    *p = lo;
    *j = 2 * lo + (int)(t - ((long long)lo * T - (long long)lo * (lo - 1)));
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

// Output of the epilogue, one instance each, since a runtime choice between staging stores
// slowed the epilogue about 2.8x: kOutSw16 (full square through tensor maps, or the packed
// triangle in the 128-byte swizzle), kOutSw4 (packed XOR-32, kPackedSw4), kOutHalf16 /
// kOutHalfB16 (packed FP16 / BF16 triangle, kPackedSw128H: each 64-column box is staged
// whole -- two 32-column chunks -- and stored with one bulk copy; entries past n are zeros).
constexpr int kOutSw16 = 0, kOutSw4 = 1, kOutHalf16 = 2, kOutHalfB16 = 3;

__device__ __forceinline__ uint32_t pack_half2(float x, float y, bool bf16) {
    if (bf16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    const __half2 h = __floats2half2_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float round_half(float x, bool bf16) {
    return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : __half2float(__float2half_rn(x));
}

template <int OUT>
__global__ void __launch_bounds__(NTHREADS, 1)
    kbuild_tc_kernel(const __grid_constant__ CUtensorMap map_r, const __grid_constant__ CUtensorMap map_c,
                     const __grid_constant__ CUtensorMap map_kd, const __grid_constant__ CUtensorMap map_kt,
                     TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + a.off_bar;
    const int S = a.stages;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (MAX_STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * MAX_STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * MAX_STAGES + 2 + b); };
    const uint32_t down_bar = bar0 + 8u * (2 * MAX_STAGES + 4);
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(smem + a.off_misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_misc + 4);
    float* rj_s = reinterpret_cast<float*>(smem + a.off_rj);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
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
    if (warp == 1) {   // whole warp: all 512 TMEM columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // stage layout: rows-hi (32 KB) | cols-hi (16 KB) [| rows-lo (32 KB) | cols-lo (16 KB)]
    constexpr uint32_t kRowsHi = 0, kColsHi = ROWS_BYTES, kRowsLo = ROWS_BYTES + COLS_BYTES,
                       kColsLo = 2 * ROWS_BYTES + COLS_BYTES;
    const long long G = gridDim.x;
    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_parity[MAX_STAGES];
            bool issued[MAX_STAGES];
            for (int s = 0; s < MAX_STAGES; ++s) issued[s] = false;
            bool ok = true;
            for (long long t = blockIdx.x; t < a.tiles && ok; t += G) {
                int p, j;
                pair_coords(t, a.T, a.T2, a.full, &p, &j);
                for (int kb = 0; kb < a.nkb; ++kb) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + (uint32_t)(stage * a.stage_bytes);
                    mbar_arrive_expect_tx(full_bar(stage), (uint32_t)a.stage_bytes);
                    tma_load_2d(st + kRowsHi, &map_r, kb * BK, p * 2 * BM, full_bar(stage));
                    tma_load_2d(st + kColsHi, &map_c, kb * BK, j * BM, full_bar(stage));
                    if (a.x3) {
                        tma_load_2d(st + kRowsLo, &map_r, a.dpad + kb * BK, p * 2 * BM, full_bar(stage));
                        tma_load_2d(st + kColsLo, &map_c, a.dpad + kb * BK, j * BM, full_bar(stage));
                    }
                    issued[stage] = true;
                    issued_parity[stage] = phase;
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // aborted: let this CTA's own copies land before shared memory goes away
                for (int s = 0; s < S; ++s)
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
                for (int kb = 0; kb < a.nkb; ++kb) {
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + (uint32_t)(stage * a.stage_bytes);
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t d_tmem = tmem + (uint32_t)(ab * 2 * BM + h * BM);
                        const uint32_t rh = st + kRowsHi + h * (BM * BK * 2);   // row block h of the pair
                        const uint32_t rl = st + kRowsLo + h * (BM * BK * 2);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            // 16 bf16 = 32 bytes further along K inside the 128-byte swizzled row
                            mma_bf16(d_tmem, sw128_desc(rh + kk * 32), sw128_desc(st + kColsHi + kk * 32), kIdesc,
                                     (kb | kk) ? 1u : 0u);
                            if (a.x3) {
                                mma_bf16(d_tmem, sw128_desc(rh + kk * 32), sw128_desc(st + kColsLo + kk * 32), kIdesc, 1u);
                                mma_bf16(d_tmem, sw128_desc(rl + kk * 32), sw128_desc(st + kColsHi + kk * 32), kIdesc, 1u);
                            }
                        }
                    }
                    mma_commit(empty_bar(stage));   // stage free once these MMAs have read it
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(accf_bar(ab));           // both accumulators ready for the epilogue
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
            int p, j;
            pair_coords(t, a.T, a.T2, a.full, &p, &j);
            const int ab = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            // column norms of this tile's column block j
            if (a.kp.kind == POPCORN_GAUSSIAN) {
                const int col = j * BM + et;
                epi_bar();   // previous tile finished reading rj_s
                rj_s[et] = col < a.n ? a.norms[col] : 0.f;
            }
            if (!mbar_wait(accf_bar(ab), use & 1u, abort_flag, a.err)) ok = false;
            // all epilogue threads agree (one barrier, one AND) before touching TMEM or staging
            if (!named_bar_all(1, 128, ok && !*abort_flag)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int row_local = 32 * q + lane;
            for (int h = 0; h < 2; ++h) {
                const int rb = 2 * p + h;             // 128-row block of K
                const int row = rb * BM + row_local;
                const float ri = (a.kp.kind == POPCORN_GAUSSIAN && row < a.n) ? a.norms[row] : 0.f;
                // blocks past the matrix and block (2p + 1, 2p) below the diagonal are not stored
                const bool store = rb < a.T && (a.full || rb <= j);
                const bool diag = (rb == j);
                for (int c = 0; c < BM / 32; ++c) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * 2 * BM + h * BM + 32 * c), v);
                    if (h == 1 && c == BM / 32 - 1) {
                        // both accumulators fully read: hand the buffer back to the MMA warp
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acce_bar(ab));
                    }
                    if (!store) continue;
                    constexpr bool HALF = OUT == kOutHalf16 || OUT == kOutHalfB16;
                    constexpr bool HB16 = OUT == kOutHalfB16;
#pragma unroll
                    for (int x = 0; x < 32; ++x) {
                        v[x] = kappa(v[x], ri, rj_s[32 * c + x], a.kp);
                        if (diag && 32 * c + x == row_local) {
                            if (a.kp.kind == POPCORN_GAUSSIAN) v[x] = 1.f;
                            if (row < a.n) a.kdiag[row] = HALF ? round_half(v[x], HB16) : v[x];
                        }
                    }
                    if constexpr (HALF) {
                        // box c / 2 of the half tile: staged over two chunks, stored after the second
                        const int sbuf = a.nstg == 2 ? ((chunk_ctr >> 1) & 1) : 0;
                        ++chunk_ctr;
                        if ((c & 1) == 0) {
                            // the store that last used this staging buffer has read it
                            if (et == 0) {
                                if (a.nstg == 2) bulk_wait_read<1>();
                                else bulk_wait_read<0>();
                            }
                            epi_bar();
                        }
                        unsigned char* sb = smem + a.off_sd + sbuf * STG_BYTES;
                        const int col0 = j * BM + 32 * c;
                        const bool rv = row < a.n;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            // logical 16-byte chunk 4 (c mod 2) + i of the row, at its swizzled place
                            uint32_t w[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int x = 8 * i + 2 * e;
                                const float x0 = (rv && col0 + x < a.n) ? v[x] : 0.f;
                                const float x1 = (rv && col0 + x + 1 < a.n) ? v[x + 1] : 0.f;
                                w[e] = pack_half2(x0, x1, HB16);
                            }
                            const int pc = (4 * (c & 1) + i) ^ (row_local & 7);
                            *reinterpret_cast<uint4*>(sb + row_local * 128 + 16 * pc) = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                        if (c & 1) {
                            fence_proxy_async();
                            epi_bar();
                            if (et == 0) {
                                const long long tri = (long long)rb * a.T - (long long)rb * (rb - 1) / 2 + (j - rb);
                                bulk_store_1d(reinterpret_cast<unsigned char*>(a.Kp) + tri * 32768 + (c >> 1) * 16384,
                                              smem_u32(sb), (uint32_t)STG_BYTES);
                                bulk_commit();
                            }
                        }
                        continue;
                    }
                    const int sbuf = a.nstg == 2 ? (chunk_ctr & 1) : 0;
                    ++chunk_ctr;
                    // the store that last used this staging buffer has read it
                    if (et == 0) {
                        if (a.nstg == 2) bulk_wait_read<1>();
                        else bulk_wait_read<0>();
                    }
                    epi_bar();
                    float* sd = reinterpret_cast<float*>(smem + a.off_sd + sbuf * STG_BYTES);
                    float* sx = reinterpret_cast<float*>(smem + a.off_st + sbuf * STG_BYTES);
                    if constexpr (OUT == kOutSw4) {
                        // packed XOR-32 layout: element x of row row_local at x ^ (row_local mod 32)
                        // (the 32 lanes hold 32 consecutive rows: 32 different banks per store)
#pragma unroll
                        for (int x = 0; x < 32; ++x) sd[row_local * 32 + (x ^ lane)] = v[x];
                    } else {
                        // direct chunk: row row_local, 8 x 16-byte pieces, piece i at i ^ (row % 8)
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float4 w = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                            *reinterpret_cast<float4*>(sd + row_local * 32 + ((i ^ (row_local & 7)) * 4)) = w;
                        }
                    }
                    const bool transpose = !diag && !a.Kp && !a.full;
                    if (transpose) {
#pragma unroll
                        for (int x = 0; x < 32; ++x) sx[x * 128 + row_local] = v[x];
                    }
                    fence_proxy_async();
                    epi_bar();
                    if (et == 0) {
                        if (a.Kp) {
                            // the staged chunk is box c of packed tile (rb, j), byte for byte
                            const long long tri = (long long)rb * a.T - (long long)rb * (rb - 1) / 2 + (j - rb);
                            bulk_store_1d(a.Kp + tri * (BM * BM) + c * (BM * 32), smem_u32(sd), (uint32_t)STG_BYTES);
                        } else {
                            tma_store_2d(&map_kd, j * BM + 32 * c, rb * BM, smem_u32(sd));
                            if (transpose) tma_store_2d(&map_kt, rb * BM, j * BM + 32 * c, smem_u32(sx));
                        }
                        bulk_commit();
                    }
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// FP32 rows -> BF16 operand rows W (BF16X3: [hi | lo]), zero padding, FP32 norms
// of the represented rows.  One warp per row.
__global__ void __launch_bounds__(256) prep_operands_kernel(const float* __restrict__ P, int n, int d, int64_t ldp,
                                                            int dpad, int x3, __nv_bfloat16* __restrict__ W,
                                                            float* __restrict__ norms) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int64_t ldw = (int64_t)(x3 ? 2 : 1) * dpad;
    __nv_bfloat16* wr = W + (int64_t)warp * ldw;
    float nrm = 0.f;
    for (int l = lane; l < dpad; l += 32) {
        const float p = l < d ? P[(int64_t)warp * ldp + l] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(p);
        const float hf = __bfloat162float(hi);
        wr[l] = hi;
        if (!x3) {
            nrm = fmaf(hf, hf, nrm);
        } else {
            const __nv_bfloat16 lo = __float2bfloat16_rn(p - hf);
            const float rep = hf + __bfloat162float(lo);
            wr[dpad + l] = lo;
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
    const size_t ldw = (precision == POPCORN_BF16X3 ? 2 : 1) * dpad;
    const size_t ops = (size_t)n * ldw * 2;
    return ((ops + 255) & ~(size_t)255) + (size_t)n * 4 + 256;
}

// shared memory the kernel is configured for: the largest layout below (BF16X3:
// a full 192 KB ring and one staging buffer of each kind), the column norms,
// barriers and slack for the 1024-byte alignment
constexpr int kSmemBytes = RING_BYTES + 2 * STG_BYTES + BM * 4 + 16 * 8 + 16 + 1024;

cudaError_t configure_kbuild_tc() {
    encode_fn();
    decltype(&kbuild_tc_kernel<kOutSw16>) fs[4] = {kbuild_tc_kernel<kOutSw16>, kbuild_tc_kernel<kOutSw4>,
                                                   kbuild_tc_kernel<kOutHalf16>, kbuild_tc_kernel<kOutHalfB16>};
    for (auto f : fs) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_kbuild_tc(const float* P, int n, int d, int64_t ldp, KernParams kp, int precision, float* K,
                             int64_t ldk, float* kdiag, void* workspace, int* err, int num_sms, cudaStream_t s,
                             int* launches, int packed, int full, int k_storage) {
    // packed kPackedSw128H: K is the FP16 / BF16 packed triangle (k_storage)
    const int half = packed == kPackedSw128H ? (k_storage == POPCORN_K_BF16 ? 2 : 1) : 0;
    if (packed == kPackedSw128H && k_storage != POPCORN_K_FP16 && k_storage != POPCORN_K_BF16)
        return cudaErrorInvalidValue;
    const int dpad = (d + BK - 1) / BK * BK;
    const int x3 = precision == POPCORN_BF16X3 ? 1 : 0;
    const int64_t ldw = (int64_t)(x3 ? 2 : 1) * dpad;
    __nv_bfloat16* W = static_cast<__nv_bfloat16*>(workspace);
    const size_t ops = (size_t)n * ldw * 2;
    float* norms = reinterpret_cast<float*>(static_cast<char*>(workspace) + ((ops + 255) & ~(size_t)255));

    prep_operands_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(P, n, d, ldp, dpad, x3, W, norms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;

    CUtensorMap mr, mc, mkd, mkt;
    memset(&mkd, 0, sizeof mkd);
    memset(&mkt, 0, sizeof mkt);
    if (!make_tensor_map_2d(&mr, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, W, (uint64_t)ldw, (uint64_t)n, (uint64_t)ldw * 2, BK,
                            2 * BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tensor_map_2d(&mc, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, W, (uint64_t)ldw, (uint64_t)n, (uint64_t)ldw * 2, BK,
                            BM, CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorInvalidValue;
    // the full-square stores go through tensor maps; the packed stores are plain bulk copies
    if (!packed && (!make_tensor_map_2d(&mkd, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, K, (uint64_t)n, (uint64_t)n,
                                        (uint64_t)ldk * 4, 32, BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
                    !make_tensor_map_2d(&mkt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, K, (uint64_t)n, (uint64_t)n,
                                        (uint64_t)ldk * 4, BM, 32, CU_TENSOR_MAP_SWIZZLE_NONE)))
        return cudaErrorInvalidValue;

    TcArgs a;
    a.n = n;
    a.T = (n + BM - 1) / BM;
    a.T2 = (a.T + 1) / 2;
    a.dpad = dpad;
    a.nkb = dpad / BK;
    a.x3 = x3;
    // BF16: 3 stages of 48 KB; BF16X3: 2 stages of 96 KB (hi and lo of both operands)
    a.stage_bytes = x3 ? 2 * (ROWS_BYTES + COLS_BYTES) : ROWS_BYTES + COLS_BYTES;
    a.stages = x3 ? 2 : 3;
    // staging: two buffers of each kind when the ring leaves room, else one
    const int ring = a.stages * a.stage_bytes;
    a.nstg = ring + 4 * STG_BYTES <= RING_BYTES + 2 * STG_BYTES ? 2 : 1;
    a.off_sd = ring;
    a.off_st = a.off_sd + a.nstg * STG_BYTES;
    a.off_rj = a.off_st + a.nstg * STG_BYTES;
    a.off_bar = a.off_rj + BM * 4;
    a.off_misc = a.off_bar + 16 * 8;
    a.full = full && !packed ? 1 : 0;
    a.tiles = a.full ? (long long)a.T2 * a.T : (long long)a.T2 * a.T - (long long)a.T2 * (a.T2 - 1);
    a.Kp = packed ? K : nullptr;
    a.sw4 = packed == kPackedSw4 ? 1 : 0;
    a.kp = kp;
    a.norms = norms;
    a.kdiag = kdiag;
    a.err = err;
    const int smem = a.off_misc + 16 + 1024;
    if (smem > kSmemBytes) return cudaErrorInvalidConfiguration;
    const int grid = (int)(a.tiles < num_sms ? a.tiles : num_sms);
    if (half == 1)
        kbuild_tc_kernel<kOutHalf16><<<grid, NTHREADS, smem, s>>>(mr, mc, mkd, mkt, a);
    else if (half == 2)
        kbuild_tc_kernel<kOutHalfB16><<<grid, NTHREADS, smem, s>>>(mr, mc, mkd, mkt, a);
    else if (a.sw4)
        kbuild_tc_kernel<kOutSw4><<<grid, NTHREADS, smem, s>>>(mr, mc, mkd, mkt, a);
    else
        kbuild_tc_kernel<kOutSw16><<<grid, NTHREADS, smem, s>>>(mr, mc, mkd, mkt, a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace popcorn
