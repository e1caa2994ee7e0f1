// Symmetric K stream on the tensor cores, for a K stored in FP16 or BF16.
//
// The segment sums of a pass are the paper's SpMM E = K V^T (Alg. 2 line 7) with V the
// one-hot label matrix of Eq. 8 (its 1 / |L_c| scale is applied later, by the fold): for
// every row i and cluster c, S_ic = sum_{j in L_c} K_ij.  The symmetric pass (reduce_sym.cu)
// splits S by 128-blocks and reads only the blocks (I, J), I <= J: the row sums of block
// (I, J) are its part for the rows of I, its column sums the part for the rows of J.  Per
// block both are small products:
//   row sums     R = K_IJ V_J^T      (128 x 128) x (128 x N),
//   column sums  C = K_IJ^T V_I^T    (128 x 128) x (128 x N),
// with V_X the one-hot rows of block X's points (N = 16 or 32 >= k columns).  A half entry
// times 1 or 0 is exact, and the tensor cores add in FP32, so on a K rounded to FP16 /
// BF16 the products are the cluster sums the CUDA-core forms compute, up to the order of
// the FP32 additions.
//
// Why tensor cores for a stream that HBM bounds: a half tile is 32 KB, half the bytes of
// an FP32 tile, but a CUDA-core walk spends the same instructions per element (address,
// load, convert, add) as on FP32, so it falls to about half of HBM speed.  Here one
// thread issues 16 MMAs a block; the SMs only move bytes.
//
// Layout.  A tile of the packed triangle (kPackedSw128H, kpack.cu) is two boxes of
// 128 rows x 64 columns in the 128-byte swizzle of the MMA shared-memory operands.  The
// same bytes are the A operand of both products: K-major for R (M = rows r, reduction
// over columns C: 16 columns = 32 bytes further along a row, the second box 16 KB on)
// and MN-major for C (M = columns C, the two boxes 16 KB apart; reduction over rows r:
// 16 rows = 2 KB further on).  The one-hot operand of block X (sym_onehot_kernel, once a
// pass, [T][N x 128 halves]) is K-major: N rows c of 128 point entries in the same
// swizzle.
//
// The kernel: persistent, one CTA an SM, super-tiles of a x a blocks round-robin (the
// slot scheme of the sorted form: row sums of super-tile (Is, Js) to slot Js, column sums
// to slot Is, or to slot Ts from a super-tile on the diagonal).  Warp 0: one thread
// bulk-copies each block with V_J and V_I into a ring of stages.  Warp 1: one thread
// issues the MMAs, R into the TMEM accumulator of the block's row, C (off the diagonal)
// into that of its column; the accumulators (2a of N columns) stay in TMEM over the
// super-tile, double-buffered so that the next super-tile's MMAs overlap this one's
// stores.  Warps 2-5: read the accumulators (one TMEM lane quadrant each: a lane is a
// row) and store each row's k sums to its slot.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "popcorn_internal.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

constexpr int kB = 128;                  // block edge
constexpr int kTileBytes = 32768;        // a 128 x 128 tile of half entries
constexpr int kMmaThreads = 192;         // producer, MMA issuer, 4 epilogue warps
constexpr int kOneHotThreads = 128;
constexpr int kMaxStages = 6;

__host__ __device__ constexpr int onehot_bytes(int N) { return N * kB * 2; }   // N rows x 128 halves

struct MmaUnit {
    int Is, Js, I0, J0;
};
__device__ __forceinline__ MmaUnit mma_unit(long long u, int a, int Ts) {
    MmaUnit w;
    tri_coords(u, Ts, &w.Is, &w.Js);
    w.I0 = w.Is * a;
    w.J0 = w.Js * a;
    return w;
}

// The one-hot operand of every block: V_X[c][i] = 1 if point 128 X + i has label c (0 past
// n), stored K-major in the 128-byte swizzle: 16-byte chunk q = (box, c, ch) at byte 16 q
// holds the points 64 box + 8 (ch ^ (c mod 8)) + 0..7.
template <typename TH>
__global__ void __launch_bounds__(kOneHotThreads) sym_onehot_kernel(const uint8_t* __restrict__ lab8, int n, int k,
                                                                    int N, uint4* __restrict__ V,
                                                                    const LoopState* st, int eval_only) {
    grid_dependency_wait();   // the labels come from the previous pass
    if (pass_skip(st, eval_only)) return;
    __shared__ uint8_t lab[kB];
    const int X = blockIdx.x, t = threadIdx.x;
    const int i = X * kB + t;
    lab[t] = (i < n && (int)lab8[i] < k) ? lab8[i] : (uint8_t)0xFF;
    __syncthreads();
    const uint32_t one = std::is_same<TH, __half>::value ? 0x3C00u : 0x3F80u;   // 1.0
    uint4* dst = V + (size_t)X * (onehot_bytes(N) / 16);
    for (int q = t; q < N * 16; q += kOneHotThreads) {
        const int box = q / (N * 8), c = (q >> 3) % N, ch = q & 7;
        const int i0 = 64 * box + 8 * (ch ^ (c & 7));
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            w[e] = (lab[i0 + 2 * e] == c ? one : 0u) | ((lab[i0 + 2 * e + 1] == c ? one : 0u) << 16);
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Instruction descriptor of kind::f16 with FP32 accumulation: A and B both FP16 (format 0)
// or both BF16 (format 1); A MN-major when a_mn (bit 15), B K-major; N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_half(bool bf16, bool a_mn, int M, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((a_mn ? 1u : 0u) << 15) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory descriptor of an MN-major operand in the 128-byte swizzle: atoms of 64
// elements along M (one 128-byte row) by 8 along the reduction; lbo = bytes between atoms
// along M, sbo = bytes between groups of 8 reduction rows; version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// N consecutive TMEM columns of this thread's lane (32x32b shape), as floats.
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[N]) {
    uint32_t r[N];
    if constexpr (N == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(taddr));
    } else {
        static_assert(N == 32, "16 or 32 columns");
        tc::tmem_ld32_nowait(taddr, r);
    }
    tc::tmem_ld_wait();
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = __uint_as_float(r[x]);
}

struct MmaArgs {
    const unsigned char* Kh;   // block-packed K, kPackedSw128H
    const unsigned char* V;    // [T][onehot_bytes(N)] one-hot operands of this pass
    int n, k, N, T, a, Ts;
    long long units;
    int stages, stage_bytes, vbytes, off_bars;
    uint32_t tmem_cols;
    float* Spart;              // [Ts + 1][k][n]
    const LoopState* st;
    int* err;
    int eval_only;
    // Test hook for the error path (0 in every ordinary launch): CTA 0 never issues the
    // copies of its block number stall_block - 1, so the waits for it run out after
    // wait_ns and the launch reports a timed-out wait.
    int stall_block;
    unsigned long long wait_ns;
    const int* order;          // super-tiles in processing order (larger first), or null
};

template <bool BF16, int N>
__global__ void __launch_bounds__(kMmaThreads, 1) reduce_sym_mma_kernel(MmaArgs a) {
    grid_dependency_wait();   // the one-hot operands and the loop state come from before this pass
    if (pass_skip(a.st, a.eval_only)) return;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment: the swizzle pattern follows address bits 4-9
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = tc::smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = a.a, S = a.stages, T = a.T;
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
    const long long G = gridDim.x;
    // blocks of a super-tile, row by row: (I0 + m, J0 + i) on or above the diagonal
    auto block_of = [&](const MmaUnit& w, int m, int i, int* I, int* J) {
        *I = w.I0 + m;
        *J = w.J0 + i;
        return *I < T && *J < T && *J >= *I;
    };
    // TMEM column of accumulator x of buffer b: x < a for block rows, a + y for block columns
    auto acc_col = [&](int b, int x) { return (uint32_t)((b * 2 * A + x) * N); };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: each block with V_J (row sums) and V_I (column sums)
            const uint64_t stream_once = tc::l2_evict_first();   // K is read once per pass
            const long long skip = blockIdx.x == 0 ? (long long)a.stall_block - 1 : -1;
            long long t = 0;
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (long long u = blockIdx.x; u < a.units && ok; u += G) {
                const MmaUnit w = mma_unit(a.order ? a.order[u] : u, A, a.Ts);
                for (int m = 0; m < A && ok; ++m)
                    for (int i = 0; i < A; ++i) {
                        int I, J;
                        if (!block_of(w, m, i, &I, &J)) continue;
                        if (t >= S && !tc::mbar_wait_for(empty_bar(s), ph ^ 1u, abort_flag, a.err, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        if (t != skip) {   // the test hook: this block never arrives
                            tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)(kTileBytes + 2 * a.vbytes));
                            const uint32_t dst = sbase + (uint32_t)s * (uint32_t)a.stage_bytes;
                            const long long tri = (long long)I * T - (long long)I * (I - 1) / 2 + (J - I);
                            tc::bulk_load_1d_hint(dst, a.Kh + tri * kTileBytes, (uint32_t)kTileBytes, full_bar(s),
                                                  stream_once);
                            tc::bulk_load_1d(dst + kTileBytes, a.V + (size_t)J * a.vbytes, (uint32_t)a.vbytes,
                                             full_bar(s));
                            tc::bulk_load_1d(dst + kTileBytes + a.vbytes, a.V + (size_t)I * a.vbytes,
                                             (uint32_t)a.vbytes, full_bar(s));
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
            // ---------------- MMA issuer ----------------
            constexpr uint32_t kIdescRow = idesc_half(BF16, false, kB, N);
            constexpr uint32_t kIdescCol = idesc_half(BF16, true, kB, N);
            int s = 0;
            uint32_t ph = 0;
            int lt = 0;
            bool ok = true;
            for (long long u = blockIdx.x; u < a.units && ok; u += G, ++lt) {
                const int buf = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!tc::mbar_wait_for(acce_bar(buf), (use & 1u) ^ 1u, abort_flag, a.err, a.wait_ns)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const MmaUnit w = mma_unit(a.order ? a.order[u] : u, A, a.Ts);
                uint32_t touched = 0;   // accumulators written in this super-tile
                for (int m = 0; m < A && ok; ++m)
                    for (int i = 0; i < A; ++i) {
                        int I, J;
                        if (!block_of(w, m, i, &I, &J)) continue;
                        if (!tc::mbar_wait_for(full_bar(s), ph, abort_flag, a.err, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t st = sbase + (uint32_t)s * (uint32_t)a.stage_bytes;
                        const uint32_t vJ = st + kTileBytes, vI = st + kTileBytes + (uint32_t)a.vbytes;
                        const int x = I - w.I0, y = J - w.J0;
                        // row sums: A = the tile K-major; 16 columns = 32 bytes on, box 2 at 16 KB
                        const uint32_t drow = tmem + acc_col(buf, x);
                        const uint32_t acc_r = (touched >> x) & 1u;   // accumulate onto earlier blocks
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk)
                            tc::mma_bf16(drow, tc::sw128_desc(st + (kk >> 2) * 16384 + (kk & 3) * 32),
                                         tc::sw128_desc(vJ + (kk >> 2) * (N * 128) + (kk & 3) * 32), kIdescRow,
                                         (acc_r | (uint32_t)kk) ? 1u : 0u);
                        touched |= 1u << x;
                        if (I != J) {
                            // column sums: A = the tile MN-major; 16 rows = 2 KB on
                            const uint32_t dcol = tmem + acc_col(buf, A + y);
                            const uint32_t acc_c = (touched >> (A + y)) & 1u;
#pragma unroll
                            for (int kk = 0; kk < 8; ++kk)
                                tc::mma_bf16(dcol, sw128_desc_mn(st + kk * 2048, 16384, 1024),
                                             tc::sw128_desc(vI + (kk >> 2) * (N * 128) + (kk & 3) * 32), kIdescCol,
                                             (acc_c | (uint32_t)kk) ? 1u : 0u);
                            touched |= 1u << (A + y);
                        }
                        tc::mma_commit(empty_bar(s));   // the stage is free once these MMAs have read it
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                if (!ok) break;
                tc::mma_commit(accf_bar(buf));   // this super-tile's sums are complete
            }
            // every MMA this thread issued completes before TMEM is released
            tc::mma_commit(down_bar);
            const unsigned long long t0 = tc::globaltimer();
            while (!tc::mbar_try_wait(down_bar, 0) && tc::globaltimer() - t0 < a.wait_ns) {
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lanes 32 (warp % 4) + lane = tile rows
        const uint64_t keep = tc::l2_evict_last();   // the slots are read back by the fold
        const int q = warp & 3;
        const int n = a.n, k = a.k;
        int lt = 0;
        for (long long u = blockIdx.x; u < a.units; u += G, ++lt) {
            const int buf = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            const bool ok = tc::mbar_wait_for(accf_bar(buf), use & 1u, abort_flag, a.err, a.wait_ns);
            // all epilogue threads agree before touching TMEM
            if (!tc::named_bar_all(1, 128, ok && !*abort_flag)) break;
            tc::tc_fence_after();
            const MmaUnit w = mma_unit(a.order ? a.order[u] : u, A, a.Ts);
            for (int z = 0; z < 2 * A; ++z) {
                const bool rowsum = z < A;
                const int X = rowsum ? w.I0 + z : w.J0 + (z - A);   // the block whose rows take these sums
                if (X >= T) continue;
                // written in this super-tile: a row sum when a block (X, J), J >= X, lies in it; a
                // column sum when a block (I, X), I < X, does
                const bool touched = rowsum ? (X > w.J0 ? X : w.J0) < (T < w.J0 + A ? T : w.J0 + A) : w.I0 < X;
                float v[N];
                if (touched) {
                    tmem_ld_cols<N>(tmem + ((uint32_t)(32 * q) << 16) + acc_col(buf, z), v);
                } else {
#pragma unroll
                    for (int c = 0; c < N; ++c) v[c] = 0.f;
                }
                const int slot = rowsum ? w.Js : (w.Is == w.Js ? a.Ts : w.Is);
                const int row = X * kB + 32 * q + lane;
                if (row < n) {
                    float* out = a.Spart + (size_t)slot * k * n + row;
#pragma unroll
                    for (int c = 0; c < N; ++c)
                        if (c < k) tc::st_hint(out + (size_t)c * n, v[c], keep);
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

int sym_mma_bars_bytes(int stages) { return 8 * (2 * stages + 5) + 8; }

}  // namespace

bool plan_sym_mma(SymPlan* p, int k, int num_sms, int smem_optin, int a_req, int stages_req) {
    if (k < 1 || k > 32) return false;
    const int N = k <= 16 ? 16 : 32;
    const int vbytes = onehot_bytes(N);
    const int stage_bytes = kTileBytes + 2 * vbytes;
    // TMEM: two buffers of 2a accumulators of N columns in 512
    const int amax = 512 / (4 * N);
    p->mma = true;
    p->sorted = false;
    p->kb = N;
    p->layout = kPackedSw128H;
    p->rpl = p->pw = 0;
    int cand_a[8] = {8, 7, 6, 5, 4, 3, 2, 1}, na = 8;
    if (a_req > 0) {
        cand_a[0] = a_req;
        na = 1;
    }
    for (int ia = 0; ia < na; ++ia) {
        const int A = cand_a[ia];
        if (A < 1 || A > amax) continue;
        const int Ts = (p->T + A - 1) / A;
        const long long units = (long long)Ts * (Ts + 1) / 2;
        // at least 8 super-tiles an SM, so the static round-robin stays near balance
        if (a_req == 0 && A > 1 && units < 8LL * num_sms) continue;
        for (int S = kMaxStages; S >= 2; --S) {
            if (stages_req > 0 && S != stages_req) continue;
            const int bytes = S * stage_bytes + sym_mma_bars_bytes(S) + 1024;   // + 1024-byte alignment slack
            if (bytes > smem_optin) continue;
            p->a = A;
            p->Ts = Ts;
            p->units = units;
            p->stages = S;
            p->smem = (size_t)bytes;
            p->nslots = Ts + 1;
            p->grid = (int)(units < num_sms ? units : num_sms);
            p->meta_bytes = (size_t)p->T * vbytes;
            p->ok = true;
            return true;
        }
    }
    return false;
}

cudaError_t configure_sym_mma(int smem_optin) {
    void (*fs[4])(MmaArgs) = {reduce_sym_mma_kernel<false, 16>, reduce_sym_mma_kernel<false, 32>,
                              reduce_sym_mma_kernel<true, 16>, reduce_sym_mma_kernel<true, 32>};
    for (auto f : fs) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sym_mma_stream(const PassBuffers& b, const SymPlan& p, int* err, int eval_only, cudaStream_t s,
                                  int stall_ms) {
    if (!p.mma || !p.packed || p.layout != kPackedSw128H || !b.sym_meta) return cudaErrorInvalidValue;
    const bool bf16 = b.k_storage == POPCORN_K_BF16;
    if (!bf16 && b.k_storage != POPCORN_K_FP16) return cudaErrorInvalidValue;
    const int N = p.kb;
    cudaError_t e = launch_pdl(bf16 ? sym_onehot_kernel<__nv_bfloat16> : sym_onehot_kernel<__half>, dim3((unsigned)p.T),
                               dim3(kOneHotThreads), 0, s, (const uint8_t*)b.lab8, b.n, b.k, N,
                               reinterpret_cast<uint4*>(b.sym_meta), (const LoopState*)b.st, eval_only);
    if (e != cudaSuccess) return e;
    MmaArgs a;
    a.Kh = static_cast<const unsigned char*>(b.K);
    a.V = b.sym_meta;
    a.n = b.n;
    a.k = b.k;
    a.N = N;
    a.T = p.T;
    a.a = p.a;
    a.Ts = p.Ts;
    a.units = p.units;
    a.stages = p.stages;
    a.vbytes = onehot_bytes(N);
    a.stage_bytes = kTileBytes + 2 * a.vbytes;
    a.off_bars = p.stages * a.stage_bytes;
    uint32_t cols = 32;
    while (cols < (uint32_t)(4 * p.a * N)) cols <<= 1;
    a.tmem_cols = cols;
    a.Spart = b.Spart;
    a.st = b.st;
    a.err = err;
    a.eval_only = eval_only;
    a.stall_block = stall_ms > 0 ? 1 : 0;
    a.wait_ns = stall_ms > 0 ? (unsigned long long)stall_ms * 1000000ull : tc::kWaitLimitNs;
    a.order = b.sym_order;
    void (*f)(MmaArgs) = bf16 ? (N == 16 ? reduce_sym_mma_kernel<true, 16> : reduce_sym_mma_kernel<true, 32>)
                              : (N == 16 ? reduce_sym_mma_kernel<false, 16> : reduce_sym_mma_kernel<false, 32>);
    return launch_pdl(f, dim3((unsigned)p.grid), dim3(kMmaThreads), p.smem, s, a);
}

}  // namespace popcorn
