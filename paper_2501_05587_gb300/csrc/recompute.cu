// Recompute path: Kernel K-means passes without a stored K.
//
// The paper stores K (Sec. 4.2), which caps n at what HBM holds.  This path
// recomputes, every pass, the tiles of B = Q Q^T that the K stream would read
// (Q = the points in BF16, or FP8 E4M3 with a per-row scale), applies kappa in
// the epilogue and folds the result straight into the per-row cluster sums
// S_ic = sum_{j in L_c} K_ij -- the quantity the paper's SpMM produces (Alg. 2
// line 7).  The columns are visited in cluster order: each pass first sorts
// the points by label (a stable counting sort) and gathers their operand rows,
// so a 128-column block spans only a few runs of equal labels and every
// thread adds kappa into a running register sum, flushing it to its
// shared-memory accumulator only when the (warp-uniform) label changes.
//
// Per pass:  sort_hist -> sort_scan -> sort_scatter (gather) -> recompute_kernel
//            -> zreduce (iterate.cu) -> assign (iterate.cu).
//
// recompute_kernel: one persistent CTA per SM, 192 threads:
//   warp 0   TMA: the unit's 128-row block of Q once (resident), then the
//            column blocks' k-blocks through a ring;
//   warp 1   tcgen05.mma (kind::f16 for BF16, kind::f8f6f4 for E4M3) into one
//            of two 128-column TMEM accumulators;
//   warps 2-5  epilogue: tcgen05.ld, dequantize (FP8: s_i s_j), kappa, run sums.
// A unit is (row block(s), column segment); its sums go to Spart[s][c][i],
// the layout the assign kernel reads.  All waits are bounded as in kbuild_tc.cu.
#include <cmath>
#include <type_traits>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "popcorn_internal.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

using namespace tc;

constexpr int RM = 128;                 // rows per block (MMA M)
constexpr int RN = 128;                 // columns per block (MMA N)
constexpr int KBB = 128;                // operand bytes per row per k-block (64 BF16 / 128 E4M3)
constexpr int KB_TILE = RM * KBB;       // 16 KB
constexpr int kNoLabel = 0xFF;          // padding columns beyond n
constexpr int MS = 16;                  // column-metadata ring slots: deep enough that the epilogue,
                                        // which frees them, never limits how far the copies run ahead
constexpr int NBAR = 96;                // mbarrier slots reserved (2 stages + 4 + 2 MS + 3 used)
constexpr int META_LAB = 0, META_KN = 128, META_SC = 128 + 512, META_BYTES = 128 + 512 + 512;

struct RcArgs {
    int n, ncols, nseg, seglen, nkb, k, fp8;   // ncols: padded column space (multiple of 128)
    int rbp;                            // 128-row blocks per unit (1 or 2): each column tile feeds rbp MMAs
    int stages;                         // B ring depth
    int off_b, off_meta, off_bar, off_misc;   // shared-memory layout (bytes from the aligned base)
    float fact_limit;                   // Gaussian: factor exp2(c2 r_i) out when max_i |c2| r_i is below this
    KernParams kp;
    const float* rnorm;                 // row norms of the represented rows, original order
    const float* rscale;                // FP8 row scales, original order (1 for BF16)
    const uint8_t* slab;                // npad labels in sorted order, kNoLabel past n
    const float* sknorm;                // npad: c2 * norm (Gaussian; raw norm otherwise), sorted order, 0 past n
    const float* sscale;                // npad scales in sorted order, 0 past n
    const int* maxkn;                   // bits of max_i |c2| r_i (Gaussian)
    float* Spart;                       // [nseg * (kEpiGroups / rbp)][k][n]
    LoopState* st;
    int* err;
    int eval;                           // 1: the final objective pass (runs after the loop stopped)
};

constexpr int kEpiGroups = 4;           // epilogue warpgroups

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per-thread view of one 32-column chunk in the 16x256b TMEM fragments: thread
// t = 4 g + m of a warp holds rows g, g + 8 (fragment ra, lanes 0-15 of the warp's
// 32) and g + 16, g + 24 (rb, lanes 16-31), each at columns 8 rep + 2 m + {0, 1},
// rep = 0..3.  Row slot ri = 2 (half) + (row >= +8).  Each column constant then
// serves four rows of a thread instead of one, which keeps the shared-memory
// reads of kn_j / s_j (one 8-byte pair per rep, four distinct addresses per
// warp) far below the exp2 rate.
struct RowConsts {
    float rowc[4];   // -2 c2 (BF16) or -2 c2 s_i (FP8): the coefficient of b in the exponent
    float ar[4];     // c2 r_i (Gaussian, clamped form)
    float si[4];     // s_i (FP8 dot kernels)
};

__device__ __forceinline__ uint32_t frag(const uint32_t (&ra)[16], const uint32_t (&rb)[16], int ri, int x) {
    return ri < 2 ? ra[x] : rb[x];
}

// Adds this thread's share of the chunk to run[ri] (packed pairs of partial sums).
//  Gaussian, factored: exp2(kn_j + coef b) with kn_j = c2 r_j; the caller later
//    multiplies by exp2(c2 r_i).  Padding columns (kn = -inf) give exp2(-inf) = 0.
//  Gaussian, clamped:  exp2(min(c2 (r_i + r_j) - 2 c2 b', 0)) (distance >= 0), used
//    when exp2(|c2| r_i) could overflow.
//  Linear / polynomial of b' = b (BF16) or s_i s_j b (FP8); padding masked.
template <bool FP8, int KIND, bool FACT>
__device__ __forceinline__ void chunk_accumulate(const uint32_t (&ra)[16], const uint32_t (&rb)[16],
                                                 const float2 (&knp)[4], const float2 (&scp)[4], const RowConsts& rc,
                                                 const KernParams& kp, unsigned long long (&run)[4]) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
#pragma unroll
        for (int ri = 0; ri < 4; ++ri) {
            const int x = 4 * rep + 2 * (ri & 1);
            const float b0 = __uint_as_float(frag(ra, rb, ri, x)), b1 = __uint_as_float(frag(ra, rb, ri, x + 1));
            if (KIND == POPCORN_GAUSSIAN && FACT) {
                const unsigned long long rc2 = f2pack(rc.rowc[ri], rc.rowc[ri]);
                const unsigned long long coef = FP8 ? f2mul(rc2, f2pack(scp[rep].x, scp[rep].y)) : rc2;
                const unsigned long long t = f2fma(coef, f2pack(b0, b1), f2pack(knp[rep].x, knp[rep].y));
                float e0, e1;
                f2unpack(t, e0, e1);
                run[ri] = f2add(run[ri], f2pack(ex2(e0), ex2(e1)));
            } else if (KIND == POPCORN_GAUSSIAN) {
                const float c0 = FP8 ? rc.rowc[ri] * scp[rep].x : rc.rowc[ri];
                const float c1 = FP8 ? rc.rowc[ri] * scp[rep].y : rc.rowc[ri];
                const float v0 = ex2(fminf(fmaf(c0, b0, rc.ar[ri] + knp[rep].x), 0.f));
                const float v1 = ex2(fminf(fmaf(c1, b1, rc.ar[ri] + knp[rep].y), 0.f));
                run[ri] = f2add(run[ri], f2pack(v0, v1));
            } else {
                const float bb0 = FP8 ? b0 * (rc.si[ri] * scp[rep].x) : b0;
                const float bb1 = FP8 ? b1 * (rc.si[ri] * scp[rep].y) : b1;
                float v0 = bb0, v1 = bb1;
                if (KIND == POPCORN_POLYNOMIAL) {
                    const float base0 = fmaf(kp.gamma, bb0, kp.coef0), base1 = fmaf(kp.gamma, bb1, kp.coef0);
                    v0 = base0;
                    v1 = base1;
                    for (int e = 1; e < kp.degree; ++e) {
                        v0 *= base0;
                        v1 *= base1;
                    }
                }
                v0 = knp[rep].x == -INFINITY ? 0.f : v0;
                v1 = knp[rep].y == -INFINITY ? 0.f : v1;
                run[ri] = f2add(run[ri], f2pack(v0, v1));
            }
        }
    }
}

template <bool FP8, int KIND>
__global__ void __launch_bounds__(64 + 128 * kEpiGroups, 1)
    recompute_kernel(const __grid_constant__ CUtensorMap map_rows, const __grid_constant__ CUtensorMap map_cols,
                     RcArgs a) {
    if (pass_skip(a.st, a.eval)) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    const int S = a.stages;
    constexpr int EW = 4 * kEpiGroups;  // epilogue warps
    const uint32_t bar0 = sbase + a.off_bar;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (S + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * S + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * S + 2 + b); };
    auto mfull_bar = [&](int m) { return bar0 + 8u * (2 * S + 4 + m); };
    auto mempty_bar = [&](int m) { return bar0 + 8u * (2 * S + 4 + MS + m); };
    const uint32_t afull_bar = bar0 + 8u * (2 * S + 4 + 2 * MS);
    const uint32_t aempty_bar = afull_bar + 8u;
    const uint32_t down_bar = afull_bar + 16u;
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(smem + a.off_misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_misc + 4);
    unsigned char* meta = smem + a.off_meta;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), EW);
        }
        for (int m = 0; m < MS; ++m) {
            mbar_init(mfull_bar(m), 1);
            mbar_init(mempty_bar(m), EW);
        }
        mbar_init(afull_bar, 1);
        mbar_init(aempty_bar, 1);
        mbar_init(down_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t tmem_cols = a.rbp == 2 ? 512u : 256u;   // 2 buffers x rbp accumulators x 128 columns
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int T = (a.n + RM * a.rbp - 1) / (RM * a.rbp);   // row-block groups
    const int units = T * a.nseg;
    const int G = gridDim.x;
    auto unit_cols = [&](int u, int* I, int* s, int* jb0, int* jb1) {
        *I = u / a.nseg;
        *s = u - *I * a.nseg;
        const int c0 = *s * a.seglen;
        const int c1 = min(a.ncols, c0 + a.seglen);
        *jb0 = c0 / RN;
        *jb1 = (c1 + RN - 1) / RN;
    };
    constexpr uint32_t idesc = FP8 ? idesc_e4m3(RM, RN) : idesc_bf16(RM, RN);
    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: row block, column metadata, column k-blocks ----------------
            int stage = 0;
            uint32_t phase = 0;
            int ucount = 0, bc = 0;
            bool ok = true;
            bool a_issued = false;
            uint32_t a_parity = 0;
            uint32_t issued_mask = 0, issued_par = 0;    // per B stage
            uint32_t missued_mask = 0, missued_par = 0;  // per metadata slot
            for (int u = blockIdx.x; u < units && ok; u += G, ++ucount) {
                int I, s, jb0, jb1;
                unit_cols(u, &I, &s, &jb0, &jb1);
                if (!mbar_wait(aempty_bar, ((uint32_t)ucount & 1u) ^ 1u, abort_flag, a.err)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(afull_bar, (uint32_t)(a.rbp * a.nkb * KB_TILE));
                for (int h = 0; h < a.rbp; ++h)
                    for (int kb = 0; kb < a.nkb; ++kb)
                        tma_load_2d(sbase + (h * a.nkb + kb) * KB_TILE, &map_rows, kb * (FP8 ? KBB : KBB / 2),
                                    (I * a.rbp + h) * RM, afull_bar);
                a_issued = true;
                a_parity = (uint32_t)ucount & 1u;
                for (int jb = jb0; jb < jb1 && ok; ++jb, ++bc) {
                    const int ms = bc % MS;
                    const uint32_t mpar = (uint32_t)(bc / MS) & 1u;
                    if (!mbar_wait(mempty_bar(ms), mpar ^ 1u, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t mdst = sbase + a.off_meta + ms * META_BYTES;
                    mbar_arrive_expect_tx(mfull_bar(ms), META_BYTES);
                    bulk_load_1d(mdst + META_LAB, a.slab + (size_t)jb * RN, 128, mfull_bar(ms));
                    bulk_load_1d(mdst + META_KN, a.sknorm + (size_t)jb * RN, 512, mfull_bar(ms));
                    bulk_load_1d(mdst + META_SC, a.sscale + (size_t)jb * RN, 512, mfull_bar(ms));
                    missued_mask |= 1u << ms;
                    missued_par = (missued_par & ~(1u << ms)) | (mpar << ms);
                    for (int kb = 0; kb < a.nkb; ++kb) {
                        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(full_bar(stage), KB_TILE);
                        tma_load_2d(sbase + a.off_b + stage * KB_TILE, &map_cols, kb * (FP8 ? KBB : KBB / 2),
                                    jb * RN, full_bar(stage));
                        issued_mask |= 1u << stage;
                        issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                // aborted: let this CTA's own copies land before shared memory goes away
                auto drain = [&](uint32_t bar, uint32_t par) {
                    const unsigned long long t0 = globaltimer();
                    while (!mbar_try_wait(bar, par) && globaltimer() - t0 < kWaitLimitNs) {
                    }
                };
                for (int s2 = 0; s2 < S; ++s2)
                    if (issued_mask >> s2 & 1u) drain(full_bar(s2), issued_par >> s2 & 1u);
                for (int m = 0; m < MS; ++m)
                    if (missued_mask >> m & 1u) drain(mfull_bar(m), missued_par >> m & 1u);
                if (a_issued) drain(afull_bar, a_parity);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            // This thread shares its sub-partition with four busy epilogue warps, so the
            // loop keeps its own instructions few: descriptors are advanced by adds (the
            // 14-bit address field of a 1024-aligned tile never carries).
            int stage = 0;
            uint32_t phase = 0;
            int ucount = 0, bc = 0;
            bool ok = true;
            const uint64_t bdesc0 = sw128_desc(sbase + a.off_b);   // stage 0, first 32 bytes of K
            const uint64_t adesc0 = sw128_desc(sbase);             // resident rows in shared memory
            constexpr uint32_t kStageStep = KB_TILE >> 4;          // descriptor units per 16 KB tile
            for (int u = blockIdx.x; u < units && ok; u += G, ++ucount) {
                int I, s, jb0, jb1;
                unit_cols(u, &I, &s, &jb0, &jb1);
                // the unit's resident row blocks have landed in shared memory
                if (!mbar_wait(afull_bar, (uint32_t)ucount & 1u, abort_flag, a.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int jb = jb0; jb < jb1 && ok; ++jb, ++bc) {
                    const int ab = bc & 1;
                    if (!mbar_wait(acce_bar(ab), ((uint32_t)(bc >> 1) & 1u) ^ 1u, abort_flag, a.err)) {
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
                        const uint64_t bd = bdesc0 + (uint64_t)(stage * kStageStep);
                        for (int h = 0; h < a.rbp; ++h) {
                            // accumulator (buffer ab, row block h) at TMEM column (ab * rbp + h) * 128
                            const uint32_t d_tmem = tmem + (uint32_t)((ab * a.rbp + h) * RN);
                            const uint64_t ad = adesc0 + (uint64_t)((h * a.nkb + kb) * kStageStep);
                            const uint32_t acc0 = kb ? 1u : 0u;
                            // 32 bytes of K per instruction: +2 in the descriptor's address field
                            if (FP8) {
                                mma_e4m3(d_tmem, ad, bd, idesc, acc0);
                                mma_e4m3(d_tmem, ad + 2, bd + 2, idesc, 1u);
                                mma_e4m3(d_tmem, ad + 4, bd + 4, idesc, 1u);
                                mma_e4m3(d_tmem, ad + 6, bd + 6, idesc, 1u);
                            } else {
                                mma_bf16(d_tmem, ad, bd, idesc, acc0);
                                mma_bf16(d_tmem, ad + 2, bd + 2, idesc, 1u);
                                mma_bf16(d_tmem, ad + 4, bd + 4, idesc, 1u);
                                mma_bf16(d_tmem, ad + 6, bd + 6, idesc, 1u);
                            }
                        }
                        mma_commit(empty_bar(stage));
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(accf_bar(ab));
                }
                mma_commit(aempty_bar);   // the resident row block is free once these MMAs finish
            }
            mma_commit(down_bar);
            const unsigned long long t0 = globaltimer();
            while (!mbar_try_wait(down_bar, 0) && globaltimer() - t0 < kWaitLimitNs) {
            }
        }
    } else if (warp < 2 + EW) {
        // ---------------- epilogue ----------------
        // Warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31, i.e. 32 rows.  Group
        // g = (w - 2) / 4 takes row block g % rbp of the pair and the 32-column chunks
        // [gsub nch, gsub nch + nch) of every column block, gsub = g / rbp, nch = rbp.
        // The columns arrive in cluster order, so each (row, cluster) sum of a unit is
        // one run: it is written to Spart once, when the label changes, and the
        // clusters the unit does not meet get zeros -- no shared-memory accumulators.
        const int g = (warp - 2) >> 2;
        const int q = warp & 3;
        const int hb = g % a.rbp;
        const int gpr = kEpiGroups / a.rbp;          // groups per row block: Spart slots per segment
        const int gsub = g / a.rbp;
        const int nch = a.rbp;                       // = 4 / gpr
        const int ch0 = gsub * nch;
        const int gq = lane >> 2, m = lane & 3;      // fragment row group and column pair
        const float c2 = a.kp.neg_gamma_over_sigma2 * 1.4426950408889634f;
        const float m2c2 = -2.f * c2;
        const KernParams kp = a.kp;
        auto body = [&](auto fact_tag) {
            constexpr bool FACT = decltype(fact_tag)::value;
            int bc = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += G) {
                int I, s, jb0, jb1;
                unit_cols(u, &I, &s, &jb0, &jb1);
                const int rbase = (I * a.rbp + hb) * RM + 32 * q;
                RowConsts rc;
#pragma unroll
                for (int ri = 0; ri < 4; ++ri) {
                    const int row = rbase + 16 * (ri >> 1) + gq + 8 * (ri & 1);
                    const bool v = row < a.n;
                    const float si = v ? a.rscale[row] : 0.f;
                    rc.si[ri] = si;
                    rc.rowc[ri] = FP8 ? m2c2 * si : m2c2;
                    rc.ar[ri] = v && KIND == POPCORN_GAUSSIAN ? c2 * a.rnorm[row] : 0.f;
                }
                // lane 4 gq + m writes row slot m of its quad: the warp's 32 rows, once each
                const int wrow = rbase + 16 * (m >> 1) + gq + 8 * (m & 1);
                const bool wvalid = wrow < a.n;
                const float wfin = FACT ? ex2(m == 0 ? rc.ar[0] : m == 1 ? rc.ar[1] : m == 2 ? rc.ar[2] : rc.ar[3])
                                        : 1.f;
                float* out = a.Spart + (size_t)(s * gpr + gsub) * a.k * a.n + wrow;   // [slot][c][i]
                int cur = -1, nextc = 0;
                unsigned long long run[4] = {0ull, 0ull, 0ull, 0ull};
                // write the finished run of cluster c (and zeros for the clusters skipped before it)
                auto emit = [&](int c) {
                    float v[4];
#pragma unroll
                    for (int ri = 0; ri < 4; ++ri) {
                        float lo, hi;
                        f2unpack(run[ri], lo, hi);
                        v[ri] = lo + hi;
                        v[ri] += __shfl_xor_sync(0xffffffffu, v[ri], 1);
                        v[ri] += __shfl_xor_sync(0xffffffffu, v[ri], 2);
                    }
                    const float mine = (m == 0 ? v[0] : m == 1 ? v[1] : m == 2 ? v[2] : v[3]) * wfin;
                    if (wvalid) {
                        for (int z = nextc; z < c; ++z) out[(size_t)z * a.n] = 0.f;
                        out[(size_t)c * a.n] = mine;
                    }
                    nextc = c + 1;
                };
                for (int jb = jb0; jb < jb1; ++jb, ++bc) {
                    const int ab = bc & 1;
                    const int ms = bc % MS;
                    bool got = mbar_wait(mfull_bar(ms), (uint32_t)(bc / MS) & 1u, abort_flag, a.err);
                    got = got && mbar_wait(accf_bar(ab), (uint32_t)(bc >> 1) & 1u, abort_flag, a.err);
                    if (__any_sync(0xffffffffu, !got)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* mp = meta + ms * META_BYTES;
                    const uint8_t* ml = mp + META_LAB;
                    const float* mk = reinterpret_cast<const float*>(mp + META_KN);
                    const float* msc = reinterpret_cast<const float*>(mp + META_SC);
                    const uint32_t tacc =
                        tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((ab * a.rbp + hb) * RN + 32 * ch0);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h >= nch) break;
                        uint32_t ra[16], rb[16];
                        tmem_ld16x256_x4_nowait(tacc + 32u * h, ra);
                        tmem_ld16x256_x4_nowait(tacc + 32u * h + (16u << 16), rb);
                        tmem_ld_wait();
                        if (h == nch - 1) {
                            // this warp has read its share of the accumulator
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(acce_bar(ab));
                        }
                        // every cluster's run of columns is padded to a multiple of 32, so a
                        // chunk holds one label (kNoLabel: padding past the last cluster)
                        const int ch = ch0 + h;
                        const int lab = ml[32 * ch];
                        if (lab == kNoLabel) continue;
                        if (lab != cur) {   // warp-uniform
                            if (cur >= 0) emit(cur);
                            cur = lab;
#pragma unroll
                            for (int ri = 0; ri < 4; ++ri) run[ri] = 0ull;
                        }
                        float2 knp[4], scp[4];
#pragma unroll
                        for (int rep = 0; rep < 4; ++rep) {
                            knp[rep] = *reinterpret_cast<const float2*>(mk + 32 * ch + 8 * rep + 2 * m);
                            scp[rep] = FP8 || KIND != POPCORN_GAUSSIAN
                                           ? *reinterpret_cast<const float2*>(msc + 32 * ch + 8 * rep + 2 * m)
                                           : make_float2(1.f, 1.f);
                        }
                        chunk_accumulate<FP8, KIND, FACT>(ra, rb, knp, scp, rc, kp, run);
                    }
                    // this warp is done with the metadata slot
                    __syncwarp();
                    if (lane == 0) mbar_arrive(mempty_bar(ms));
                }
                if (!ok) break;
                if (cur >= 0) emit(cur);
                if (wvalid)
                    for (int z = nextc; z < a.k; ++z) out[(size_t)z * a.n] = 0.f;
            }
        };
        if (KIND == POPCORN_GAUSSIAN && __int_as_float(*a.maxkn) < a.fact_limit)
            body(std::true_type{});
        else
            body(std::false_type{});
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------- operand preparation (once per fit)
// One warp per row: BF16 copy (or E4M3 with scale amax/448), the represented
// row's FP32 norm, its scale, and diag K = kappa(p_i, p_i).
__global__ void __launch_bounds__(256) quantize_kernel(const float* __restrict__ P, int n, int d, int64_t ldp,
                                                       int dpad, int fp8, KernParams kp, unsigned char* __restrict__ Q,
                                                       float* __restrict__ norms, float* __restrict__ knorms,
                                                       float* __restrict__ scales, float* __restrict__ kdiag,
                                                       int* __restrict__ maxkn) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const float* p = P + (int64_t)w * ldp;
    float scale = 1.f;
    if (fp8) {
        float amax = 0.f;
        for (int l = lane; l < d; l += 32) amax = fmaxf(amax, fabsf(p[l]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        scale = amax > 0.f ? amax / 448.f : 1.f;
    }
    float nrm = 0.f;
    for (int l = lane; l < dpad; l += 32) {
        const float x = l < d ? p[l] : 0.f;
        float rep;
        if (fp8) {
            const __nv_fp8_storage_t qv = __nv_cvt_float_to_fp8(x / scale, __NV_SATFINITE, __NV_E4M3);
            Q[(int64_t)w * dpad + l] = qv;
            const __half_raw hr = __nv_cvt_fp8_to_halfraw(qv, __NV_E4M3);
            rep = __half2float(__half(hr)) * scale;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            reinterpret_cast<__nv_bfloat16*>(Q)[(int64_t)w * dpad + l] = h;
            rep = __bfloat162float(h);
        }
        nrm = fmaf(rep, rep, nrm);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) {
        norms[w] = nrm;
        // the epilogue works in base 2: c2 * r with c2 = -gamma log2(e) / sigma^2
        const float kn = kp.kind == POPCORN_GAUSSIAN ? kp.neg_gamma_over_sigma2 * 1.4426950408889634f * nrm : nrm;
        knorms[w] = kn;
        // max_i |c2| r_i (non-negative floats order like their bit patterns)
        if (kp.kind == POPCORN_GAUSSIAN) atomicMax(maxkn, __float_as_int(fabsf(kn)));
        scales[w] = scale;
        float kd;
        if (kp.kind == POPCORN_GAUSSIAN) {
            kd = 1.f;
        } else if (kp.kind == POPCORN_POLYNOMIAL) {
            const float base = fmaf(kp.gamma, nrm, kp.coef0);
            kd = base;
            for (int e = 1; e < kp.degree; ++e) kd *= base;
        } else {
            kd = nrm;
        }
        kdiag[w] = kd;
    }
}

// ---------------------------------------------------------------- stable counting sort by label
constexpr int SORT_THREADS = 1024;

__global__ void __launch_bounds__(SORT_THREADS) sort_hist_kernel(const uint8_t* __restrict__ lab, int n, int k,
                                                                 int* __restrict__ blockhist, const LoopState* st,
                                                                 int eval) {
    if (pass_skip(st, eval)) return;
    __shared__ int h[kMaxClusters];
    for (int c = threadIdx.x; c < k; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&h[lab[i]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) blockhist[(size_t)blockIdx.x * k + c] = h[c];
}

// blockoff[b][c] = (padded start of cluster c) + (points with label c in blocks < b),
// where cluster c starts at sum_{c' < c} round_up(|L_c'|, 32): every cluster's
// columns fill whole 32-column chunks.
__global__ void __launch_bounds__(kMaxClusters) sort_scan_kernel(const int* __restrict__ blockhist, int nb, int k,
                                                                 int* __restrict__ blockoff, int ncols,
                                                                 uint8_t* __restrict__ slab, float* __restrict__ snorm,
                                                                 float* __restrict__ sscale, const LoopState* st,
                                                                 int eval) {
    if (pass_skip(st, eval)) return;
    __shared__ int tot[kMaxClusters];
    __shared__ int total;
    const int c = threadIdx.x;
    int t = 0;
    if (c < k)
        for (int b = 0; b < nb; ++b) t += blockhist[(size_t)b * k + c];
    tot[c] = c < k ? t : 0;
    __syncthreads();
    if (c < k) {
        int base = 0;
        for (int c2 = 0; c2 < c; ++c2) base += (tot[c2] + 31) & ~31;
        int run = base;
        for (int b = 0; b < nb; ++b) {
            blockoff[(size_t)b * k + c] = run;
            run += blockhist[(size_t)b * k + c];
        }
        // this cluster's padding up to its next 32-column boundary: no cluster, zero weight
        for (int pos = base + t; pos < base + ((t + 31) & ~31); ++pos) {
            slab[pos] = (uint8_t)kNoLabel;
            snorm[pos] = -INFINITY;
            sscale[pos] = 0.f;
        }
        if (c == k - 1) total = base + ((t + 31) & ~31);
    }
    __syncthreads();
    for (int pos = total + c; pos < ncols; pos += blockDim.x) {
        slab[pos] = (uint8_t)kNoLabel;
        snorm[pos] = -INFINITY;
        sscale[pos] = 0.f;
    }
}

// Position of every point in cluster order (stable: by block, then warp, then
// lane) and a gather of its operand row, norm, scale and label.
__global__ void __launch_bounds__(SORT_THREADS) sort_scatter_kernel(
    const uint8_t* __restrict__ lab, int n, int k, const int* __restrict__ blockoff, const unsigned char* __restrict__ Q,
    int row_bytes, const float* __restrict__ norms, const float* __restrict__ scales, unsigned char* __restrict__ Qs,
    float* __restrict__ snorm, float* __restrict__ sscale, uint8_t* __restrict__ slab, const LoopState* st, int eval) {
    if (pass_skip(st, eval)) return;
    __shared__ int wcount[SORT_THREADS / 32][kMaxClusters];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < (SORT_THREADS / 32) * kMaxClusters; t += blockDim.x) (&wcount[0][0])[t] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const int l = valid ? lab[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcount[warp][l] = __popc(peers);
    __syncthreads();
    // exclusive prefix over warps, per label
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        int run = 0;
        for (int w = 0; w < SORT_THREADS / 32; ++w) {
            const int v = wcount[w][c];
            wcount[w][c] = run;
            run += v;
        }
    }
    __syncthreads();
    if (!valid) return;
    const int pos = blockoff[(size_t)blockIdx.x * k + l] + wcount[warp][l] + rank;
    const uint4* src = reinterpret_cast<const uint4*>(Q + (int64_t)i * row_bytes);
    uint4* dst = reinterpret_cast<uint4*>(Qs + (int64_t)pos * row_bytes);
    for (int t = 0; t < row_bytes / 16; ++t) dst[t] = src[t];
    snorm[pos] = norms[i];   // (the c2-scaled norm for the Gaussian)
    sscale[pos] = scales[i];
    slab[pos] = (uint8_t)l;
}

using RcFn = void (*)(const CUtensorMap, const CUtensorMap, RcArgs);

RcFn recompute_fn(bool fp8, int kind) {
    switch (kind) {
        case POPCORN_LINEAR: return fp8 ? recompute_kernel<true, POPCORN_LINEAR> : recompute_kernel<false, POPCORN_LINEAR>;
        case POPCORN_POLYNOMIAL:
            return fp8 ? recompute_kernel<true, POPCORN_POLYNOMIAL> : recompute_kernel<false, POPCORN_POLYNOMIAL>;
        default: return fp8 ? recompute_kernel<true, POPCORN_GAUSSIAN> : recompute_kernel<false, POPCORN_GAUSSIAN>;
    }
}

bool make_map_u8(CUtensorMap* m, void* base, uint64_t inner_bytes, uint64_t rows, bool fp8) {
    // BF16 maps count elements of 2 bytes, E4M3 maps elements of 1 byte
    return make_tensor_map_2d(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base,
                              fp8 ? inner_bytes : inner_bytes / 2, rows, inner_bytes, fp8 ? KBB : KBB / 2, RM,
                              CU_TENSOR_MAP_SWIZZLE_128B);
}

}  // namespace

// ---------------------------------------------------------------- host side

RecomputePlan plan_recompute(int n, int d, int k, int precision, int num_sms, int smem_budget, int rbp_req,
                             int units_per_sm) {
    RecomputePlan p{};
    p.fp8 = precision == POPCORN_FP8;
    const int elem = p.fp8 ? 1 : 2;
    const int per_kb = KBB / elem;                         // elements per k-block
    p.dpad = (d + per_kb - 1) / per_kb * per_kb;
    p.row_bytes = p.dpad * elem;
    p.nkb = p.row_bytes / KBB;
    p.npad = (n + RN - 1) / RN * RN;
    // sorted column space: clusters padded to 32-column chunks
    p.ncols = (n + 31 * k + RN - 1) / RN * RN;
    // shared memory: resident row blocks, B ring, metadata ring, barriers.  Prefer two
    // row blocks per unit (each column tile then feeds two MMAs, halving the operand
    // traffic from L2 per flop); fall back to one when fewer than 3 ring stages fit.
    const int meta = MS * META_BYTES;
    const int fixed = meta + NBAR * 8 + 64 + 1024;
    int rbp = rbp_req == 1 ? 1 : 2;
    int stages = (smem_budget - rbp * p.nkb * KB_TILE - fixed) / KB_TILE;
    if (stages < 3 && rbp_req == 0) {
        rbp = 1;
        stages = (smem_budget - rbp * p.nkb * KB_TILE - fixed) / KB_TILE;
    }
    if (stages > 12) stages = 12;
    p.rbp = rbp;
    p.eg = kEpiGroups;
    p.threads = 64 + 128 * kEpiGroups;
    p.stages = stages;
    p.off_b = rbp * p.nkb * KB_TILE;
    p.off_meta = p.off_b + stages * KB_TILE;
    p.off_bar = p.off_meta + meta;
    // units: groups of rbp row blocks x column segments, about units_per_sm per SM
    {
        const int Tg = (p.npad / RM + rbp - 1) / rbp;
        p.units_per_sm = units_per_sm > 0 ? units_per_sm : 16;
        long long ns = ((long long)p.units_per_sm * num_sms + Tg - 1) / Tg;
        const long long maxseg = p.ncols / RN;
        if (ns > maxseg) ns = maxseg;
        if (ns < 1) ns = 1;
        long long sl = (p.ncols + ns - 1) / ns;
        sl = (sl + RN - 1) / RN * RN;
        p.seglen = (int)sl;
        p.nseg = (int)((p.ncols + sl - 1) / sl);
    }
    // every epilogue group writes its own slot of each segment
    p.nslot = p.nseg * (kEpiGroups / rbp);
    // factored Gaussian: exp2(x_ij) with x_ij <= |c2| r_i summed over up to ncols
    // columns must stay finite: |c2| r_i + log2(ncols) well below 128
    p.fact_limit = 120.f - std::log2((float)p.ncols);
    p.off_misc = p.off_bar + NBAR * 8;
    p.smem = p.off_misc + 64 + 1024;
    p.ok = p.nkb <= 4 && stages >= 2 && k <= 255;
    p.grid = num_sms;
    return p;
}

cudaError_t configure_recompute(int smem_optin, int* usable) {
    size_t st = 0;
    for (int f = 0; f < 2; ++f)
        for (int kind = 0; kind < 3; ++kind) {
            cudaFuncAttributes fa;
            cudaError_t e = cudaFuncGetAttributes(&fa, recompute_fn(f != 0, kind));
            if (e != cudaSuccess) return e;
            if (fa.sharedSizeBytes > st) st = fa.sharedSizeBytes;
        }
    const int bytes = optin_minus_static(smem_optin, st);
    for (int f = 0; f < 2; ++f)
        for (int kind = 0; kind < 3; ++kind) {
            cudaError_t e = cudaFuncSetAttribute(recompute_fn(f != 0, kind), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 bytes);
            if (e != cudaSuccess) return e;
        }
    *usable = bytes;
    return cudaSuccess;
}

cudaError_t launch_quantize(const float* P, int n, int d, int64_t ldp, KernParams kp, const RecomputePlan& p,
                            const RecomputeBuffers& rb, float* kdiag, cudaStream_t s) {
    quantize_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(P, n, d, ldp, p.dpad, p.fp8, kp, rb.Q, rb.norms, rb.knorms,
                                                         rb.scales, kdiag, rb.maxkn);
    return cudaGetLastError();
}

int recompute_sort_blocks(int n) { return (n + SORT_THREADS - 1) / SORT_THREADS; }

cudaError_t launch_recompute_pass(const PassBuffers& b, KernParams kp, const RecomputePlan& p,
                                  const RecomputeBuffers& rb, int* err, int eval, cudaStream_t s) {
    const int n = b.n, k = b.k;
    const int nb = recompute_sort_blocks(n);
    sort_hist_kernel<<<nb, SORT_THREADS, 0, s>>>(b.lab8, n, k, rb.blockhist, b.st, eval);
    sort_scan_kernel<<<1, kMaxClusters, 0, s>>>(rb.blockhist, nb, k, rb.blockoff, p.ncols, rb.slab, rb.snorm,
                                                rb.sscale, b.st, eval);
    sort_scatter_kernel<<<nb, SORT_THREADS, 0, s>>>(b.lab8, n, k, rb.blockoff, rb.Q, p.row_bytes, rb.knorms,
                                                    rb.scales, rb.Qs, rb.snorm, rb.sscale, rb.slab, b.st, eval);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RcArgs a;
    a.n = n;
    a.ncols = p.ncols;
    a.nseg = p.nseg;
    a.seglen = p.seglen;
    a.nkb = p.nkb;
    a.k = k;
    a.fp8 = p.fp8;
    a.rbp = p.rbp;
    a.stages = p.stages;
    a.off_b = p.off_b;
    a.off_meta = p.off_meta;
    a.off_bar = p.off_bar;
    a.off_misc = p.off_misc;
    a.kp = kp;
    a.rnorm = rb.norms;
    a.rscale = rb.scales;
    a.slab = rb.slab;
    a.sknorm = rb.snorm;
    a.sscale = rb.sscale;
    a.maxkn = rb.maxkn;
    a.fact_limit = p.fact_limit;
    a.Spart = b.Spart;
    a.st = b.st;
    a.err = err;
    a.eval = eval;
    CUtensorMap mr, mc;
    if (!make_map_u8(&mr, rb.Q, (uint64_t)p.row_bytes, (uint64_t)n, p.fp8) ||
        !make_map_u8(&mc, rb.Qs, (uint64_t)p.row_bytes, (uint64_t)p.ncols, p.fp8))
        return cudaErrorInvalidValue;
    recompute_fn(p.fp8 != 0, kp.kind)<<<p.grid, p.threads, p.smem, s>>>(mr, mc, a);
    return cudaGetLastError();
}

}  // namespace popcorn
