// Symmetric K stream: one pass over the upper triangle of K.
//
// K is symmetric (K = kappa(P P^T), Sec. 3.2), so S_ic = sum_{j in L_c} K_ij
// (the paper's SpMM, Alg. 2 line 7) splits into the part with j in or after
// row i's 128-column block, read along row i, and the part with j before it,
// which equals the column sums sum_{j in L_c} K_ji over rows j of earlier
// blocks.  Reading only the blocks on and above the diagonal gives both: every
// element K_ij of an off-diagonal block is added to row i's sum of cluster
// cl(j) AND to column j's sum of cluster cl(i).  The diagonal blocks are read
// whole and feed row sums only.  That halves the bytes a pass reads.
//
// Work: column segments of L columns; an item is (segment s, a range of
// 128-row blocks whose rows reach into s).  A CTA takes items in turn; its
// warps take the item's rows.  Per row the warp streams float4s from the
// start of the row's block (or the segment) to the segment end:
//   * row sums in lane-private shared-memory columns acc[c][lane] (as in
//     reduce_kernel), reduced at the row's end into Spart[s][c][i];
//   * column sums (blocks after the row's own) into the CTA's colacc[c][j]
//     with shared-memory atomic adds: cl(i) is the same for the whole row,
//     so a lane's adds go to its own columns.  Warps add to the same columns
//     in no fixed order, so the adds are 64-bit integer (fixed point, F
//     fractional bits of max_i K_ii): integer sums do not depend on order,
//     and for a PSD kernel |K_ij| <= max_i K_ii keeps n terms inside 63 bits.
//     colacc is stored [c][e][q] (column c0 + 4 q + e): a warp's adds for one
//     element e of its float4s hit 32 consecutive words.
// At an item's end colacc goes to Cpart[item]; sym_fold_kernel then sums the
// items of each segment into Spart[nseg][c][j] (fixed order).  The distance
// and z kernels read, for row i, the segments from the one holding row i's
// block on, plus slot nseg.
#include <algorithm>
#include <vector>

#include "popcorn_internal.cuh"
#include "stream_common.cuh"

namespace popcorn {
namespace {

using namespace stream;

struct SymArgs {
    const float* K;           // FP32 rows, pitch ldk (multiple of 4)
    int64_t ldk;
    int n, k, seglen, nseg;   // seglen: multiple of 128
    const int4* items;        // {segment, first row block, end row block, 0}
    int nitems;
    const uint8_t* lab8;
    float* Spart;             // [nseg + 1][k][n]
    unsigned long long* Cpart;   // [nitems][k][4][seglen / 4], fixed point
    int fbits;                // fractional bits: 61 - ceil(log2 n)
    const LoopState* st;
    int eval_only;
};

// Fixed-point scale 2^F / max_i |K_ii| (capped so that a zero diagonal stays finite);
// the K stream and the fold compute it the same way.
__device__ __forceinline__ float fixed_scale(const LoopState* st, int fbits) {
    return fminf(exp2f((float)fbits) / fmaxf((float)st->kdiag_max, 1e-30f), 0x1p100f);
}

template <int KB, int UNR, bool LAB_SMEM>
__global__ void __launch_bounds__(kReduceMaxWarps * 32, 1) reduce_sym_kernel(SymArgs a) {
    if (pass_skip(a.st, a.eval_only)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, k = a.k, L = a.seglen, L4 = a.seglen / 4;
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nlab = LAB_SMEM ? ((n + 15) & ~15) : 0;
    uint8_t* slab = smem;
    unsigned long long* colacc = reinterpret_cast<unsigned long long*>(smem + nlab);   // [k][4][L4]
    float* sacc = reinterpret_cast<float*>(colacc + (size_t)k * L);                     // [W][k][32]
    const float scale = fixed_scale(a.st, a.fbits);
    if (LAB_SMEM) {
        const uint4* src = reinterpret_cast<const uint4*>(a.lab8);
        uint4* dst = reinterpret_cast<uint4*>(slab);
        for (int t = threadIdx.x; t < nlab / 16; t += blockDim.x) dst[t] = src[t];
    }
    for (int t = threadIdx.x; t < k * L; t += blockDim.x) colacc[t] = 0ull;
    for (int t = threadIdx.x; t < W * k * 32; t += blockDim.x) sacc[t] = 0.f;
    __syncthreads();
    const uint8_t* labs = LAB_SMEM ? slab : a.lab8;
    const uint32_t* lab4 = reinterpret_cast<const uint32_t*>(labs);
    float* accw = sacc + (size_t)warp * k * 32;
    float* accl = accw + lane;

    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const int4 item = a.items[it];
        const int s = item.x;
        const int c0 = s * L, c1 = min(n, c0 + L);
        const int q1 = c1 >> 2;                       // full float4s of the segment
        const int row_end = min(n, item.z * 128);
        // cursor of this warp: row i, float4 base qb (lane 0's), diagonal end dend
        struct Cur {
            int i, qb, dend, li;
            const float4* row4;
        };
        auto open_row = [&](int i, Cur& c) -> bool {
            if (i >= row_end) return false;
            const int blk0 = (i >> 7) << 7;
            c.i = i;
            c.qb = max(c0, blk0) >> 2;
            c.dend = blk0 + 128;
            c.li = labs[i];
            c.row4 = reinterpret_cast<const float4*>(a.K + (int64_t)i * a.ldk);
            return true;
        };
        auto load = [&](const Cur& c, float4 (&v)[UNR], uint32_t (&Lb)[UNR]) {
#pragma unroll
            for (int t = 0; t < UNR; ++t) {
                const int q = c.qb + lane + 32 * t;
                if (q < q1) {
                    v[t] = ld_stream(c.row4 + q);
                    Lb[t] = LAB_SMEM ? lab4[q] : __ldg(lab4 + q);
                } else {
                    v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                    Lb[t] = 0u;
                }
            }
        };
        Cur cur;
        if (open_row(item.y * 128 + warp, cur)) {
            float4 v[UNR];
            uint32_t Lb[UNR];
            load(cur, v, Lb);
            while (true) {
                const bool last = cur.qb + 32 * UNR >= q1;
                Cur nxt = cur;
                bool more = true;
                if (last) more = open_row(cur.i + W, nxt);
                else nxt.qb = cur.qb + 32 * UNR;
                float4 vn[UNR];
                uint32_t Ln[UNR];
                if (more) load(nxt, vn, Ln);
                unsigned long long* colrow = colacc + (size_t)cur.li * L - (c0 >> 2);   // [e * L4 + q]
#pragma unroll
                for (int t = 0; t < UNR; ++t) {
                    const int q = cur.qb + lane + 32 * t;
                    const float e4[4] = {v[t].x, v[t].y, v[t].z, v[t].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) accl[((Lb[t] >> (8 * e)) & 0xffu) * 32] += e4[e];
                    // a float4 never straddles the block boundary (both multiples of 4)
                    if (q < q1 && 4 * q >= cur.dend) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            atomicAdd(colrow + e * L4 + q, (unsigned long long)__float2ll_rn(e4[e] * scale));
                    }
                }
                if (last) {
                    {   // ragged tail of the row (n not a multiple of 4)
                        const int j = 4 * q1 + lane;
                        if (j < c1) {
                            const float x = a.K[(int64_t)cur.i * a.ldk + j];
                            accl[(int)labs[j] * 32] += x;
                            if (j >= cur.dend)
                                atomicAdd(colacc + (size_t)cur.li * L + ((j - c0) & 3) * L4 + ((j - c0) >> 2),
                                          (unsigned long long)__float2ll_rn(x * scale));
                        }
                    }
                    float* out = a.Spart + (size_t)s * k * n + cur.i;   // [s][c][i]
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
                        if ((lane & (32 / KB - 1)) == 0 && c < k) out[(size_t)c * n] = tot;
                    } else {
                        for (int cb = 0; cb < k; cb += 32) {
                            const int c = cb + lane;
                            if (c < k) {
                                float tot = 0.f;
                                float* rowp = accw + (size_t)c * 32;
#pragma unroll 8
                                for (int j = 0; j < 32; ++j) {
                                    const int idx = (j + lane) & 31;
                                    tot += rowp[idx];
                                    rowp[idx] = 0.f;
                                }
                                out[(size_t)c * n] = tot;
                            }
                        }
                    }
                    __syncwarp();
                    if (!more) break;
                }
                cur = nxt;
#pragma unroll
                for (int t = 0; t < UNR; ++t) {
                    v[t] = vn[t];
                    Lb[t] = Ln[t];
                }
            }
        }
        // this item's column sums: to Cpart, and cleared for the next item
        __syncthreads();
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(a.Cpart + (size_t)it * k * L);
        ulonglong2* src = reinterpret_cast<ulonglong2*>(colacc);
        for (int t = threadIdx.x; t < k * L / 2; t += blockDim.x) {
            dst[t] = src[t];
            src[t] = make_ulonglong2(0ull, 0ull);
        }
        __syncthreads();
    }
}

// Spart[nseg][c][j] = the column sums of j over the items of j's segment: an exact
// integer sum, then scaled back.
__global__ void __launch_bounds__(256) sym_fold_kernel(const unsigned long long* __restrict__ Cpart,
                                                        const int* __restrict__ seg_item, int n, int k, int seglen,
                                                        int nseg, int fbits, float* __restrict__ Spart,
                                                        const LoopState* st, int eval_only) {
    if (pass_skip(st, eval_only)) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (j >= n) return;
    const int s = j / seglen, jj = j - s * seglen, L4 = seglen / 4;
    const size_t off = (size_t)c * seglen + (size_t)(jj & 3) * L4 + (jj >> 2);
    unsigned long long acc = 0ull;
    for (int it = seg_item[s]; it < seg_item[s + 1]; ++it) acc += Cpart[(size_t)it * k * seglen + off];
    const double scale = (double)fixed_scale(st, fbits);
    Spart[((size_t)nseg * k + c) * n + j] = (float)((double)(long long)acc / scale);
}

using SymFn = void (*)(SymArgs);

SymFn sym_fn(int k, bool lab_smem) {
    if (k <= 4) return lab_smem ? reduce_sym_kernel<4, 4, true> : reduce_sym_kernel<4, 4, false>;
    if (k <= 8) return lab_smem ? reduce_sym_kernel<8, 4, true> : reduce_sym_kernel<8, 4, false>;
    return lab_smem ? reduce_sym_kernel<0, 4, true> : reduce_sym_kernel<0, 4, false>;
}

}  // namespace

cudaError_t configure_reduce_sym(int smem_optin, int* usable) {
    size_t st = 0;
    for (int kk : {4, 8, 16})
        for (int ls = 0; ls < 2; ++ls) {
            cudaFuncAttributes fa;
            cudaError_t e = cudaFuncGetAttributes(&fa, sym_fn(kk, ls != 0));
            if (e != cudaSuccess) return e;
            if (fa.sharedSizeBytes > st) st = fa.sharedSizeBytes;
        }
    const int bytes = optin_minus_static(smem_optin, st);
    for (int kk : {4, 8, 16})
        for (int ls = 0; ls < 2; ++ls) {
            cudaError_t e = cudaFuncSetAttribute(sym_fn(kk, ls != 0), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
        }
    *usable = bytes;
    return cudaSuccess;
}

// Segment length, shared memory and the item list (host side, once per fit).
SymPlan plan_reduce_sym(int n, int k, int num_sms, int smem_budget) {
    SymPlan p{};
    p.warps = kReduceMaxWarps;
    const size_t nlab = ((size_t)n + 15) & ~(size_t)15;
    const size_t rowacc = (size_t)p.warps * k * 32 * 4;
    // labels in shared memory when a useful segment still fits beside them
    p.labels_in_smem = nlab + rowacc + (size_t)k * 1024 * 8 <= (size_t)smem_budget;
    const size_t base = (p.labels_in_smem ? nlab : 0) + rowacc;
    if (base + (size_t)k * 128 * 8 > (size_t)smem_budget) return p;   // ok = false: k too large
    long long L = (long long)(((size_t)smem_budget - base) / ((size_t)k * 8)) / 128 * 128;
    const long long npad = (n + 127) / 128 * 128;
    if (L > 8192) L = 8192;
    if (L > npad) L = npad;
    p.seglen = (int)L;
    p.nseg = (int)((n + L - 1) / L);
    p.smem = base + (size_t)k * L * 8;
    int lg = 0;
    while ((1LL << lg) < (long long)n) ++lg;
    p.fbits = 61 - lg;
    // items: per segment, runs of row blocks of about equal work (elements read),
    // about three items per CTA in all
    const int T = (n + 127) / 128;
    std::vector<double> seg_work(p.nseg, 0.0);
    double total = 0.0;
    for (int s = 0; s < p.nseg; ++s) {
        const long long c0 = (long long)s * L, c1 = std::min<long long>(n, c0 + L);
        for (int r = 0; r < T && 128LL * r < c1; ++r) {
            const double w = 128.0 * (double)(c1 - std::max<long long>(c0, 128LL * r));
            seg_work[s] += w;
        }
        total += seg_work[s];
    }
    const double target = total / (3.0 * num_sms);
    p.seg_item.assign(p.nseg + 1, 0);
    for (int s = 0; s < p.nseg; ++s) {
        p.seg_item[s] = (int)p.items.size();
        const long long c0 = (long long)s * L, c1 = std::min<long long>(n, c0 + L);
        int r0 = 0;
        double acc = 0.0;
        int r = 0;
        for (; r < T && 128LL * r < c1; ++r) {
            acc += 128.0 * (double)(c1 - std::max<long long>(c0, 128LL * r));
            if (acc >= target) {
                p.items.push_back({s, r0, r + 1, 0});
                r0 = r + 1;
                acc = 0.0;
            }
        }
        if (r0 < r) p.items.push_back({s, r0, r, 0});
    }
    p.seg_item[p.nseg] = (int)p.items.size();
    p.grid = (int)std::min<size_t>((size_t)num_sms, p.items.size());
    p.ok = p.grid > 0;
    return p;
}

cudaError_t launch_reduce_sym(const PassBuffers& b, const SymPlan& p, const int4* d_items, const int* d_seg_item,
                              unsigned long long* Cpart, int eval_only, cudaStream_t s) {
    SymArgs a;
    a.K = static_cast<const float*>(b.K);
    a.ldk = b.ldk;
    a.n = b.n;
    a.k = b.k;
    a.seglen = p.seglen;
    a.nseg = p.nseg;
    a.items = d_items;
    a.nitems = (int)p.items.size();
    a.lab8 = b.lab8;
    a.Spart = b.Spart;
    a.Cpart = Cpart;
    a.fbits = p.fbits;
    a.st = b.st;
    a.eval_only = eval_only;
    sym_fn(b.k, p.labels_in_smem)<<<p.grid, p.warps * 32, p.smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 fg((b.n + 255) / 256, b.k);
    sym_fold_kernel<<<fg, 256, 0, s>>>(Cpart, d_seg_item, b.n, b.k, p.seglen, p.nseg, p.fbits, b.Spart, b.st,
                                        eval_only);
    return cudaGetLastError();
}

}  // namespace popcorn
