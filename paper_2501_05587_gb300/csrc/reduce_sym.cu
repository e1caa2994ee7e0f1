// Symmetric K stream: one pass over the 128 x 128 blocks of K on and above
// the diagonal.
//
// K is symmetric (K = kappa(P P^T), Sec. 3.2).  The segment sums of the
// paper's SpMM (Alg. 2 line 7), S_ic = sum_{j in L_c} K_ij, split by the
// 128-column block J that holds j.  For J >= I (I: the block of row i) the
// part is a row sum of block (I, J); for J < I it equals
// sum_{j in L_c, j in J} K_ji, a column sum of block (J, I).  So one read of
// every block (I, J), I <= J, gives all parts, and a pass reads about half of K.
//
// Work is handed out in super-tiles of a x a blocks (a = 1, 2 or 4): super-tile
// (Is, Js), Is <= Js, of the ceil(T / a)-wide triangle holds the blocks (I, J),
// I <= J, with I in super-row Is and J in super-column Js.  A CTA walks its
// super-tile row by row, so the row sums of a block row accumulate in registers
// over the super-tile's columns and the column sums of a block column in shared
// memory over its rows; each is stored once per super-tile: the row sums of the
// rows of super-row Is to slot Js, the column sums of the rows of super-column Js
// to slot Is (or, for a diagonal super-tile with a > 1, to the extra slot Ts).
// Every (slot, cluster, row) of Spart is written exactly once, and there are
// Ts (+1) slots instead of T: a times fewer slot bytes to write and fold.
//
// reduce_sym_kernel: persistent and warp-specialized, one CTA per SM.  One
//   producer thread loads each block (four 32-column boxes, 128-byte swizzle)
//   and its 2 x 128 labels into a ring 2 or 3 blocks deep: four TMA tensor loads
//   from a full-square K, or one 64 KB bulk copy when K is stored block-packed
//   (upper triangle only, each block already in the box layout: half the
//   memory, and a K build that writes each value once).  The row group (8
//   warps, a lane owns rows) reads its rows as float4 chunks, conflict-free
//   under the swizzle, and adds each element to the sum of its column's
//   cluster.  The column group (8 warps) takes the rows one at a time: a lane
//   holds 4 (k <= 8) or 2 (k <= 16) columns and adds the row to the sums of the
//   row's cluster.  Either way the cluster is a label byte that is the same for
//   the whole warp, so the bucketing of V is a uniform branch into registers: no
//   data-dependent addressing, no atomics.  Each group's warps split its work
//   and their partials are added in a fixed order.  Deterministic.
// sym_fold_kernel: S_ic = the slots summed in slot order (float-float),
//   written to slot 0, the per-block FP64 partials of sum_{i in L_c} S_ic (z,
//   Eq. 14), and in its last block the pass finalization (||c||^2, J).  The
//   assignment then reads slot 0 alone.
#include <cstring>

#include "popcorn_internal.cuh"
#include "stream_common.cuh"
#include "tc_common.cuh"

namespace popcorn {
namespace {

using namespace stream;

constexpr int kB = 128;                        // block edge
constexpr int kBoxCols = 32;                   // TMA box: 32 floats (one 128-byte swizzle row) x 128 rows
constexpr int kBoxBytes = kBoxCols * kB * 4;   // 16 KB
constexpr int kTileBytes = 4 * kBoxBytes;      // 64 KB: one block
constexpr int kGroup = 256;                    // threads of the row group and of the column group
constexpr int kSymThreads = 2 * kGroup + 32;   // + the producer warp
constexpr int kConsumerWarps = 2 * kGroup / 32;
constexpr int kBarRows = 1, kBarCols = 2;      // named barriers of the two groups
constexpr int kFoldThreads = 256;
constexpr int kMaxA = 4;                       // largest super-tile edge

constexpr int align128(int x) { return (x + 127) & ~127; }

// Register shapes by cluster bound KB (4, 8 or 16).
template <int KB>
struct SymShape {
    static constexpr int rpl = KB <= 4 ? 4 : 2;        // rows per lane in the row group
    static constexpr int nparts = 8 * rpl / 4;         // column parts of the row group (8 warps)
    static constexpr int cpl = KB <= 8 ? 4 : 2;        // columns per lane in the column group
    static constexpr int cparts = cpl == 4 ? 8 : 4;    // row parts of the column group
};

// Dynamic shared memory, in order: the block ring (1024-byte aligned for the
// swizzle), the label ring (row labels, then column labels), the two groups'
// partial sums, the column accumulators of a super-tile ([a][KB][128]),
// barriers and the abort flag.
struct SymLayout {
    int labels, rowpart, colpart, colacc, bars, flag, bytes;
};

template <int KB>
SymLayout sym_layout(int stages, int a) {
    using Sh = SymShape<KB>;
    SymLayout L;
    L.labels = stages * kTileBytes;
    L.rowpart = align128(L.labels + stages * 2 * kB);
    L.colpart = align128(L.rowpart + Sh::nparts * KB * kB * 4);
    L.colacc = align128(L.colpart + Sh::cparts * KB * kB * 4);
    L.bars = align128(L.colacc + a * KB * kB * 4);
    L.flag = L.bars + 2 * stages * 8;
    L.bytes = L.flag + 16 + 1024;   // + slack for the 1024-byte alignment
    return L;
}

struct SymArgs {
    const float* Kp;           // block-packed K (one bulk copy per block), or null: TMA from the full square
    int64_t ldk;
    int n, k, T, nlab;
    int a, Ts;                 // super-tile edge in blocks, super-tiles per side
    long long units;           // super-tiles on and above the diagonal
    int stages;
    int off_labels, off_rowpart, off_colpart, off_colacc, off_bars, off_flag;
    const uint8_t* lab8;
    float* Spart;              // [nslots][k][n]
    const LoopState* st;
    int* err;
    int eval_only;
};

// 16 bytes at (row r, 16-byte chunk j) of a 32-column box under the 128-byte
// swizzle (chunk j of row r sits at chunk j ^ (r mod 8)); xr = r mod 8
__device__ __forceinline__ ulonglong2 box_ld(const unsigned char* box, int r, int j, int xr) {
    return *reinterpret_cast<const ulonglong2*>(box + r * 128 + ((j ^ xr) << 4));
}

// acc[c] += v for the one c equal to the warp-uniform label l (nothing for l
// outside [0, KB)): a uniform branch, no one-hot arithmetic
template <int KB, typename T, typename F>
__device__ __forceinline__ void add_to_cluster(int l, T (&acc)[KB], F&& add) {
    switch (l) {
#define POPCORN_SYM_CASE(c) \
    case c:                 \
        if (c < KB) add(acc[c < KB ? c : 0]); \
        break;
        POPCORN_SYM_CASE(0)
        POPCORN_SYM_CASE(1)
        POPCORN_SYM_CASE(2)
        POPCORN_SYM_CASE(3)
        POPCORN_SYM_CASE(4)
        POPCORN_SYM_CASE(5)
        POPCORN_SYM_CASE(6)
        POPCORN_SYM_CASE(7)
        POPCORN_SYM_CASE(8)
        POPCORN_SYM_CASE(9)
        POPCORN_SYM_CASE(10)
        POPCORN_SYM_CASE(11)
        POPCORN_SYM_CASE(12)
        POPCORN_SYM_CASE(13)
        POPCORN_SYM_CASE(14)
        POPCORN_SYM_CASE(15)
#undef POPCORN_SYM_CASE
        default:
            break;
    }
}

// The blocks of super-tile (Is, Js): rows I0 <= I < I1, columns max(I, J0) <= J < J1.
struct Unit {
    int Is, Js, I0, I1, J0, J1;
};
__device__ __forceinline__ Unit unit_of(long long u, const SymArgs& a) {
    Unit t;
    tri_coords(u, a.Ts, &t.Is, &t.Js);
    t.I0 = t.Is * a.a;
    t.I1 = min(t.I0 + a.a, a.T);
    t.J0 = t.Js * a.a;
    t.J1 = min(t.J0 + a.a, a.T);
    return t;
}

template <int KB>
__global__ void __launch_bounds__(kSymThreads, 1)
    reduce_sym_kernel(const __grid_constant__ CUtensorMap map, SymArgs a) {
    using Sh = SymShape<KB>;
    static_assert(KB <= 16, "add_to_cluster has 16 cases");
    grid_dependency_wait();   // the labels and the loop state come from the previous pass
    if (pass_skip(a.st, a.eval_only)) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = tc::smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = a.n, k = a.k, S = a.stages;
    auto full_bar = [&](int s) { return sbase + (uint32_t)a.off_bars + 8u * s; };
    auto empty_bar = [&](int s) { return sbase + (uint32_t)a.off_bars + 8u * (S + s); };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_flag);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full_bar(s), 1);
            tc::mbar_init(empty_bar(s), kConsumerWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const long long G = gridDim.x;

    if (warp == kConsumerWarps) {
        // producer: one thread loads block after block (and its labels) into the ring
        if (lane == 0) {
            const uint64_t stream_once = tc::l2_evict_first();   // K is read once per pass
            long long t = 0;
            bool ok = true;
            for (long long u = blockIdx.x; u < a.units && ok; u += G) {
                const Unit w = unit_of(u, a);
                for (int I = w.I0; I < w.I1 && ok; ++I)
                    for (int J = max(I, w.J0); J < w.J1; ++J, ++t) {
                        const int s = (int)(t % S);
                        if (t >= S && !tc::mbar_wait(empty_bar(s), (uint32_t)((t / S) - 1) & 1u, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        const int lbI = min(kB, a.nlab - I * kB), lbJ = min(kB, a.nlab - J * kB);
                        tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)(kTileBytes + lbI + lbJ));
                        const uint32_t dst = sbase + (uint32_t)s * kTileBytes;
                        if (a.Kp) {
                            // the block is stored in exactly the swizzled box layout the loads below produce
                            const long long tri = (long long)I * a.T - (long long)I * (I - 1) / 2 + (J - I);
                            tc::bulk_load_1d_hint(dst, a.Kp + tri * (kB * kB), (uint32_t)kTileBytes, full_bar(s),
                                                  stream_once);
                        } else {
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                tc::tma_load_2d_hint(dst + b * kBoxBytes, &map, J * kB + kBoxCols * b, I * kB,
                                                     full_bar(s), stream_once);
                        }
                        const uint32_t ldst = sbase + (uint32_t)a.off_labels + (uint32_t)s * 2 * kB;
                        tc::bulk_load_1d(ldst, a.lab8 + (size_t)I * kB, (uint32_t)lbI, full_bar(s));
                        tc::bulk_load_1d(ldst + kB, a.lab8 + (size_t)J * kB, (uint32_t)lbJ, full_bar(s));
                    }
            }
            if (*abort_flag) {
                // leaving early: let this thread's copies land before the CTA's memory goes
                // (bounded; the consumers may never have waited for them)
                for (long long t2 = t > S ? t - S : 0; t2 < t; ++t2) {
                    const uint32_t bar = full_bar((int)(t2 % S)), par = (uint32_t)(t2 / S) & 1u;
                    const unsigned long long t0 = tc::globaltimer();
                    while (!tc::mbar_try_wait(bar, par) && tc::globaltimer() - t0 < tc::kWaitLimitNs) {
                    }
                }
            }
        }
        return;
    }

    const uint64_t keep = tc::l2_evict_last();   // the slots are read back by the fold
    const bool rowg = warp < kConsumerWarps / 2;
    const int u = threadIdx.x & (kGroup - 1);   // thread within its group
    const int bar_id = rowg ? kBarRows : kBarCols;
    const int gw = u >> 5;                      // warp within its group
    const int diag_slot = a.Ts;                 // column sums of a diagonal super-tile (a > 1)

    // row group: the 32 four-column chunks are split into NPART parts; a part's 128 rows
    // go to WPR warps, RPL rows a lane (lane + 32 e)
    constexpr int RPL = Sh::rpl, NPART = Sh::nparts, WPR = 4 / RPL, CH = 32 / NPART;
    const int part = gw / WPR;
    const int r0 = 32 * RPL * (gw % WPR) + lane;
    float acc[KB][RPL];   // row group: per cluster, this lane's rows (kept over a block row of a super-tile)

    int t = 0;
    bool alive = true;
    // A group's barrier at the top of block t + 1 also orders the reads of its
    // partials (block t) before their next writes.
    for (long long uu = blockIdx.x; uu < a.units && alive; uu += G) {
        const Unit w = unit_of(uu, a);
        for (int I = w.I0; I < w.I1 && alive; ++I)
            for (int J = max(I, w.J0); J < w.J1; ++J, ++t) {
                const int s = t % S;
                const bool ok = tc::mbar_wait(full_bar(s), (uint32_t)(t / S) & 1u, abort_flag, a.err);
                if (!tc::named_bar_all(bar_id, kGroup, ok)) {   // the group leaves together
                    alive = false;
                    break;
                }
                const unsigned char* tile = smem + (size_t)s * kTileBytes;
                const uint8_t* lab = smem + a.off_labels + s * 2 * kB;
                if (rowg) {
                    // row sums of block I over the columns of block J, accumulated over the
                    // super-tile's columns and stored to slot Js after its last one.  A chunk's
                    // 4 labels come in one broadcast word; one uniform branch per column.
                    const int xr = lane & 7;             // every row this lane reads is r0 mod 8
                    const int cols_left = n - J * kB;    // columns of block J inside K
                    if (J == max(I, w.J0)) {
#pragma unroll
                        for (int e = 0; e < RPL; ++e)
#pragma unroll
                            for (int c = 0; c < KB; ++c) acc[c][e] = 0.f;
                    }
#pragma unroll 2
                    for (int jj = 0; jj < CH; ++jj) {
                        const int q = part * CH + jj;    // chunk: columns 4 q .. 4 q + 3
                        const unsigned char* box = tile + (q >> 3) * kBoxBytes;
                        const uint32_t lw = *reinterpret_cast<const uint32_t*>(lab + kB + 4 * q);
                        float4 v[RPL];
#pragma unroll
                        for (int e = 0; e < RPL; ++e) {
                            const ulonglong2 raw = box_ld(box, r0 + 32 * e, q & 7, xr);
                            v[e] = *reinterpret_cast<const float4*>(&raw);
                        }
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            const int l = 4 * q + x < cols_left ? (int)((lw >> (8 * x)) & 0xffu) : -1;
                            float col[RPL];
#pragma unroll
                            for (int e = 0; e < RPL; ++e) col[e] = (&v[e].x)[x];
                            add_to_cluster<KB>(l, acc, [&](float (&dst)[RPL]) {
#pragma unroll
                                for (int e = 0; e < RPL; ++e) dst[e] += col[e];
                            });
                        }
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(empty_bar(s));   // this warp is done with the stage
                    if (J == w.J1 - 1) {
                        float* prt = reinterpret_cast<float*>(smem + a.off_rowpart);
#pragma unroll
                        for (int c = 0; c < KB; ++c)
#pragma unroll
                            for (int e = 0; e < RPL; ++e) prt[(part * KB + c) * kB + r0 + 32 * e] = acc[c][e];
                        tc::named_bar<kGroup>(kBarRows);
                        if (u < kB && I * kB + u < n) {
                            float* out = a.Spart + (size_t)w.Js * k * n + I * kB + u;
                            for (int c = 0; c < k; ++c) {
                                const float* pp = prt + c * kB + u;
                                float v = pp[0];
#pragma unroll
                                for (int p = 1; p < NPART; ++p) v += pp[p * KB * kB];
                                tc::st_hint(out + (size_t)c * n, v, keep);
                            }
                        }
                    }
                } else {
                    const bool diag = I == J;
                    if (diag && a.a == 1) {
                        // a diagonal block on its own: its row sums already cover it
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(empty_bar(s));
                        continue;
                    }
                    // column sums of block J over the rows of block I, accumulated in shared
                    // memory over the super-tile's rows (colacc[J - J0]) and stored after the
                    // last one: to slot Is, or the extra slot for a diagonal super-tile.  A
                    // diagonal block adds nothing (its row sums cover it).
                    const int rows_left = n - I * kB;
                    float* cpart = reinterpret_cast<float*>(smem + a.off_colpart);
                    if constexpr (Sh::cpl == 4) {
                        // warp gw: rows 16 gw .. 16 gw + 15; lane: columns 4 lane .. 4 lane + 3
                        if (!diag) {
                            const unsigned char* box = tile + (lane >> 3) * kBoxBytes;
                            const int j = lane & 7;
                            unsigned long long pq[KB][2];   // columns (4 lane, +1) and (4 lane + 2, +3)
#pragma unroll
                            for (int c = 0; c < KB; ++c) pq[c][0] = pq[c][1] = 0ull;
#pragma unroll
                            for (int r4 = 0; r4 < 4; ++r4) {
                                const int rb = 16 * gw + 4 * r4;
                                const uint32_t lw = *reinterpret_cast<const uint32_t*>(lab + rb);
                                ulonglong2 v[4];
#pragma unroll
                                for (int x = 0; x < 4; ++x) v[x] = box_ld(box, rb + x, j, (rb + x) & 7);
#pragma unroll
                                for (int x = 0; x < 4; ++x) {
                                    const int l = rb + x < rows_left ? (int)((lw >> (8 * x)) & 0xffu) : -1;
                                    add_to_cluster<KB>(l, pq, [&](unsigned long long (&dst)[2]) {
                                        dst[0] = tc::f2add(dst[0], v[x].x);
                                        dst[1] = tc::f2add(dst[1], v[x].y);
                                    });
                                }
                            }
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(empty_bar(s));
#pragma unroll
                            for (int c = 0; c < KB; ++c) {
                                float x0, y0, x1, y1;
                                tc::f2unpack(pq[c][0], x0, y0);
                                tc::f2unpack(pq[c][1], x1, y1);
                                *reinterpret_cast<float4*>(cpart + (gw * KB + c) * kB + 4 * lane) =
                                    make_float4(x0, y0, x1, y1);
                            }
                        } else {
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(empty_bar(s));
                        }
                    } else {
                        // warp gw: column half gw & 1 (64 columns), rows 32 (gw >> 1) .. + 31;
                        // lane: columns 64 (gw & 1) + 2 lane, + 1
                        const int ch = gw & 1, rq = gw >> 1;
                        if (!diag) {
                            const unsigned char* box = tile + (2 * ch + (lane >> 4)) * kBoxBytes;
                            const int j = (lane & 15) >> 1, half = (lane & 1) * 8;
                            unsigned long long pq[KB];
#pragma unroll
                            for (int c = 0; c < KB; ++c) pq[c] = 0ull;
#pragma unroll 2
                            for (int r4 = 0; r4 < 8; ++r4) {
                                const int rb = 32 * rq + 4 * r4;
                                const uint32_t lw = *reinterpret_cast<const uint32_t*>(lab + rb);
                                unsigned long long v[4];
#pragma unroll
                                for (int x = 0; x < 4; ++x)
                                    v[x] = *reinterpret_cast<const unsigned long long*>(
                                        box + (rb + x) * 128 + ((j ^ ((rb + x) & 7)) << 4) + half);
#pragma unroll
                                for (int x = 0; x < 4; ++x) {
                                    const int l = rb + x < rows_left ? (int)((lw >> (8 * x)) & 0xffu) : -1;
                                    add_to_cluster<KB>(l, pq,
                                                       [&](unsigned long long& dst) { dst = tc::f2add(dst, v[x]); });
                                }
                            }
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(empty_bar(s));
#pragma unroll
                            for (int c = 0; c < KB; ++c) {
                                float x0, y0;
                                tc::f2unpack(pq[c], x0, y0);
                                *reinterpret_cast<float2*>(cpart + (rq * KB + c) * kB + 64 * ch + 2 * lane) =
                                    make_float2(x0, y0);
                            }
                        } else {
                            __syncwarp();
                            if (lane == 0) tc::mbar_arrive(empty_bar(s));
                        }
                    }
                    tc::named_bar<kGroup>(kBarCols);
                    if (u < kB) {
                        // the group's partials in part order, then into the super-tile's accumulator
                        float* ca = reinterpret_cast<float*>(smem + a.off_colacc) + (size_t)(J - w.J0) * KB * kB + u;
                        const bool first = I == w.I0, last = I == min(J, w.I1 - 1);
                        for (int c = 0; c < k; ++c) {
                            float v = 0.f;
                            if (!diag) {
                                const float* pp = cpart + c * kB + u;
                                v = pp[0];
#pragma unroll
                                for (int p = 1; p < Sh::cparts; ++p) v += pp[p * KB * kB];
                            }
                            ca[c * kB] = first ? v : ca[c * kB] + v;
                        }
                        if (last && J * kB + u < n) {
                            const int slot = w.Is == w.Js ? diag_slot : w.Is;
                            float* out = a.Spart + (size_t)slot * k * n + J * kB + u;
                            for (int c = 0; c < k; ++c) tc::st_hint(out + (size_t)c * n, ca[c * kB], keep);
                        }
                    }
                }
            }
    }
}

struct FoldArgs {
    int n, k, nslots;
    float* Spart;
    const uint8_t* lab8;
    double* zpart;             // [gridDim.x][k]
    double* zsum;
    double* cnorm;
    double* invm;
    const int32_t* counts;
    LoopState* st;
    double* J_hist;
    int eval_only;
};

// Block (x, c): rows x * 256 ... of cluster c.
__global__ void __launch_bounds__(kFoldThreads) sym_fold_kernel(FoldArgs a) {
    grid_dependency_wait();   // the slots come from the stream kernel
    LoopState* st = a.st;
    if (pass_skip(st, a.eval_only)) {
        if (a.eval_only && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) st->J_eval = st->J_last;
        return;
    }
    __shared__ double wsum[kFoldThreads / 32];
    __shared__ int am_last;
    const int c = blockIdx.y;
    const int i = blockIdx.x * kFoldThreads + threadIdx.x;
    const int n = a.n;
    double zc = 0.0;
    if (i < n) {
        float* p = a.Spart + (size_t)c * n + i;
        const size_t ss = (size_t)a.k * n;
        // two interleaved float-float sums keep more loads in flight
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        int s = 0;
#pragma unroll 4
        for (; s + 2 <= a.nslots; s += 2) {
            ff_add(h0, l0, p[(size_t)s * ss]);
            ff_add(h1, l1, p[(size_t)(s + 1) * ss]);
        }
        if (s < a.nslots) ff_add(h0, l0, p[(size_t)s * ss]);
        const double S = ((double)h0 + (double)l0) + ((double)h1 + (double)l1);
        *p = (float)S;
        if ((int)a.lab8[i] == c) zc = S;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zc += __shfl_xor_sync(0xffffffffu, zc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = zc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kFoldThreads / 32; ++w) t += wsum[w];
        a.zpart[(size_t)blockIdx.x * a.k + c] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(&st->reduce_ticket, 1u) == gridDim.x * gridDim.y - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    finalize_pass(a.zpart, (int)gridDim.x, a.k, a.counts, a.zsum, a.cnorm, a.invm, st, a.J_hist, a.eval_only);
}

int sym_kb(int k) { return k <= 4 ? 4 : k <= 8 ? 8 : 16; }

SymLayout sym_layout_rt(int kb, int stages, int a) {
    return kb == 4 ? sym_layout<4>(stages, a) : kb == 8 ? sym_layout<8>(stages, a) : sym_layout<16>(stages, a);
}

}  // namespace

cudaError_t configure_reduce_sym(int smem_optin) {
    // every instance may use up to the opt-in limit; plan_reduce_sym keeps each layout within it
    const int bytes = smem_optin;
    cudaError_t e = cudaFuncSetAttribute(reduce_sym_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(reduce_sym_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(reduce_sym_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

SymPlan plan_reduce_sym(int n, int k, int num_sms, int smem_optin, int a_req, int stages_req) {
    SymPlan p{};
    if (k < 1 || k > kSymMaxK || n < 1) return p;
    p.kb = sym_kb(k);
    p.T = (n + kB - 1) / kB;
    // automatic: single blocks (a = 1) with the deepest ring that fits, the configuration
    // measured fastest for k <= 8; a forced super-tile edge takes the deepest ring that fits
    const int A = a_req > 0 ? a_req : 1;
    if (A > kMaxA) return p;
    const int Ts = (p.T + A - 1) / A;
    int cand_s[2] = {3, 2};
    if (stages_req > 0) cand_s[0] = cand_s[1] = stages_req;
    for (int is = 0; is < 2; ++is) {
        const int S = cand_s[is];
        if (S < 2 || S > 3) continue;
        const SymLayout L = sym_layout_rt(p.kb, S, A);
        if (L.bytes > smem_optin) continue;
        p.a = A;
        p.Ts = Ts;
        p.units = (long long)Ts * (Ts + 1) / 2;
        p.stages = S;
        p.smem = (size_t)L.bytes;
        p.nslots = Ts + (A > 1 ? 1 : 0);
        p.items = (long long)p.T * (p.T + 1) / 2;
        p.grid = (int)(p.units < num_sms ? p.units : num_sms);
        p.fold_blocks = (n + kFoldThreads - 1) / kFoldThreads;
        p.ok = true;
        return p;
    }
    return p;
}

cudaError_t launch_reduce_sym(const PassBuffers& b, const SymPlan& p, int* err, int eval_only, cudaStream_t s,
                              cudaEvent_t between) {
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    if (!p.packed && !make_tensor_map_2d(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<void*>(b.K),
                                         (uint64_t)b.n, (uint64_t)b.n, (uint64_t)b.ldk * 4, kBoxCols, kB,
                                         CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorInvalidValue;
    const SymLayout L = sym_layout_rt(p.kb, p.stages, p.a);
    SymArgs a;
    a.Kp = p.packed ? static_cast<const float*>(b.K) : nullptr;
    a.ldk = b.ldk;
    a.n = b.n;
    a.k = b.k;
    a.T = p.T;
    a.nlab = (b.n + 15) & ~15;
    a.a = p.a;
    a.Ts = p.Ts;
    a.units = p.units;
    a.stages = p.stages;
    a.off_labels = L.labels;
    a.off_rowpart = L.rowpart;
    a.off_colpart = L.colpart;
    a.off_colacc = L.colacc;
    a.off_bars = L.bars;
    a.off_flag = L.flag;
    a.lab8 = b.lab8;
    a.Spart = b.Spart;
    a.st = b.st;
    a.err = err;
    a.eval_only = eval_only;
    cudaError_t e;
    if (p.kb == 4)
        e = launch_pdl(reduce_sym_kernel<4>, dim3(p.grid), dim3(kSymThreads), p.smem, s, map, a);
    else if (p.kb == 8)
        e = launch_pdl(reduce_sym_kernel<8>, dim3(p.grid), dim3(kSymThreads), p.smem, s, map, a);
    else
        e = launch_pdl(reduce_sym_kernel<16>, dim3(p.grid), dim3(kSymThreads), p.smem, s, map, a);
    if (e != cudaSuccess) return e;
    if (between && (e = cudaEventRecord(between, s)) != cudaSuccess) return e;
    FoldArgs f;
    f.n = b.n;
    f.k = b.k;
    f.nslots = p.nslots;
    f.Spart = b.Spart;
    f.lab8 = b.lab8;
    f.zpart = b.zpart;
    f.zsum = b.zsum;
    f.cnorm = b.cnorm;
    f.invm = b.invm;
    f.counts = b.counts;
    f.st = b.st;
    f.J_hist = b.J_hist;
    f.eval_only = eval_only;
    return launch_pdl(sym_fold_kernel, dim3((unsigned)p.fold_blocks, (unsigned)b.k), dim3(kFoldThreads), 0, s, f);
}

}  // namespace popcorn
