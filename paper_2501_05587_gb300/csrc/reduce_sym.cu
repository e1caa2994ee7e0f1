// Symmetric K stream: one pass over the 128 x 128 blocks of K on and above
// the diagonal.
//
// K is symmetric (K = kappa(P P^T), Sec. 3.2).  The segment sums of the
// paper's SpMM (Alg. 2 line 7), S_ic = sum_{j in L_c} K_ij, split by the
// 128-column block J that holds j.  For J >= I (I: the block of row i) the
// part is a row sum of block (I, J); for J < I it equals
// sum_{j in L_c, j in J} K_ji, a column sum of block (J, I).  So one read of
// every block (I, J), I <= J, gives all parts, and a pass reads about half of K.
// The parts go to slots of Spart [slot][cluster][row]; every (slot, cluster,
// row) is written exactly once, and sym_fold_kernel adds a row's slots.
//
// Two forms, by the number of clusters.
//
// Branch form (k <= 8), reduce_sym_kernel: persistent and warp-specialized, one
//   CTA per SM, single blocks taken in turn; block (I, J) writes its row sums to
//   slot J of the rows of block I and, off the diagonal, its column sums to slot
//   I of the rows of block J (T slots).  One producer thread loads each block (four
//   32-column boxes, 128-byte swizzle) and its 2 x 128 labels into a ring 3
//   blocks deep (2 for k > 4): four TMA tensor loads from a full-square K, or one
//   64 KB bulk copy when K is stored block-packed (upper triangle only, each block
//   already in the box layout, kPackedSw16).  The row group (8 warps, a lane owns
//   rows) reads its rows as float4 chunks, conflict-free under the swizzle, and
//   adds each element to the sum of its column's cluster.  The column group (8
//   warps) takes the rows one at a time: lane l holds columns 4l..4l+3 and adds
//   the row to the sums of the row's cluster.  Either way the cluster is a label
//   byte that is the same for the whole warp, so the bucketing of V is a uniform
//   branch into registers: no data-dependent addressing, no atomics.
//
// Sorted form (k <= kSymMaxK; also k <= 8 with a forced super-tile edge > 1),
//   sym_sort_kernel + reduce_sym_sorted_kernel: a per-pass stable sort of every
//   128-block's labels into lists of tile offsets, cluster after cluster; super-tiles
//   of a x a blocks, a row warp per block row and a column warp per block column, each
//   walking its blocks' lists with the per-cluster sums in registers over the whole
//   super-tile (the loop over clusters is unrolled): see below.
//
// Every partial is added in a fixed order and stored once: deterministic.
// sym_fold_kernel: S_ic = the slots summed in slot order (float-float), written to
// slot 0, the per-block FP64 partials of sum_{i in L_c} S_ic (z, Eq. 14), and in its
// last block the pass finalization (||c||^2, J).  The assignment then reads slot 0
// alone.
#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

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

constexpr int align128(int x) { return (x + 127) & ~127; }

// ---------------------------------------------------------------------------
// The branch form (k <= 8).

// Dynamic shared memory, in order: the block ring (1024-byte aligned for the
// swizzle), the label ring (row labels, then column labels), the block
// coordinates of each stage, the two groups' partial sums, barriers and the
// abort flag.  KB <= 4 keeps 3 blocks in flight, KB = 8 two.

template <int KB>
struct BranchLayout {
    static constexpr int stages = KB <= 4 ? 3 : 2;
    static constexpr int rpl = KB <= 4 ? 4 : 2;      // rows per lane in the row group
    static constexpr int nparts = 8 * rpl / 4;        // column parts of the row group (8 warps)
    static constexpr int tiles = 0;
    static constexpr int labels = tiles + stages * kTileBytes;
    static constexpr int ij = align128(labels + stages * 2 * kB);
    static constexpr int rowpart = align128(ij + stages * 8);
    static constexpr int colpart = align128(rowpart + nparts * KB * kB * 4);
    static constexpr int bars = align128(colpart + 8 * KB * kB * 4);
    static constexpr int flag = bars + 2 * stages * 8;
    static constexpr int bytes = flag + 16 + 1024;   // + slack for the 1024-byte alignment
};

struct BranchArgs {
    const float* Kp;           // block-packed K (one bulk copy per block), or null: TMA from the full square
    int64_t ldk;
    int n, k, T, nlab;
    long long items;
    const uint8_t* lab8;
    float* Spart;              // [T][k][n]
    const LoopState* st;
    int* err;
    int eval_only;
    // Test hook for the error path (0 in every ordinary launch): CTA 0 never issues the
    // copies of its block number stall_block - 1, so the waits for it run out after
    // wait_ns and the launch reports a timed-out wait.
    int stall_block;
    unsigned long long wait_ns;
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
#undef POPCORN_SYM_CASE
        default:
            break;
    }
}

template <int KB>
__global__ void __launch_bounds__(kSymThreads, 1)
    reduce_sym_kernel(const __grid_constant__ CUtensorMap map, BranchArgs a) {
    using L = BranchLayout<KB>;
    constexpr int S = L::stages;
    static_assert(KB <= 8, "add_to_cluster has 8 cases");
    grid_dependency_wait();   // the labels and the loop state come from the previous pass
    if (pass_skip(a.st, a.eval_only)) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = tc::smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = a.n, k = a.k;
    auto full_bar = [&](int s) { return sbase + L::bars + 8u * s; };
    auto empty_bar = [&](int s) { return sbase + L::bars + 8u * (S + s); };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::flag);
    int2* ij = reinterpret_cast<int2*>(smem + L::ij);
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
    const long long nmine = (long long)blockIdx.x < a.items ? (a.items - 1 - blockIdx.x) / G + 1 : 0;

    if (warp == kConsumerWarps) {
        // producer: one thread loads block after block (and its labels) into the ring
        if (lane == 0) {
            const uint64_t stream_once = tc::l2_evict_first();   // K is read once per pass
            long long t = 0;
            const long long skip = blockIdx.x == 0 ? (long long)a.stall_block - 1 : -1;
            for (; t < nmine; ++t) {
                const int s = (int)(t % S);
                if (t >= S &&
                    !tc::mbar_wait_for(empty_bar(s), (uint32_t)((t / S) - 1) & 1u, abort_flag, a.err, a.wait_ns))
                    break;
                if (t == skip) continue;   // the test hook: this block never arrives
                int I, J;
                tri_coords(blockIdx.x + t * G, a.T, &I, &J);
                ij[s] = make_int2(I, J);   // published by the arrive below (release)
                const int lbI = min(kB, a.nlab - I * kB), lbJ = min(kB, a.nlab - J * kB);
                tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)(kTileBytes + lbI + lbJ));
                const uint32_t dst = sbase + L::tiles + (uint32_t)s * kTileBytes;
                if (a.Kp) {
                    // the block is stored in exactly the swizzled box layout the loads below produce
                    const long long tri = (long long)I * a.T - (long long)I * (I - 1) / 2 + (J - I);
                    tc::bulk_load_1d_hint(dst, a.Kp + tri * (kB * kB), (uint32_t)kTileBytes, full_bar(s), stream_once);
                } else {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        tc::tma_load_2d_hint(dst + b * kBoxBytes, &map, J * kB + kBoxCols * b, I * kB, full_bar(s),
                                             stream_once);
                }
                const uint32_t ldst = sbase + L::labels + (uint32_t)s * 2 * kB;
                tc::bulk_load_1d(ldst, a.lab8 + (size_t)I * kB, (uint32_t)lbI, full_bar(s));
                tc::bulk_load_1d(ldst + kB, a.lab8 + (size_t)J * kB, (uint32_t)lbJ, full_bar(s));
            }
            if (*abort_flag) {
                // leaving early: let this thread's copies land before the CTA's memory goes
                // (bounded; the consumers may never have waited for them)
                for (long long t2 = t > S ? t - S : 0; t2 < t; ++t2) {
                    if (t2 == skip) continue;   // nothing was issued for it
                    const uint32_t bar = full_bar((int)(t2 % S)), par = (uint32_t)(t2 / S) & 1u;
                    const unsigned long long t0 = tc::globaltimer();
                    while (!tc::mbar_try_wait(bar, par) && tc::globaltimer() - t0 < a.wait_ns) {
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
    // A group's barrier at the top of block t + 1 also orders the reads of its
    // partials (block t) before their next writes.
    for (long long t = 0; t < nmine; ++t) {
        const int s = (int)(t % S);
        const bool ok = tc::mbar_wait_for(full_bar(s), (uint32_t)(t / S) & 1u, abort_flag, a.err, a.wait_ns);
        if (!tc::named_bar_all(bar_id, kGroup, ok)) break;   // the group leaves together
        const int2 bij = ij[s];
        const int I = bij.x, J = bij.y;
        const unsigned char* tile = smem + L::tiles + (size_t)s * kTileBytes;
        const uint8_t* lab = smem + L::labels + s * 2 * kB;
        if (rowg) {
            // row sums of block I over the columns of block J -> slot J.  The 32 four-column
            // chunks are split into NPART parts; a part's 128 rows go to WPR warps, RPL rows
            // a lane (lane + 32 e).  A chunk's one-hot weights are built in registers from
            // its 4 labels (one broadcast word), pairs of columns per fma.rn.f32x2.
            constexpr int RPL = L::rpl, NPART = L::nparts, WPR = 4 / RPL, CH = 32 / NPART;
            const int part = gw / WPR;
            const int r0 = 32 * RPL * (gw % WPR) + lane;
            const int xr = lane & 7;             // every row this lane reads is r0 mod 8
            const int cols_left = n - J * kB;    // columns of block J inside K
            float acc[KB][RPL];   // per cluster, this lane's rows
#pragma unroll
            for (int e = 0; e < RPL; ++e)
#pragma unroll
                for (int c = 0; c < KB; ++c) acc[c][e] = 0.f;
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
                    // the column's cluster takes the element of each of this lane's rows (one
                    // uniform branch per column)
                    add_to_cluster<KB>(l, acc, [&](float (&dst)[RPL]) {
#pragma unroll
                        for (int e = 0; e < RPL; ++e) dst[e] += col[e];
                    });
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(empty_bar(s));   // this warp is done with the stage
            float* prt = reinterpret_cast<float*>(smem + L::rowpart);
#pragma unroll
            for (int c = 0; c < KB; ++c)
#pragma unroll
                for (int e = 0; e < RPL; ++e) {
                    prt[(part * KB + c) * kB + r0 + 32 * e] = acc[c][e];
                }
            tc::named_bar<kGroup>(kBarRows);
            if (u < kB && I * kB + u < n) {
                float* out = a.Spart + (size_t)J * k * n + I * kB + u;
                for (int c = 0; c < k; ++c) {
                    const float* pp = prt + c * kB + u;
                    float v = pp[0];
#pragma unroll
                    for (int p = 1; p < NPART; ++p) v += pp[p * KB * kB];
                    tc::st_hint(out + (size_t)c * n, v, keep);
                }
            }
        } else if (I == J) {
            // a diagonal block: its row sums already cover it
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(empty_bar(s));
        } else {
            // column sums of block J over the rows of block I -> slot I.  Warp gw: rows
            // 16 gw .. 16 gw + 15; lane: columns 4 lane .. 4 lane + 3.  A row's one-hot
            // weight comes from its label (a broadcast word per 4 rows), in registers.
            const unsigned char* box = tile + (lane >> 3) * kBoxBytes;
            const int j = lane & 7;
            const int rows_left = n - I * kB;
            unsigned long long pq[KB][2];   // columns (4 lane, 4 lane + 1) and (4 lane + 2, 4 lane + 3)
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
                    // the row's cluster takes the row
                    add_to_cluster<KB>(l, pq, [&](unsigned long long (&dst)[2]) {
                        dst[0] = tc::f2add(dst[0], v[x].x);
                        dst[1] = tc::f2add(dst[1], v[x].y);
                    });
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(empty_bar(s));
            // the 8 warps' partials, added in warp order
            float* part = reinterpret_cast<float*>(smem + L::colpart);
#pragma unroll
            for (int c = 0; c < KB; ++c) {
                float x0, y0, x1, y1;
                tc::f2unpack(pq[c][0], x0, y0);
                tc::f2unpack(pq[c][1], x1, y1);
                *reinterpret_cast<float4*>(part + (gw * KB + c) * kB + 4 * lane) = make_float4(x0, y0, x1, y1);
            }
            tc::named_bar<kGroup>(kBarCols);
            if (u < kB && J * kB + u < n) {
                float* out = a.Spart + (size_t)I * k * n + J * kB + u;
                for (int c = 0; c < k; ++c) {
                    const float* pp = part + c * kB + u;
                    float v = pp[0];
#pragma unroll
                    for (int w = 1; w < 8; ++w) v += pp[w * KB * kB];
                    tc::st_hint(out + (size_t)c * n, v, keep);
                }
            }
        }
    }
}

// The blocks of super-tile (Is, Js): block rows I0 <= I < I0 + a, block columns
// J0 <= J < J0 + a, those with I <= J < T.
struct Unit {
    int Is, Js, I0, J0;
};
__device__ __forceinline__ Unit unit_of(long long u, int a, int Ts) {
    Unit t;
    tri_coords(u, Ts, &t.Is, &t.Js);
    t.I0 = t.Is * a;
    t.J0 = t.Js * a;
    return t;
}

// ---------------------------------------------------------------------------
// The sorted form of the symmetric pass (k <= kSymMaxK).
//
// Per pass, sym_sort_kernel sorts the points of every 128-block by label (stable) and
// writes two lists for the block: the byte offsets of its points as columns of a tile
// (column list) and as rows of a tile (row list), cluster after cluster, each cluster's
// entries padded to a multiple of 4, after a header with each cluster's start and count.
//
// The stream takes super-tiles of a x a blocks, one per CTA at a time.  The rows of
// block row I0 + i are owned by 4 / R row warps (lane l of part h: rows
// l + 32 (R h + e), e < R), the columns of block column J0 + j by 4 / R column warps
// the same way.  On its block (I, J) a row warp walks the column list of J cluster by
// cluster: the columns of cluster c are added into one register per row, and that
// into acc[c][e], the row's running sum for c -- a register, since the loop over the
// clusters is unrolled up to KMAX.  A column warp walks the row list of I the same
// way.  The inner loop is a load of 4 list entries, per entry one XOR for the element
// offset, and per row (column) a shared-memory load and an add (f32x2, two rows a
// time): no run-end test, no register indexed by data, no shared-memory accumulator.
// The sums stay in registers over the super-tile and are stored once per row and
// cluster (slots shrink a-fold).
// All consumer warps wait for and release every block of the ring (the two that own it
// after their work), so no warp runs a phase ahead of another.
//
// K is packed in the XOR-32 layout (kPackedSw4): element c of row r of a box at
// c ^ (r mod 32), so the 32 rows of a column and the 32 columns of a row sit in 32
// different banks.  In bytes, element (r, C) of the tile is at
//   16384 (C >> 5) + 128 r + 4 ((C & 31) ^ (r & 31)).
// Column C's list entry is 16384 (C >> 5) + 4 (C & 31); for row r = l + 32 e of lane l
// the offset is (entry ^ 132 l) + 4096 e.  Row r's list entry is 128 r + 4 (r & 31); for
// column C = l + 32 e of lane l it is (entry ^ 4 l) + 16384 e.
constexpr int kSortHdr = 128;   // bytes: u32 per cluster c < 32, (start << 8) | count
// Rows (columns) a lane owns in a block: 2, i.e. two warps share a block row (column) --
// measured on the images workload (n = 70,000, k = 10): 1.67 ms a stream at a = 4 against
// 2.04 ms with 4 rows a lane at a = 8 (a block's two owners take half as long, so its
// ring stage comes back sooner).
constexpr int kSortedRowsPerLane = 2;

// Entries of one list: every cluster padded to a multiple of 4, plus one chunk of 4
// that the loop below may read ahead (never used).
__host__ __device__ constexpr int sort_list_len(int k) { return ((kB + 3 * k + 3) & ~3) + 4; }
__host__ __device__ constexpr int sort_meta_bytes(int k) { return kSortHdr + 4 * sort_list_len(k); }

__global__ void __launch_bounds__(kB) sym_sort_kernel(const uint8_t* __restrict__ lab8, int n, int k, uint8_t* metaC,
                                                      uint8_t* metaR, const LoopState* st, int eval_only) {
    grid_dependency_wait();   // the labels come from the previous pass
    if (pass_skip(st, eval_only)) return;
    __shared__ uint8_t lab[kB];
    __shared__ int cnt[kSymMaxK], start[kSymMaxK];
    __shared__ uint32_t cc[sort_list_len(kSymMaxK)], rc[sort_list_len(kSymMaxK)];
    const int b = blockIdx.x, t = threadIdx.x;
    const int i = b * kB + t;
    const int L = sort_list_len(k);
    // points past n (and, defensively, a label outside [0, k)) get no entry
    const int l = (i < n && (int)lab8[i] < k) ? (int)lab8[i] : 0xFF;
    lab[t] = (uint8_t)l;
    for (int e = t; e < L; e += kB) cc[e] = rc[e] = 0u;   // padding entries: offset 0, never added
    __syncthreads();
    int rank = 0;   // equal labels before this point (stable order)
    for (int u = 0; u < t; ++u) rank += lab[u] == l;
    if (t < k) {
        int m = 0;
        for (int u = 0; u < kB; ++u) m += lab[u] == t;
        cnt[t] = m;
    }
    __syncthreads();
    if (t < k) {
        int p = 0;
        for (int c = 0; c < t; ++c) p += (cnt[c] + 3) & ~3;
        start[t] = p;
    }
    __syncthreads();
    if (l != 0xFF) {
        const int pos = start[l] + rank;
        cc[pos] = (uint32_t)(16384 * (t >> 5) + 4 * (t & 31));
        rc[pos] = (uint32_t)(128 * t + 4 * (t & 31));
    }
    __syncthreads();
    uint32_t* hC = reinterpret_cast<uint32_t*>(metaC + (size_t)b * sort_meta_bytes(k));
    uint32_t* hR = reinterpret_cast<uint32_t*>(metaR + (size_t)b * sort_meta_bytes(k));
    if (t < kSortHdr / 4) {
        const uint32_t h = t < k ? ((uint32_t)start[t] << 8) | (uint32_t)cnt[t] : 0u;
        hC[t] = h;
        hR[t] = h;
    }
    for (int e = t; e < L; e += kB) {
        hC[kSortHdr / 4 + e] = cc[e];
        hR[kSortHdr / 4 + e] = rc[e];
    }
}

struct SortedArgs {
    const float* Kp;           // block-packed K, kPackedSw4 layout
    int n, k, T, a, Ts;
    long long units;
    int stages, stage_bytes, meta_bytes, off_bars;
    const uint8_t* metaC;      // [T][meta_bytes] column lists
    const uint8_t* metaR;      // [T][meta_bytes] row lists
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

// The lane's R rows (STRIDE 4096: rows 32 e apart) or columns (STRIDE 16384) of one
// tile, added cluster by cluster along a list: acc[c][e] += the elements of the list
// entries of cluster c.
template <int KMAX, int R, int STRIDE>
__device__ __forceinline__ void sum_sorted(const unsigned char* __restrict__ tile, const uint32_t* __restrict__ hdr,
                                           int k, uint32_t key, float (&acc)[KMAX][R]) {
    const uint32_t* __restrict__ codes = hdr + kSortHdr / 4;
    auto ld = [&](uint32_t entry, int e) {
        return *reinterpret_cast<const float*>(tile + (entry ^ key) + STRIDE * e);
    };
#pragma unroll
    for (int c = 0; c < KMAX; ++c) {
        if (c < k) {
            const uint32_t h = hdr[c];
            const int p0 = (int)(h >> 8), cnt = (int)(h & 0xffu);
            const int pe = p0 + (cnt & ~3);
            float s[R];
#pragma unroll
            for (int e = 0; e < R; ++e) s[e] = 0.f;
            uint4 cw = *reinterpret_cast<const uint4*>(codes + p0);
#pragma unroll 1
            for (int p = p0; p < pe; p += 4) {
                const uint4 cur = cw;
                cw = *reinterpret_cast<const uint4*>(codes + p + 4);   // the next chunk (or the tail)
#pragma unroll
                for (int e = 0; e < R; e += 2) {
                    // rows (columns) e and e + 1 as one f32x2 pair: half the add instructions
                    const unsigned long long w0 = tc::f2pack(ld(cur.x, e), ld(cur.x, e + 1));
                    const unsigned long long w1 = tc::f2pack(ld(cur.y, e), ld(cur.y, e + 1));
                    const unsigned long long w2 = tc::f2pack(ld(cur.z, e), ld(cur.z, e + 1));
                    const unsigned long long w3 = tc::f2pack(ld(cur.w, e), ld(cur.w, e + 1));
                    float x, y;
                    tc::f2unpack(tc::f2add(tc::f2add(w0, w1), tc::f2add(w2, w3)), x, y);
                    const unsigned long long t = tc::f2add(tc::f2pack(s[e], s[e + 1]), tc::f2pack(x, y));
                    tc::f2unpack(t, s[e], s[e + 1]);
                }
            }
            const int rem = cnt & 3;   // the last 1-3 entries of the cluster (uniform)
            if (rem) {
#pragma unroll
                for (int e = 0; e < R; ++e) {
                    float v = ld(cw.x, e);
                    if (rem > 1) v += ld(cw.y, e);
                    if (rem > 2) v += ld(cw.z, e);
                    s[e] += v;
                }
            }
#pragma unroll
            for (int e = 0; e < R; ++e) acc[c][e] += s[e];
        }
    }
}

// Register sums per lane (P R KMAX) against the register file: an SM sub-partition holds
// 16384 registers for its share of the CTA's warps (2a (4 / R) / P consumers + 1), so the
// widest super-tile edge with 4 rows a lane is 8 for KMAX = 12 (96 registers a thread),
// 7 for 16 (128) and 3 for 32 (255); with 2 rows a lane (two warps share a block row or
// column) it is 4 for KMAX <= 16 (96) and 3 for 32 (128), and 8 for KMAX = 12 when each
// warp owns two block rows (columns) of the super-tile (P = 2: rows i and i + a / 2).
__host__ __device__ constexpr int sorted_max_a(int kmax, int rpl, int pw = 1) {
    return rpl == 4 ? (kmax <= 12 ? 8 : kmax <= 16 ? 7 : 3)
                    : (pw == 2 ? (kmax <= 12 ? 8 : 0) : (kmax <= 16 ? 4 : 3));
}
__host__ __device__ constexpr int sorted_threads(int a, int rpl, int pw = 1) {
    return 32 * (2 * a * (4 / rpl) / pw + 1);
}

template <int KMAX, int R, int P>
__global__ void __launch_bounds__(sorted_threads(sorted_max_a(KMAX, R, P), R, P), 1)
    reduce_sym_sorted_kernel(SortedArgs a) {
    grid_dependency_wait();   // the block lists and the loop state come from before this pass
    if (pass_skip(a.st, a.eval_only)) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const uint32_t sbase = tc::smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int H = 4 / R;   // warps per block row (column)
    const int A = a.a, nw = 2 * A * H / P, S = a.stages;
    const int AP = A / P;      // a warp owns block rows (columns) mine + AP q, q < P
    const int n = a.n, k = a.k, T = a.T;
    auto full_bar = [&](int s) { return sbase + (uint32_t)a.off_bars + 8u * s; };
    auto empty_bar = [&](int s) { return sbase + (uint32_t)a.off_bars + 8u * (S + s); };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + a.off_bars + 16 * S);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full_bar(s), 1);
            tc::mbar_init(empty_bar(s), (uint32_t)nw);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long G = gridDim.x;
    // the blocks of a super-tile in a Latin-square order: consecutive blocks lie in
    // different block rows and block columns, so the blocks in the ring keep different
    // row and column warps busy
    auto block_of = [&](const Unit& w, int m, int i, int* I, int* J) {
        const int jj = i + m < A ? i + m : i + m - A;
        *I = w.I0 + i;
        *J = w.J0 + jj;
        return *I < T && *J < T && *J >= *I;
    };

    if (warp == nw) {
        // producer: one thread bulk-copies each block and the lists of its column and row blocks
        if (lane == 0) {
            const uint64_t stream_once = tc::l2_evict_first();   // K is read once per pass
            const long long skip = blockIdx.x == 0 ? (long long)a.stall_block - 1 : -1;
            long long t = 0;
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (long long u = blockIdx.x; u < a.units && ok; u += G) {
                const Unit w = unit_of(a.order ? a.order[u] : u, A, a.Ts);
                for (int m = 0; m < A && ok; ++m)
                    for (int i = 0; i < A; ++i) {
                        int I, J;
                        if (!block_of(w, m, i, &I, &J)) continue;
                        if (t >= S && !tc::mbar_wait_for(empty_bar(s), ph ^ 1u, abort_flag, a.err, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        if (t == skip) {   // the test hook: this block never arrives
                            ++t;
                            if (++s == S) {
                                s = 0;
                                ph ^= 1u;
                            }
                            continue;
                        }
                        tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)(kTileBytes + 2 * a.meta_bytes));
                        const uint32_t dst = sbase + (uint32_t)s * (uint32_t)a.stage_bytes;
                        const long long tri = (long long)I * T - (long long)I * (I - 1) / 2 + (J - I);
                        tc::bulk_load_1d_hint(dst, a.Kp + tri * (kB * kB), (uint32_t)kTileBytes, full_bar(s),
                                              stream_once);
                        tc::bulk_load_1d(dst + kTileBytes, a.metaC + (size_t)J * a.meta_bytes, (uint32_t)a.meta_bytes,
                                         full_bar(s));
                        tc::bulk_load_1d(dst + kTileBytes + a.meta_bytes, a.metaR + (size_t)I * a.meta_bytes,
                                         (uint32_t)a.meta_bytes, full_bar(s));
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
        return;
    }

    const uint64_t keep = tc::l2_evict_last();   // the slots are read back by the fold
    const bool roww = warp < AP * H;
    const int wr = roww ? warp : warp - AP * H;
    const int mine = wr / H;          // block row (column) of the super-tile, + AP q
    const int part = wr % H;          // this warp's rows (columns): 32 (R part + e) + lane, e < R
    const uint32_t key = roww ? 132u * (uint32_t)lane : 4u * (uint32_t)lane;
    int s = 0;
    uint32_t ph = 0;
    bool alive = true;
    for (long long u = blockIdx.x; u < a.units && alive; u += G) {
        const Unit w = unit_of(a.order ? a.order[u] : u, A, a.Ts);
        float acc[P][KMAX][R];
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int c = 0; c < KMAX; ++c)
#pragma unroll
                for (int e = 0; e < R; ++e) acc[q][c][e] = 0.f;
        for (int m = 0; m < A && alive; ++m)
            for (int i = 0; i < A; ++i) {
                int I, J;
                if (!block_of(w, m, i, &I, &J)) continue;
                if (!tc::mbar_wait_for(full_bar(s), ph, abort_flag, a.err, a.wait_ns)) {
                    alive = false;
                    break;
                }
                const unsigned char* stage = smem + (size_t)s * a.stage_bytes;
                // the accumulator set of this block row (column) when this warp owns it
                const int x = roww ? i : J - w.J0;
                const int q = x / AP;
                if (x - AP * q == mine && (roww || I != J)) {
                    // row warps: row sums of block I over the columns of block J, by the column
                    // list of J; column warps: column sums of block J over the rows of block I,
                    // by the row list of I (a diagonal block's row sums already cover it)
                    const unsigned char* tile = stage + (roww ? 4096 : 16384) * R * part;
                    const uint32_t* hdr =
                        reinterpret_cast<const uint32_t*>(stage + kTileBytes + (roww ? 0 : a.meta_bytes));
                    if (roww) {
                        if (P == 1 || q == 0)
                            sum_sorted<KMAX, R, 4096>(tile, hdr, k, key, acc[0]);
                        else
                            sum_sorted<KMAX, R, 4096>(tile, hdr, k, key, acc[P - 1]);
                    } else {
                        if (P == 1 || q == 0)
                            sum_sorted<KMAX, R, 16384>(tile, hdr, k, key, acc[0]);
                        else
                            sum_sorted<KMAX, R, 16384>(tile, hdr, k, key, acc[P - 1]);
                    }
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(empty_bar(s));
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        if (!alive) break;
        // one store per row (column) and cluster: row sums to slot Js of the rows of block
        // row I; column sums to slot Is of the rows of block column J, or to the extra slot
        // Ts from a super-tile on the diagonal (its rows also take row sums into slot Js)
        const int slot = roww ? w.Js : (w.Is == w.Js ? a.Ts : w.Is);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int X = (roww ? w.I0 : w.J0) + mine + AP * q;
            if (X < T) {
                const int r0 = X * kB + 32 * R * part + lane;   // this lane's rows (columns): r0 + 32 e
                float* out = a.Spart + (size_t)slot * k * n + r0;
#pragma unroll
                for (int c = 0; c < KMAX; ++c) {
                    if (c < k) {
#pragma unroll
                        for (int e = 0; e < R; ++e)
                            if (r0 + 32 * e < n) tc::st_hint(out + (size_t)c * n + 32 * e, acc[q][c][e], keep);
                    }
                }
            }
        }
    }
}

// Dynamic shared memory of the sorted form, in order: the ring of stages (a 64 KB tile,
// the column list of its block column, the row list of its block row), barriers and the
// abort flag.
struct SortedLayout {
    int stage_bytes, meta_bytes, bars, bytes;
};
SortedLayout sorted_layout(int k, int stages) {
    SortedLayout L;
    L.meta_bytes = sort_meta_bytes(k);
    L.stage_bytes = kTileBytes + 2 * L.meta_bytes;
    L.bars = stages * L.stage_bytes;
    L.bytes = L.bars + 16 * stages + 16 + 128;   // + slack for the 128-byte alignment
    return L;
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

}  // namespace

cudaError_t configure_reduce_sym(int smem_optin) {
    // every instance may use up to the opt-in limit; plan_reduce_sym keeps each layout within it
    const int bytes = smem_optin;
    cudaError_t e = cudaFuncSetAttribute(reduce_sym_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(reduce_sym_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    void (*sorted[7])(SortedArgs) = {reduce_sym_sorted_kernel<12, 4, 1>, reduce_sym_sorted_kernel<16, 4, 1>,
                                     reduce_sym_sorted_kernel<32, 4, 1>, reduce_sym_sorted_kernel<12, 2, 1>,
                                     reduce_sym_sorted_kernel<16, 2, 1>, reduce_sym_sorted_kernel<32, 2, 1>,
                                     reduce_sym_sorted_kernel<12, 2, 2>};
    for (auto f : sorted)
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

SymPlan plan_reduce_sym(int n, int k, int num_sms, int smem_optin, int a_req, int stages_req, int ebytes) {
    SymPlan p{};
    if (k < 1 || k > kSymMaxK || n < 1 || (ebytes != 4 && ebytes != 2)) return p;
    p.ebytes = ebytes;
    p.T = (n + kB - 1) / kB;
    p.items = (long long)p.T * (p.T + 1) / 2;
    p.fold_blocks = (n + kFoldThreads - 1) / kFoldThreads;
    // an FP16 / BF16 K: the tensor-core form (reduce_sym_mma.cu)
    if (ebytes == 2) {
        if (!plan_sym_mma(&p, k, num_sms, smem_optin, a_req, stages_req)) p.ok = false;
        return p;
    }
    // the branch form (k <= 8, single blocks) when asked for with a super-tile edge of 1;
    // otherwise the sorted form (measured faster on the rings workload too: 0.152 ms a
    // stream against 0.160)
    if (k <= kSymBranchMaxK && a_req == 1) {
        const int bytes = k <= 4 ? BranchLayout<4>::bytes : BranchLayout<8>::bytes;
        if (bytes > smem_optin) return p;
        p.sorted = false;
        p.kb = k <= 4 ? 4 : 8;
        p.layout = kPackedSw16;
        p.a = 1;
        p.Ts = p.T;
        p.units = p.items;
        p.stages = k <= 4 ? BranchLayout<4>::stages : BranchLayout<8>::stages;
        p.smem = (size_t)bytes;
        p.nslots = p.T;
        p.grid = (int)(p.items < num_sms ? p.items : num_sms);
        p.meta_bytes = 0;
        p.ok = true;
        return p;
    }
    p.sorted = true;
    p.kb = k <= 12 ? 12 : k <= 16 ? 16 : 32;   // register sums a lane: KMAX clusters x 4 rows
    p.layout = kPackedSw4;
    // the widest super-tile whose consumer warps fit the register file and that leaves at
    // least 4 super-tiles per SM for balance
    p.rpl = kSortedRowsPerLane;
    // edges above 4 with 2 rows a lane: each warp owns two block rows (columns), even edges only
    auto pw_of = [&](int A) { return p.rpl == 2 && A > 4 ? 2 : 1; };
    auto fits = [&](int A) {
        const int pw = pw_of(A);
        return A >= 1 && A % pw == 0 && A <= sorted_max_a(p.kb, p.rpl, pw);
    };
    // automatic: 4 x 4 at most with 2 rows a lane -- the 8 x 8 form (two block rows a warp)
    // halves the slots but measured slower on images (stream 1.94 ms against 1.70 ms, fold
    // 0.059 against 0.089), so it runs only when asked for
    int cand_a[6] = {8, 7, 4, 3, 2, 1}, na = 6;
    if (p.rpl == 2) cand_a[0] = cand_a[1] = 4;
    if (a_req > 0) {
        cand_a[0] = a_req;
        na = 1;
    }
    for (int ia = 0; ia < na; ++ia) {
        const int A = cand_a[ia];
        if (!fits(A)) continue;
        const int Ts = (p.T + A - 1) / A;
        const long long units = (long long)Ts * (Ts + 1) / 2;
        // at least 8 super-tiles an SM, so the static round-robin stays near balance (rings,
        // n = 20,000: edge 3 with 9.4 a SM streams in 0.145 ms, edge 4 with 5.4 in 0.154)
        if (a_req == 0 && A > 1 && units < 8LL * num_sms) continue;
        int cand_s[2] = {3, 2};
        if (stages_req > 0) cand_s[0] = cand_s[1] = stages_req;
        for (int is = 0; is < 2; ++is) {
            const int S = cand_s[is];
            if (S < 2 || S > 3) continue;
            const int bytes = sorted_layout(k, S).bytes;
            if (bytes > smem_optin) continue;
            p.a = A;
            p.pw = pw_of(A);
            p.Ts = Ts;
            p.units = units;
            p.stages = S;
            p.smem = (size_t)bytes;
            p.nslots = Ts + 1;
            p.grid = (int)(units < num_sms ? units : num_sms);
            p.meta_bytes = 2 * (size_t)p.T * sort_meta_bytes(k);
            p.ok = true;
            return p;
        }
    }
    return p;
}

void sym_unit_order(const SymPlan& p, std::vector<int>* order) {
    // blocks (I, J), J >= I, of super-tile (Is, Js) inside the T x T block triangle
    std::vector<std::pair<int, int>> size_id;
    size_id.reserve((size_t)p.units);
    long long u = 0;
    for (int Is = 0; Is < p.Ts; ++Is)
        for (int Js = Is; Js < p.Ts; ++Js, ++u) {
            int blocks = 0;
            for (int I = Is * p.a; I < (Is + 1) * p.a && I < p.T; ++I)
                for (int J = Js * p.a; J < (Js + 1) * p.a && J < p.T; ++J) blocks += J >= I;
            size_id.push_back({-blocks, (int)u});
        }
    std::stable_sort(size_id.begin(), size_id.end(),
                     [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first < y.first; });
    order->resize(size_id.size());
    for (size_t q = 0; q < size_id.size(); ++q) (*order)[q] = size_id[q].second;
}

cudaError_t launch_reduce_sym(const PassBuffers& b, const SymPlan& p, int* err, int eval_only, cudaStream_t s,
                              cudaEvent_t between, int stall_ms) {
    cudaError_t e;
    if (p.mma) {
        e = launch_sym_mma_stream(b, p, err, eval_only, s, stall_ms);
    } else if (p.sorted) {
        if (!p.packed || p.layout != kPackedSw4 || !b.sym_meta) return cudaErrorInvalidValue;
        const SortedLayout L = sorted_layout(b.k, p.stages);
        uint8_t* metaC = b.sym_meta;
        uint8_t* metaR = b.sym_meta + (size_t)p.T * L.meta_bytes;
        e = launch_pdl(sym_sort_kernel, dim3((unsigned)p.T), dim3(kB), 0, s, (const uint8_t*)b.lab8, b.n, b.k, metaC,
                       metaR, (const LoopState*)b.st, eval_only);
        if (e != cudaSuccess) return e;
        SortedArgs r;
        r.Kp = static_cast<const float*>(b.K);
        r.n = b.n;
        r.k = b.k;
        r.T = p.T;
        r.a = p.a;
        r.Ts = p.Ts;
        r.units = p.units;
        r.stages = p.stages;
        r.stage_bytes = L.stage_bytes;
        r.meta_bytes = L.meta_bytes;
        r.off_bars = L.bars;
        r.metaC = metaC;
        r.metaR = metaR;
        r.Spart = b.Spart;
        r.st = b.st;
        r.err = err;
        r.eval_only = eval_only;
        r.stall_block = stall_ms > 0 ? 1 : 0;
        r.wait_ns = stall_ms > 0 ? (unsigned long long)stall_ms * 1000000ull : tc::kWaitLimitNs;
        r.order = b.sym_order;
        const dim3 block((unsigned)sorted_threads(p.a, p.rpl, p.pw));
        void (*f)(SortedArgs) = p.rpl == 4 ? (p.kb == 12   ? reduce_sym_sorted_kernel<12, 4, 1>
                                              : p.kb == 16 ? reduce_sym_sorted_kernel<16, 4, 1>
                                                           : reduce_sym_sorted_kernel<32, 4, 1>)
                                : p.pw == 2 ? reduce_sym_sorted_kernel<12, 2, 2>
                                           : (p.kb == 12   ? reduce_sym_sorted_kernel<12, 2, 1>
                                              : p.kb == 16 ? reduce_sym_sorted_kernel<16, 2, 1>
                                                           : reduce_sym_sorted_kernel<32, 2, 1>);
        e = launch_pdl(f, dim3(p.grid), block, p.smem, s, r);
    } else {
        CUtensorMap map;
        memset(&map, 0, sizeof map);
        if (!p.packed && !make_tensor_map_2d(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<void*>(b.K),
                                             (uint64_t)b.n, (uint64_t)b.n, (uint64_t)b.ldk * 4, kBoxCols, kB,
                                             CU_TENSOR_MAP_SWIZZLE_128B))
            return cudaErrorInvalidValue;
        if (p.packed && p.layout != kPackedSw16) return cudaErrorInvalidValue;
        BranchArgs a;
        a.Kp = p.packed ? static_cast<const float*>(b.K) : nullptr;
        a.ldk = b.ldk;
        a.n = b.n;
        a.k = b.k;
        a.T = p.T;
        a.nlab = (b.n + 15) & ~15;
        a.items = p.items;
        a.lab8 = b.lab8;
        a.Spart = b.Spart;
        a.st = b.st;
        a.err = err;
        a.eval_only = eval_only;
        a.stall_block = stall_ms > 0 ? 1 : 0;
        a.wait_ns = stall_ms > 0 ? (unsigned long long)stall_ms * 1000000ull : tc::kWaitLimitNs;
        e = b.k <= 4 ? launch_pdl(reduce_sym_kernel<4>, dim3(p.grid), dim3(kSymThreads), p.smem, s, map, a)
                     : launch_pdl(reduce_sym_kernel<8>, dim3(p.grid), dim3(kSymThreads), p.smem, s, map, a);
    }
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
