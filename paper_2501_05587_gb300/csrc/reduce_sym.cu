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
// Run form (k <= kSymMaxK), reduce_sym_runs_kernel: blocks in label order (a
//   per-pass sort of every block's labels), one shared-memory add per run of one
//   label, on super-tiles of a x a blocks whose row and column sums are kept over
//   the super-tile before one store per row: see below.
//
// Each group's warps split the work and their partials are added in a fixed
// order: deterministic.  sym_fold_kernel: S_ic = the slots summed in slot order
// (float-float), written to slot 0, the per-block FP64 partials of
// sum_{i in L_c} S_ic (z, Eq. 14), and in its last block the pass finalization
// (||c||^2, J).  The assignment then reads slot 0 alone.
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
constexpr int kMaxA = 4;                       // largest super-tile edge (run form)

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

// The blocks of super-tile (Is, Js) of the run form: rows I0 <= I < I1, columns
// max(I, J0) <= J < J1.
struct Unit {
    int Is, Js, I0, I1, J0, J1;
};
__device__ __forceinline__ Unit unit_of(long long u, int T, int a, int Ts) {
    Unit t;
    tri_coords(u, Ts, &t.Is, &t.Js);
    t.I0 = t.Is * a;
    t.I1 = min(t.I0 + a, T);
    t.J0 = t.Js * a;
    t.J1 = min(t.J0 + a, T);
    return t;
}

// ---------------------------------------------------------------------------
// The run form of the symmetric pass (k up to kSymRunsMaxK).
//
// Per pass, sym_meta_kernel sorts the labels of every 128-block (a stable counting
// sort) and writes the block's metadata: for each sorted position p, the box offset
// of the local index it holds when the block is a column block (colcode) and when it
// is a row block (rowcode), its label, and a mask of the positions that end a run of
// one label.  The stream then walks a block in label order: a row-group lane owns a
// row and adds the row's elements column after column, in sorted order, into one
// register, and only at the end of a run of one label adds that register to the row's
// cluster sum in shared memory; a column-group lane owns a column and does the same
// over the rows.  So shared memory sees one read-add-write per run (at most k per
// half-block) instead of one per element, and a cluster sum is the same whatever k
// is.  K is packed in the XOR-32 layout (kPackedSw4): element c of row r of a box at
// c ^ (r mod 32), so that both the 32 rows of a column and the 32 columns of a row
// sit in 32 different banks.
constexpr int kMetaBytes = 768;        // per 128-block
constexpr int kMetaColcode = 0;        // u16[128]: (box << 12) | (l mod 32)   of local index l
constexpr int kMetaRowcode = 256;      // u16[128]: 32 l + (l mod 32)
constexpr int kMetaLabel = 512;        // u8[128]: the label at sorted position p (0xFF past the block's rows)
constexpr int kMetaMask = 640;         // u64[2]: bit p set where position p ends a run (half 0 also at 63)

__global__ void __launch_bounds__(kB) sym_meta_kernel(const uint8_t* __restrict__ lab8, int n, int k, uint8_t* meta,
                                                      const LoopState* st, int eval_only) {
    grid_dependency_wait();   // the labels come from the previous pass
    if (pass_skip(st, eval_only)) return;
    __shared__ uint8_t lab[kB];
    __shared__ unsigned long long ends[2];
    const int b = blockIdx.x, t = threadIdx.x;
    const int i = b * kB + t;
    // rows past n, and (defensively) any label outside [0, k), take no part in a run: the
    // stream adds a run into the cluster sum its label indexes
    const int l = (i < n && (int)lab8[i] < k) ? (int)lab8[i] : 0xFF;
    lab[t] = (uint8_t)l;
    if (t < 2) ends[t] = 0ull;
    __syncthreads();
    // stable rank: labels below mine, then equal labels before me; is a later one equal?
    int pos = 0;
    bool last = true;
    for (int u = 0; u < kB; ++u) {
        const int lu = lab[u];
        pos += (lu < l) || (lu == l && u < t);
        last = last && !(lu == l && u > t);
    }
    uint8_t* m = meta + (size_t)b * kMetaBytes;
    reinterpret_cast<uint16_t*>(m + kMetaColcode)[pos] = (uint16_t)(((t >> 5) << 12) | (t & 31));
    reinterpret_cast<uint16_t*>(m + kMetaRowcode)[pos] = (uint16_t)(32 * t + (t & 31));
    m[kMetaLabel + pos] = (uint8_t)l;
    // a run of a real label ends here; the first half also ends at position 63 (its
    // partial sum is stored before the second half's part of the same run)
    if (l != 0xFF && (last || pos == 63)) atomicOr(&ends[pos >> 6], 1ull << (pos & 63));
    __syncthreads();
    if (t < 2) reinterpret_cast<unsigned long long*>(m + kMetaMask)[t] = ends[t];
}

struct RunArgs {
    const float* Kp;           // block-packed K, kPackedSw4 layout
    int n, k, T;
    int a, Ts;
    long long units;
    int stages;
    int off_meta, off_accr, off_colacc, off_bars, off_flag;
    const uint8_t* meta;       // [T][kMetaBytes]
    float* Spart;              // [nslots][k][n]
    const LoopState* st;
    int* err;
    int eval_only;
};

// Runs of one half-block (64 sorted positions): v(p) = tile[code(p) ^ key] for this lane;
// at the end of a run of label c (a set bit of `mask`), acc[c * 128] += the run's sum.
// The run structure is the same for every lane; the end test is taken as a warp vote so
// that the add into shared memory is a branch the warp takes together (a run ends at
// about one position in six at k = 10), not predicated code every position pays for.
__device__ __forceinline__ void sum_runs(const float* __restrict__ tile, const uint16_t* __restrict__ codes,
                                         const uint8_t* __restrict__ labels, unsigned long long mask, uint32_t key,
                                         float* acc) {
    float run = 0.f;
#pragma unroll 1
    for (int pc = 0; pc < 8; ++pc) {
        const uint4 cw = *reinterpret_cast<const uint4*>(codes + 8 * pc);   // 8 codes, the same for every lane
        const uint32_t c32[4] = {cw.x, cw.y, cw.z, cw.w};
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t code = (c32[e >> 1] >> (16 * (e & 1))) & 0xffffu;
            v[e] = tile[code ^ key];
        }
        const uint32_t mb = (uint32_t)(mask >> (8 * pc)) & 0xffu;
        if (mb == 0u) {   // no run ends in these 8 positions (uniform)
            run += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
            continue;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            run += v[e];
            if (__any_sync(0xffffffffu, (mb >> e) & 1u)) {
                float* dst = acc + (uint32_t)labels[8 * pc + e] * kB;
                *dst += run;
                run = 0.f;
            }
        }
    }
}

__global__ void __launch_bounds__(kSymThreads, 1) reduce_sym_runs_kernel(RunArgs a) {
    grid_dependency_wait();   // the block metadata and the loop state come from before this pass
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
        // producer: one thread bulk-copies each block and the metadata of its row and column blocks
        if (lane == 0) {
            const uint64_t stream_once = tc::l2_evict_first();
            long long t = 0;
            bool ok = true;
            for (long long u = blockIdx.x; u < a.units && ok; u += G) {
                const Unit w = unit_of(u, a.T, a.a, a.Ts);
                for (int I = w.I0; I < w.I1 && ok; ++I)
                    for (int J = max(I, w.J0); J < w.J1; ++J, ++t) {
                        const int s = (int)(t % S);
                        if (t >= S && !tc::mbar_wait(empty_bar(s), (uint32_t)((t / S) - 1) & 1u, abort_flag, a.err)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(full_bar(s), (uint32_t)(kTileBytes + 2 * kMetaBytes));
                        const long long tri = (long long)I * a.T - (long long)I * (I - 1) / 2 + (J - I);
                        tc::bulk_load_1d_hint(sbase + (uint32_t)s * kTileBytes, a.Kp + tri * (kB * kB),
                                              (uint32_t)kTileBytes, full_bar(s), stream_once);
                        const uint32_t mdst = sbase + (uint32_t)a.off_meta + (uint32_t)s * 2 * kMetaBytes;
                        tc::bulk_load_1d(mdst, a.meta + (size_t)I * kMetaBytes, (uint32_t)kMetaBytes, full_bar(s));
                        tc::bulk_load_1d(mdst + kMetaBytes, a.meta + (size_t)J * kMetaBytes, (uint32_t)kMetaBytes,
                                         full_bar(s));
                    }
            }
            if (*abort_flag) {
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

    const uint64_t keep = tc::l2_evict_last();
    const bool rowg = warp < kConsumerWarps / 2;
    const int u = threadIdx.x & (kGroup - 1);
    const int bar_id = rowg ? kBarRows : kBarCols;
    const int gw = u >> 5;
    const int h = gw >> 2;                      // half of the sorted order: positions 64 h .. 64 h + 63
    const int q = gw & 3;                       // row group: rows 32 q + lane; column group: box q
    // this lane's row (row group) or column (column group) inside the block, and the XOR key
    // that turns a code into its element's offset: row group 32 r + (r mod 32) with r its row,
    // column group 4096 q + lane
    const int mine = 32 * q + lane;
    const uint32_t key = rowg ? (uint32_t)(32 * mine + lane) : (uint32_t)(4096 * q + lane);
    float* accr = reinterpret_cast<float*>(smem + a.off_accr);     // [2][k][128] row sums of the block row
    // column sums of the super-tile's block columns, per half: [a][2][k][128]
    float* colacc = reinterpret_cast<float*>(smem + a.off_colacc);
    float* my = accr + (size_t)h * k * kB + mine;                  // row group: this lane's sums my[c * 128]
    const int diag_slot = a.Ts;

    int t = 0;
    bool alive = true;
    for (long long uu = blockIdx.x; uu < a.units && alive; uu += G) {
        const Unit w = unit_of(uu, a.T, a.a, a.Ts);
        for (int I = w.I0; I < w.I1 && alive; ++I)
            for (int J = max(I, w.J0); J < w.J1; ++J, ++t) {
                const int s = t % S;
                const bool ok = tc::mbar_wait(full_bar(s), (uint32_t)(t / S) & 1u, abort_flag, a.err);
                if (!tc::named_bar_all(bar_id, kGroup, ok)) {
                    alive = false;
                    break;
                }
                const float* tile = reinterpret_cast<const float*>(smem + (size_t)s * kTileBytes);
                const uint8_t* mI = smem + a.off_meta + s * 2 * kMetaBytes;
                const uint8_t* mJ = mI + kMetaBytes;
                if (rowg) {
                    // row sums of block I over the columns of block J (sorted by label), kept per
                    // half over the super-tile's columns; the halves are added and stored to slot
                    // Js after the last one
                    if (J == max(I, w.J0))
                        for (int c = 0; c < k; ++c) my[c * kB] = 0.f;
                    sum_runs(tile, reinterpret_cast<const uint16_t*>(mJ + kMetaColcode) + 64 * h,
                             mJ + kMetaLabel + 64 * h, reinterpret_cast<const unsigned long long*>(mJ + kMetaMask)[h],
                             key, my);
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(empty_bar(s));
                    if (J == w.J1 - 1) {
                        tc::named_bar<kGroup>(kBarRows);
                        if (u < kB && I * kB + u < n) {
                            float* out = a.Spart + (size_t)w.Js * k * n + I * kB + u;
                            const float* __restrict__ h0 = accr + u;
                            const float* __restrict__ h1 = accr + (size_t)k * kB + u;
#pragma unroll 4
                            for (int c = 0; c < k; ++c) tc::st_hint(out + (size_t)c * n, h0[c * kB] + h1[c * kB], keep);
                        }
                    }
                } else {
                    const bool diag = I == J;
                    if (diag && a.a == 1) {
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(empty_bar(s));
                        continue;
                    }
                    // column sums of block J over the rows of block I (sorted by label), kept per
                    // half over the super-tile's rows in colacc[J - J0]; after the last of those
                    // rows the halves are added and stored to slot Is (the extra slot for a
                    // diagonal super-tile).  A diagonal block adds nothing.
                    float* myc = colacc + ((size_t)(J - w.J0) * 2 + h) * k * kB + mine;
                    if (I == w.I0)
                        for (int c = 0; c < k; ++c) myc[c * kB] = 0.f;
                    if (!diag)
                        sum_runs(tile, reinterpret_cast<const uint16_t*>(mI + kMetaRowcode) + 64 * h,
                                 mI + kMetaLabel + 64 * h,
                                 reinterpret_cast<const unsigned long long*>(mI + kMetaMask)[h], key, myc);
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(empty_bar(s));
                    if (I == min(J, w.I1 - 1)) {
                        tc::named_bar<kGroup>(kBarCols);
                        if (u < kB && J * kB + u < n) {
                            const int slot = w.Is == w.Js ? diag_slot : w.Is;
                            float* out = a.Spart + (size_t)slot * k * n + J * kB + u;
                            const float* __restrict__ h0 = colacc + (size_t)(J - w.J0) * 2 * k * kB + u;
                            const float* __restrict__ h1 = h0 + (size_t)k * kB;
#pragma unroll 4
                            for (int c = 0; c < k; ++c) tc::st_hint(out + (size_t)c * n, h0[c * kB] + h1[c * kB], keep);
                        }
                    }
                }
            }
    }
}

// Dynamic shared memory of the run form, in order: the block ring (1024-byte aligned),
// the metadata ring (row block, column block), the row sums of a block row per half
// ([2][k][128]), the column sums of the super-tile's block columns per half
// ([a][2][k][128]), barriers and the abort flag.
struct RunLayout {
    int meta, accr, colacc, bars, flag, bytes;
};
RunLayout run_layout(int k, int stages, int a) {
    RunLayout L;
    L.meta = stages * kTileBytes;
    L.accr = align128(L.meta + stages * 2 * kMetaBytes);
    L.colacc = align128(L.accr + 2 * k * kB * 4);
    L.bars = align128(L.colacc + a * 2 * k * kB * 4);
    L.flag = L.bars + 2 * stages * 8;
    L.bytes = L.flag + 16 + 1024;
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
    return cudaFuncSetAttribute(reduce_sym_runs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

SymPlan plan_reduce_sym(int n, int k, int num_sms, int smem_optin, int a_req, int stages_req) {
    SymPlan p{};
    if (k < 1 || k > kSymMaxK || n < 1) return p;
    p.T = (n + kB - 1) / kB;
    p.items = (long long)p.T * (p.T + 1) / 2;
    p.fold_blocks = (n + kFoldThreads - 1) / kFoldThreads;
    // k <= 8 on single blocks: the branch form (register sums, the deepest ring that fits);
    // above, or for a forced super-tile edge > 1: the run form
    if (k <= kSymBranchMaxK && a_req <= 1) {
        const int bytes = k <= 4 ? BranchLayout<4>::bytes : BranchLayout<8>::bytes;
        if (bytes > smem_optin) return p;
        p.runs = false;
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
    p.runs = true;
    p.kb = 0;
    p.layout = kPackedSw4;
    int cand_a[3] = {4, 2, 1}, na = 3;
    if (a_req > 0) {
        cand_a[0] = a_req;
        na = 1;
    }
    for (int ia = 0; ia < na; ++ia) {
        const int A = cand_a[ia];
        if (A < 1 || A > kMaxA) continue;
        const int Ts = (p.T + A - 1) / A;
        const long long units = (long long)Ts * (Ts + 1) / 2;
        // leave about 16 super-tiles per SM, so the static round-robin stays near balance
        if (a_req == 0 && A > 1 && units < 16LL * num_sms) continue;
        int cand_s[2] = {3, 2};
        if (stages_req > 0) cand_s[0] = cand_s[1] = stages_req;
        for (int is = 0; is < 2; ++is) {
            const int S = cand_s[is];
            if (S < 2 || S > 3) continue;
            const int bytes = run_layout(k, S, A).bytes;
            if (bytes > smem_optin) continue;
            p.a = A;
            p.Ts = Ts;
            p.units = units;
            p.stages = S;
            p.smem = (size_t)bytes;
            p.nslots = Ts + (A > 1 ? 1 : 0);
            p.grid = (int)(units < num_sms ? units : num_sms);
            p.meta_bytes = (size_t)p.T * kMetaBytes;
            p.ok = true;
            return p;
        }
    }
    return p;
}

cudaError_t launch_reduce_sym(const PassBuffers& b, const SymPlan& p, int* err, int eval_only, cudaStream_t s,
                              cudaEvent_t between, int stall_ms) {
    cudaError_t e;
    if (p.runs) {
        if (!p.packed || p.layout != kPackedSw4 || !b.sym_meta) return cudaErrorInvalidValue;
        e = launch_pdl(sym_meta_kernel, dim3((unsigned)p.T), dim3(kB), 0, s, (const uint8_t*)b.lab8, b.n, b.k,
                       b.sym_meta, (const LoopState*)b.st, eval_only);
        if (e != cudaSuccess) return e;
    const RunLayout L = run_layout(b.k, p.stages, p.a);
        RunArgs r;
        r.Kp = static_cast<const float*>(b.K);
        r.n = b.n;
        r.k = b.k;
        r.T = p.T;
        r.a = p.a;
        r.Ts = p.Ts;
        r.units = p.units;
        r.stages = p.stages;
        r.off_meta = L.meta;
        r.off_accr = L.accr;
        r.off_colacc = L.colacc;
        r.off_bars = L.bars;
        r.off_flag = L.flag;
        r.meta = b.sym_meta;
        r.Spart = b.Spart;
        r.st = b.st;
        r.err = err;
        r.eval_only = eval_only;
        e = launch_pdl(reduce_sym_runs_kernel, dim3(p.grid), dim3(kSymThreads), p.smem, s, r);
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
