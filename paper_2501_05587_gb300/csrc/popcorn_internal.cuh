// Internal declarations of the CUDA path (not part of the public ABI).
#pragma once

#include <utility>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "popcorn.h"

namespace popcorn {

constexpr int kMaxClusters = 256;       // labels are bytes on the device
constexpr int kReduceMaxWarps = 16;     // K-streaming reduction: warps per block
constexpr int kAssignThreads = 128;     // distance/argmin kernel: threads per block

// Kernel-function parameters in the precision the epilogues use.
struct KernParams {
    int kind;          // popcorn_kernel_kind
    int degree;
    float gamma;
    float coef0;
    float neg_gamma_over_sigma2;   // -gamma / sigma^2 (Gaussian)
};

// Device-resident loop state.  All passes of a fit read and update it on the
// device, so the host never has to synchronize between passes.
struct LoopState {
    int32_t iter;          // passes completed
    int32_t done;          // nonzero: later passes return immediately
    int32_t converged;     // a pass changed no label
    int32_t max_iter;
    int32_t check_conv;
    int32_t last_changed;  // labels changed by the last pass
    uint32_t reduce_ticket;  // last-block-done counters (reset by the last block)
    uint32_t assign_ticket;
    uint32_t changed_acc;    // labels changed in the running pass
    int32_t bad_label;       // an input label was outside [0, k)
    int32_t wait_err;      // a bounded wait ran out (tensor-core K build, recompute or symmetric stream)
    int32_t pad0;
    double tol;
    double trace;          // sum_i K_ii in FP64
    double J_last;         // J(labels before the last pass)
    double J_prev;         // J(labels before the pass before)
    double J_eval;         // J(final labels)
};

// Variants of the K-streaming reduction, by how a warp reduces its per-lane
// partials at the end of a unit: butterfly over 4 or 8 clusters, or the
// rotated row walk for larger k.
enum { kReduceBfly4 = 0, kReduceBfly8 = 1, kReduceRotated = 2 };

// Launch geometry of the K-streaming reduction (segment-split rows).
struct ReducePlan {
    int variant;     // kReduceBfly4 / kReduceBfly8 / kReduceRotated
    int k_storage;   // element type of K (popcorn_k_storage)
    int grid;        // blocks
    int warps;       // warps per block
    int nseg;        // column segments per row
    int seglen;      // columns per segment (multiple of 128)
    size_t smem;     // dynamic shared memory per block
    bool labels_in_smem;
};

// Symmetric K stream (reduce_sym.cu): each 128 x 128 block on and above the
// diagonal is read once.  Blocks are handed out in super-tiles of a x a blocks;
// a super-tile's row sums go to one slot of its rows and its column sums to one
// slot of its columns' rows, so Spart holds nslots = ceil(T / a) (+1 in the sorted
// form) slots; the fold sums them into slot 0 (the assignment then reads slot 0
// only) and forms z and J.  FP32 K, k <= kSymMaxK: up to kSymBranchMaxK clusters on
// single blocks a uniform branch per column / row adds into register sums; otherwise
// the sorted form walks each block's columns and rows in label order (a per-pass sort
// of every 128-block's labels) with the sums in registers over a super-tile, K packed
// in the XOR-32 layout.
constexpr int kSymMaxK = 32;
constexpr int kSymBranchMaxK = 8;
constexpr int kSymAutoMinN = 8192;   // the automatic choice takes the symmetric pass from here
struct SymPlan {
    bool ok;
    bool sorted;        // the sorted form (k > kSymBranchMaxK, or a forced super-tile edge > 1)
    bool mma;           // the tensor-core form (FP16 / BF16 K): E parts as MMAs against one-hot labels
    int layout;         // packed tile layout the pass reads: kPackedSw16 (branch), kPackedSw4 (sorted)
                        // or kPackedSw128H (tensor-core form)
    size_t meta_bytes;  // sorted form: per-pass label-sorted lists of every block (column and row lists);
                        // tensor-core form: per-pass one-hot label operand of every block
    int kb;             // sums per row / column: 4 or 8 (branch form), 12, 16 or 32 (sorted form),
                        // 16 or 32 (tensor-core form: accumulator columns, the MMA's N); >= k
    int rpl;            // sorted form: rows (columns) a lane owns in a block, 4 or 2 (2: two warps a block row)
    int pw;             // sorted form: block rows (columns) of the super-tile a warp owns, 1 or 2
    int ebytes;         // bytes a stored K entry: 4, or 2 for FP16 / BF16 K in the half layout
    int T;              // 128-blocks per side
    int a;              // super-tile edge in blocks (1 to 8)
    int Ts;             // super-tiles per side
    int nslots;         // Spart slots
    int stages;         // block ring depth
    long long items;    // blocks on and above the diagonal
    long long units;    // super-tiles on and above the diagonal
    int grid;           // persistent CTAs of the stream kernel
    int fold_blocks;    // row chunks of the fold (zpart rows)
    size_t smem;
    bool packed;        // K is block-packed in `layout` (set by the caller with the K build it chose)
};
// a_req / stages_req: 0 = the heuristic choice, else that super-tile edge / ring depth
// (ok = false if it does not fit)
// ebytes: 4 (FP32 K: branch or sorted form) or 2 (FP16 / BF16 K: the tensor-core form)
SymPlan plan_reduce_sym(int n, int k, int num_sms, int smem_optin, int a_req = 0, int stages_req = 0,
                        int ebytes = 4);
cudaError_t configure_reduce_sym(int smem_optin);
// The super-tiles of a sorted-form or tensor-core plan by decreasing number of blocks (stable):
// the diagonal and edge super-tiles hold fewer blocks, so in this order every round of the
// stream's static round-robin takes units of one size and the small ones come last.
void sym_unit_order(const SymPlan& p, std::vector<int>* order);
// The tensor-core form (reduce_sym_mma.cu): plan fields for an FP16 / BF16 K, the per-pass
// one-hot operand and the stream launch (the fold is shared with the other forms).
bool plan_sym_mma(SymPlan* p, int k, int num_sms, int smem_optin, int a_req, int stages_req);
cudaError_t configure_sym_mma(int smem_optin);
cudaError_t launch_sym_mma_stream(const struct PassBuffers& b, const SymPlan& p, int* err, int eval_only,
                                  cudaStream_t s, int stall_ms);
// err: set when a bounded wait of the stream kernel runs out; `between` (may be
// null) is recorded on s after the stream kernel, before the fold.  stall_ms > 0
// (either form; error-path tests only): CTA 0 leaves its first block's copies out,
// and every wait of the launch gives up after stall_ms, so the launch reports a
// timed-out wait and the context stays usable.
cudaError_t launch_reduce_sym(const struct PassBuffers& b, const SymPlan& p, int* err, int eval_only,
                              cudaStream_t s, cudaEvent_t between, int stall_ms = 0);

// Launch with programmatic dependent launch: the grid may be scheduled while the
// previous kernel in the stream is still finishing, and it must call
// grid_dependency_wait() before it touches anything that kernel wrote.  This
// hides the launch latency between the kernels of a pass.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Waits until the grids this one depends on have completed and their writes are
// visible (returns at once for a launch without a programmatic dependency).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Upper-triangle block (bi, bj), bi <= bj, of number t when the T x T block
// triangle is enumerated row by row (row b starts at b T - b (b - 1) / 2).  An
// FP32 estimate of the quadratic's root, then exact integer correction (no
// FP64: GB300 runs FP64 at a small fraction of the FP32 rate).
__device__ __forceinline__ void tri_coords(long long t, int T, int* bi, int* bj) {
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

// Sets the message popcorn_last_error_message() returns on this thread (api.cu).
void set_error_message(const char* msg);

// Layouts of the block-packed upper triangle of K (tile t of the row-by-row triangle
// of 128 x 128 tiles at K + t * 16384 floats, as four boxes of 128 rows x 32 columns,
// 16 KB each).  kPackedSw16: 16-byte chunk j of row r at chunk j ^ (r mod 8) (the TMA
// 128-byte swizzle; rows read as float4 chunks).  kPackedSw4: element c of row r at
// c ^ (r mod 32) (a row and a column of a box are both read conflict-free as scalars).
constexpr int kPackedSw16 = 1, kPackedSw4 = 2;
// kPackedSw128H: the same triangle with FP16 / BF16 entries, 32 KB a tile (kpack.cu):
// element (r, C) at byte 16384 (C >> 6) + 128 r + 16 (((C >> 3) & 7) ^ (r & 7)) + 2 (C & 7),
// the tensor cores' 128-byte swizzle; entries past n are zeros.
constexpr int kPackedSw128H = 4;
// The FP32 triangle (kPackedSw4) Kf rounded into kPackedSw128H Kh (k_storage FP16 or BF16);
// diag K rounded the same way.
cudaError_t configure_pack_half();
cudaError_t launch_pack_half(const float* Kf, void* Kh, int k_storage, int n, float* kdiag, cudaStream_t s);

// ---- K build (kbuild_simt.cu) ------------------------------------------------
// K is float, __half or __nv_bfloat16 by k_storage (popcorn_k_storage); ldk in elements.
// packed: 0 = full square; kPackedSw16 / kPackedSw4 = FP32 K as the block-packed upper
// triangle in that layout, read by the symmetric pass (ldk is then unused).
// full = 1 (full square only): every tile of the square computed and stored once (the
// GEMM form) instead of the upper-triangle tiles stored with their transposes (SYRK form).
// rn (n floats) and maxr (one word), both device workspace: for a Gaussian kernel the row
// norms, from which the build decides on the device whether the norm expansion is accurate
// enough; null keeps the coordinate-difference form.
cudaError_t launch_kbuild_simt(const float* P, int n, int d, int64_t ldp, KernParams kp,
                               void* K, int64_t ldk, int k_storage, float* kdiag, cudaStream_t s, int* launches,
                               int packed = 0, int full = 0, float* rn = nullptr, unsigned* maxr = nullptr);

// ---- K build on tensor cores (kbuild_tc.cu) ---------------------------------
// Workspace bytes for the BF16 operand copies and row norms.
size_t kbuild_tc_workspace(int n, int d, int precision);
// Opt the tcgen05 kernel into its shared memory (once per device) and look up
// the driver's tensor-map encoder (so no lookup happens during stream capture).
cudaError_t configure_kbuild_tc();
// precision POPCORN_BF16 or POPCORN_BF16X3; *err (device) becomes nonzero if a
// bounded wait inside the kernel ran out.
// packed: 0 = full square; kPackedSw16 / kPackedSw4 = the block-packed upper triangle
// in that layout (as the FP32 build writes it for the symmetric pass); kPackedSw128H = the
// FP16 / BF16 packed triangle (k_storage), written directly with diag K rounded the same
// way; ldk is then unused.
cudaError_t launch_kbuild_tc(const float* P, int n, int d, int64_t ldp, KernParams kp, int precision, float* K,
                             int64_t ldk, float* kdiag, void* workspace, int* err, int num_sms, cudaStream_t s,
                             int* launches, int packed = 0, int full = 0, int k_storage = POPCORN_K_FP32);

// 2-D tiled TMA descriptor over a row-major matrix (inner = contiguous extent
// in elements, row_bytes = pitch); false if the driver entry point is missing
// or rejects the arguments.
bool make_tensor_map_2d(CUtensorMap* m, CUtensorMapDataType dt, void* base, uint64_t inner, uint64_t outer,
                        uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw);

// Dynamic shared memory a kernel may request next to `static_bytes` of its own.
inline int optin_minus_static(int optin, size_t static_bytes) {
    return optin - (int)((static_bytes + 127) / 128 * 128);
}

// A pass kernel returns at once when the loop has stopped (ordinary passes) or
// when the final objective is already known (eval pass: the last pass
// changed no label, so J(labels_out) = J of that pass).
__device__ __forceinline__ bool pass_skip(const LoopState* st, int eval) {
    return eval ? (st->iter > 0 && st->last_changed == 0) : (st->done != 0);
}

// ---- whole fits in one cooperative launch (fused_fit.cu) ----------------------
// For a stored FP32 K that sits in L2 (n <= kFusedMaxN, k <= kFusedMaxK): every pass of
// the fit and the final objective in one launch of one CTA per SM, two exchanges between
// the CTAs a pass; same pass semantics and outputs (labels, LoopState, J / change
// histories, E) as the launched passes.  zpart: num_sms x k doubles; xchg:
// fused_xchg_words(num_sms, k) words of workspace.
constexpr int kFusedMaxN = 6144;
constexpr int kFusedMaxK = 32;
bool fused_fit_applies(int n, int k, int num_sms, int smem_optin);
size_t fused_fit_smem(int n, int k, int num_sms, int64_t ldk, int cache_k);
size_t fused_xchg_words(int num_sms, int k);
cudaError_t configure_fused_fit(int smem_optin);
// stall_ms > 0 (error-path tests only): CTA 0 leaves before the first grid barrier and every
// barrier wait gives up after stall_ms, so the fit reports a timed-out wait.
cudaError_t launch_fused_fit(const struct PassBuffers& b, double* zpart, unsigned* xchg, int num_sms, int smem_optin,
                             cudaStream_t s, int stall_ms = 0);

// ---- K-means++ seeding (seeding.cu) --------------------------------------------
// One cooperative launch (one CTA per SM) for all k steps; kappa in FP64 from the points.
// u: k draws (device); labels: n, centers: k (device); part: num_sms doubles, chosen: one
// int, bar: 32 words of workspace; *err (device) set when a grid-barrier wait runs out.
bool kmeanspp_fits(int n, int d, int num_sms, int smem_optin);
size_t kmeanspp_smem(int n, int d, int num_sms);
cudaError_t configure_kmeanspp(int smem_optin);
cudaError_t launch_kmeanspp(const float* P, int n, int d, int64_t ldp, int k, const popcorn_kernel& kern,
                            const double* u, int32_t* labels, int32_t* centers, double* part, int* chosen,
                            unsigned* bar, int* err, int num_sms, cudaStream_t s);

// ---- recompute path (recompute.cu): K never stored ---------------------------
struct RecomputePlan {
    int fp8;            // 1: E4M3 operands with per-row scales; 0: BF16
    int dpad;           // padded feature count (elements)
    int row_bytes;      // operand row pitch in bytes (multiple of 128)
    int nkb;            // 128-byte k-blocks per row
    int npad;           // n rounded up to 128
    int ncols;          // sorted column space: n + 31 k rounded up to 128 (clusters padded to 32)
    int nseg, seglen;   // column segments (units = row blocks x segments)
    int stages;         // column k-block ring depth
    int nslot;          // Spart slots: nseg x epilogue groups per row block
    int units_per_sm;   // the unit-count target nseg was derived from
    int eg;             // epilogue warpgroups
    int rbp;            // 128-row blocks per unit (2: each column tile feeds two MMAs)
    int threads;        // 64 + 128 * eg
    float fact_limit;   // Gaussian: row factor exp2(c2 r_i) taken out while max |c2| r_i < this
    int off_b, off_meta, off_bar, off_misc;
    int smem;
    int grid;
    bool ok;            // false: d or k too large for this path
};

struct RecomputeBuffers {
    unsigned char* Q;     // n x row_bytes operand rows, original order
    float* norms;         // n FP32 norms of the represented rows
    float* knorms;        // n norms as the epilogue uses them (c2-scaled for the Gaussian)
    float* scales;        // n row scales (1 for BF16)
    unsigned char* Qs;    // ncols x row_bytes, cluster order, each cluster padded to 32 rows
    float* snorm;         // ncols epilogue norms in cluster order
    float* sscale;        // ncols scales in cluster order
    uint8_t* slab;        // ncols labels in cluster order (0xFF on padding)
    int* blockhist;       // sort blocks x k
    int* blockoff;        // sort blocks x k
    int* maxkn;           // bits of max_i |c2| r_i (Gaussian; zeroed before quantize)
};

// rbp_req: 0 = two row blocks per tile when 3 ring stages fit, else one; 1 or 2 = that
// many (ok = false if it does not fit).  units_per_sm: column-segment target (0 = 16).
RecomputePlan plan_recompute(int n, int d, int k, int precision, int num_sms, int smem_budget, int rbp_req = 0,
                             int units_per_sm = 0);
cudaError_t configure_recompute(int smem_optin, int* usable);
int recompute_sort_blocks(int n);

// ---- iteration kernels (iterate.cu) -----------------------------------------
// Opt the reduction kernels into the largest dynamic shared memory the device
// allows (call once per device, with it current, before plan_reduce);
// *usable receives the dynamic bytes plan_reduce may use.
cudaError_t configure_reduce_smem(int optin, int* usable);
ReducePlan plan_reduce(int n, int k, int num_sms, int smem_optin, int k_storage = 0);

cudaError_t launch_init_state(LoopState* st, int max_iter, int check_conv, double tol,
                              cudaStream_t s);
cudaError_t launch_trace(const float* kdiag, int n, LoopState* st, cudaStream_t s);
cudaError_t launch_init_labels(const int32_t* in, int n, int k, int32_t* lab32, uint8_t* lab8,
                               int32_t* counts, LoopState* st, cudaStream_t s);

struct PassBuffers {
    const void* K;        // float / __half / __nv_bfloat16 by k_storage
    int64_t ldk;          // elements
    int k_storage;        // popcorn_k_storage
    const float* kdiag;
    int n, k;
    int32_t* lab32;
    uint8_t* lab8;        // n rounded up to 16, zero padded
    int32_t* counts;      // [2][k] ping-pong, indexed by pass parity
    float* Spart;         // [nseg][k][n] per-segment cluster sums (row index fastest)
    double* zpart;        // [grid][k]
    double* zsum;         // [k]
    double* cnorm;        // [k]
    double* invm;         // [k] 1/|L_c| (0 for empty clusters)
    LoopState* st;
    double* J_hist;       // [max(1, max_iter)]
    int32_t* changed_hist;
    float* E_out;         // optional n x k
    uint8_t* sym_meta;    // sorted form of the symmetric pass: the label-sorted lists of every block
    const int* sym_order; // symmetric pass: super-tiles in processing order (larger first), or null
};

// Operand rows for the recompute path, their norms and scales, and diag K.
cudaError_t launch_quantize(const float* P, int n, int d, int64_t ldp, KernParams kp, const RecomputePlan& p,
                            const RecomputeBuffers& rb, float* kdiag, cudaStream_t s);
// Sort by label + fused tile/kernel/segment-sum kernel -> b.Spart.
cudaError_t launch_recompute_pass(const PassBuffers& b, KernParams kp, const RecomputePlan& p,
                                  const RecomputeBuffers& rb, int* err, int eval, cudaStream_t s);
// sum_{i in L_c} S_ic from b.Spart (nseg segments) and the pass finalization
// (||c||^2, 1/|L_c|, J); blocks of kZReduceRows rows.
constexpr int kZReduceRows = 1024;
cudaError_t launch_zreduce(const PassBuffers& b, int nseg, int eval, cudaStream_t s);

// One assignment pass = reduction (E, z, J) + distance/argmin.
cudaError_t launch_reduce(const PassBuffers& b, const ReducePlan& plan, int eval_only,
                          cudaStream_t s);
cudaError_t launch_assign(const PassBuffers& b, const ReducePlan& plan, cudaStream_t s);
cudaError_t launch_assign_nseg(const PassBuffers& b, int nseg, cudaStream_t s);

// ---- batched mode (iterate.cu, kbuild_simt.cu) --------------------------------
// One clustering instance of a batch, device-resident.  Flattened work of all
// instances (K tiles, K-stream units, z blocks, assign blocks, label blocks)
// is located by binary search over the *0 prefix fields.
struct BatchInst {
    const float* P;
    int64_t ldp;
    int d;
    KernParams kp;
    int T;                    // 128-row tiles of K
    long long tile0;          // first flattened upper-triangle tile
    float* K;
    int64_t ldk;
    float* kdiag;
    int n, k, nseg, seglen;
    uint8_t* lab8;
    int32_t* lab32;
    int32_t* counts;
    float* Spart;
    double* zpart;
    double* zsum;
    double* cnorm;
    double* invm;
    LoopState* st;
    double* J_hist;
    int32_t* changed_hist;
    const int32_t* init_labels;
    int32_t* labels_out;
    int unit0, zblock0, ablock0, lblock0;
    // FP16 / BF16 K (batched_mma.cu): every tile of the square in kPackedSw128H, tile (I, J) at
    // Kh + (I T + J) 32 KB; the per-pass one-hot operands of the T blocks, N rows each
    unsigned char* Kh;
    unsigned char* V;
    int N;                    // accumulator columns: k rounded up to 16
    long long htile0;         // first flattened tile of the square
    int vblock0;              // first flattened 128-block
};

struct BatchPlan {
    int count;
    long long tiles;          // K tiles of all instances
    int units, zblocks, ablocks, lblocks;
    int kmax;
    int warps, grid, per_sm;  // batched K-stream launch
    size_t smem;
    // FP16 / BF16 K: the tensor-core stream over (instance, row block) units
    int half;                 // 0, or the k_storage of every instance's K
    long long htiles;         // tiles of every instance's square
    int vblocks;              // 128-blocks of every instance
    int nunits;               // (instance, row block) units
    int Nmax;                 // widest accumulator
    int mstages, mgrid;
    size_t msmem;
};

constexpr int kBatchLabelThreads = 256;
constexpr int kBatchSeg = 8192;       // columns per K-stream unit in batched mode (whole rows for n <= 8192)
// K-stream units of one instance in batched mode
inline int batch_units(int n, int nseg) { return n * nseg; }

// per instance: loop state, labels/counts, (after the K build) trace of K
cudaError_t launch_batched_init(const BatchInst* dI, const BatchPlan& bp, int max_iter, int check_conv, double tol,
                                cudaStream_t s);
cudaError_t launch_batched_trace(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s);
cudaError_t launch_batched_kbuild_simt(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s);
// one pass over every instance that has not stopped (K stream, z, argmin)
cudaError_t launch_batched_pass(const BatchInst* dI, const BatchPlan& bp, int eval, cudaStream_t s);
// the rest of a pass after its K stream: z (with per-instance finalization) and the argmin
cudaError_t launch_batched_finish(const BatchInst* dI, const BatchPlan& bp, int eval, cudaStream_t s);
cudaError_t launch_batched_copy_labels(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s);
// FP16 / BF16 K in batched mode (batched_mma.cu).  Plan: ring depth, grid and shared memory of
// the stream for accumulators up to Nmax columns (false if it does not fit).  Pack: every
// instance's FP32 square (K, ldk) rounded into its half tiles Kh, diag K rounded with it.
// Pass: the one-hot operands, then the stream over the units (instance, row block), ordered
// by the caller (larger instances first), writing each row's k sums to Spart (one segment);
// *err is set when a bounded wait runs out.  stall_ms > 0 (error-path tests only): CTA 0
// leaves its first tile's copies out and every wait gives up after stall_ms.
bool plan_batched_mma(BatchPlan* bp, int num_sms, int smem_optin);
cudaError_t configure_batched_mma(int smem_optin);
cudaError_t launch_batched_pack_half(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s);
cudaError_t launch_batched_mma_stream(const BatchInst* dI, const int2* units, const BatchPlan& bp, int* err,
                                      int eval, cudaStream_t s, int stall_ms = 0);
// warps / grid / shared memory of the batched K stream for clusters up to kmax;
// warps = 0 / per_sm = 0 pick the largest that fits / the occupancy limit
void plan_batched_reduce(BatchPlan* bp, int num_sms, int smem_budget, int warps = 0, int per_sm = 0);
// the batched K stream alone (what the autotuner times)
cudaError_t launch_batched_reduce(const BatchInst* dI, const BatchPlan& bp, int eval, cudaStream_t s);

// ---- autotune cache (autotune.cu) ---------------------------------------------
struct TuneKey {
    int32_t target;       // 1: batched K stream, 2: recompute pass
    int32_t precision;
    int32_t a, b, c, d, e;   // target-specific size buckets
    int32_t sms;
};
struct TuneValue {
    int32_t p[4];         // the chosen schedule (target-specific)
    float ms;             // its measured time
};
int32_t log2_bucket(double x);   // round(4 log2 x): quarter-octave buckets
bool tune_lookup(const TuneKey& k, TuneValue* v);
void tune_store(const TuneKey& k, const TuneValue& v);
cudaError_t configure_batched(int smem_optin);

}  // namespace popcorn
