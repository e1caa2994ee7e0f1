// Internal declarations of the CUDA path (not part of the public ABI).
#pragma once

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
    int32_t kbuild_err;      // the tensor-core K build timed out in a bounded wait
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
    int grid;        // blocks
    int warps;       // warps per block
    int nseg;        // column segments per row
    int seglen;      // columns per segment (multiple of 128)
    size_t smem;     // dynamic shared memory per block
    bool labels_in_smem;
};

// Sets the message popcorn_last_error_message() returns on this thread (api.cu).
void set_error_message(const char* msg);

// ---- K build (kbuild_simt.cu) ------------------------------------------------
cudaError_t launch_kbuild_simt(const float* P, int n, int d, int64_t ldp, KernParams kp,
                               float* K, int64_t ldk, float* kdiag, cudaStream_t s, int* launches);

// ---- K build on tensor cores (kbuild_tc.cu) ---------------------------------
// Workspace bytes for the BF16 operand copies and row norms.
size_t kbuild_tc_workspace(int n, int d, int precision);
// Opt the tcgen05 kernel into its shared memory (once per device).
cudaError_t configure_kbuild_tc();
// precision POPCORN_BF16 or POPCORN_BF16X3; *err (device) becomes nonzero if a
// bounded wait inside the kernel ran out.
cudaError_t launch_kbuild_tc(const float* P, int n, int d, int64_t ldp, KernParams kp, int precision, float* K,
                             int64_t ldk, float* kdiag, void* workspace, int* err, int num_sms, cudaStream_t s,
                             int* launches);

// ---- iteration kernels (iterate.cu) -----------------------------------------
// Opt the reduction kernels into the largest dynamic shared memory the device
// allows (call once per device, with it current, before plan_reduce);
// *usable receives the dynamic bytes plan_reduce may use.
cudaError_t configure_reduce_smem(int optin, int* usable);
ReducePlan plan_reduce(int n, int k, int num_sms, int smem_optin);

cudaError_t launch_init_state(LoopState* st, int max_iter, int check_conv, double tol,
                              cudaStream_t s);
cudaError_t launch_trace(const float* kdiag, int n, LoopState* st, cudaStream_t s);
cudaError_t launch_init_labels(const int32_t* in, int n, int k, int32_t* lab32, uint8_t* lab8,
                               int32_t* counts, LoopState* st, cudaStream_t s);

struct PassBuffers {
    const float* K;
    int64_t ldk;
    const float* kdiag;
    int n, k;
    int32_t* lab32;
    uint8_t* lab8;        // n rounded up to 16, zero padded
    int32_t* counts;      // [2][k] ping-pong, indexed by pass parity
    float* Spart;         // [n][nseg][k] per-segment cluster sums
    double* zpart;        // [grid][k]
    double* zsum;         // [k]
    double* cnorm;        // [k]
    double* invm;         // [k] 1/|L_c| (0 for empty clusters)
    LoopState* st;
    double* J_hist;       // [max(1, max_iter)]
    int32_t* changed_hist;
    float* E_out;         // optional n x k
};

// One assignment pass = reduction (E, z, J) + distance/argmin.
cudaError_t launch_reduce(const PassBuffers& b, const ReducePlan& plan, int eval_only,
                          cudaStream_t s);
cudaError_t launch_assign(const PassBuffers& b, const ReducePlan& plan, cudaStream_t s);

}  // namespace popcorn
