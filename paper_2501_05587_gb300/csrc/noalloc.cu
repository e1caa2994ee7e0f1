// popcorn_assign_step_noalloc: the assignment step with its scratch in a
// fixed, statically allocated device array instead of a workspace.
//
// Some callers may not allocate device memory at all, for example a host
// framework that owns every byte of device memory through its own allocator,
// or a long-running loop that forbids allocation once it has started.  This
// entry point serves them: it runs exactly the kernels of popcorn_assign_step
// (same launch plan, so the same results), but every temporary buffer is
// carved out of `g_assign_scratch` below.  It calls no cudaMalloc, cudaFree,
// pool or pinned-host allocation.
//
// `g_assign_scratch` is a file-scope __device__ array: each GPU that loads
// this library holds its kNoallocScratchBytes until the process exits.  On the
// host its name is only a stand-in, so the device address is obtained once
// per device with cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "popcorn.h"
#include "popcorn_internal.cuh"

using namespace popcorn;

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)POPCORN_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_assign_scratch[kNoallocScratchBytes];

popcorn_status nfail(popcorn_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_error_message(buf);
    return s;
}

#define NOALLOC_CUDA(call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return nfail(POPCORN_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
        }                                                                                    \
    } while (0)

struct NoallocDevice {
    bool ready = false;
    int sms = 0;
    int reduce_smem = 0;
    unsigned char* scratch = nullptr;   // device address of g_assign_scratch on this device
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

// Once per device, with it current: attributes, the reduction kernels'
// shared-memory opt-in, and the device address of the static scratch array.
popcorn_status noalloc_setup(NoallocDevice** out) {
    int dev = 0;
    NOALLOC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return nfail(POPCORN_ERR_UNSUPPORTED, "device ordinal %d >= 64", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        int optin = 0;
        NOALLOC_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        NOALLOC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        NOALLOC_CUDA(configure_reduce_smem(optin, &d.reduce_smem));
        void* p = nullptr;
        NOALLOC_CUDA(cudaGetSymbolAddress(&p, g_assign_scratch));
        if (p == nullptr) return nfail(POPCORN_ERR_CUDA, "cudaGetSymbolAddress returned a null scratch address");
        d.scratch = static_cast<unsigned char*>(p);
        d.ready = true;
    }
    *out = &d;
    return POPCORN_OK;
}

// Carves 256-byte-aligned pieces off the front of the scratch array.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base + used);
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        used += (bytes + 255) & ~(size_t)255;
        return p;
    }
};

// Scratch bytes one step needs for (n, k) under `plan` (same carve order as below).
size_t scratch_bytes(int n, int k, const ReducePlan& plan) {
    Carver c{nullptr};
    const size_t nlab = ((size_t)n + 15) & ~(size_t)15;
    c.take<int32_t>(n);
    c.take<uint8_t>(nlab);
    c.take<int32_t>(2 * (size_t)k);
    c.take<float>((size_t)plan.nseg * n * k);
    c.take<double>((size_t)plan.grid * k);
    c.take<double>(k);
    c.take<double>(k);
    c.take<double>(k);
    c.take<LoopState>(1);
    c.take<double>(1);
    c.take<int32_t>(1);
    return c.used;
}

}  // namespace

extern "C" {

popcorn_status popcorn_assign_step_noalloc(const float* K, int64_t ldk, const float* kdiag, int64_t n,
                                           int32_t k, const int32_t* labels, int32_t* new_labels,
                                           int32_t* counts, float* E, double* cnorm, double* objective,
                                           int32_t* changed, popcorn_stream_t stream) {
    set_error_message("");
    cudaStream_t s = (cudaStream_t)stream;
    if (!K || !kdiag || !labels || !new_labels) return nfail(POPCORN_ERR_INVALID, "null pointer argument");
    if (n < 2 || n >= (1LL << 31)) return nfail(POPCORN_ERR_INVALID, "n = %lld outside [2, 2^31)", (long long)n);
    if (k < 1 || k > n || k > kMaxClusters)
        return nfail(POPCORN_ERR_INVALID, "k = %d outside [1, min(n, %d)]", k, kMaxClusters);
    if (ldk < n || ldk % 4 != 0)
        return nfail(POPCORN_ERR_INVALID, "ldk = %lld must be >= n and a multiple of 4", (long long)ldk);
    if (reinterpret_cast<uintptr_t>(K) % 16 != 0) return nfail(POPCORN_ERR_INVALID, "K must be 16-byte aligned");
    NoallocDevice* dev;
    popcorn_status st = noalloc_setup(&dev);
    if (st != POPCORN_OK) return st;
    const int ni = (int)n;
    const ReducePlan plan = plan_reduce(ni, k, dev->sms, dev->reduce_smem);
    if (plan.grid == 0) return nfail(POPCORN_ERR_UNSUPPORTED, "n = %d is too large for the materialized path", ni);
    const size_t need = scratch_bytes(ni, k, plan);
    if (need > kNoallocScratchBytes)
        return nfail(POPCORN_ERR_INVALID,
                     "n = %d, k = %d needs %zu bytes of scratch; the static scratch holds %zu bytes "
                     "(use popcorn_assign_step, which allocates)",
                     ni, k, need, kNoallocScratchBytes);

    Carver cv{dev->scratch};
    PassBuffers b{};
    b.K = K;
    b.ldk = ldk;
    b.kdiag = kdiag;
    b.n = ni;
    b.k = k;
    const size_t nlab = ((size_t)ni + 15) & ~(size_t)15;
    b.lab32 = cv.take<int32_t>(ni);
    b.lab8 = cv.take<uint8_t>(nlab);
    b.counts = cv.take<int32_t>(2 * (size_t)k);
    b.Spart = cv.take<float>((size_t)plan.nseg * ni * k);
    b.zpart = cv.take<double>((size_t)plan.grid * k);
    b.zsum = cv.take<double>(k);
    b.cnorm = cv.take<double>(k);
    b.invm = cv.take<double>(k);
    b.st = cv.take<LoopState>(1);
    b.J_hist = cv.take<double>(1);
    b.changed_hist = cv.take<int32_t>(1);
    b.E_out = E;

    // the array keeps the previous call's contents: counts must start at zero,
    // the loop state is rewritten by launch_init_state, the rest is overwritten
    NOALLOC_CUDA(cudaMemsetAsync(b.counts, 0, 2 * (size_t)k * sizeof(int32_t), s));
    NOALLOC_CUDA(launch_init_state(b.st, 1, 0, 0.0, s));
    NOALLOC_CUDA(launch_init_labels(labels, ni, k, b.lab32, b.lab8, b.counts, b.st, s));
    NOALLOC_CUDA(launch_trace(kdiag, ni, b.st, s));
    NOALLOC_CUDA(launch_reduce(b, plan, 0, s));
    if (cnorm) NOALLOC_CUDA(cudaMemcpyAsync(cnorm, b.cnorm, (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice, s));
    NOALLOC_CUDA(launch_assign(b, plan, s));
    NOALLOC_CUDA(cudaMemcpyAsync(new_labels, b.lab32, (size_t)ni * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (counts) NOALLOC_CUDA(cudaMemcpyAsync(counts, b.counts + k, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    LoopState hs;
    NOALLOC_CUDA(cudaMemcpyAsync(&hs, b.st, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
    NOALLOC_CUDA(cudaStreamSynchronize(s));
    if (hs.bad_label) return nfail(POPCORN_ERR_INVALID, "a label is outside [0, %d)", k);
    if (objective) *objective = hs.J_last;
    if (changed) *changed = hs.last_changed;
    return POPCORN_OK;
}

}  // extern "C"
