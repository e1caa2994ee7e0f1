// Half-precision copy of the block-packed upper triangle of K.
//
// The symmetric pass reads K once a pass; stored in FP16 or BF16 (the K storage option,
// an extension of the paper's FP32 K), the packed triangle is half the bytes again.  The K
// builds write the FP32 triangle in the XOR-32 layout (kPackedSw4); pack_half_kernel rounds
// it, once a fit, into kPackedSw128H, 32 KB a tile:
//   element (r, C) at byte 16384 (C >> 6) + 128 r + 16 (((C >> 3) & 7) ^ (r & 7)) + 2 (C & 7),
// two boxes of 128 rows x 64 columns in the 128-byte swizzle of the tensor cores' shared-
// memory operands: the tile is, byte for byte, the A operand of the symmetric pass's MMAs --
// K-major for the row sums (rows r, reduction over C) and MN-major for the column sums
// (rows C, reduction over r).  Entries past n (a ragged last block) are stored as zeros, so
// that the one-hot operand's zeros meet finite values.  The diagonal tiles also round
// diag K, so that K_ii and K agree.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "half_common.cuh"
#include "popcorn_internal.cuh"

namespace popcorn {
namespace {

constexpr int kPackThreads = 256;

using hstore::pack2;
using hstore::round_trip;

// element (r, C) of an FP32 tile in the XOR-32 layout, in floats
__device__ __forceinline__ int sw4(int r, int C) { return 4096 * (C >> 5) + 32 * r + ((C & 31) ^ (r & 31)); }

template <typename TH>
__global__ void __launch_bounds__(kPackThreads) pack_half_kernel(const float* __restrict__ Kf, uint32_t* Kh,
                                                                 int T, int n, float* kdiag) {
    extern __shared__ __align__(16) float tile[];   // 16384 floats
    const long long t = blockIdx.x;
    const float4* src = reinterpret_cast<const float4*>(Kf + t * 16384);
    for (int q = threadIdx.x; q < 4096; q += kPackThreads) reinterpret_cast<float4*>(tile)[q] = __ldcs(src + q);
    __syncthreads();
    int I, J;
    tri_coords(t, T, &I, &J);
    const int rows = n - I * 128, cols = n - J * 128;   // valid rows and columns of the tile
    uint32_t* dst = Kh + t * 8192;
    for (int o = threadIdx.x; o < 8192; o += kPackThreads) {
        // word o: box o >> 12, row (o >> 5) & 127, 16-byte chunk (o >> 2) & 7 of the row (the
        // swizzled position of logical chunk ((o >> 2) & 7) ^ (row & 7)), columns 2 (o & 3) + {0, 1}
        const int b = o >> 12, r = (o >> 5) & 127;
        const int C = 64 * b + 8 * (((o >> 2) & 7) ^ (r & 7)) + 2 * (o & 3);
        const float x0 = (r < rows && C < cols) ? tile[sw4(r, C)] : 0.f;
        const float x1 = (r < rows && C + 1 < cols) ? tile[sw4(r, C + 1)] : 0.f;
        dst[o] = pack2<TH>(x0, x1);
    }
    if (I == J && threadIdx.x < 128) {
        const int i = I * 128 + threadIdx.x;
        if (i < n) kdiag[i] = round_trip<TH>(tile[sw4(threadIdx.x, threadIdx.x)]);
    }
}

}  // namespace

cudaError_t configure_pack_half() {
    cudaError_t e = cudaFuncSetAttribute(pack_half_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pack_half_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
}

cudaError_t launch_pack_half(const float* Kf, void* Kh, int k_storage, int n, float* kdiag, cudaStream_t s) {
    const int T = (n + 127) / 128;
    const long long tiles = (long long)T * (T + 1) / 2;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (k_storage == POPCORN_K_FP16)
        pack_half_kernel<__half><<<(unsigned)tiles, kPackThreads, 65536, s>>>(Kf, static_cast<uint32_t*>(Kh), T, n,
                                                                              kdiag);
    else
        pack_half_kernel<__nv_bfloat16><<<(unsigned)tiles, kPackThreads, 65536, s>>>(
            Kf, static_cast<uint32_t*>(Kh), T, n, kdiag);
    return cudaGetLastError();
}

}  // namespace popcorn
