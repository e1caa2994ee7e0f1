// FP32 CUDA-core build of the kernel matrix K = kappa(P P^T).
//
// Sec. 3.2: B = P P^T, then the kernel function elementwise (polynomial:
// (gamma B + c)^r; Gaussian: exp(-gamma ||p_i - p_j||^2 / sigma^2)).  The
// paper forms B with GEMM or SYRK plus a triangle copy and a separate
// transform pass (Sec. 4.2); here one kernel computes each upper-triangle
// 128 x 128 tile once, applies kappa in registers and stores the tile and its
// transpose, so B never exists in memory and no copy pass runs.
//
// The Gaussian squared distance takes one of two forms, decided on the device
// per launch from the largest row norm.  The norm expansion of Eq. 12,
// r_i + r_j - 2 p_i.p_j, costs one multiply-add per pair and coordinate; its
// rounding error in a kernel value is about 4 sqrt(d) u max_i r_i gamma /
// sigma^2 (u = 2^-24: the dot product's and the norms' roundings, the
// cancellation bounded by the norms), and it is used when that stays below
// 1e-6, the FP32 parity bar on K.  Otherwise (points far from the origin
// relative to sigma, where the expansion cancels) the distance is summed from
// coordinate differences, a subtract and a multiply-add per pair and
// coordinate, which keeps full relative accuracy for near-duplicate points.
#include "popcorn_internal.cuh"
#include "tc_common.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <type_traits>

namespace popcorn {
namespace {

constexpr int TILE = 128;
constexpr int KC = 16;          // depth of one shared-memory slice (double-buffered)
constexpr int LDS = TILE + 4;   // padded row

// Internal kernel kind: the Gaussian with its distance from the norm expansion (Eq. 12).
constexpr int kGaussExpand = 3;

template <int KIND>
__device__ __forceinline__ float apply_kernel(float v, const KernParams& kp) {
    if (KIND == POPCORN_LINEAR) return v;
    if (KIND == POPCORN_POLYNOMIAL) {
        float base = fmaf(kp.gamma, v, kp.coef0);
        float r = base;
        for (int e = 1; e < kp.degree; ++e) r *= base;
        return r;
    }
    return expf(kp.neg_gamma_over_sigma2 * v);   // v = ||p_i - p_j||^2
}

// Row norms r_i = sum_l p_il^2 (one warp a row, a fixed reduction order) and the largest
// of them (positive floats order like their bit patterns).
__global__ void __launch_bounds__(256) row_norms_kernel(const float* __restrict__ P, int n, int d, int64_t ldp,
                                                        float* __restrict__ rn, unsigned* __restrict__ maxr) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float* p = P + (int64_t)row * ldp;
    float s = 0.f;
    for (int l = lane; l < d; l += 32) s = fmaf(p[l], p[l], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        rn[row] = s;
        atomicMax(maxr, __float_as_uint(s));
    }
}

// Stored element type of K and its 4-wide packed store.
template <typename TK> struct KStore;
template <> struct KStore<float> {
    __device__ static float round(float v) { return v; }
    __device__ static void put4(float* p, float a, float b, float c, float d) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    }
    __device__ static void put1(float* p, float a) { *p = a; }
};
template <> struct KStore<__half> {
    __device__ static float round(float v) { return __half2float(__float2half_rn(v)); }
    __device__ static void put4(__half* p, float a, float b, float c, float d) {
        __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&lo);
        u.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(p) = u;
    }
    __device__ static void put1(__half* p, float a) { *p = __float2half_rn(a); }
};
template <> struct KStore<__nv_bfloat16> {
    __device__ static float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    __device__ static void put4(__nv_bfloat16* p, float a, float b, float c, float d) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&lo);
        u.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(p) = u;
    }
    __device__ static void put1(__nv_bfloat16* p, float a) { *p = __float2bfloat16_rn(a); }
};

// One upper-triangle tile (number `tile`) of K: RPT x 8 outputs a thread, 256 threads
// (RPT = 8) or 128 (RPT = 16).  The depth loop runs over KC-wide slices of the two
// 128-row operand blocks, double-buffered in shared memory: while a slice is consumed,
// the next one is already in flight into registers (float4 loads when rows are 16-byte
// aligned).  A thread reads RPT / 4 + 2 float4 a depth step for 8 RPT multiply-adds:
// RPT = 16 halves the shared-memory traffic a multiply-add, which is what bounds the
// dot-product kinds (one multiply-add a pair and coordinate) at RPT = 8; the
// coordinate-difference Gaussian (two operations) keeps RPT = 8.
// kdiag receives the stored (rounded) diagonal so that diag K and K agree.
struct TileSmem {
    float As[2][KC][LDS];
    float Bs[2][KC][LDS];
};

// PACKED: 0 = row-major full square (tile and transpose); kPackedSw16 / kPackedSw4 = the
// block-packed upper triangle in the tile layout of that name (popcorn_internal.cuh).
template <int KIND, typename TK = float, bool ONE_SLICE = false, int PACKED = 0, int RPT = 8>
__device__ __forceinline__ void kbuild_tile(const float* __restrict__ P, int n, int d, int64_t ldp,
                                            const KernParams& kp, TK* __restrict__ K, int64_t ldk,
                                            float* __restrict__ kdiag, int T, long long tile, TileSmem& sm,
                                            int full = 0, const float* __restrict__ rn = nullptr) {
    auto& As = sm.As;
    auto& Bs = sm.Bs;
    int bi, bj;
    if (full) {   // every tile of the square, row by row (the GEMM form): no transposes
        bi = (int)(tile / T);
        bj = (int)(tile % T);
    } else {
        tri_coords(tile, T, &bi, &bj);
    }
    static_assert(RPT == 8 || RPT == 16, "8 or 16 rows a thread");
    constexpr int NT = RPT == 8 ? 256 : 128;       // threads
    constexpr int RS = TILE / (RPT / 4);           // rows between a thread's groups of 4 rows
    constexpr int NF = (KC / 4) / (NT / 128);      // float4 a thread fetches per operand and slice
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int row0 = bi * TILE, col0 = bj * TILE;
    const bool vec = (ldp & 3) == 0 && ((uintptr_t)P & 15) == 0;

    // slice fill: thread tid carries float4 f = (tid >> 7) + (NT / 128) rep of row tid & 127
    const int fr = tid & 127;
    auto fetch = [&](int base, int l0, int rep) -> float4 {
        const int r = base + fr, gl = l0 + 4 * ((tid >> 7) + (NT / 128) * rep);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < n) {
            const float* p = P + (int64_t)r * ldp + gl;
            if (vec && gl + 3 < d) {
                v = __ldg(reinterpret_cast<const float4*>(p));
            } else {
                if (gl < d) v.x = __ldg(p);
                if (gl + 1 < d) v.y = __ldg(p + 1);
                if (gl + 2 < d) v.z = __ldg(p + 2);
                if (gl + 3 < d) v.w = __ldg(p + 3);
            }
        }
        return v;
    };
    auto put = [&](float (*S)[LDS], int rep, const float4& v) {
        const int l = 4 * ((tid >> 7) + (NT / 128) * rep);
        S[l][fr] = v.x;
        S[l + 1][fr] = v.y;
        S[l + 2][fr] = v.z;
        S[l + 3][fr] = v.w;
    };

    // The dot-product kinds on 16 x 8 outputs keep their sums as f32x2 pairs (rows 2i and
    // 2i + 1 of column y): one fma.rn.f32x2 does two multiply-adds, which halves the
    // instructions the FMA pipe is fed with (each lane rounds exactly as fma.rn.f32).
    constexpr bool PAIRS = RPT == 16 && KIND != POPCORN_GAUSSIAN;
    float acc[RPT][8];
    unsigned long long acc2[PAIRS ? RPT / 2 : 1][8];
#pragma unroll
    for (int x = 0; x < RPT; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
#pragma unroll
    for (int i = 0; i < (PAIRS ? RPT / 2 : 1); ++i)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc2[i][y] = 0ull;

    float4 na[NF], nb[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        na[q] = fetch(row0, 0, q);
        nb[q] = fetch(col0, 0, q);
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        put(As[0], q, na[q]);
        put(Bs[0], q, nb[q]);
    }
    __syncthreads();
    int buf = 0;
    for (int l0 = 0; l0 < d; l0 += KC) {
        const bool more = !ONE_SLICE && l0 + KC < d;
        if (more) {
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                na[q] = fetch(row0, l0 + KC, q);
                nb[q] = fetch(col0, l0 + KC, q);
            }
        }
#pragma unroll
        for (int l = 0; l < KC; ++l) {
            float a[RPT], b[8];
#pragma unroll
            for (int m = 0; m < RPT / 4; ++m) {
                const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][l][RS * m + ty * 4]);
                a[4 * m] = a4.x;
                a[4 * m + 1] = a4.y;
                a[4 * m + 2] = a4.z;
                a[4 * m + 3] = a4.w;
            }
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][l][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][l][64 + tx * 4]);
            b[0] = b0.x, b[1] = b0.y, b[2] = b0.z, b[3] = b0.w, b[4] = b1.x, b[5] = b1.y, b[6] = b1.z, b[7] = b1.w;
            if constexpr (PAIRS) {
                unsigned long long bb[8];
#pragma unroll
                for (int y = 0; y < 8; ++y) bb[y] = tc::f2pack(b[y], b[y]);
#pragma unroll
                for (int i = 0; i < RPT / 2; ++i) {
                    const unsigned long long aa = tc::f2pack(a[2 * i], a[2 * i + 1]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) acc2[i][y] = tc::f2fma(aa, bb[y], acc2[i][y]);
                }
            } else {
#pragma unroll
                for (int x = 0; x < RPT; ++x)
#pragma unroll
                    for (int y = 0; y < 8; ++y) {
                        if constexpr (KIND == POPCORN_GAUSSIAN) {
                            float t = a[x] - b[y];
                            acc[x][y] = fmaf(t, t, acc[x][y]);
                        } else {
                            acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
                        }
                    }
            }
        }
        if (more) {
            // the other buffer was last read before the previous barrier
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                put(As[buf ^ 1], q, na[q]);
                put(Bs[buf ^ 1], q, nb[q]);
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    if constexpr (PAIRS) {
#pragma unroll
        for (int i = 0; i < RPT / 2; ++i)
#pragma unroll
            for (int y = 0; y < 8; ++y) tc::f2unpack(acc2[i][y], acc[2 * i][y], acc[2 * i + 1][y]);
    }
    // epilogue: kappa, diagonal, store tile and (off-diagonal tiles) its transpose
    if constexpr (KIND == kGaussExpand) {
        // d2 = r_i + r_j - 2 b (Eq. 12), clamped at 0; rows / columns past n take 0
        float ri[RPT], rj[8];
#pragma unroll
        for (int x = 0; x < RPT; ++x) {
            const int r = row0 + ty * 4 + (x & 3) + RS * (x >> 2);
            ri[x] = r < n ? rn[r] : 0.f;
        }
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int c = col0 + tx * 4 + (y & 3) + 64 * (y >> 2);
            rj[y] = c < n ? rn[c] : 0.f;
        }
#pragma unroll
        for (int x = 0; x < RPT; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y)
                acc[x][y] = apply_kernel<POPCORN_GAUSSIAN>(fmaxf(fmaf(-2.f, acc[x][y], ri[x] + rj[y]), 0.f), kp);
    } else {
#pragma unroll
        for (int x = 0; x < RPT; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = apply_kernel<KIND>(acc[x][y], kp);
    }

    if (bi == bj) {
#pragma unroll
        for (int x = 0; x < RPT; ++x) {
            int r = row0 + ty * 4 + (x & 3) + RS * (x >> 2);
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                int c = col0 + tx * 4 + (y & 3) + 64 * (y >> 2);
                if (r == c && r < n) {
                    if (KIND == POPCORN_GAUSSIAN || KIND == kGaussExpand) acc[x][y] = 1.0f;
                    kdiag[r] = KStore<TK>::round(acc[x][y]);
                }
            }
        }
    }

    if constexpr (PACKED == kPackedSw128H) {
        // FP16 / BF16 square as 32 KB tiles (batched mode): tile (I, J) at K + (I T + J) 32 KB,
        // two boxes of 128 rows x 64 columns in the 128-byte swizzle, element (r, c) at byte
        // 16384 (c >> 6) + 128 r + 16 (((c >> 3) & 7) ^ (r & 7)) + 2 (c & 7); entries past n
        // are zeros.  A thread's 4 consecutive columns (4-aligned) are 8 bytes of one 16-byte
        // chunk; so are its 4 consecutive rows in the transposed tile (J, I).
        static_assert(sizeof(TK) == 2, "half tiles hold FP16 / BF16 K");
        unsigned char* base = reinterpret_cast<unsigned char*>(K);
        auto off = [](int r, int c) { return 16384 * (c >> 6) + 128 * r + 16 * (((c >> 3) & 7) ^ (r & 7)) + 2 * (c & 7); };
        auto put = [](unsigned char* p, float a, float b, float c, float d) {
            uint2 u;
            if constexpr (std::is_same<TK, __half>::value) {
                __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
            } else {
                __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
            }
            *reinterpret_cast<uint2*>(p) = u;
        };
        unsigned char* Bd = base + ((size_t)bi * T + bj) * 32768;
#pragma unroll
        for (int x = 0; x < RPT; ++x) {
            const int rl = ty * 4 + (x & 3) + RS * (x >> 2);
            const bool rv = row0 + rl < n;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cl = 64 * h + tx * 4, c = col0 + cl;
                const float* v = &acc[x][4 * h];
                put(Bd + off(rl, cl), rv && c < n ? v[0] : 0.f, rv && c + 1 < n ? v[1] : 0.f,
                    rv && c + 2 < n ? v[2] : 0.f, rv && c + 3 < n ? v[3] : 0.f);
            }
        }
        if (bi != bj) {   // rows of block bi < bj are all below n
            unsigned char* Bt = base + ((size_t)bj * T + bi) * 32768;
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                const int cl = tx * 4 + (y & 3) + 64 * (y >> 2);
                const bool cv = col0 + cl < n;
#pragma unroll
                for (int g = 0; g < RPT / 4; ++g) {
                    const int rl = RS * g + ty * 4;
                    put(Bt + off(cl, rl), cv ? acc[4 * g][y] : 0.f, cv ? acc[4 * g + 1][y] : 0.f,
                        cv ? acc[4 * g + 2][y] : 0.f, cv ? acc[4 * g + 3][y] : 0.f);
                }
            }
        }
        return;
    } else if constexpr (PACKED != 0) {
        // block-packed upper triangle: tile t is 64 KB at K + t * 128 * 128, as four boxes of
        // 128 rows x 32 columns, the layout the symmetric pass loads with one bulk copy.
        // kPackedSw16: 16-byte chunk j of row r stored at chunk j ^ (r mod 8) (the 128-byte
        // swizzle).  kPackedSw4: element c of row r stored at c ^ (r mod 32), so that both a
        // row and a column of a box are read without bank conflicts.  This thread's 4
        // consecutive columns (4-aligned) stay in one 16-byte chunk under either layout; under
        // kPackedSw4 they are permuted inside it by (r mod 4), which is x mod 4 here (a
        // compile-time constant), so each store is still one float4.  The whole tile is
        // written: entries past n are finite and no pass reads them.
        static_assert(sizeof(TK) == 4, "packed storage holds FP32 K");
        float* B = reinterpret_cast<float*>(K) + (size_t)tile * (TILE * TILE);
#pragma unroll
        for (int x = 0; x < RPT; ++x) {
            const int rl = ty * 4 + (x & 3) + RS * (x >> 2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cl = 64 * h + tx * 4;
                const float* v = &acc[x][4 * h];
                if constexpr (PACKED == kPackedSw16) {
                    const int j = (cl & 31) >> 2;
                    *reinterpret_cast<float4*>(B + (cl >> 5) * (TILE * 32) + rl * 32 + ((j ^ (rl & 7)) << 2)) =
                        make_float4(v[0], v[1], v[2], v[3]);
                } else {
                    const int q = x & 3;   // == rl & 3 (the loop is unrolled: a constant)
                    *reinterpret_cast<float4*>(B + (cl >> 5) * (TILE * 32) + rl * 32 +
                                               ((cl & 31) ^ (rl & 28))) = make_float4(v[q], v[1 ^ q], v[2 ^ q], v[3 ^ q]);
                }
            }
        }
        return;
    }
#pragma unroll
    for (int x = 0; x < RPT; ++x) {
        int r = row0 + ty * 4 + (x & 3) + RS * (x >> 2);
        if (r >= n) continue;
        TK* Kr = K + (int64_t)r * ldk;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int c = col0 + 64 * h + tx * 4;
            const float v0 = acc[x][4 * h], v1 = acc[x][4 * h + 1], v2 = acc[x][4 * h + 2], v3 = acc[x][4 * h + 3];
            if (c + 3 < n) {
                KStore<TK>::put4(Kr + c, v0, v1, v2, v3);
            } else {
                if (c < n) KStore<TK>::put1(Kr + c, v0);
                if (c + 1 < n) KStore<TK>::put1(Kr + c + 1, v1);
                if (c + 2 < n) KStore<TK>::put1(Kr + c + 2, v2);
            }
        }
    }
    if (bi != bj && !full) {
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            int c = col0 + tx * 4 + (y & 3) + 64 * (y >> 2);
            if (c >= n) continue;
            TK* Kc = K + (int64_t)c * ldk;
#pragma unroll
            for (int g = 0; g < RPT / 4; ++g) {
                int r = row0 + RS * g + ty * 4;   // row0 tiles are full (bi < bj => rows < n)
                KStore<TK>::put4(Kc + r, acc[4 * g][y], acc[4 * g + 1][y], acc[4 * g + 2][y], acc[4 * g + 3][y]);
            }
        }
    }
}

// The Gaussian instances choose the distance form here, uniformly for the launch: the norm
// expansion when expand_coef * max_i r_i <= 1e-6 (rn / maxr from row_norms_kernel).  With
// dot_expands set, a separate kbuild_dot_kernel launch takes the expansion and this one
// returns at once when it applies.
__device__ __forceinline__ bool expansion_applies(const float* rn, const unsigned* maxr, float expand_coef) {
    return rn && __uint_as_float(*maxr) * expand_coef <= 1e-6f;
}

template <int KIND, typename TK, int PACKED>
__global__ void __launch_bounds__(256) kbuild_simt_kernel(const float* __restrict__ P, int n, int d, int64_t ldp,
                                                          KernParams kp, TK* __restrict__ K, int64_t ldk,
                                                          float* __restrict__ kdiag, int T, int full,
                                                          const float* __restrict__ rn, const unsigned* maxr,
                                                          float expand_coef, int dot_expands) {
    __shared__ __align__(16) TileSmem sm;
    const bool expand = KIND == POPCORN_GAUSSIAN && expansion_applies(rn, maxr, expand_coef);
    if (expand && dot_expands) return;
    if (expand)
        kbuild_tile<kGaussExpand, TK, false, PACKED>(P, n, d, ldp, kp, K, ldk, kdiag, T, (long long)blockIdx.x, sm,
                                                     full, rn);
    else
        kbuild_tile<KIND, TK, false, PACKED>(P, n, d, ldp, kp, K, ldk, kdiag, T, (long long)blockIdx.x, sm, full);
}

// The dot-product kinds (linear, polynomial, the Gaussian by the norm expansion) on FP32 K:
// 16 x 8 outputs a thread, 128 threads.  The Gaussian instance returns at once when the
// expansion does not apply (the 256-thread kernel then forms coordinate differences).
template <int KIND, int PACKED>
__global__ void __launch_bounds__(128, 2) kbuild_dot_kernel(const float* __restrict__ P, int n, int d, int64_t ldp,
                                                            KernParams kp, float* __restrict__ K, int64_t ldk,
                                                            float* __restrict__ kdiag, int T, int full,
                                                            const float* __restrict__ rn, const unsigned* maxr,
                                                            float expand_coef) {
    __shared__ __align__(16) TileSmem sm;
    if (KIND == kGaussExpand && !expansion_applies(rn, maxr, expand_coef)) return;
    kbuild_tile<KIND, float, false, PACKED, 16>(P, n, d, ldp, kp, K, ldk, kdiag, T, (long long)blockIdx.x, sm, full,
                                                rn);
}

// d <= KC: the depth loop is one slice, so no next slice is held in registers;
// the lighter kernel fits two blocks per SM, which overlaps one block's stores
// with the other's loads (small d is store-bound)
template <int KIND, typename TK, int PACKED>
__global__ void __launch_bounds__(256, 2) kbuild_simt_small_kernel(const float* __restrict__ P, int n, int d,
                                                                   int64_t ldp, KernParams kp, TK* __restrict__ K,
                                                                   int64_t ldk, float* __restrict__ kdiag, int T,
                                                                   int full, const float* __restrict__ rn,
                                                                   const unsigned* maxr, float expand_coef) {
    __shared__ __align__(16) TileSmem sm;
    if (KIND == POPCORN_GAUSSIAN && expansion_applies(rn, maxr, expand_coef))
        kbuild_tile<kGaussExpand, TK, true, PACKED>(P, n, d, ldp, kp, K, ldk, kdiag, T, (long long)blockIdx.x, sm,
                                                    full, rn);
    else
        kbuild_tile<KIND, TK, true, PACKED>(P, n, d, ldp, kp, K, ldk, kdiag, T, (long long)blockIdx.x, sm, full);
}

template <typename TK, int PACKED>
cudaError_t launch_simt_typed(const float* P, int n, int d, int64_t ldp, KernParams kp, TK* K, int64_t ldk,
                              float* kdiag, cudaStream_t s, int full, float* rn, unsigned* maxr, int* launches) {
    const int T = (n + TILE - 1) / TILE;
    // Gaussian: row norms and their maximum first (the build then picks the distance form);
    // 4 sqrt(d) u gamma / sigma^2 bounds the expansion's error per unit of max_i r_i
    float expand_coef = 0.f;
    if (kp.kind == POPCORN_GAUSSIAN && rn && maxr) {
        cudaError_t e = cudaMemsetAsync(maxr, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        row_norms_kernel<<<(unsigned)(((int64_t)n * 32 + 255) / 256), 256, 0, s>>>(P, n, d, ldp, rn, maxr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) ++*launches;
        expand_coef = (float)(4.0 * sqrt((double)d) * ldexp(1.0, -24) * fabs((double)kp.neg_gamma_over_sigma2));
    } else {
        rn = nullptr;
    }
    const long long tiles = full ? (long long)T * T : (long long)T * (T + 1) / 2;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)tiles), block(256);
    if (d <= KC) {
        switch (kp.kind) {
            case POPCORN_LINEAR:
                kbuild_simt_small_kernel<POPCORN_LINEAR, TK, PACKED>
                    <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef);
                break;
            case POPCORN_POLYNOMIAL:
                kbuild_simt_small_kernel<POPCORN_POLYNOMIAL, TK, PACKED>
                    <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef);
                break;
            default:
                kbuild_simt_small_kernel<POPCORN_GAUSSIAN, TK, PACKED>
                    <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef);
                break;
        }
        return cudaGetLastError();
    }
    if constexpr (std::is_same<TK, float>::value) {
        // FP32 K, d > KC: the dot-product kinds on the 16 x 8 kernel; the Gaussian launches both
        // forms, and the one whose distance form does not apply returns at once
        dim3 dblock(128);
        switch (kp.kind) {
            case POPCORN_LINEAR:
                kbuild_dot_kernel<POPCORN_LINEAR, PACKED>
                    <<<grid, dblock, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef);
                return cudaGetLastError();
            case POPCORN_POLYNOMIAL:
                kbuild_dot_kernel<POPCORN_POLYNOMIAL, PACKED>
                    <<<grid, dblock, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef);
                return cudaGetLastError();
            default:
                if (rn) {
                    kbuild_dot_kernel<kGaussExpand, PACKED>
                        <<<grid, dblock, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef);
                    cudaError_t e = cudaGetLastError();
                    if (e != cudaSuccess) return e;
                    if (launches) ++*launches;
                }
                kbuild_simt_kernel<POPCORN_GAUSSIAN, TK, PACKED>
                    <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef, 1);
                return cudaGetLastError();
        }
    }
    switch (kp.kind) {
        case POPCORN_LINEAR:
            kbuild_simt_kernel<POPCORN_LINEAR, TK, PACKED>
                <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef, 0);
            break;
        case POPCORN_POLYNOMIAL:
            kbuild_simt_kernel<POPCORN_POLYNOMIAL, TK, PACKED>
                <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef, 0);
            break;
        default:
            kbuild_simt_kernel<POPCORN_GAUSSIAN, TK, PACKED>
                <<<grid, block, 0, s>>>(P, n, d, ldp, kp, K, ldk, kdiag, T, full, rn, maxr, expand_coef, 0);
            break;
    }
    return cudaGetLastError();
}

// All instances of a batch: flattened tile b belongs to the instance whose
// tile0 is the largest one <= b.
// TK float: each instance's FP32 square, row-major (K, ldk); TK __half / __nv_bfloat16: its
// square as half tiles (Kh, kPackedSw128H), for the tensor-core batched stream.
template <typename TK>
__global__ void __launch_bounds__(256, 2) batched_kbuild_kernel(const BatchInst* I, int count) {
    const long long b = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (I[mid].tile0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const BatchInst& x = I[lo];
    const long long t = b - x.tile0;
    __shared__ __align__(16) TileSmem sm;   // one copy for the three kernel functions
    constexpr int PK = sizeof(TK) == 2 ? kPackedSw128H : 0;
    TK* K = sizeof(TK) == 2 ? reinterpret_cast<TK*>(x.Kh) : reinterpret_cast<TK*>(x.K);
    switch (x.kp.kind) {
        case POPCORN_LINEAR:
            kbuild_tile<POPCORN_LINEAR, TK, false, PK>(x.P, x.n, x.d, x.ldp, x.kp, K, x.ldk, x.kdiag, x.T, t, sm);
            break;
        case POPCORN_POLYNOMIAL:
            kbuild_tile<POPCORN_POLYNOMIAL, TK, false, PK>(x.P, x.n, x.d, x.ldp, x.kp, K, x.ldk, x.kdiag, x.T, t, sm);
            break;
        default:
            kbuild_tile<POPCORN_GAUSSIAN, TK, false, PK>(x.P, x.n, x.d, x.ldp, x.kp, K, x.ldk, x.kdiag, x.T, t, sm);
            break;
    }
}

}  // namespace

cudaError_t launch_batched_kbuild_simt(const BatchInst* dI, const BatchPlan& bp, cudaStream_t s) {
    if (bp.tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (bp.half == POPCORN_K_FP16)
        batched_kbuild_kernel<__half><<<(unsigned)bp.tiles, 256, 0, s>>>(dI, bp.count);
    else if (bp.half == POPCORN_K_BF16)
        batched_kbuild_kernel<__nv_bfloat16><<<(unsigned)bp.tiles, 256, 0, s>>>(dI, bp.count);
    else
        batched_kbuild_kernel<float><<<(unsigned)bp.tiles, 256, 0, s>>>(dI, bp.count);
    return cudaGetLastError();
}

cudaError_t launch_kbuild_simt(const float* P, int n, int d, int64_t ldp, KernParams kp, void* K, int64_t ldk,
                               int k_storage, float* kdiag, cudaStream_t s, int* launches, int packed, int full,
                               float* rn, unsigned* maxr) {
    if (launches) ++*launches;
    if (packed) {
        if (k_storage != POPCORN_K_FP32) return cudaErrorInvalidValue;
        if (packed == kPackedSw4)
            return launch_simt_typed<float, kPackedSw4>(P, n, d, ldp, kp, static_cast<float*>(K), ldk, kdiag, s, 0,
                                                        rn, maxr, launches);
        return launch_simt_typed<float, kPackedSw16>(P, n, d, ldp, kp, static_cast<float*>(K), ldk, kdiag, s, 0, rn,
                                                     maxr, launches);
    }
    if (k_storage == POPCORN_K_FP16)
        return launch_simt_typed<__half, 0>(P, n, d, ldp, kp, static_cast<__half*>(K), ldk, kdiag, s, 0, rn, maxr,
                                            launches);
    if (k_storage == POPCORN_K_BF16)
        return launch_simt_typed<__nv_bfloat16, 0>(P, n, d, ldp, kp, static_cast<__nv_bfloat16*>(K), ldk, kdiag, s, 0,
                                                   rn, maxr, launches);
    return launch_simt_typed<float, 0>(P, n, d, ldp, kp, static_cast<float*>(K), ldk, kdiag, s, full, rn, maxr,
                                       launches);
}

}  // namespace popcorn
