// ensf_conv.cu -- the U-Net surrogate's 3x3 circular convolutions on the
// tensor cores (sm_103a): the forward convolution and the data gradient as one
// implicit-GEMM kernel over TMA boxes of the haloed NHWC input (k_conv3x3),
// the weight gradient as nine GEMMs over the pixels of column-shifted input
// copies (k_conv3x3_wgrad), and their helper kernels.  The MMAs are
// tcgen05.mma kind::f16 (BF16 operands, FP32 accumulators in TMEM); every
// mbarrier wait is bounded (ENSF_ETIMEOUT in the error word on expiry).
#include <cuda_bf16.h>

#include <algorithm>

#include "ensf_internal.h"
#include "ensf_ptx.cuh"
#include "ensf_tc.h"

namespace ensf {

namespace {

// ------------------------------------------------ 3x3 convolution (implicit GEMM)
// out[p][n] = sum over taps (dy, dx) and input channels c of
//             xpad[b][y + dy][x + dx][c] * wt[n][(dy * 3 + dx) * C + c]
// for output pixel p = (b, y, x) of an image of h x w pixels, xpad the input
// with a one-pixel circular halo ((h + 2) x (w + 2) per image, NHWC, BF16).
// One CTA computes 128 pixels (128 / w whole image rows) x BN output
// channels: k-block kb = tap * (C / 32) + channel block is one TMA box of
// 32 channels x w pixels x 128 / w rows read at the tap's offset from xpad,
// plus 32 columns of the K-major weights, so no im2col matrix exists.  The
// epilogue adds the bias and applies SiLU (act) or stores the plain sums
// (the data gradient, with the weights' taps mirrored by the caller).
struct ConvParams {
    int P;          // output pixels (a multiple of 128)
    int N;          // output channels
    int cblk;       // input channels / 32
    int h, w, hp;   // image rows and columns, padded rows h + 2
    int rows;       // image rows per 128-pixel tile (128 / w)
    const float *bias;  // [N] or NULL
    int act;            // 1: z = sum + bias, y = SiLU(z); 0: the sum alone
    float *out32;       // [P][N] FP32 (the pre-activation z, or the data gradient)
    __nv_bfloat16 *out16;  // [P][N] BF16 SiLU(z), or NULL
    int *err;
};

constexpr int kConvKB = 32;     // input channels per k-block (64-byte rows)
constexpr int kConvStages = 6;
struct ConvPlan {
    static constexpr int kA = BM * kConvKB * 2;      // 8 KB: 128 pixels x 32 channels
    static constexpr int kBmax = 256 * kConvKB * 2;  // 16 KB: up to 256 output channels
    static constexpr int kStage = kA + kBmax;
    static constexpr int kBarOff = kStage * kConvStages;
    static constexpr int kBytes = kBarOff + 256 + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__global__ void __launch_bounds__(192, 1)
k_conv3x3(const __grid_constant__ CUtensorMap a_map, const __grid_constant__ CUtensorMap b_map, ConvParams p, int BN,
          uint32_t tmem_cols) {
    using P = ConvPlan;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(p.err) != 0) return;
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = smem_raw + pad;
    const int sstride = P::kA + BN * kConvKB * 2;  // stage bytes for this BN (a multiple of 1024)
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + sstride * kConvStages);
    uint64_t *empty = full + kConvStages;
    uint64_t *accum = empty + kConvStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kConvStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int p0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int img = p0 / (p.h * p.w), y0 = (p0 / p.w) % p.h;
    const int nkb = 9 * p.cblk;
    const uint32_t stage_bytes = P::kA + BN * kConvKB * 2;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kConvStages;
                const uint32_t ph = (kb / kConvStages) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.err)) break;
                const uint32_t st = smem_u32(tiles + s * sstride);
                mbar_expect_tx(&full[s], stage_bytes);
                const int tap = kb / p.cblk, cb = kb % p.cblk;
                tma_load_3d(st, &a_map, &full[s], cb * kConvKB, tap % 3, img * p.hp + y0 + tap / 3);
                tma_load_2d(st + P::kA, &b_map, &full[s], kb * kConvKB, n0);
                issued = kb + 1;
            }
            if (*abort_flag) {
                const uint64_t t0 = globaltimer();
                for (int i = issued > kConvStages ? issued - kConvStages : 0; i < issued; ++i) {
                    const int s = i % kConvStages;
                    while (!mbar_try_wait(&full[s], (i / kConvStages) & 1) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, BN);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kConvStages;
                const uint32_t ph = (kb / kConvStages) & 1;
                if (!mbar_wait(&full[s], ph, abort_flag, p.err)) break;
                tc_fence_after();
                const uint32_t a = smem_u32(tiles + s * sstride);
                const uint32_t b = a + P::kA;
#pragma unroll
                for (int kk = 0; kk < kConvKB / 16; ++kk)
                    mma_bf16(tmem, desc_sw64(a + kk * 32), desc_sw64(b + kk * 32), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            mma_commit(accum);
        }
    } else {
        const int q = warp & 3;  // TMEM lane quarter
        const int pix = p0 + q * 32 + lane;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(accum, 0, abort_flag, p.err));
        tc_fence_after();
        if (ok) {
            for (int cc = 0; cc < BN; cc += 32) {
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + cc, v);
                const int nb = n0 + cc;
                if (nb >= p.N) continue;
                if (p.act) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = __fadd_rn(v[e], p.bias[nb + e]);
                }
                if (p.out32) {
                    float *o32 = p.out32 + static_cast<int64_t>(pix) * p.N + nb;
#pragma unroll
                    for (int e = 0; e < 32; e += 4)
                        *reinterpret_cast<float4 *>(o32 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                }
                if (p.out16) {
                    __nv_bfloat16 *o16 = p.out16 + static_cast<int64_t>(pix) * p.N + nb;
#pragma unroll
                    for (int e = 0; e < 32; e += 8) {
                        __align__(16) __nv_bfloat16 t8[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float z = v[e + k];
                            t8[k] = __float2bfloat16_rn(z * (1.f / (1.f + __expf(-z))));
                        }
                        *reinterpret_cast<uint4 *>(o16 + e) = *reinterpret_cast<const uint4 *>(t8);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// ---------------------------------------- 3x3 convolution, weight gradient
// dW[n][tap][c] = sum_p dZ[p][n] * x[b][y + dy - 1][x + dx - 1][c]  (circular)
// as GEMMs over the pixels, one per tap: A = dZ^T [N][P] (K-major), B = the
// input transposed with the tap's column shift applied in advance:
// xs[dx][c][b * (h + 2) + yy][x] = x[b][(yy - 1) mod h][(x + dx - 1) mod w][c]
// (three copies, one per dx, with a one-row circular halo), read as 4-D TMA
// boxes whose innermost coordinate (the pixel column) is always a multiple of
// the k-block; the tap's row shift lands on a non-innermost coordinate.  A
// k-block is KB pixels of one image row.  Split-K over the pixels: CTA
// (tap, channel tile, output tile, split) writes its partial
// partial[split][tap][n][c] (FP32), summed in split order by k_wgrad_reduce.
struct WgradParams {
    int P, N, C, h, w, hp;
    int kbps;        // k-blocks per split
    int nkb;         // P / KB
    int ctiles, otiles, BNc;
    float *partial;  // [S][9][N][C]
    int *err;
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                            int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

template <int KB>
struct WgradPlan {
    static constexpr int kStages = 4;
    static constexpr int kA = BM * KB * 2;
    static constexpr int kBmax = 256 * KB * 2;
    static constexpr int kStage = kA + kBmax;
    static constexpr int kBarOff = kStage * kStages;
    static constexpr int kBytes = kBarOff + 256 + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
};

template <int KB>
__global__ void __launch_bounds__(192, 1)
k_conv3x3_wgrad(const __grid_constant__ CUtensorMap a_map, const __grid_constant__ CUtensorMap b_map, WgradParams p,
                uint32_t tmem_cols) {
    using P = WgradPlan<KB>;
    constexpr int NST = P::kStages;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(p.err) != 0) return;
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = smem_raw + pad;
    const int sstride = P::kA + p.BNc * KB * 2;  // stage bytes for this channel tile (a multiple of 1024)
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + sstride * NST);
    uint64_t *empty = full + NST;
    uint64_t *accum = empty + NST;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int tap = blockIdx.x % 9;
    const int rest = blockIdx.x / 9;
    const int ct = rest % p.ctiles, ot = rest / p.ctiles;
    const int split = blockIdx.y;
    const int n0 = ot * BM, c0 = ct * p.BNc;
    const int kb0 = split * p.kbps;
    const int nkb = min(p.nkb, kb0 + p.kbps) - kb0;
    const int dy = tap / 3, dx = tap % 3;
    const uint32_t stage_bytes = P::kA + p.BNc * KB * 2;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % NST;
                const uint32_t ph = (i / NST) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.err)) break;
                const uint32_t st = smem_u32(tiles + s * sstride);
                mbar_expect_tx(&full[s], stage_bytes);
                const int pix = (kb0 + i) * KB;
                const int img = pix / (p.h * p.w), y = (pix / p.w) % p.h, x0 = pix % p.w;
                tma_load_2d(st, &a_map, &full[s], pix, n0);
                tma_load_4d(st + P::kA, &b_map, &full[s], x0, img * p.hp + y + dy, c0, dx);
                issued = i + 1;
            }
            if (*abort_flag) {
                const uint64_t t0 = globaltimer();
                for (int i = issued > NST ? issued - NST : 0; i < issued; ++i) {
                    const int s = i % NST;
                    while (!mbar_try_wait(&full[s], (i / NST) & 1) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, p.BNc);
            for (int i = 0; i < nkb; ++i) {
                const int s = i % NST;
                const uint32_t ph = (i / NST) & 1;
                if (!mbar_wait(&full[s], ph, abort_flag, p.err)) break;
                tc_fence_after();
                const uint32_t a = smem_u32(tiles + s * sstride);
                const uint32_t b = a + P::kA;
#pragma unroll
                for (int kk = 0; kk < KB / 16; ++kk)
                    mma_bf16(tmem, desc_kmajor<KB * 2>(a + kk * 32), desc_kmajor<KB * 2>(b + kk * 32), idesc,
                             (i > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            mma_commit(accum);
        }
    } else {
        const int q = warp & 3;
        const int n = n0 + q * 32 + lane;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(accum, 0, abort_flag, p.err));
        tc_fence_after();
        if (ok && nkb > 0) {
            for (int cc = 0; cc < p.BNc; cc += 32) {
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + cc, v);
                if (n < p.N) {  // rows past N are the zero fill of the A box
                    float *dst = p.partial + ((static_cast<int64_t>(split) * 9 + tap) * p.N + n) * p.C + c0 + cc;
#pragma unroll
                    for (int e = 0; e < 32; e += 4)
                        *reinterpret_cast<float4 *>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

// dw[(n * 9 + tap) * C + c] = sum over splits s (in order) of partial[s][tap][n][c]
__global__ void k_wgrad_reduce(const float *__restrict__ partial, int S, int N, int C, float *__restrict__ dw) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t total = static_cast<int64_t>(N) * 9 * C;
    if (i >= total) return;
    const int c = static_cast<int>(i % C);
    const int tap = static_cast<int>((i / C) % 9);
    const int n = static_cast<int>(i / (static_cast<int64_t>(9) * C));
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += partial[((static_cast<int64_t>(s) * 9 + tap) * N + n) * C + c];
    dw[i] = acc;
}

// xs[dx][c][b * (h + 2) + yy][x] = x[b][(yy - 1) mod h][(x + dx - 1) mod w][c].
// A block takes one haloed row (b, yy), TW columns and 32 channels: it reads
// the TW + 2 source columns around them (circularly) once, 16 bytes per load,
// and writes the three column-shifted copies from shared memory, eight
// columns (16 bytes) per store.
template <int TW>
__global__ void __launch_bounds__(256) k_shift3_transpose(const __nv_bfloat16 *__restrict__ x, int B, int h, int w,
                                                          int C, __nv_bfloat16 *__restrict__ xs) {
    __shared__ __nv_bfloat16 tile[TW + 2][34];  // [source column - x0 + 1][channel], rows padded to 17 words
    const int ctiles = C / 32, xtiles = w / TW, hp = h + 2;
    int64_t blk = blockIdx.x;
    const int ct = static_cast<int>(blk % ctiles);
    blk /= ctiles;
    const int xt = static_cast<int>(blk % xtiles);
    const int64_t row = blk / xtiles;  // b * (h + 2) + yy
    const int b = static_cast<int>(row / hp), yy = static_cast<int>(row % hp);
    const int sy = (yy - 1 + h) % h;
    const int x0 = xt * TW, c0 = ct * 32;
    const __nv_bfloat16 *src = x + (static_cast<int64_t>(b) * h + sy) * w * C + c0;
    for (int t = threadIdx.x; t < (TW + 2) * 4; t += blockDim.x) {
        const int col = t >> 2, q = t & 3;
        const int sx = (x0 + col - 1 + w) % w;
        const uint4 v = *reinterpret_cast<const uint4 *>(src + static_cast<int64_t>(sx) * C + q * 8);
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int k = 0; k < 8; ++k) tile[col][q * 8 + k] = e[k];
    }
    __syncthreads();
    constexpr int G = TW / 8;
    const int64_t plane = static_cast<int64_t>(B) * hp * w;  // elements of one (dx, c) plane
    for (int t = threadIdx.x; t < 3 * 32 * G; t += blockDim.x) {
        const int g = t % G, c = (t / G) % 32, dx = t / (32 * G);
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = tile[g * 8 + k + dx][c];
        *reinterpret_cast<uint4 *>(xs + (static_cast<int64_t>(dx) * C + c0 + c) * plane + row * w + x0 + g * 8) =
            *reinterpret_cast<const uint4 *>(o);
    }
}

}  // namespace

bool conv3x3_supported(int C, int N, int h, int w, int P) {
    // output tiles of N (<= 256) or N / 2 channels, a multiple of 32 either way:
    // the epilogue drains the accumulator 32 columns at a time
    return C % kConvKB == 0 && C > 0 && N % 32 == 0 && N > 0 && N <= 512 && (N <= 256 || N % 64 == 0) &&
           w <= BM && BM % w == 0 && (BM / w) <= h && h % (BM / w) == 0 && P % BM == 0;
}

cudaError_t launch_conv3x3(TcContext *ctx, const __nv_bfloat16 *xpad, int C, int B, int h, int w,
                           const __nv_bfloat16 *wt, int N, const float *bias, int act, float *out32,
                           __nv_bfloat16 *out16, int *err, cudaStream_t s) {
    const int P = B * h * w;
    if (!ctx || !conv3x3_supported(C, N, h, w, P) || (!out32 && !out16)) return cudaErrorInvalidValue;
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tc_encoder(ctx);
    CUtensorMap am, bm;
    {
        const int wp = w + 2, hp = h + 2;
        cuuint64_t dims[3] = {static_cast<cuuint64_t>(C), static_cast<cuuint64_t>(wp),
                              static_cast<cuuint64_t>(B) * hp};
        cuuint64_t strides[2] = {static_cast<cuuint64_t>(C) * 2, static_cast<cuuint64_t>(wp) * C * 2};
        cuuint32_t box[3] = {static_cast<cuuint32_t>(kConvKB), static_cast<cuuint32_t>(w),
                             static_cast<cuuint32_t>(BM / w)};
        cuuint32_t estr[3] = {1, 1, 1};
        if (encode(&am, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(xpad), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const int BN = N <= 256 ? N : N / 2;
    if (BN % 16 != 0) return cudaErrorInvalidValue;
    {
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(9) * C, static_cast<cuuint64_t>(N)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(9) * C * 2};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(kConvKB), static_cast<cuuint32_t>(BN)};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&bm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(wt), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    ConvParams prm;
    prm.P = P;
    prm.N = N;
    prm.cblk = C / kConvKB;
    prm.h = h;
    prm.w = w;
    prm.hp = h + 2;
    prm.rows = BM / w;
    prm.bias = bias;
    prm.act = act;
    prm.out32 = out32;
    prm.out16 = out16;
    prm.err = err;
    uint32_t cols = 32;
    while (static_cast<int>(cols) < BN) cols <<= 1;
    // shared memory sized for this BN: narrow layers fit two or three CTAs per
    // SM, so one CTA's epilogue overlaps another's loads and MMAs
    const int smem = (ConvPlan::kA + BN * kConvKB * 2) * kConvStages + 256 + 1024;
    cudaError_t e = set_smem(k_conv3x3, ConvPlan::kBytes);
    if (e != cudaSuccess) return e;
    k_conv3x3<<<dim3(P / BM, (N + BN - 1) / BN), 192, smem, s>>>(am, bm, prm, BN, cols);
    return cudaGetLastError();
}

namespace {
// Channel tile of the weight-gradient kernel: all C channels, else half of
// them (at most 256 either way, a multiple of 32); 0 when neither fits.
int wgrad_channel_tile(int C) {
    if (C > 0 && C % 32 == 0 && C <= 256) return C;
    if (C % 64 == 0 && C / 2 <= 256) return C / 2;
    return 0;
}
}  // namespace

bool conv3x3_wgrad_supported(int C, int N, int h, int w, int P) {
    const int KB = w >= 64 ? 64 : 32;
    return h > 0 && w >= 32 && w % KB == 0 && P % KB == 0 && wgrad_channel_tile(C) > 0 && N > 0 && N % 8 == 0;
}

cudaError_t launch_shift3_transpose(const __nv_bfloat16 *x, int B, int h, int w, int C, __nv_bfloat16 *xs,
                                    cudaStream_t s) {
    if (B < 1 || h < 1 || w % 32 != 0 || C % 32 != 0 || C < 32) return cudaErrorInvalidValue;
    const int64_t blocks = static_cast<int64_t>(B) * (h + 2) * (C / 32);
    if (w % 64 == 0)
        k_shift3_transpose<64><<<static_cast<unsigned>(blocks * (w / 64)), 256, 0, s>>>(x, B, h, w, C, xs);
    else
        k_shift3_transpose<32><<<static_cast<unsigned>(blocks * (w / 32)), 256, 0, s>>>(x, B, h, w, C, xs);
    return cudaGetLastError();
}

cudaError_t launch_conv3x3_wgrad(TcContext *ctx, const __nv_bfloat16 *dzT, const __nv_bfloat16 *xs, int B, int h,
                                 int w, int C, int N, float *partial, int64_t partial_cap, float *dw, int *err,
                                 cudaStream_t s) {
    const int P = B * h * w;
    if (!ctx || !conv3x3_wgrad_supported(C, N, h, w, P)) return cudaErrorInvalidValue;
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tc_encoder(ctx);
    const int KB = w >= 64 ? 64 : 32;
    const int BNc = wgrad_channel_tile(C);
    const int ctiles = C / BNc, otiles = (N + BM - 1) / BM;
    const int nkb = P / KB;
    // split-K over the pixels: about two CTAs per SM, at least 8 k-blocks each
    const int base = 9 * ctiles * otiles;
    int S = std::max(1, std::min(nkb / 8, (2 * 152 + base - 1) / base));
    const int64_t per = static_cast<int64_t>(9) * N * C;
    if (per > partial_cap) return cudaErrorInvalidValue;
    while (S > 1 && static_cast<int64_t>(S) * per > partial_cap) --S;
    const int kbps = (nkb + S - 1) / S;
    S = (nkb + kbps - 1) / kbps;
    CUtensorMap am, bm;
    {
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(P), static_cast<cuuint64_t>(N)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(P) * 2};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(KB), static_cast<cuuint32_t>(BM)};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&am, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(dzT), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        KB == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const int64_t rows = static_cast<int64_t>(B) * (h + 2);
        cuuint64_t dims[4] = {static_cast<cuuint64_t>(w), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(C),
                              3};
        cuuint64_t strides[3] = {static_cast<cuuint64_t>(w) * 2, static_cast<cuuint64_t>(rows) * w * 2,
                                 static_cast<cuuint64_t>(C) * rows * w * 2};
        cuuint32_t box[4] = {static_cast<cuuint32_t>(KB), 1, static_cast<cuuint32_t>(BNc), 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (encode(&bm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(xs), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        KB == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    WgradParams prm;
    prm.P = P;
    prm.N = N;
    prm.C = C;
    prm.h = h;
    prm.w = w;
    prm.hp = h + 2;
    prm.kbps = kbps;
    prm.nkb = nkb;
    prm.ctiles = ctiles;
    prm.otiles = otiles;
    prm.BNc = BNc;
    prm.partial = partial;
    prm.err = err;
    uint32_t cols = 32;
    while (static_cast<int>(cols) < BNc) cols <<= 1;
    cudaError_t e;
    dim3 grid(base, S);
    // shared memory sized for this channel tile (several CTAs per SM when narrow)
    const int smem = (BM * KB * 2 + BNc * KB * 2) * (KB == 64 ? WgradPlan<64>::kStages : WgradPlan<32>::kStages) +
                     256 + 1024;
    if (KB == 64) {
        if ((e = set_smem(k_conv3x3_wgrad<64>, WgradPlan<64>::kBytes)) != cudaSuccess) return e;
        k_conv3x3_wgrad<64><<<grid, 192, smem, s>>>(am, bm, prm, cols);
    } else {
        if ((e = set_smem(k_conv3x3_wgrad<32>, WgradPlan<32>::kBytes)) != cudaSuccess) return e;
        k_conv3x3_wgrad<32><<<grid, 192, smem, s>>>(am, bm, prm, cols);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t total = static_cast<int64_t>(N) * 9 * C;
    k_wgrad_reduce<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(partial, S, N, C, dw);
    return cudaGetLastError();
}

}  // namespace ensf
