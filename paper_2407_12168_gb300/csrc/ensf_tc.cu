// ensf_tc.cu -- tensor-core stages of the EnSF analysis step on sm_103a.
//
// Both contractions of an Euler-Maruyama step are "TN" GEMMs over BF16
// operands stored K-major, D[m][n] = sum_k A[m][k] B[n][k]:
//
//   Gram   G = Z X^T     A = particles Z  [n][d],   B = forecast X   [n_x][d],
//                        K = d, split over d (split-K), FP32 partials out;
//                        the cross term z_i . x_j of the Gaussian kernel (Eq. 12)
//   Sum    U = W X       A = weights W    [n][n_x], B = X^T          [d][n_x],
//                        K = n_x, epilogue = score (Eq. 15, 17) + the
//                        Euler-Maruyama update of Eq. 7 on the FP32 particles.
//
// Split-BF16x3: an FP32 operand a is carried as a = a_hi + a_lo with
// a_hi = bf16(a), a_lo = bf16(a - a_hi); the product uses a_hi b_hi + a_hi b_lo
// + a_lo b_hi (the a_lo b_lo term is below FP32 rounding), accumulated in FP32.
//
// Kernel structure (one output tile of 128 x BN per CTA, 6 warps):
//   warp 0     TMA producer: 128B-swizzled tiles of A and B (hi, lo planes)
//              into a STAGES-deep shared-memory ring, mbarrier transaction counts
//   warp 1     allocates BN TMEM columns; one thread issues tcgen05.mma
//              (kind::f16, BF16 in, FP32 accumulate in TMEM), 4 MMAs of K = 16
//              per 64-wide k-block and operand product; tcgen05.commit frees
//              each ring slot and finally signals the accumulator
//   warps 2-5  epilogue: tcgen05.ld 32 columns at a time from their TMEM lane
//              quarter, then the per-kernel epilogue
// Every mbarrier wait is bounded by %globaltimer: on expiry the CTA records
// ENSF_ETIMEOUT in the error word, drains its own copies, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "ensf_tc.h"

namespace ensf {

namespace {

constexpr int BM = 128;        // tile rows (particles)
constexpr int BK = 64;         // k-block: 64 BF16 = one 128-byte swizzle row
constexpr int kThreads = 192;  // 6 warps
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr int kStatusTimeout = 5;  // ENSF_ETIMEOUT

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false when the
// CTA is aborting (another role timed out) or when this wait times out, in
// which case it raises the abort flag and records ENSF_ETIMEOUT.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > kTimeoutNs) {
                *abort_flag = 1;
                atomicCAS(err, 0, kStatusTimeout);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO),
// leading offset unused for this layout, descriptor version 1, layout 2.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(1) << 16;
    d |= static_cast<uint64_t>(1024 >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A and B BF16, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    __syncwarp();  // the load is warp-collective: reconverge after per-lane branches
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------- shared-memory plan
template <int BN, int STAGES, bool SPLIT>
struct Plan {
    static constexpr int kA = BM * BK * 2;  // one A plane of a stage
    static constexpr int kB = BN * BK * 2;  // one B plane
    static constexpr int kPlanes = SPLIT ? 2 : 1;
    static constexpr int kStage = (kA + kB) * kPlanes;
    static constexpr int kBarOff = kStage * STAGES;
    static constexpr int kBytes = kBarOff + 256 + 1024;  // barriers + alignment slack
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN");
};

struct Ctl {
    uint64_t *full, *empty, *accum;
    uint32_t *tmem_slot;
    volatile int *abort_flag;
    uint8_t *tiles;
};

template <class P>
__device__ __forceinline__ Ctl carve(uint8_t *raw, int stages) {
    uintptr_t base = reinterpret_cast<uintptr_t>(raw);
    uint32_t s = smem_u32(raw);
    uint32_t pad = (1024u - (s & 1023u)) & 1023u;
    Ctl c;
    c.tiles = reinterpret_cast<uint8_t *>(base + pad);
    uint64_t *bars = reinterpret_cast<uint64_t *>(c.tiles + P::kBarOff);
    c.full = bars;
    c.empty = bars + stages;
    c.accum = bars + 2 * stages;
    c.tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages + 1);
    c.abort_flag = reinterpret_cast<volatile int *>(c.tmem_slot + 1);
    return c;
}

// Set-up common to both kernels: barriers, abort flag, TMEM allocation.
template <int BN, int STAGES>
__device__ __forceinline__ uint32_t setup(const Ctl &c, int warp) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&c.full[s], 1);
            mbar_init(&c.empty[s], 1);
        }
        mbar_init(c.accum, 1);
        *c.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(c.tmem_slot, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *c.tmem_slot;
}

// Producer (one thread): k-blocks kb0 .. kb0+nkb-1 of A rows m0.. and B rows n0..
template <int BN, int STAGES, bool SPLIT>
__device__ void produce(const Ctl &c, const CUtensorMap *a_hi, const CUtensorMap *a_lo, const CUtensorMap *b_hi,
                        const CUtensorMap *b_lo, int m0, int n0, int kb0, int nkb, int *err) {
    using P = Plan<BN, STAGES, SPLIT>;
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(&c.empty[s], ph ^ 1u, c.abort_flag, err)) break;
        const uint32_t st = smem_u32(c.tiles + s * P::kStage);
        mbar_expect_tx(&c.full[s], P::kStage);
        const int kx = (kb0 + i) * BK;
        tma_load_2d(st, a_hi, &c.full[s], kx, m0);
        if (SPLIT) tma_load_2d(st + P::kA, a_lo, &c.full[s], kx, m0);
        tma_load_2d(st + P::kA * P::kPlanes, b_hi, &c.full[s], kx, n0);
        if (SPLIT) tma_load_2d(st + P::kA * P::kPlanes + P::kB, b_lo, &c.full[s], kx, n0);
        ++issued;
    }
    if (*c.abort_flag) {
        // drain: wait (bounded) for the copies this thread issued to land
        const uint64_t t0 = globaltimer();
        for (int i = std::max(0, issued - STAGES); i < issued; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (i / STAGES) & 1;
            while (!mbar_try_wait(&c.full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
            }
        }
    }
}

// MMA issuer (one thread): accumulate the tile in TMEM, then signal accum.
template <int BN, int STAGES, bool SPLIT>
__device__ void mma_loop(const Ctl &c, uint32_t tmem, int nkb, int *err) {
    using P = Plan<BN, STAGES, SPLIT>;
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int i = 0; i < nkb; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(&c.full[s], ph, c.abort_flag, err)) break;
        tc_fence_after();
        const uint32_t a_hi = smem_u32(c.tiles + s * P::kStage);
        const uint32_t a_lo = a_hi + P::kA;
        const uint32_t b_hi = a_hi + P::kA * P::kPlanes;
        const uint32_t b_lo = b_hi + P::kB;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;  // 16 BF16 = 32 bytes along the swizzled row
            mma_bf16(tmem, desc_sw128(a_hi + off), desc_sw128(b_hi + off), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            if (SPLIT) {
                mma_bf16(tmem, desc_sw128(a_hi + off), desc_sw128(b_lo + off), idesc, 1u);
                mma_bf16(tmem, desc_sw128(a_lo + off), desc_sw128(b_hi + off), idesc, 1u);
            }
        }
        mma_commit(&c.empty[s]);
    }
    mma_commit(c.accum);
}

template <int BN>
__device__ __forceinline__ void teardown(uint32_t tmem, int warp) {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

// ------------------------------------------------------------------- Gram
struct GramParams {
    int n, n_x;
    int kblocks;       // ceil(d / BK)
    int kb_per_split;  // k-blocks per split (last split may hold fewer)
    float *partial;    // [splits][n][n_x]
    int *err;
};

template <int BN, int STAGES, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const __grid_constant__ CUtensorMap a_hi, const __grid_constant__ CUtensorMap a_lo,
          const __grid_constant__ CUtensorMap b_hi, const __grid_constant__ CUtensorMap b_lo, GramParams p) {
    using P = Plan<BN, STAGES, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    const Ctl c = carve<P>(smem_raw, STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, split = blockIdx.z;
    const int kb0 = split * p.kb_per_split;
    const int nkb = min(p.kblocks, kb0 + p.kb_per_split) - kb0;
    if (*reinterpret_cast<volatile int *>(p.err) != 0) return;  // an earlier launch failed: skip
    const uint32_t tmem = setup<BN, STAGES>(c, warp);

    if (warp == 0) {
        if (lane == 0) produce<BN, STAGES, SPLIT>(c, &a_hi, &a_lo, &b_hi, &b_lo, m0, n0, kb0, nkb, p.err);
    } else if (warp == 1) {
        if (lane == 0) mma_loop<BN, STAGES, SPLIT>(c, tmem, nkb, p.err);
    } else {
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        const int row = m0 + q * 32 + lane;
        const bool ok = mbar_wait(c.accum, 0, c.abort_flag, p.err);
        tc_fence_after();
        if (ok) {
            float *dst = p.partial + (static_cast<int64_t>(split) * p.n + row) * p.n_x;
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + cc, v);
                const int col0 = n0 + cc;
                if (row < p.n && col0 < p.n_x) {
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        if (col0 + e < p.n_x) dst[col0 + e] = v[e];
                }
            }
        }
    }
    teardown<BN>(tmem, warp);
}

// ------------------------------------------------------- W X + EM update
// Persistent kernel over tiles of U^T = X^T W^T: MMA rows (TMEM lanes) are 128
// state columns c, MMA columns are BN particles i.  An epilogue thread owns one
// state column, so for each particle the 32 lanes of a warp touch 32
// consecutive floats of z[i][:] (coalesced), and y[c], mask[c] are read once
// per tile.  Two TMEM accumulators (columns 0 and 256) let the epilogue of one
// tile run while the MMAs of the next accumulate.
constexpr int kEpiWarps = 8;                       // two per TMEM lane quarter
constexpr int kWxThreads = 64 + 32 * kEpiWarps;    // producer, MMA, epilogue
constexpr int kWxTmemCols = 512;

template <int BN, int STAGES, bool SPLIT>
struct WxPlan {
    static constexpr int kA = BM * BK * 2;  // X^T rows (state columns)
    static constexpr int kB = BN * BK * 2;  // W rows (particles)
    static constexpr int kPlanes = SPLIT ? 2 : 1;
    static constexpr int kStage = (kA + kB) * kPlanes;
    static constexpr int kBarOff = kStage * STAGES;
    static constexpr int kBytes = kBarOff + 512 + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
    static_assert(BN == 64 || BN == 128 || BN == 256, "BN");
};

struct WxParams {
    int n;
    int64_t d;
    int kblocks;   // ceil(n_x / BK)
    int m_tiles;   // ceil(d / 128)
    int n_tiles;   // ceil(n / BN)
    float *z;
    __nv_bfloat16 *zb_hi, *zb_lo;
    const float *y;
    const uint8_t *mask;
    const float *noise_buf;
    uint64_t seed;
    uint32_t offset;
    StepCoef coef;
    int *err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int BN, int STAGES, bool SPLIT>
__global__ void __launch_bounds__(kWxThreads, 1)
k_wx_em_tc(const __grid_constant__ CUtensorMap xt_hi, const __grid_constant__ CUtensorMap xt_lo,
           const __grid_constant__ CUtensorMap w_hi, const __grid_constant__ CUtensorMap w_lo, WxParams p) {
    using P = WxPlan<BN, STAGES, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(p.err) != 0) return;  // an earlier launch failed: skip

    uintptr_t base = reinterpret_cast<uintptr_t>(smem_raw);
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = reinterpret_cast<uint8_t *>(base + pad);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + P::kBarOff);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;   // [2] accumulator ready
    uint64_t *tempty = tfull + 2;       // [2] accumulator drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kEpiWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, kWxTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int total = p.m_tiles * p.n_tiles;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            int issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int m0 = (t / p.n_tiles) * BM, n0 = (t % p.n_tiles) * BN;
                for (int kb = 0; kb < p.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.err)) { ok = false; break; }
                    const uint32_t st = smem_u32(tiles + s * P::kStage);
                    mbar_expect_tx(&full[s], P::kStage);
                    const int kx = kb * BK;
                    tma_load_2d(st, &xt_hi, &full[s], kx, m0);
                    if (SPLIT) tma_load_2d(st + P::kA, &xt_lo, &full[s], kx, m0);
                    tma_load_2d(st + P::kA * P::kPlanes, &w_hi, &full[s], kx, n0);
                    if (SPLIT) tma_load_2d(st + P::kA * P::kPlanes + P::kB, &w_lo, &full[s], kx, n0);
                    issued = it + 1;
                }
            }
            if (*abort_flag) {
                const uint64_t t0 = globaltimer();
                for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i) {
                    const int s = i % STAGES;
                    while (!mbar_try_wait(&full[s], (i / STAGES) & 1) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            int it = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++lt) {
                const int slot = lt & 1;
                const uint32_t use = lt >> 1;
                if (!mbar_wait(&tempty[slot], (use & 1u) ^ 1u, abort_flag, p.err)) break;
                tc_fence_after();
                const uint32_t acc = tmem + slot * 256;
                for (int kb = 0; kb < p.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&full[s], ph, abort_flag, p.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_hi = smem_u32(tiles + s * P::kStage);
                    const uint32_t a_lo = a_hi + P::kA;
                    const uint32_t b_hi = a_hi + P::kA * P::kPlanes;
                    const uint32_t b_lo = b_hi + P::kB;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        mma_bf16(acc, desc_sw128(a_hi + off), desc_sw128(b_hi + off), idesc,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                        if (SPLIT) {
                            mma_bf16(acc, desc_sw128(a_hi + off), desc_sw128(b_lo + off), idesc, 1u);
                            mma_bf16(acc, desc_sw128(a_lo + off), desc_sw128(b_hi + off), idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[slot]);
            }
        }
    } else {
        const int ew = warp - 2;            // 0 .. kEpiWarps-1
        const int q = warp & 3;             // TMEM lane quarter this warp may read
        const int half = ew >> 2;           // which half of the BN particle columns
        constexpr int kCols = BN / 2;
        const StepCoef &cf = p.coef;
        int lt = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++lt) {
            const int slot = lt & 1;
            const uint32_t use = lt >> 1;
            const int m0 = (t / p.n_tiles) * BM, n0 = (t % p.n_tiles) * BN;
            if (!mbar_wait(&tfull[slot], use & 1u, abort_flag, p.err)) break;
            tc_fence_after();
            const int64_t c = static_cast<int64_t>(m0) + q * 32 + lane;  // this thread's state column
            const bool cok = c < p.d;
            const float yc = cok ? p.y[c] : 0.f;
            const bool obs = cok && (p.mask == nullptr || p.mask[c] != 0);
#pragma unroll 1
            for (int cc = half * kCols; cc < (half + 1) * kCols; cc += 32) {
                float u[32];
                tmem_ld32(tmem + slot * 256 + (static_cast<uint32_t>(q * 32) << 16) + cc, u);
                const int i0 = n0 + cc;
                if (!cok || i0 >= p.n) continue;
                float zv[32];
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    zv[e] = (i0 + e < p.n) ? p.z[static_cast<int64_t>(i0 + e) * p.d + c] : 0.f;
#pragma unroll
                for (int e4 = 0; e4 < 8; ++e4) {
                    const int ib = i0 + e4 * 4;
                    if (ib >= p.n) break;
                    float xi[4];
                    if (p.noise_buf) {
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            xi[r] = (ib + r < p.n)
                                        ? p.noise_buf[(static_cast<int64_t>(cf.k + 1) * p.n + ib + r) * p.d + c]
                                        : 0.f;
                    } else {
                        const float4 v = noise4(p.seed, p.offset, cf.k + 1, c, ib >> 2);
                        xi[0] = v.x; xi[1] = v.y; xi[2] = v.z; xi[3] = v.w;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int i = ib + r;
                        if (i >= p.n) break;
                        const int e = e4 * 4 + r;
                        const float g = obs ? lik_score(cf.obs_op, zv[e], yc, cf.inv_r) : 0.f;
                        const float zn = em_update(cf, zv[e], u[e], g, xi[r]);
                        const int64_t off = static_cast<int64_t>(i) * p.d + c;
                        p.z[off] = zn;
                        if (p.zb_hi) {
                            const __nv_bfloat16 hi = __float2bfloat16_rn(zn);
                            p.zb_hi[off] = hi;
                            if (p.zb_lo) p.zb_lo[off] = __float2bfloat16_rn(zn - __bfloat162float(hi));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[slot]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kWxTmemCols);
    }
}

}  // namespace

// =================================================================== host
struct TcContext {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};

cudaError_t tc_context_create(TcContext **out) {
    *out = nullptr;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    TcContext *c = new TcContext;
    c->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    *out = c;
    return cudaSuccess;
}

void tc_context_destroy(TcContext *ctx) { delete ctx; }

int64_t tc_partial_floats(int max_n, int /*sms*/) {
    const int64_t sq = static_cast<int64_t>(max_n) * max_n;
    return std::min<int64_t>(64 * sq, std::max<int64_t>(int64_t(32) << 20, sq));
}

namespace {

// 2-D BF16 tensor map: rows x cols (cols contiguous), row pitch `pitch`
// elements, box = BK columns x box_rows rows, 128-byte swizzle, zero fill.
cudaError_t make_map(const TcContext *ctx, CUtensorMap *m, const void *base, int64_t cols, int64_t rows,
                     int64_t pitch, int box_rows) {
    if (!base) {  // an unused plane: point at nothing valid but keep the map well formed
        memset(m, 0, sizeof(*m));
        return cudaSuccess;
    }
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ctx->encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int BN, int STAGES, bool SPLIT>
cudaError_t run_gram(const CUtensorMap (&maps)[4], const GramParams &p, dim3 grid, cudaStream_t s) {
    using P = Plan<BN, STAGES, SPLIT>;
    auto kern = k_gram_tc<BN, STAGES, SPLIT>;
    cudaError_t e = set_smem(kern, P::kBytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, P::kBytes, s>>>(maps[0], maps[1], maps[2], maps[3], p);
    return cudaGetLastError();
}

template <int BN, int STAGES, bool SPLIT>
cudaError_t run_wx(const CUtensorMap (&maps)[4], WxParams p, int sms, cudaStream_t s) {
    using P = WxPlan<BN, STAGES, SPLIT>;
    auto kern = k_wx_em_tc<BN, STAGES, SPLIT>;
    cudaError_t e = set_smem(kern, P::kBytes);
    if (e != cudaSuccess) return e;
    p.n_tiles = (p.n + BN - 1) / BN;
    const int total = p.m_tiles * p.n_tiles;
    const int grid = total < sms ? total : sms;
    kern<<<grid, kWxThreads, P::kBytes, s>>>(maps[0], maps[1], maps[2], maps[3], p);
    return cudaGetLastError();
}

// Split count minimising (waves) x (k-blocks per split + epilogue cost), with
// the partials within the scratch capacity.
int choose_splits(int tiles, int kblocks, int sms, int64_t per_split_floats, int64_t cap) {
    int best = 1;
    double best_cost = 1e300;
    const int smax = static_cast<int>(std::min<int64_t>({64, kblocks, std::max<int64_t>(1, cap / per_split_floats)}));
    for (int s = 1; s <= smax; ++s) {
        const int kb = (kblocks + s - 1) / s;
        const int used = (kblocks + kb - 1) / kb;  // splits that actually hold work
        if (used != s) continue;
        const double waves = std::ceil(static_cast<double>(tiles) * s / sms);
        const double cost = waves * (kb + 4.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = s;
        }
    }
    return best;
}

}  // namespace

cudaError_t launch_gram_tc(TcContext *ctx, const TcGramArgs &a, int sms, int *splits, int64_t *part_stride, int *ldp,
                           cudaStream_t s) {
    if (!ctx) return cudaErrorInvalidValue;
    const int BN = a.n_x <= 128 ? 128 : 256;
    CUtensorMap maps[4];
    cudaError_t e;
    if ((e = make_map(ctx, &maps[0], a.zb_hi, a.d, a.n, a.d, BM)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[1], a.split3 ? a.zb_lo : nullptr, a.d, a.n, a.d, BM)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[2], a.xb_hi, a.d, a.n_x, a.d, BN)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[3], a.split3 ? a.xb_lo : nullptr, a.d, a.n_x, a.d, BN)) != cudaSuccess) return e;
    const int mt = (a.n + BM - 1) / BM, nt = (a.n_x + BN - 1) / BN;
    GramParams p;
    p.n = a.n;
    p.n_x = a.n_x;
    p.kblocks = static_cast<int>((a.d + BK - 1) / BK);
    const int S = choose_splits(mt * nt, p.kblocks, sms, static_cast<int64_t>(a.n) * a.n_x, a.partial_cap);
    p.kb_per_split = (p.kblocks + S - 1) / S;
    p.partial = a.partial;
    p.err = a.err;
    *splits = S;
    *part_stride = static_cast<int64_t>(a.n) * a.n_x;
    *ldp = a.n_x;
    dim3 grid(mt, nt, S);
    if (a.split3) {
        if (BN == 256) return run_gram<256, 2, true>(maps, p, grid, s);
        return run_gram<128, 3, true>(maps, p, grid, s);
    }
    if (BN == 256) return run_gram<256, 4, false>(maps, p, grid, s);
    return run_gram<128, 6, false>(maps, p, grid, s);
}

cudaError_t launch_wx_em_tc(TcContext *ctx, const TcWxArgs &a, int sms, cudaStream_t s) {
    if (!ctx) return cudaErrorInvalidValue;
    const bool split = a.wb_lo != nullptr && a.xt_lo != nullptr;
    const int BN = a.n <= 64 ? 64 : (a.n <= 128 ? 128 : 256);
    // A = X^T [d][ldw] (state columns; K = n_x members), B = W [n][ldw] (particles)
    const int n_x = a.n;
    CUtensorMap maps[4];
    cudaError_t e;
    if ((e = make_map(ctx, &maps[0], a.xt_hi, n_x, a.d, a.ldw, BM)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[1], split ? a.xt_lo : nullptr, n_x, a.d, a.ldw, BM)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[2], a.wb_hi, n_x, a.n, a.ldw, BN)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[3], split ? a.wb_lo : nullptr, n_x, a.n, a.ldw, BN)) != cudaSuccess) return e;
    WxParams p;
    p.n = a.n;
    p.d = a.d;
    p.kblocks = (n_x + BK - 1) / BK;
    p.m_tiles = static_cast<int>((a.d + BM - 1) / BM);
    p.n_tiles = 0;
    p.z = a.z;
    p.zb_hi = a.zb_hi;
    p.zb_lo = a.zb_lo;
    p.y = a.y;
    p.mask = a.mask;
    p.noise_buf = a.noise_buf;
    p.seed = a.seed;
    p.offset = a.offset;
    p.coef = a.coef;
    p.err = a.err;
    if (split) {
        if (BN == 256) return run_wx<256, 2, true>(maps, p, sms, s);
        if (BN == 128) return run_wx<128, 3, true>(maps, p, sms, s);
        return run_wx<64, 4, true>(maps, p, sms, s);
    }
    if (BN == 256) return run_wx<256, 4, false>(maps, p, sms, s);
    if (BN == 128) return run_wx<128, 6, false>(maps, p, sms, s);
    return run_wx<64, 8, false>(maps, p, sms, s);
}

}  // namespace ensf
