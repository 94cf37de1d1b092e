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
// Gram kernel structure (one output tile of 128 x BN per CTA, 10 warps):
//   warp 0     TMA producer: 128B-swizzled tiles of A and B (hi, lo planes)
//              into a STAGES-deep shared-memory ring, mbarrier transaction counts
//   warp 1     allocates BN TMEM columns; one thread issues tcgen05.mma
//              (kind::f16, BF16 in, FP32 accumulate in TMEM), 4 MMAs of K = 16
//              per 64-wide k-block and operand product; tcgen05.commit frees
//              each ring slot and finally signals the accumulator
//   warps 2-5  epilogue: tcgen05.ld 32 columns at a time from their TMEM lane
//              quarter, then the per-kernel epilogue
//   warps 6-9  (with warps 2-5 while the MMAs run) the next step's noise slice
// The pair form (k_gram_tc_pair) runs a 256 x 256 tile on a cluster of two
// CTAs with tcgen05.mma.cta_group::2: each CTA stages half of A and half of
// B, so the B traffic through each SM's shared memory halves -- the resource
// that bounds the single-CTA split-BF16x3 Gram (three products re-read both
// operands while TMA refills the ring).
// The W X kernel is persistent with 16 epilogue warps (see below).
// Every mbarrier wait is bounded by %globaltimer: on expiry the CTA records
// ENSF_ETIMEOUT in the error word, drains its own copies, frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ensf_internal.h"
#include "ensf_ptx.cuh"
#include "ensf_tc.h"

namespace ensf {

namespace {

constexpr int kGramThreads = 320;  // Gram: 6 warps + 4 warps that only generate noise

// ----------------------------------------------------- shared-memory plan
template <int BN, int STAGES, bool SPLIT, int KB = BK, int ES = 2>
struct Plan {
    static constexpr int kA = BM * KB * ES;  // one A plane of a stage
    static constexpr int kB = BN * KB * ES;  // one B plane
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

// Producer (one thread): k-blocks kb0 .. kb0+nkb-1 (KB elements wide) of A
// rows m0.. and B rows n0..
template <int BN, int STAGES, bool SPLIT, int KB = BK, int ES = 2>
__device__ void produce(const Ctl &c, const CUtensorMap *a_hi, const CUtensorMap *a_lo, const CUtensorMap *b_hi,
                        const CUtensorMap *b_lo, int m0, int n0, int kb0, int nkb, int *err) {
    using P = Plan<BN, STAGES, SPLIT, KB, ES>;
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
        const int s = i % STAGES;
        const uint32_t ph = (i / STAGES) & 1;
        if (!mbar_wait(&c.empty[s], ph ^ 1u, c.abort_flag, err)) break;
        const uint32_t st = smem_u32(c.tiles + s * P::kStage);
        mbar_expect_tx(&c.full[s], P::kStage);
        const int kx = (kb0 + i) * KB;
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
template <int BN, int STAGES, bool SPLIT, int KB = BK, int ES = 2>
__device__ void mma_loop(const Ctl &c, uint32_t tmem, int nkb, int *err) {
    using P = Plan<BN, STAGES, SPLIT, KB, ES>;
    constexpr int kRowB = KB * ES;  // bytes per k-block row (one swizzle row)
    constexpr uint32_t idesc = ES == 4 ? idesc_tf32(BM, BN) : idesc_bf16(BM, BN);
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
        for (int kk = 0; kk < kRowB / 32; ++kk) {
            // one MMA covers 32 bytes along the swizzled row: K = 16 BF16 or K = 8 TF32
            const uint32_t off = kk * 32;
            if (ES == 4) {
                mma_tf32(tmem, desc_kmajor<kRowB>(a_hi + off), desc_kmajor<kRowB>(b_hi + off), idesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
                continue;
            }
            mma_bf16(tmem, desc_kmajor<kRowB>(a_hi + off), desc_kmajor<kRowB>(b_hi + off), idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
            if (SPLIT) {
                mma_bf16(tmem, desc_kmajor<kRowB>(a_hi + off), desc_kmajor<kRowB>(b_lo + off), idesc, 1u);
                mma_bf16(tmem, desc_kmajor<kRowB>(a_lo + off), desc_kmajor<kRowB>(b_hi + off), idesc, 1u);
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
    int kblocks;       // ceil(d / k-block width)
    int kb_per_split;  // k-blocks per split (last split may hold fewer)
    float *partial;    // [splits][n][n_x]
    int *err;
    // optional: the noise slice xi[noise_k][i][c] of the next Euler-Maruyama
    // step, written by the epilogue warps while the MMAs run (NULL: none)
    float *noise;
    uint64_t seed;
    uint32_t offset;
    int noise_k;
    int64_t d;
    int64_t noise_col0;  // global index of state column 0 (noise counters use global columns)
    int noise_warp0;   // first warp that generates noise (2: warps 2-9, 6: warps 6-9)
    // FP32-operand form: A = z - alpha m split in the kernel (centre m, [d])
    float alpha;
    const float *centre;
    bool pdl;  // host: launched with programmatic stream serialization
    // row softmax fused into the epilogue (pair tiles; sm_L NULL: a separate launch)
    int splits;                 // split-K slices of this launch
    DF *sm_L;                   // [n][n_x] log-kernels
    float4 *sm_stats;           // [n][n_x / 256] tile statistics
    int *sm_cnt;                // arrival counters: [n / 128][n_x / 256] blocks, then [n / 128] bands
    const double *sm_norms;     // |x_j - m|^2
    double sm_alpha, sm_inv_2beta2;
    float *sm_w;                // FP32 weights [n][sm_ldw] or NULL
    int sm_ldw;
    __nv_bfloat16 *sm_w_hi, *sm_w_lo;
    int sm_ldwb;
};

// The row softmax of Eq. 16 fused into the pair Gram: every CTA counts its
// finished 128 x 256 block of partials; the last of the block's split-K CTAs
// sums them (fixed order), forms the block's log-kernels and per-row tile
// statistics; the last block of each 128-row band normalises the band's rows.
// Arrival counters only (reset by the last arriver): nothing waits.  The
// arithmetic is that of the separate tiled softmax launch.
__device__ void gram_softmax_tail(const GramParams &p, int rb, int cb) {
    __shared__ int s_last;
    const int tid = threadIdx.x, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nt = (p.n_x + kSoftTile - 1) / kSoftTile;
    const int bands = (p.n + 127) / 128;
    int *blk_cnt = p.sm_cnt + rb * nt + cb;
    int *band_cnt = p.sm_cnt + bands * nt + rb;
    if (tid == 0) s_last = atomicAdd(blk_cnt, 1) == p.splits - 1;
    __syncthreads();
    if (!s_last) return;
    if (tid == 0) *blk_cnt = 0;
    __threadfence();
    const LogitCoef kc = logit_coef(p.sm_alpha, p.sm_inv_2beta2);
    const int64_t stride = static_cast<int64_t>(p.n) * p.n_x;
    for (int r = warp; r < 128; r += nwarps) {
        const int i = rb * 128 + r;
        if (i < p.n)
            softmax_tile_stats(i, cb, p.partial, p.splits, stride, p.n_x, p.n_x, p.sm_norms, kc, p.sm_L, p.n_x,
                               p.sm_stats, nt);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(band_cnt, 1) == nt - 1;
    __syncthreads();
    if (!s_last) return;
    if (tid == 0) *band_cnt = 0;
    __threadfence();
    for (int r = warp; r < 128; r += nwarps) {
        const int i = rb * 128 + r;
        if (i < p.n)
            softmax_finalize_row(i, p.n_x, nt, p.sm_L, p.n_x, p.sm_stats, p.sm_w, p.sm_ldw, p.sm_w_hi, p.sm_w_lo,
                                 p.sm_ldwb);
    }
}

// This CTA's share of the next step's noise slice, written while the MMAs
// run by warps noise_warp0..9 (the epilogue warps 2-5 are idle then too and
// may join): a contiguous range of state columns for every particle quad, two
// independent Philox blocks per iteration.
__device__ __forceinline__ void gram_noise_share(const GramParams &p) {
    const int blocks = gridDim.x * gridDim.y * gridDim.z;
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int64_t per = (p.d + blocks - 1) / blocks;
    const int64_t c0 = static_cast<int64_t>(b) * per;
    const int64_t c1 = c0 + per < p.d ? c0 + per : p.d;
    const int quads = (p.n + 3) / 4;
    const int et = threadIdx.x - 32 * p.noise_warp0;
    const int kStride = static_cast<int>(blockDim.x) - 32 * p.noise_warp0;
    for (int qd = 0; qd < quads; ++qd) {
        for (int64_t col = c0 + et; col < c1; col += 2 * kStride) {
            const int64_t col2 = col + kStride;
            const float4 v = noise4(p.seed, p.offset, p.noise_k, col + p.noise_col0, qd);
            const float4 v2 = col2 < c1 ? noise4(p.seed, p.offset, p.noise_k, col2 + p.noise_col0, qd) : v;
            const float vv[4] = {v.x, v.y, v.z, v.w}, vv2[4] = {v2.x, v2.y, v2.z, v2.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = qd * 4 + r;
                if (i < p.n) {
                    p.noise[static_cast<int64_t>(i) * p.d + col] = vv[r];
                    if (col2 < c1) p.noise[static_cast<int64_t>(i) * p.d + col2] = vv2[r];
                }
            }
        }
    }
}

template <int BN, int STAGES, bool SPLIT, int KB, int ES = 2>
__global__ void __launch_bounds__(kGramThreads, 1)
k_gram_tc(const __grid_constant__ CUtensorMap a_hi, const __grid_constant__ CUtensorMap a_lo,
          const __grid_constant__ CUtensorMap b_hi, const __grid_constant__ CUtensorMap b_lo, GramParams p) {
    pdl_wait();  // reads the particle planes of the previous step's W X
    pdl_launch_dependents();
    using P = Plan<BN, STAGES, SPLIT, KB, ES>;
    extern __shared__ uint8_t smem_raw[];
    const Ctl c = carve<P>(smem_raw, STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, split = blockIdx.z;
    const int kb0 = split * p.kb_per_split;
    const int nkb = min(p.kblocks, kb0 + p.kb_per_split) - kb0;
    if (*reinterpret_cast<volatile int *>(p.err) != 0) return;  // an earlier launch failed: skip
    const uint32_t tmem = setup<BN, STAGES>(c, warp);

    if (warp == 0) {
        if (lane == 0) produce<BN, STAGES, SPLIT, KB, ES>(c, &a_hi, &a_lo, &b_hi, &b_lo, m0, n0, kb0, nkb, p.err);
    } else if (warp == 1) {
        if (lane == 0) mma_loop<BN, STAGES, SPLIT, KB, ES>(c, tmem, nkb, p.err);
    } else {
        if (p.noise && warp >= p.noise_warp0) gram_noise_share(p);
        if (warp >= 6) {
            // noise-only warps: nothing else to do
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
    }
    teardown<BN>(tmem, warp);
}

// ------------------------------------------------------------- Pair Gram
// A cluster of two CTAs computes one 256 x 256 tile of the split-BF16x3 Gram
// with tcgen05.mma.cta_group::2 (M = 256 across the pair).  CTA r of the pair
// loads rows m0 + 128 r of A (particles) and rows n0 + 128 r of B (forecast
// members) into its own ring; the leader (r = 0) issues the MMAs, which read
// the A and B halves of both CTAs and write 128 accumulator rows into each
// CTA's TMEM.  Per SM this halves the B operand traffic through shared
// memory, which bounds the single-CTA Gram.
//
// Readiness of a stage: each CTA's TMA completes on its own full barrier; the
// peer's warp 1 forwards its completion to the leader's full barrier (count 2:
// the leader's own expect_tx arrival and the peer's remote arrival).  The
// leader's commits arrive on the empty and accumulator barriers of both CTAs
// (multicast).  Every wait is bounded; TMEM allocation, the cluster barriers
// and the deallocation are reached by every thread of both CTAs (no early
// exit), and the decision to skip the work after an earlier failure is taken
// jointly by the pair.
constexpr int kPairStages = 3;      // split-BF16x3: 64 KB per k-block
constexpr int kPairStagesTf32 = 6;  // TF32: 32 KB per k-block
constexpr int kPairTile = 256;

// Per k-block of 128 bytes per row (64 BF16 or 32 FP32 elements): this CTA's
// 128 rows of A and of B, as hi and lo planes (split-BF16x3) or one FP32
// plane each (TF32).
template <bool TF32>
struct PairPlan {
    static constexpr int kStages = TF32 ? kPairStagesTf32 : kPairStages;
    static constexpr int kA = 128 * 128;  // this CTA's 128 rows of A, one plane
    static constexpr int kB = 128 * 128;  // this CTA's 128 rows of B, one plane
    static constexpr int kStage = (kA + kB) * (TF32 ? 1 : 2);
    static constexpr int kBarOff = kStage * kStages + 32 * 1024;  // + guard after the ring
    static constexpr int kBytes = kBarOff + 256 + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the variable at shared::cta address `addr` in CTA `rank`
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Cluster-wide barrier of every thread of both CTAs (the non-aligned form:
// lanes may arrive from divergent paths).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait with cluster-scope acquire (arrivals come from the other CTA).
__device__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cl(bar, parity)) return true;
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

__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_tf32_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive on the barrier at this offset in both CTAs of the pair once the
// leader's MMAs issued so far have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(static_cast<uint16_t>(3))
        : "memory");
}

// TF32: one FP32 plane per operand (a_hi, b_hi; a_lo, b_lo unused), k-blocks
// of 32 elements, one kind::tf32 product (K = 8 per MMA).
template <bool TF32>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGramThreads, 1)
k_gram_tc_pair(const __grid_constant__ CUtensorMap a_hi, const __grid_constant__ CUtensorMap a_lo,
               const __grid_constant__ CUtensorMap b_hi, const __grid_constant__ CUtensorMap b_lo, GramParams p) {
    pdl_wait();  // reads the particle planes of the previous step's W X
    pdl_launch_dependents();
    using P = PairPlan<TF32>;
    constexpr int NST = P::kStages;          // ring depth
    constexpr int KBW = TF32 ? 32 : BK;      // k-block width in elements
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = smem_raw + pad;
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + P::kBarOff);
    uint64_t *empty = full + NST;
    uint64_t *accum = empty + NST;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *skip_own = abort_flag + 1;
    volatile int *skip_pair = abort_flag + 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    const int m_own = (blockIdx.x >> 1) * kPairTile + static_cast<int>(rank) * 128;
    const int n0 = blockIdx.y * kPairTile;
    const int n_own = n0 + static_cast<int>(rank) * 128;
    const int split = blockIdx.z;
    const int kb0 = split * p.kb_per_split;
    int nkb = min(p.kblocks, kb0 + p.kb_per_split) - kb0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], leader ? 2 : 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        *skip_own = *reinterpret_cast<volatile int *>(p.err) != 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, kPairTile);
    tc_fence_before();
    cluster_sync_all();
    tc_fence_after();
    if (threadIdx.x == 0) {
        uint32_t peer_flag = mapa_shared(smem_u32(const_cast<int *>(skip_own)), rank ^ 1u);
        int other;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(other) : "r"(peer_flag) : "memory");
        *skip_pair = (*skip_own | other) != 0;
    }
    __syncthreads();
    const bool skip = *skip_pair != 0;
    if (skip) nkb = 0;
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % NST;
                const uint32_t ph = (i / NST) & 1;
                if (!mbar_wait_cl(&empty[s], ph ^ 1u, abort_flag, p.err)) break;
                const uint32_t st = smem_u32(tiles + s * P::kStage);
                mbar_expect_tx(&full[s], P::kStage);
                const int kx = (kb0 + i) * KBW;
                if (TF32) {
                    tma_load_2d(st, &a_hi, &full[s], kx, m_own);
                    tma_load_2d(st + P::kA, &b_hi, &full[s], kx, n_own);
                } else {
                    tma_load_2d(st, &a_hi, &full[s], kx, m_own);
                    tma_load_2d(st + P::kA, &a_lo, &full[s], kx, m_own);
                    tma_load_2d(st + 2 * P::kA, &b_hi, &full[s], kx, n_own);
                    tma_load_2d(st + 2 * P::kA + P::kB, &b_lo, &full[s], kx, n_own);
                }
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
            if (leader) {
                constexpr uint32_t idesc = TF32 ? idesc_tf32(2 * BM, kPairTile) : idesc_bf16(2 * BM, kPairTile);
                for (int i = 0; i < nkb; ++i) {
                    const int s = i % NST;
                    const uint32_t ph = (i / NST) & 1;
                    if (!mbar_wait_cl(&full[s], ph, abort_flag, p.err)) break;
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(tiles + s * P::kStage);
                    if (TF32) {
                        const uint32_t b0 = a0 + P::kA;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {  // K = 8 FP32 = 32 bytes per MMA
                            const uint32_t off = kk * 32;
                            mma_tf32_pair(tmem, desc_sw128(a0 + off), desc_sw128(b0 + off), idesc,
                                          (i > 0 || kk > 0) ? 1u : 0u);
                        }
                    } else {
                        const uint32_t a1 = a0 + P::kA;
                        const uint32_t b0 = a0 + 2 * P::kA;
                        const uint32_t b1 = b0 + P::kB;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint32_t off = kk * 32;
                            mma_bf16_pair(tmem, desc_sw128(a0 + off), desc_sw128(b0 + off), idesc,
                                          (i > 0 || kk > 0) ? 1u : 0u);
                            mma_bf16_pair(tmem, desc_sw128(a0 + off), desc_sw128(b1 + off), idesc, 1u);
                            mma_bf16_pair(tmem, desc_sw128(a1 + off), desc_sw128(b0 + off), idesc, 1u);
                        }
                    }
                    mma_commit_pair(&empty[s]);
                }
                mma_commit_pair(accum);
            } else {
                // forward the completion of this CTA's loads to the leader
                for (int i = 0; i < nkb; ++i) {
                    const int s = i % NST;
                    if (!mbar_wait(&full[s], (i / NST) & 1, abort_flag, p.err)) break;
                    mbar_arrive_cluster(mapa_shared(smem_u32(&full[s]), 0));
                }
            }
        }
    } else {
        if (p.noise && !skip && warp >= p.noise_warp0) gram_noise_share(p);
        if (warp < 6 && nkb > 0) {
            const int q = warp & 3;
            const int row = m_own + q * 32 + lane;
            const bool ok = mbar_wait_cl(accum, 0, abort_flag, p.err);
            tc_fence_after();
            if (ok) {
                float *dst = p.partial + (static_cast<int64_t>(split) * p.n + row) * p.n_x;
#pragma unroll 1
                for (int cc = 0; cc < kPairTile; cc += 32) {
                    float v[32];
                    tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + cc, v);
                    const int col0 = n0 + cc;
                    if (row < p.n && col0 < p.n_x) {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (col0 + e < p.n_x) dst[col0 + e] = v[e];
                    }
                }
                if (p.sm_L) __threadfence();  // the partials reach L2 before this block is counted
            }
        }
    }
    tc_fence_before();
    cluster_sync_all();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem, kPairTile);
    }
    if (p.sm_L && !skip && nkb > 0 && *abort_flag == 0) gram_softmax_tail(p, m_own >> 7, blockIdx.y);
}

// ------------------------------------------------ Pair Gram, FP32 particles
// The same 256 x 256 pair tile, but the particle operand arrives as FP32 z
// (two 128-byte-swizzled 32-column boxes per k-block) instead of BF16 hi/lo
// planes: warps 2-5 form a = z - alpha m for their 32 rows, split it into
// a_hi + a_lo and store both into TMEM with tcgen05.st; the MMAs take A from
// TMEM (tcgen05.mma ... [a_tmem], b_desc).  The W X kernel then no longer
// writes Z hi/lo planes (4 bytes per particle element per step less HBM
// traffic), and shared memory carries only B for the MMAs.  The split is the
// one the W X epilogue would have written, so results are bitwise those of
// the plane-fed kernels.
constexpr int kPairF32Stages = 3;

struct PairF32Plan {
    static constexpr int kZBox = 128 * 32 * 4;  // one 32-column FP32 box of this CTA's 128 rows
    static constexpr int kB = 128 * BK * 2;     // this CTA's 128 rows of B, one plane
    static constexpr int kStage = 2 * kZBox + 2 * kB;
    static constexpr int kBarOff = kStage * kPairF32Stages;
    static constexpr int kBytes = kBarOff + 256 + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
};
constexpr int kPairF32TmemCols = 512;   // accumulator 0-255, A slots 256 + 64 s (hi 32, lo 32)
// warps: 0 producer, 1 MMA issuer (leader) / forwarder (peer), 2-9 split the
// particle operand (warp w: TMEM lane quarter w % 4, 32-column box (w - 2) / 4)
// and then run the epilogue, 10-15 generate the next step's noise
constexpr int kPairF32Threads = 512;
constexpr int kPairF32Convert = 8;

__device__ __forceinline__ void mma_bf16_pair_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                 uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    __syncwarp();
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo_k, __nv_bfloat16 hi_k) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(lo_k)) |
           (static_cast<uint32_t>(__bfloat16_as_ushort(hi_k)) << 16);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairF32Threads, 1)
k_gram_tc_pair_f32(const __grid_constant__ CUtensorMap z32, const __grid_constant__ CUtensorMap unused,
                   const __grid_constant__ CUtensorMap b_hi, const __grid_constant__ CUtensorMap b_lo, GramParams p) {
    pdl_wait();  // reads the particles written by the previous step's W X
    pdl_launch_dependents();
    using P = PairF32Plan;
    constexpr int S = kPairF32Stages;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = smem_raw + pad;
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + P::kBarOff);
    uint64_t *empty = full + S;
    uint64_t *aready = empty + S;
    uint64_t *accum = aready + S;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *skip_own = abort_flag + 1;
    volatile int *skip_pair = abort_flag + 2;
    (void)unused;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    const int m_own = (blockIdx.x >> 1) * kPairTile + static_cast<int>(rank) * 128;
    const int n0 = blockIdx.y * kPairTile;
    const int n_own = n0 + static_cast<int>(rank) * 128;
    const int split = blockIdx.z;
    const int kb0 = split * p.kb_per_split;
    int nkb = min(p.kblocks, kb0 + p.kb_per_split) - kb0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&aready[s], leader ? kPairF32Convert + 1 : kPairF32Convert);  // (+ the peer's forward)
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        *skip_own = *reinterpret_cast<volatile int *>(p.err) != 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc_pair(tmem_slot, kPairF32TmemCols);
    tc_fence_before();
    cluster_sync_all();
    tc_fence_after();
    if (threadIdx.x == 0) {
        uint32_t peer_flag = mapa_shared(smem_u32(const_cast<int *>(skip_own)), rank ^ 1u);
        int other;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(other) : "r"(peer_flag) : "memory");
        *skip_pair = (*skip_own | other) != 0;
    }
    __syncthreads();
    const bool skip = *skip_pair != 0;
    if (skip) nkb = 0;
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % S;
                const uint32_t ph = (i / S) & 1;
                if (!mbar_wait_cl(&empty[s], ph ^ 1u, abort_flag, p.err)) break;
                const uint32_t st = smem_u32(tiles + s * P::kStage);
                mbar_expect_tx(&full[s], P::kStage);
                const int kx = (kb0 + i) * BK;
                tma_load_2d(st, &z32, &full[s], kx, m_own);
                tma_load_2d(st + P::kZBox, &z32, &full[s], kx + 32, m_own);
                tma_load_2d(st + 2 * P::kZBox, &b_hi, &full[s], kx, n_own);
                tma_load_2d(st + 2 * P::kZBox + P::kB, &b_lo, &full[s], kx, n_own);
                issued = i + 1;
            }
            if (*abort_flag) {
                const uint64_t t0 = globaltimer();
                for (int i = issued > S ? issued - S : 0; i < issued; ++i) {
                    const int s = i % S;
                    while (!mbar_try_wait(&full[s], (i / S) & 1) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            if (leader) {
                constexpr uint32_t idesc = idesc_bf16(2 * BM, kPairTile);
                for (int i = 0; i < nkb; ++i) {
                    const int s = i % S;
                    const uint32_t ph = (i / S) & 1;
                    if (!mbar_wait_cl(&aready[s], ph, abort_flag, p.err)) break;
                    tc_fence_after();
                    const uint32_t a_hi = tmem + 256 + 64 * s;
                    const uint32_t b0 = smem_u32(tiles + s * P::kStage + 2 * P::kZBox);
                    const uint32_t b1 = b0 + P::kB;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t ta = a_hi + 8 * kk;  // 16 BF16 = 8 columns per K = 16 chunk
                        const uint32_t off = kk * 32;
                        mma_bf16_pair_ta(tmem, ta, desc_sw128(b0 + off), idesc, (i > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16_pair_ta(tmem, ta, desc_sw128(b1 + off), idesc, 1u);
                        mma_bf16_pair_ta(tmem, ta + 32, desc_sw128(b0 + off), idesc, 1u);
                    }
                    mma_commit_pair(&empty[s]);
                }
                mma_commit_pair(accum);
            } else {
                // forward this CTA's A-ready signals to the leader
                for (int i = 0; i < nkb; ++i) {
                    const int s = i % S;
                    if (!mbar_wait(&aready[s], (i / S) & 1, abort_flag, p.err)) break;
                    mbar_arrive_cluster(mapa_shared(smem_u32(&aready[s]), 0));
                }
            }
        }
    } else if (warp < 2 + kPairF32Convert) {
        const int q = warp & 3;             // TMEM lane quarter of this warp
        const int box = (warp - 2) >> 2;    // which 32-column half of the k-block
        const int r = q * 32 + lane;        // this thread's row within the CTA's 128
        const uint32_t lane_base = static_cast<uint32_t>(q * 32) << 16;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            if (!mbar_wait(&full[s], (i / S) & 1, abort_flag, p.err)) break;
            // alpha m for the 32 columns of this box: one coalesced load per
            // warp, handed to every lane by shuffles
            const int64_t c_lane = static_cast<int64_t>(kb0 + i) * BK + box * 32 + lane;
            const float shift_lane =
                (p.centre && c_lane < p.d) ? __fmul_rn(p.alpha, __ldg(p.centre + c_lane)) : 0.f;
            const bool tail = static_cast<int64_t>(kb0 + i) * BK + box * 32 + 32 > p.d;
            const uint8_t *zrow = tiles + s * P::kStage + box * P::kZBox + r * 128;
            float4 v[8];
#pragma unroll
            for (int ch = 0; ch < 8; ++ch)  // 128-byte swizzle: chunk ch of row r sits at ch ^ (r & 7)
                v[ch] = *reinterpret_cast<const float4 *>(zrow + ((ch ^ (r & 7)) << 4));
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
                const float vv[4] = {v[ch].x, v[ch].y, v[ch].z, v[ch].w};
                __nv_bfloat16 h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = ch * 4 + e;
                    const float sh = __shfl_sync(0xffffffffu, shift_lane, j);
                    // past the end of the state the tile holds zeros: keep them
                    const bool in = !tail || (static_cast<int64_t>(kb0 + i) * BK + box * 32 + j < p.d);
                    const float a = in ? __fsub_rn(vv[e], sh) : 0.f;
                    h[e] = __float2bfloat16_rn(a);
                    l[e] = __float2bfloat16_rn(__fsub_rn(a, __bfloat162float(h[e])));
                }
                hw[ch * 2] = pack_bf16x2(h[0], h[1]);
                hw[ch * 2 + 1] = pack_bf16x2(h[2], h[3]);
                lw[ch * 2] = pack_bf16x2(l[0], l[1]);
                lw[ch * 2 + 1] = pack_bf16x2(l[2], l[3]);
            }
            const uint32_t ta = tmem + lane_base + 256 + 64 * s + 16 * box;
            tmem_st16(ta, hw);
            tmem_st16(ta + 32, lw);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&aready[s]);
        }
        if (nkb > 0) {
            // epilogue: the two warps of a lane quarter take 128 columns each
            const int row = m_own + r;
            const bool ok = mbar_wait_cl(accum, 0, abort_flag, p.err);
            tc_fence_after();
            if (ok) {
                float *dst = p.partial + (static_cast<int64_t>(split) * p.n + row) * p.n_x;
#pragma unroll 1
                for (int cc = box * 128; cc < box * 128 + 128; cc += 32) {
                    float o[32];
                    tmem_ld32(tmem + lane_base + cc, o);
                    const int col0 = n0 + cc;
                    if (row < p.n && col0 < p.n_x) {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (col0 + e < p.n_x) dst[col0 + e] = o[e];
                    }
                }
            }
        }
    } else {
        if (p.noise && !skip) gram_noise_share(p);
    }
    tc_fence_before();
    cluster_sync_all();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem, kPairF32TmemCols);
    }
}

// ------------------------------------------------------- W X + EM update
// Persistent kernel over tiles of U^T = X^T W^T: MMA rows (TMEM lanes) are 128
// state columns c, MMA columns are BN particles i.  An epilogue thread owns one
// state column, so for each particle the 32 lanes of a warp touch 32
// consecutive floats of z[i][:] and of the noise slice (coalesced), and y[c],
// mask[c] are read once per tile.  Two TMEM accumulators (columns 0 and 256)
// let the epilogue of one tile run while the MMAs of the next accumulate.  The
// noise of the step arrives pre-generated (a [n][d] slice), so the epilogue is
// loads, the score, the update and stores.
constexpr int kEpiWarps = 16;                      // four per TMEM lane quarter
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
    float *zc32;             // FP32 z - alpha_next m for a TF32 Gram (NULL: none)
    const float *y;
    const uint8_t *mask;
    const float *noise;  // xi[k+1] slice [n][d] (pre-generated form)
    uint64_t seed;       // Philox stream (in-kernel form)
    uint32_t offset;
    const float *centre; // Gram centre m [d] or NULL
    float alpha_next;    // z_hi/z_lo carry z - alpha_next m for the next Gram
    StepCoef coef;
    int *err;
    bool pdl;  // host: launched with programmatic stream serialization
};


template <int BN, int STAGES, bool SPLIT, bool INLINE_NOISE>
__global__ void __launch_bounds__(kWxThreads, 1)
k_wx_em_tc(const __grid_constant__ CUtensorMap xt_hi, const __grid_constant__ CUtensorMap xt_lo,
           const __grid_constant__ CUtensorMap w_hi, const __grid_constant__ CUtensorMap w_lo, WxParams p) {
    pdl_wait();  // reads the weights of the row softmax
    pdl_launch_dependents();
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
        const int part = ew >> 2;           // which quarter of the BN particle columns
        constexpr int kCols = BN / 4;       // 16, 32 or 64 particle columns per warp
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
            const float shift = (cok && p.centre) ? __fmul_rn(p.alpha_next, p.centre[c]) : 0.f;
#pragma unroll 1
            for (int cc = part * kCols; cc < (part + 1) * kCols; cc += 16) {
                float u[16];
                tmem_ld16(tmem + slot * 256 + (static_cast<uint32_t>(q * 32) << 16) + cc, u);
                const int i0 = n0 + cc;
                if (!cok || i0 >= p.n) continue;
                const int cnt = p.n - i0 < 16 ? p.n - i0 : 16;
                const int64_t base = static_cast<int64_t>(i0) * p.d + c;
                float zv[16], xi[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    if (e < cnt) {
                        zv[e] = p.z[base + e * p.d];
                        if (!INLINE_NOISE) xi[e] = p.noise[base + e * p.d];
                    }
                }
                if (INLINE_NOISE) {
                    // xi[k+1][i0 .. i0+15][c]: four Philox blocks of four particles each
#pragma unroll
                    for (int e4 = 0; e4 < 4; ++e4) {
                        const float4 v = noise4(p.seed, p.offset, cf.k + 1, c + cf.col0, (i0 >> 2) + e4);
                        xi[e4 * 4 + 0] = v.x;
                        xi[e4 * 4 + 1] = v.y;
                        xi[e4 * 4 + 2] = v.z;
                        xi[e4 * 4 + 3] = v.w;
                    }
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    if (e >= cnt) break;
                    const float g = obs ? lik_score(cf.obs_op, zv[e], yc, cf.inv_r) : 0.f;
                    const float zn = em_update(cf, zv[e], u[e], g, xi[e]);
                    const int64_t off = base + e * p.d;
                    p.z[off] = zn;
                    if (p.zc32) p.zc32[off] = __fsub_rn(zn, shift);
                    if (p.zb_hi) {
                        const float zc = __fsub_rn(zn, shift);  // rounded as the FP32-operand Gram rounds it
                        const __nv_bfloat16 hi = __float2bfloat16_rn(zc);
                        p.zb_hi[off] = hi;
                        if (p.zb_lo) p.zb_lo[off] = __float2bfloat16_rn(zc - __bfloat162float(hi));
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

// ------------------------------------------- W X + EM, TMA-staged epilogue
// The persistent tile loop of k_wx_em_tc (tiles of U^T = X^T W^T: 128 state
// columns x BN particles, two TMEM accumulators), with the particle state
// moved through shared memory by TMA instead of per-thread global accesses.
// The four epilogue warps that share a quarter of the tile's particles work
// in chunks of 16 particles x 128 state columns: one thread of the four warps
// loads the chunk of z (FP32) into a staging buffer with TMA (the next chunk's
// load overlaps this chunk's arithmetic), each thread updates its column of
// the chunk in place and writes the BF16 planes of the next Gram beside it,
// and the same thread stores the chunk back with TMA.  The step's noise is
// evaluated in the epilogue from the counter-based stream.  Per element an
// epilogue thread thus issues three or four shared-memory accesses at fixed
// offsets and no address arithmetic, which leaves the issue slots the noise
// needs.  The arithmetic is that of k_wx_em_tc (bitwise).
constexpr int kStgRows = 16;    // particles per staged chunk
constexpr int kStgCols = BM;    // state columns per staged chunk (the tile's MMA rows)

template <int BN, int STAGES>
struct WxStagedPlan {
    static constexpr int kA = BM * BK * 2;  // X^T rows (state columns)
    static constexpr int kB = BN * BK * 2;  // W rows (particles)
    static constexpr int kStage = kA + kB;
    static constexpr int kStgZ = kStgRows * kStgCols * 4;   // FP32 z chunk
    static constexpr int kStgH = kStgRows * kStgCols * 2;   // one BF16 plane chunk
    static constexpr int kStgBuf = kStgZ + 2 * kStgH;
    static constexpr int kStgOff = kStage * STAGES;
    static constexpr int kBarOff = kStgOff + 4 * 2 * kStgBuf;  // four particle quarters, double-buffered
    static constexpr int kBytes = kBarOff + 512 + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory plan too large");
    static_assert(BN == 64 || BN == 128 || BN == 256, "BN");
};

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// OBS: the observation operator (0 identity, 1 arctan); PLANES: the BF16
// particle planes the next Gram reads (0 none, 1 hi, 2 hi and lo).
template <int BN, int STAGES, int OBS, int PLANES>
__global__ void __launch_bounds__(kWxThreads, 1)
k_wx_em_staged(const __grid_constant__ CUtensorMap xt_hi, const __grid_constant__ CUtensorMap w_hi,
               const __grid_constant__ CUtensorMap z_map, const __grid_constant__ CUtensorMap zh_map,
               const __grid_constant__ CUtensorMap zl_map, WxParams p) {
    pdl_wait();  // reads the weights of the row softmax
    pdl_launch_dependents();
    using P = WxStagedPlan<BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(p.err) != 0) return;  // an earlier launch failed: skip

    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = smem_raw + pad;
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + P::kBarOff);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;   // [2] accumulator ready
    uint64_t *tempty = tfull + 2;       // [2] accumulator drained
    uint64_t *zfull = tempty + 2;       // [4 quarters][2 buffers] staged z chunk landed
    uint64_t *zdone = zfull + 8;        // [4 quarters][2 buffers] chunk updated by its 128 threads
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(zdone + 8);
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
        for (int b = 0; b < 8; ++b) {
            mbar_init(&zfull[b], 1);
            mbar_init(&zdone[b], 128);
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
            int it = 0, issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int m0 = (t / p.n_tiles) * BM, n0 = (t % p.n_tiles) * BN;
                for (int kb = 0; kb < p.kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.err)) { ok = false; break; }
                    const uint32_t st = smem_u32(tiles + s * P::kStage);
                    mbar_expect_tx(&full[s], P::kStage);
                    tma_load_2d(st, &xt_hi, &full[s], kb * BK, m0);
                    tma_load_2d(st + P::kA, &w_hi, &full[s], kb * BK, n0);
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
                    const uint32_t a = smem_u32(tiles + s * P::kStage);
                    const uint32_t b = a + P::kA;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(acc, desc_sw128(a + kk * 32), desc_sw128(b + kk * 32), idesc,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[slot]);
            }
        }
    } else {
        const int ew = warp - 2;            // 0 .. kEpiWarps-1
        const int q = warp & 3;             // TMEM lane quarter this warp may read
        const int part = ew >> 2;           // which quarter of the BN particle columns
        const bool leader = (ew & 3) == 0 && lane == 0;
        constexpr int kCols = BN / 4;       // particle columns per quarter
        constexpr int kChunks = kCols / kStgRows;
        const int cl = q * 32 + lane;       // this thread's state column within the tile
        const StepCoef &cf = p.coef;
        uint8_t *stg = tiles + P::kStgOff + part * 2 * P::kStgBuf;
        uint64_t *zf = zfull + part * 2;
        uint64_t *zd = zdone + part * 2;
        constexpr bool planes = PLANES >= 1;
        constexpr bool lo_plane = PLANES == 2;
        // the chunk sequence of this quarter runs across the tiles of this CTA
        auto chunk_origin = [&](int g, int &x, int &y) {
            const int t = blockIdx.x + (g / kChunks) * gridDim.x;
            x = (t / p.n_tiles) * BM;
            y = (t % p.n_tiles) * BN + part * kCols + (g % kChunks) * kStgRows;
        };
        auto issue_load = [&](int g) {
            int x, y;
            chunk_origin(g, x, y);
            uint64_t *bar = &zf[g & 1];
            mbar_expect_tx(bar, P::kStgZ);
            tma_load_2d(smem_u32(stg + (g & 1) * P::kStgBuf), &z_map, bar, x, y);
        };
        const int my_tiles = blockIdx.x < total ? (total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const int n_chunks = my_tiles * kChunks;
        if (leader && n_chunks > 0) issue_load(0);
        int g = 0, lt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++lt) {
            const int slot = lt & 1;
            const uint32_t use = lt >> 1;
            const int m0 = (t / p.n_tiles) * BM, n0 = (t % p.n_tiles) * BN;
            // every wait's outcome is made warp-uniform: the TMEM loads are warp-collective
            if (!__all_sync(0xffffffffu, mbar_wait(&tfull[slot], use & 1u, abort_flag, p.err))) break;
            tc_fence_after();
            const int64_t c = static_cast<int64_t>(m0) + cl;  // this thread's state column
            const bool cok = c < p.d;
            const float yc = cok ? p.y[c] : 0.f;
            const bool obs = cok && (p.mask == nullptr || p.mask[c] != 0);
            const float shift = (cok && p.centre) ? __fmul_rn(p.alpha_next, p.centre[c]) : 0.f;
#pragma unroll 1
            for (int ch = 0; ch < kChunks; ++ch, ++g) {
                const int buf = g & 1;
                if (leader && g + 1 < n_chunks) {
                    bulk_wait_read_all();  // the store of chunk g - 1 has left that buffer
                    issue_load(g + 1);
                }
                const int cc = part * kCols + ch * kStgRows;  // accumulator column = particle within tile
                float u[16];
                tmem_ld16(tmem + slot * 256 + (static_cast<uint32_t>(q * 32) << 16) + cc, u);
                if (!__all_sync(0xffffffffu, mbar_wait(&zf[buf], (g >> 1) & 1u, abort_flag, p.err))) {
                    ok = false;
                    break;
                }
                float *zs = reinterpret_cast<float *>(stg + buf * P::kStgBuf);
                __nv_bfloat16 *hs = reinterpret_cast<__nv_bfloat16 *>(stg + buf * P::kStgBuf + P::kStgZ);
                __nv_bfloat16 *ls = hs + kStgRows * kStgCols;
                const int i0 = n0 + cc;
                if (i0 < p.n) {  // (a chunk wholly past the last particle is neither computed nor stored)
                float xi[16];
#pragma unroll
                for (int e4 = 0; e4 < 4; ++e4) {
                    const float4 v = noise4(p.seed, p.offset, cf.k + 1, c + cf.col0, (i0 >> 2) + e4);
                    xi[e4 * 4 + 0] = v.x;
                    xi[e4 * 4 + 1] = v.y;
                    xi[e4 * 4 + 2] = v.z;
                    xi[e4 * 4 + 3] = v.w;
                }
#pragma unroll
                for (int e = 0; e < kStgRows; ++e) {
                    const float zv = zs[e * kStgCols + cl];
                    const float gl = obs ? lik_score(OBS, zv, yc, cf.inv_r) : 0.f;
                    const float zn = em_update(cf, zv, u[e], gl, xi[e]);
                    zs[e * kStgCols + cl] = zn;
                    if (planes) {
                        const float zc = __fsub_rn(zn, shift);  // rounded as the FP32-operand Gram rounds it
                        const __nv_bfloat16 hi = __float2bfloat16_rn(zc);
                        hs[e * kStgCols + cl] = hi;
                        if (lo_plane) ls[e * kStgCols + cl] = __float2bfloat16_rn(zc - __bfloat162float(hi));
                    }
                }
                }
                // the chunk's shared-memory writes, visible to the TMA store, then
                // counted on the chunk's barrier; the leader alone waits (bounded)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&zd[buf]);
                if (leader) {
                    if (!mbar_wait(&zd[buf], (g >> 1) & 1u, abort_flag, p.err)) {
                        ok = false;
                    } else if (i0 < p.n) {  // (a chunk wholly past the last particle stores nothing)
                        tma_store_2d(&z_map, smem_u32(zs), m0, i0);
                        if (planes) tma_store_2d(&zh_map, smem_u32(hs), m0, i0);
                        if (lo_plane) tma_store_2d(&zl_map, smem_u32(ls), m0, i0);
                        bulk_commit();
                    }
                }
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[slot]);
        }
        if (leader) bulk_wait_all();  // the stores have read shared memory and landed
        (void)ok;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kWxTmemCols);
    }
}

// ================================================================ batched
// Gram tile of one instance; maps / parameters / k-range from device tables.
template <int BN, int STAGES, bool SPLIT>
__global__ void __launch_bounds__(192, 1)
k_gram_tc_batched(const CUtensorMap *__restrict__ maps, const BGramItem *__restrict__ items,
                  const BInst *__restrict__ insts, int *err) {
    using P = Plan<BN, STAGES, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    const Ctl c = carve<P>(smem_raw, STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(err) != 0) return;
    const BGramItem it = items[blockIdx.x];
    const BInst &I = insts[it.inst];
    const int n = I.n;
    const int kblocks = static_cast<int>((I.d + BK - 1) / BK);
    const int kb0 = it.split * I.kb_chunk;
    const int nkb = min(kblocks, kb0 + I.kb_chunk) - kb0;
    const CUtensorMap *m = maps + 4 * it.inst;
    const uint32_t tmem = setup<BN, STAGES>(c, warp);
    if (warp == 0) {
        if (lane == 0) produce<BN, STAGES, SPLIT>(c, m + 0, m + 1, m + 2, m + 3, it.m0, it.n0, kb0, nkb, err);
    } else if (warp == 1) {
        if (lane == 0) mma_loop<BN, STAGES, SPLIT>(c, tmem, nkb, err);
    } else {
        const int q = warp & 3;
        const int row = it.m0 + q * 32 + lane;
        const bool ok = mbar_wait(c.accum, 0, c.abort_flag, err);
        tc_fence_after();
        if (ok) {
            float *dst = I.partial + (static_cast<int64_t>(it.split) * n + row) * n;
#pragma unroll 1
            for (int cc = 0; cc < BN; cc += 32) {
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + cc, v);
                const int col0 = it.n0 + cc;
                if (row < n && col0 < n) {
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        if (col0 + e < n) dst[col0 + e] = v[e];
                }
            }
        }
    }
    teardown<BN>(tmem, warp);
}

__global__ void __launch_bounds__(256)
k_softmax_batched(const BRow *__restrict__ rows, const BInst *__restrict__ insts, double alpha, double inv_2beta2) {
    extern __shared__ double lg[];
    __shared__ double red[256];
    const BRow r = rows[blockIdx.x];
    const BInst &I = insts[r.inst];
    softmax_row<256>(r.row, I.partial, I.splits, static_cast<int64_t>(I.n) * I.n, I.n, I.n, I.norms, alpha,
                     inv_2beta2, nullptr, 0, I.wb_hi, I.wb_lo, I.ldw, lg, red);
}

// Persistent W X + EM over the tile list of all instances (U^T = X^T W^T as in
// the single-filter kernel); noise from the caller's buffer or Philox inline.
template <int BN, int STAGES, bool SPLIT>
__global__ void __launch_bounds__(kWxThreads, 1)
k_wx_em_tc_batched(const CUtensorMap *__restrict__ maps, const BWxItem *__restrict__ items, int n_items,
                   const BInst *__restrict__ insts, StepCoef cf, float alpha_next, int *err) {
    using P = WxPlan<BN, STAGES, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(err) != 0) return;

    uintptr_t base = reinterpret_cast<uintptr_t>(smem_raw);
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = reinterpret_cast<uint8_t *>(base + pad);
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + P::kBarOff);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
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

    if (warp == 0) {
        if (lane == 0) {
            int it_count = 0, issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x) {
                const BWxItem w = items[t];
                const int kblocks = (insts[w.inst].n + BK - 1) / BK;
                const CUtensorMap *m = maps + 8 * w.inst;  // eight maps per filter
                for (int kb = 0; kb < kblocks; ++kb, ++it_count) {
                    const int s = it_count % STAGES;
                    const uint32_t ph = (it_count / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, err)) { ok = false; break; }
                    const uint32_t st = smem_u32(tiles + s * P::kStage);
                    mbar_expect_tx(&full[s], P::kStage);
                    const int kx = kb * BK;
                    tma_load_2d(st, m + 0, &full[s], kx, w.m0);
                    if (SPLIT) tma_load_2d(st + P::kA, m + 1, &full[s], kx, w.m0);
                    tma_load_2d(st + P::kA * P::kPlanes, m + 2, &full[s], kx, w.n0);
                    if (SPLIT) tma_load_2d(st + P::kA * P::kPlanes + P::kB, m + 3, &full[s], kx, w.n0);
                    issued = it_count + 1;
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
            int it_count = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x, ++lt) {
                const int slot = lt & 1;
                const uint32_t use = lt >> 1;
                const int kblocks = (insts[items[t].inst].n + BK - 1) / BK;
                if (!mbar_wait(&tempty[slot], (use & 1u) ^ 1u, abort_flag, err)) break;
                tc_fence_after();
                const uint32_t acc = tmem + slot * 256;
                for (int kb = 0; kb < kblocks; ++kb, ++it_count) {
                    const int s = it_count % STAGES;
                    const uint32_t ph = (it_count / STAGES) & 1;
                    if (!mbar_wait(&full[s], ph, abort_flag, err)) { ok = false; break; }
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
        const int ew = warp - 2;
        const int q = warp & 3;
        const int part = ew >> 2;
        constexpr int kCols = BN / 4;
        int lt = 0;
        for (int t = blockIdx.x; t < n_items; t += gridDim.x, ++lt) {
            const int slot = lt & 1;
            const uint32_t use = lt >> 1;
            const BWxItem w = items[t];
            const BInst &I = insts[w.inst];
            if (!mbar_wait(&tfull[slot], use & 1u, abort_flag, err)) break;
            tc_fence_after();
            const int64_t c = static_cast<int64_t>(w.m0) + q * 32 + lane;
            const bool cok = c < I.d;
            const float yc = cok ? I.y[c] : 0.f;
            const bool obs = cok && (I.mask == nullptr || I.mask[c] != 0);
            const float shift = cok ? __fmul_rn(alpha_next, I.centre[c]) : 0.f;
#pragma unroll 1
            for (int cc = part * kCols; cc < (part + 1) * kCols; cc += 16) {
                float u[16];
                tmem_ld16(tmem + slot * 256 + (static_cast<uint32_t>(q * 32) << 16) + cc, u);
                const int i0 = w.n0 + cc;
                if (!cok || i0 >= I.n) continue;
                const int cnt = I.n - i0 < 16 ? I.n - i0 : 16;
                const int64_t base_off = static_cast<int64_t>(i0) * I.d + c;
                float zv[16], xi[16];
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    if (e < cnt) zv[e] = I.z[base_off + e * I.d];
                if (I.noise_buf) {
                    const float *nb = I.noise_buf + static_cast<int64_t>(cf.k + 1) * I.n * I.d;
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (e < cnt) xi[e] = nb[base_off + e * I.d];
                } else {
#pragma unroll
                    for (int e4 = 0; e4 < 4; ++e4) {
                        const float4 v = noise4(I.seed, I.offset, cf.k + 1, c, (i0 >> 2) + e4);
                        xi[e4 * 4 + 0] = v.x; xi[e4 * 4 + 1] = v.y; xi[e4 * 4 + 2] = v.z; xi[e4 * 4 + 3] = v.w;
                    }
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    if (e >= cnt) break;
                    const float g = obs ? lik_score(I.obs_op, zv[e], yc, I.inv_r) : 0.f;
                    const float zn = em_update(cf, zv[e], u[e], g, xi[e]);
                    const int64_t off = base_off + e * I.d;
                    I.z[off] = zn;
                    const float zc = __fsub_rn(zn, shift);
                    const __nv_bfloat16 hi = __float2bfloat16_rn(zc);
                    I.zb_hi[off] = hi;
                    if (I.zb_lo) I.zb_lo[off] = __float2bfloat16_rn(zc - __bfloat162float(hi));
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

// One staged chunk's update (16 particles of this thread's state column):
// score, Euler-Maruyama step and the next Gram's BF16 planes, the
// observation operator (OBS) and the lo plane (LO) fixed at compile time.
template <int OBS, bool LO>
__device__ __forceinline__ void staged_chunk_update(float *zs, __nv_bfloat16 *hs, __nv_bfloat16 *ls, int cl,
                                                    const float (&u)[16], const float (&xi)[16], bool obs, float yc,
                                                    float inv_r, const StepCoef &cf, float shift) {
#pragma unroll
    for (int e = 0; e < kStgRows; ++e) {
        const float zv = zs[e * kStgCols + cl];
        const float gl = obs ? lik_score(OBS, zv, yc, inv_r) : 0.f;
        const float zn = em_update(cf, zv, u[e], gl, xi[e]);
        zs[e * kStgCols + cl] = zn;
        const float zc = __fsub_rn(zn, shift);
        const __nv_bfloat16 hi = __float2bfloat16_rn(zc);
        hs[e * kStgCols + cl] = hi;
        if (LO) ls[e * kStgCols + cl] = __float2bfloat16_rn(zc - __bfloat162float(hi));
    }
}

// Batched W X + EM with the TMA-staged epilogue of k_wx_em_staged, over the
// tile list of all filters (BN = kBatchTileN particles per item).  The
// filter's maps sit at maps[8 inst + ...]: 0, 2 the W X operands (X^T, W),
// 4, 5, 6 the staging maps of z (FP32) and of its BF16 hi and lo planes.  The
// noise is the counter-based stream of each filter (no caller buffers).
__global__ void __launch_bounds__(kWxThreads, 1)
k_wx_em_staged_batched(const CUtensorMap *__restrict__ maps, const BWxItem *__restrict__ items, int n_items,
                       const BInst *__restrict__ insts, StepCoef cf, float alpha_next, int *err) {
    constexpr int BN = kBatchTileN, STAGES = 3;
    using P = WxStagedPlan<BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile int *>(err) != 0) return;
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    uint8_t *tiles = smem_raw + pad;
    uint64_t *full = reinterpret_cast<uint64_t *>(tiles + P::kBarOff);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *zfull = tempty + 2;
    uint64_t *zdone = zfull + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(zdone + 8);
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
        for (int b = 0; b < 8; ++b) {
            mbar_init(&zfull[b], 1);
            mbar_init(&zdone[b], 128);
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

    if (warp == 0) {
        if (lane == 0) {
            int it = 0, issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x) {
                const BWxItem w = items[t];
                const int kblocks = (insts[w.inst].n + BK - 1) / BK;
                const CUtensorMap *m = maps + 8 * w.inst;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, err)) { ok = false; break; }
                    const uint32_t st = smem_u32(tiles + s * P::kStage);
                    mbar_expect_tx(&full[s], P::kStage);
                    tma_load_2d(st, m + 0, &full[s], kb * BK, w.m0);
                    tma_load_2d(st + P::kA, m + 2, &full[s], kb * BK, w.n0);
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
            for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x, ++lt) {
                const int slot = lt & 1;
                const uint32_t use = lt >> 1;
                const int kblocks = (insts[items[t].inst].n + BK - 1) / BK;
                if (!mbar_wait(&tempty[slot], (use & 1u) ^ 1u, abort_flag, err)) break;
                tc_fence_after();
                const uint32_t acc = tmem + slot * 256;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&full[s], ph, abort_flag, err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a = smem_u32(tiles + s * P::kStage);
                    const uint32_t b = a + P::kA;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(acc, desc_sw128(a + kk * 32), desc_sw128(b + kk * 32), idesc,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[slot]);
            }
        }
    } else {
        const int ew = warp - 2;
        const int q = warp & 3;
        const int part = ew >> 2;
        const bool leader = (ew & 3) == 0 && lane == 0;
        constexpr int kMaxChunks = BN / kStgRows;   // 16-particle chunks of an item
        const int cl = q * 32 + lane;
        uint8_t *stg = tiles + P::kStgOff + part * 2 * P::kStgBuf;
        uint64_t *zf = zfull + part * 2;
        uint64_t *zd = zdone + part * 2;
        // An item's chunks that hold particles go round-robin to the four
        // groups of epilogue warps, starting at a group that rotates with the
        // item (chunk j of item t to group (j - t) mod 4), so that items of
        // small filters keep every group busy over consecutive items.
        auto group_slot = [&](int t) -> int { return (part + t) & 3; };  // this group's first chunk of item t
        auto chunks_of = [&](int t) -> int {
            const BWxItem w = items[t];
            const int live = min(kMaxChunks, (insts[w.inst].n - w.n0 + kStgRows - 1) / kStgRows);
            const int g0 = group_slot(t);
            return live > g0 ? (live - g0 - 1) / 4 + 1 : 0;
        };
        // the cursor of this group's next chunk to load: item nt, local chunk nc
        int nt = blockIdx.x, nc = 0;
        auto skip_empty = [&]() {
            while (nt < n_items && nc >= chunks_of(nt)) {
                nt += gridDim.x;
                nc = 0;
            }
        };
        int loads = 0;  // chunks this group has loaded (the buffer and phase of a load)
        auto issue_next = [&]() {
            skip_empty();
            if (nt >= n_items) return;
            const BWxItem w = items[nt];
            const int y = w.n0 + (group_slot(nt) + 4 * nc) * kStgRows;
            uint64_t *bar = &zf[loads & 1];
            mbar_expect_tx(bar, P::kStgZ);
            tma_load_2d(smem_u32(stg + (loads & 1) * P::kStgBuf), maps + 8 * w.inst + 4, bar, w.m0, y);
            ++loads;
            ++nc;
        };
        if (leader) issue_next();
        int g = 0, lt = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < n_items && ok; t += gridDim.x, ++lt) {
            const int slot = lt & 1;
            const uint32_t use = lt >> 1;
            const BWxItem w = items[t];
            const BInst &I = insts[w.inst];
            const CUtensorMap *m = maps + 8 * w.inst;
            if (!__all_sync(0xffffffffu, mbar_wait(&tfull[slot], use & 1u, abort_flag, err))) break;
            tc_fence_after();
            const int64_t c = static_cast<int64_t>(w.m0) + cl;
            const bool cok = c < I.d;
            const float yc = cok ? I.y[c] : 0.f;
            const bool obs = cok && (I.mask == nullptr || I.mask[c] != 0);
            const float shift = cok ? __fmul_rn(alpha_next, I.centre[c]) : 0.f;
            const bool lo_plane = I.zb_lo != nullptr;
            const int mine = chunks_of(t);
#pragma unroll 1
            for (int ch = 0; ch < mine; ++ch, ++g) {
                const int buf = g & 1;
                if (leader) {
                    bulk_wait_read_all();  // the store of this group's previous chunk has left that buffer
                    issue_next();
                }
                const int cc = (group_slot(t) + 4 * ch) * kStgRows;  // accumulator column = particle within the item
                float u[16];
                tmem_ld16(tmem + slot * 256 + (static_cast<uint32_t>(q * 32) << 16) + cc, u);
                if (!__all_sync(0xffffffffu, mbar_wait(&zf[buf], (g >> 1) & 1u, abort_flag, err))) {
                    ok = false;
                    break;
                }
                float *zs = reinterpret_cast<float *>(stg + buf * P::kStgBuf);
                __nv_bfloat16 *hs = reinterpret_cast<__nv_bfloat16 *>(stg + buf * P::kStgBuf + P::kStgZ);
                __nv_bfloat16 *ls = hs + kStgRows * kStgCols;
                const int i0 = w.n0 + cc;
                float xi[16];
#pragma unroll
                for (int e4 = 0; e4 < 4; ++e4) {
                    const float4 v = noise4(I.seed, I.offset, cf.k + 1, c, (i0 >> 2) + e4);
                    xi[e4 * 4 + 0] = v.x;
                    xi[e4 * 4 + 1] = v.y;
                    xi[e4 * 4 + 2] = v.z;
                    xi[e4 * 4 + 3] = v.w;
                }
                // the element loop specialised on the item's operator and planes
                if (I.obs_op == 1) {
                    if (lo_plane)
                        staged_chunk_update<1, true>(zs, hs, ls, cl, u, xi, obs, yc, I.inv_r, cf, shift);
                    else
                        staged_chunk_update<1, false>(zs, hs, ls, cl, u, xi, obs, yc, I.inv_r, cf, shift);
                } else {
                    if (lo_plane)
                        staged_chunk_update<0, true>(zs, hs, ls, cl, u, xi, obs, yc, I.inv_r, cf, shift);
                    else
                        staged_chunk_update<0, false>(zs, hs, ls, cl, u, xi, obs, yc, I.inv_r, cf, shift);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&zd[buf]);
                if (leader) {
                    if (!mbar_wait(&zd[buf], (g >> 1) & 1u, abort_flag, err)) {
                        ok = false;
                    } else {
                        tma_store_2d(m + 4, smem_u32(zs), w.m0, i0);
                        tma_store_2d(m + 5, smem_u32(hs), w.m0, i0);
                        if (lo_plane) tma_store_2d(m + 6, smem_u32(ls), w.m0, i0);
                        bulk_commit();
                    }
                }
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[slot]);
        }
        if (leader) bulk_wait_all();
        (void)ok;
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
    // launch shapes picked by tc_autotune, keyed by problem shape
    std::mutex mu;
    std::map<std::tuple<int, int, int64_t, bool>, GramChoice> gram_tuned;  // (n, n_x, d, split3)
    std::map<std::tuple<int, int64_t, bool>, int> wx_tuned;                 // (n, d, split) -> BN
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

PFN_cuTensorMapEncodeTiled_v12000 tc_encoder(TcContext *ctx) { return ctx ? ctx->encode : nullptr; }

int64_t tc_partial_floats(int max_n, int /*sms*/) {
    const int64_t sq = static_cast<int64_t>(max_n) * max_n;
    return std::min<int64_t>(64 * sq, std::max<int64_t>(int64_t(32) << 20, sq));
}

namespace {

// 2-D BF16 tensor map: rows x cols (cols contiguous), row pitch `pitch`
// elements, box = box_cols columns x box_rows rows, zero fill; 64-column
// boxes use the 128-byte swizzle, 32-column boxes the 64-byte swizzle.
cudaError_t make_map(const TcContext *ctx, CUtensorMap *m, const void *base, int64_t cols, int64_t rows,
                     int64_t pitch, int box_rows, int box_cols = BK) {
    if (!base) {  // an unused plane: point at nothing valid but keep the map well formed
        memset(m, 0, sizeof(*m));
        return cudaSuccess;
    }
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch) * 2};
    if (box_cols != 64 && box_cols != 32) return cudaErrorInvalidValue;
    cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ctx->encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D FP32 tensor map rows x cols (cols contiguous, pitch = cols), box of 32
// columns (128 bytes) x box_rows rows with the 128-byte swizzle, zero fill.
cudaError_t make_map_f32(const TcContext *ctx, CUtensorMap *m, const float *base, int64_t cols, int64_t rows,
                         int box_rows) {
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * 4};
    cuuint32_t box[2] = {32u, static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ctx->encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D tensor map without swizzle for the staged W X epilogue: rows x cols of
// `esize`-byte elements (cols contiguous, pitch = cols), box = kStgCols
// columns x kStgRows rows, zero fill beyond the edges (loads) and clipping
// (stores).
cudaError_t make_map_stage(const TcContext *ctx, CUtensorMap *m, const void *base, int esize, int64_t cols,
                           int64_t rows) {
    if (!base) {
        memset(m, 0, sizeof(*m));
        return cudaSuccess;
    }
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * esize};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kStgCols), static_cast<cuuint32_t>(kStgRows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ctx->encode(m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                             const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int STAGES, bool SPLIT, int KB = BK, int ES = 2>
cudaError_t run_gram(const CUtensorMap (&maps)[4], const GramParams &p, dim3 grid, cudaStream_t s) {
    using P = Plan<BN, STAGES, SPLIT, KB, ES>;
    auto kern = k_gram_tc<BN, STAGES, SPLIT, KB, ES>;
    cudaError_t e = set_smem(kern, P::kBytes);
    if (e != cudaSuccess) return e;
    return launch_k(kern, grid, dim3(kGramThreads), P::kBytes, s, p.pdl, maps[0], maps[1], maps[2], maps[3], p);
}

cudaError_t run_gram_pair_f32(const CUtensorMap (&maps)[4], const GramParams &p, dim3 grid, cudaStream_t s) {
    cudaError_t e = set_smem(k_gram_tc_pair_f32, PairF32Plan::kBytes);
    if (e != cudaSuccess) return e;
    return launch_k(k_gram_tc_pair_f32, grid, dim3(kPairF32Threads), PairF32Plan::kBytes, s, p.pdl, maps[0],
                    maps[1], maps[2], maps[3], p);
}

template <bool TF32>
cudaError_t run_gram_pair(const CUtensorMap (&maps)[4], const GramParams &p, dim3 grid, cudaStream_t s) {
    using P = PairPlan<TF32>;
    cudaError_t e = set_smem(k_gram_tc_pair<TF32>, P::kBytes);
    if (e != cudaSuccess) return e;
    return launch_k(k_gram_tc_pair<TF32>, grid, dim3(kGramThreads), P::kBytes, s, p.pdl, maps[0], maps[1],
                    maps[2], maps[3], p);
}

template <int BN, int STAGES, bool SPLIT, bool INLINE_NOISE>
cudaError_t run_wx(const CUtensorMap (&maps)[4], WxParams p, int sms, cudaStream_t s) {
    using P = WxPlan<BN, STAGES, SPLIT>;
    auto kern = k_wx_em_tc<BN, STAGES, SPLIT, INLINE_NOISE>;
    cudaError_t e = set_smem(kern, P::kBytes);
    if (e != cudaSuccess) return e;
    p.n_tiles = (p.n + BN - 1) / BN;
    const int total = p.m_tiles * p.n_tiles;
    const int grid = total < sms ? total : sms;
    return launch_k(kern, dim3(grid), dim3(kWxThreads), P::kBytes, s, p.pdl, maps[0], maps[1], maps[2], maps[3], p);
}

template <int BN, int STAGES, int OBS, int PLANES>
cudaError_t run_wx_staged(const CUtensorMap &xt, const CUtensorMap &w, const CUtensorMap (&stg)[3], WxParams p,
                          int sms, cudaStream_t s) {
    using P = WxStagedPlan<BN, STAGES>;
    auto kern = k_wx_em_staged<BN, STAGES, OBS, PLANES>;
    cudaError_t e = set_smem(kern, P::kBytes);
    if (e != cudaSuccess) return e;
    p.n_tiles = (p.n + BN - 1) / BN;
    const int total = p.m_tiles * p.n_tiles;
    const int grid = total < sms ? total : sms;
    return launch_k(kern, dim3(grid), dim3(kWxThreads), P::kBytes, s, p.pdl, xt, w, stg[0], stg[1], stg[2], p);
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

namespace {

GramChoice default_gram_choice(const TcGramArgs &a) {
    GramChoice g;
    g.bn = a.n_x <= 128 ? 128 : 256;
    g.stages = a.split3 ? (g.bn == 256 ? 2 : 3) : (g.bn == 256 ? 4 : 6);
    g.splits = 0;  // cost model
    return g;
}

// The fused-softmax fields of a launch: used when the caller supplied the
// scratch, the tuning asks for it and the launch runs pair tiles.
void set_fused_softmax(GramParams &p, const TcGramArgs &a, const GramChoice &ch, bool pair, int S) {
    const bool on = a.sm_L && ch.fused_softmax && pair;
    p.splits = S;
    p.sm_L = on ? static_cast<DF *>(a.sm_L) : nullptr;
    p.sm_stats = a.sm_stats;
    p.sm_cnt = a.sm_cnt;
    p.sm_norms = a.sm_norms;
    p.sm_alpha = a.sm_alpha;
    p.sm_inv_2beta2 = a.sm_inv_2beta2;
    p.sm_w = a.sm_w;
    p.sm_ldw = a.sm_ldw;
    p.sm_w_hi = a.sm_w_hi;
    p.sm_w_lo = a.sm_w_lo;
    p.sm_ldwb = a.sm_ldwb;
    if (a.sm_done) *a.sm_done = on;
}

// Split-K plan of a Gram launch with shape choice ch: the k-block width, the
// k-blocks per split and the number of splits that hold work (returned).
int gram_split_plan(const TcGramArgs &a, const GramChoice &ch, int sms, int *kblocks, int *kb_per_split) {
    int KB, BN;
    if (a.tf32) {
        const bool pair = ch.pair && a.n % kPairTile == 0 && a.n_x % kPairTile == 0;
        KB = 32;
        BN = (pair || ch.bn != 128) ? 256 : 128;
    } else {
        const bool pair = ch.pair && a.split3 && a.n % kPairTile == 0 && a.n_x % kPairTile == 0;
        BN = pair ? kPairTile : ch.bn;
        KB = pair ? BK : (ch.bk == 32 ? 32 : BK);
    }
    const int mt = (a.n + BM - 1) / BM, nt = (a.n_x + BN - 1) / BN;
    const int kb = static_cast<int>((a.d + KB - 1) / KB);
    const int64_t per_split = static_cast<int64_t>(a.n) * a.n_x;
    int S = ch.splits > 0 ? ch.splits : choose_splits(mt * nt, kb, sms, per_split, a.partial_cap);
    S = std::max(1, std::min<int>(S, static_cast<int>(std::min<int64_t>(kb, a.partial_cap / per_split))));
    const int kbps = (kb + S - 1) / S;
    *kblocks = kb;
    *kb_per_split = kbps;
    return (kb + kbps - 1) / kbps;  // splits that hold work
}

cudaError_t gram_launch_tf32(TcContext *ctx, const TcGramArgs &a, int sms, const GramChoice &ch, int *splits,
                             int64_t *part_stride, int *ldp, cudaStream_t s) {
    constexpr int KB = 32;  // 32 FP32 = one 128-byte swizzle row
    // the pair form needs whole 256-row tiles on both sides
    const bool pair = ch.pair && a.n % kPairTile == 0 && a.n_x % kPairTile == 0;
    const int BN = (pair || ch.bn != 128) ? 256 : 128;
    CUtensorMap maps[4];
    cudaError_t e;
    if ((e = make_map_f32(ctx, &maps[0], a.zc32, a.d, a.n, BM)) != cudaSuccess) return e;
    if ((e = make_map_f32(ctx, &maps[2], a.xc32, a.d, a.n_x, pair ? 128 : BN)) != cudaSuccess) return e;
    memset(&maps[1], 0, sizeof(maps[1]));
    memset(&maps[3], 0, sizeof(maps[3]));
    const int mt = (a.n + BM - 1) / BM, nt = (a.n_x + BN - 1) / BN;
    GramParams p;
    p.n = a.n;
    p.n_x = a.n_x;
    const int64_t per_split = static_cast<int64_t>(a.n) * a.n_x;
    int S = gram_split_plan(a, ch, sms, &p.kblocks, &p.kb_per_split);
    p.partial = a.partial;
    p.err = a.err;
    p.noise = a.noise;
    p.seed = a.seed;
    p.offset = a.offset;
    p.noise_k = a.noise_k;
    p.noise_col0 = a.noise_col0;
    p.pdl = a.pdl;
    p.d = a.d;
    p.noise_warp0 = ch.noise_warps == 4 ? 6 : 2;
    p.alpha = 0.f;
    p.centre = nullptr;
    set_fused_softmax(p, a, ch, pair, S);
    *splits = S;
    *part_stride = per_split;
    *ldp = a.n_x;
    dim3 grid(mt, nt, S);
    if (pair) return run_gram_pair<true>(maps, p, grid, s);  // mt = 2 x pair tiles: one CTA per 128 rows
    if (BN == 256) return run_gram<256, 4, false, KB, 4>(maps, p, grid, s);
    return run_gram<128, 6, false, KB, 4>(maps, p, grid, s);
}

cudaError_t gram_launch(TcContext *ctx, const TcGramArgs &a, int sms, const GramChoice &ch, int *splits,
                        int64_t *part_stride, int *ldp, cudaStream_t s) {
    if (a.tf32) return gram_launch_tf32(ctx, a, sms, ch, splits, part_stride, ldp, s);
    // the pair Gram needs whole 256-row tiles on both sides (no tile of a CTA
    // lies entirely outside the operands)
    const bool pair = ch.pair && a.split3 && a.n % kPairTile == 0 && a.n_x % kPairTile == 0;
    const bool f32a = pair && ch.a_fp32 && a.z32 != nullptr;
    const int BN = pair ? kPairTile : ch.bn;
    const int KB = pair ? BK : (ch.bk == 32 ? 32 : BK);
    const int box_a = BM, box_b = pair ? 128 : BN;
    CUtensorMap maps[4];
    cudaError_t e;
    if (f32a) {
        if ((e = make_map_f32(ctx, &maps[0], a.z32, a.d, a.n, BM)) != cudaSuccess) return e;
        memset(&maps[1], 0, sizeof(maps[1]));
    } else {
        if ((e = make_map(ctx, &maps[0], a.zb_hi, a.d, a.n, a.d, BM, KB)) != cudaSuccess) return e;
        if ((e = make_map(ctx, &maps[1], a.split3 ? a.zb_lo : nullptr, a.d, a.n, a.d, BM, KB)) != cudaSuccess)
            return e;
    }
    if ((e = make_map(ctx, &maps[2], a.xb_hi, a.d, a.n_x, a.d, box_b, KB)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[3], a.split3 ? a.xb_lo : nullptr, a.d, a.n_x, a.d, box_b, KB)) != cudaSuccess) return e;
    (void)box_a;
    // output tiles counted in single-CTA units (a pair covers two)
    const int mt = (a.n + BM - 1) / BM, nt = (a.n_x + BN - 1) / BN;
    GramParams p;
    p.n = a.n;
    p.n_x = a.n_x;
    const int64_t per_split = static_cast<int64_t>(a.n) * a.n_x;
    int S = gram_split_plan(a, ch, sms, &p.kblocks, &p.kb_per_split);
    p.partial = a.partial;
    p.err = a.err;
    p.noise = a.noise;
    p.seed = a.seed;
    p.offset = a.offset;
    p.noise_k = a.noise_k;
    p.noise_col0 = a.noise_col0;
    p.pdl = a.pdl;
    p.d = a.d;
    // the FP32 form's warps 2-9 split A and warps 10-15 generate the noise
    p.noise_warp0 = f32a ? 2 + kPairF32Convert : (ch.noise_warps == 4 ? 6 : 2);
    p.alpha = a.alpha;
    p.centre = a.centre;
    set_fused_softmax(p, a, ch, pair && !f32a, S);
    *splits = S;
    *part_stride = per_split;
    *ldp = a.n_x;
    dim3 grid(mt, nt, S);
    if (f32a) return run_gram_pair_f32(maps, p, grid, s);
    if (pair) return run_gram_pair<false>(maps, p, grid, s);  // mt = 2 x pair tiles: one CTA per 128 rows
    if (KB == 32) {  // narrow k-blocks: twice the ring depth for the same bytes in flight
        if (a.split3) {
            if (BN == 256) return ch.stages == 3 ? run_gram<256, 3, true, 32>(maps, p, grid, s)
                                                 : run_gram<256, 4, true, 32>(maps, p, grid, s);
            return run_gram<128, 6, true, 32>(maps, p, grid, s);
        }
        if (BN == 256) return run_gram<256, 8, false, 32>(maps, p, grid, s);
        return run_gram<128, 12, false, 32>(maps, p, grid, s);
    }
    if (a.split3) {
        if (BN == 256) return run_gram<256, 2, true>(maps, p, grid, s);
        return run_gram<128, 3, true>(maps, p, grid, s);
    }
    if (BN == 256) return run_gram<256, 4, false>(maps, p, grid, s);
    return run_gram<128, 6, false>(maps, p, grid, s);
}

}  // namespace

cudaError_t launch_gram_tc(TcContext *ctx, const TcGramArgs &a, int sms, int *splits, int64_t *part_stride, int *ldp,
                           cudaStream_t s) {
    if (!ctx) return cudaErrorInvalidValue;
    GramChoice ch = default_gram_choice(a);
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        auto it = ctx->gram_tuned.find(std::make_tuple(a.n, a.n_x, a.d, a.split3));
        if (it != ctx->gram_tuned.end()) ch = it->second;
    }
    return gram_launch(ctx, a, sms, ch, splits, part_stride, ldp, s);
}

cudaError_t tc_encode_stage_map(TcContext *ctx, void *out128, const void *base, int esize, int64_t cols,
                                int64_t rows) {
    return make_map_stage(ctx, static_cast<CUtensorMap *>(out128), base, esize, cols, rows);
}

int tc_gram_split_count(TcContext *ctx, const TcGramArgs &a, int sms) {
    if (!ctx) return 0;
    GramChoice ch = default_gram_choice(a);
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        auto it = ctx->gram_tuned.find(std::make_tuple(a.n, a.n_x, a.d, a.split3));
        if (it != ctx->gram_tuned.end()) ch = it->second;
    }
    int kb = 0, kbps = 0;
    return gram_split_plan(a, ch, sms, &kb, &kbps);
}

cudaError_t launch_wx_em_tc(TcContext *ctx, const TcWxArgs &a, int sms, cudaStream_t s) {
    if (!ctx) return cudaErrorInvalidValue;
    const bool split = a.wb_lo != nullptr && a.xt_lo != nullptr;
    int BN = a.n <= 64 ? 64 : (a.n <= 128 ? 128 : 256);
    if (a.force_bn) {
        BN = a.force_bn;
    } else {
        std::lock_guard<std::mutex> lock(ctx->mu);
        auto it = ctx->wx_tuned.find(std::make_tuple(a.n, a.d, split));
        if (it != ctx->wx_tuned.end()) BN = it->second;
    }
    if (BN != 64 && BN != 128 && BN != 256) return cudaErrorInvalidValue;
    // A = X^T [d][ldw] (state columns; K = n_x members), B = W [n][ldwb] (particles)
    const int n_x = a.n_x > 0 ? a.n_x : a.n;
    const int ldwb = a.ldwb > 0 ? a.ldwb : a.ldw;
    CUtensorMap maps[4];
    cudaError_t e;
    if ((e = make_map(ctx, &maps[0], a.xt_hi, n_x, a.d, a.ldw, BM)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[1], split ? a.xt_lo : nullptr, n_x, a.d, a.ldw, BM)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[2], a.wb_hi, n_x, a.n, ldwb, BN)) != cudaSuccess) return e;
    if ((e = make_map(ctx, &maps[3], split ? a.wb_lo : nullptr, n_x, a.n, ldwb, BN)) != cudaSuccess) return e;
    WxParams p;
    p.n = a.n;
    p.d = a.d;
    p.kblocks = (n_x + BK - 1) / BK;
    p.m_tiles = static_cast<int>((a.d + BM - 1) / BM);
    p.n_tiles = 0;
    p.z = a.z;
    p.zb_hi = a.zb_hi;
    p.zc32 = a.zc32;
    p.zb_lo = a.zb_lo;
    p.y = a.y;
    p.mask = a.mask;
    p.noise = a.noise;
    p.seed = a.seed;
    p.offset = a.offset;
    p.centre = a.centre;
    p.alpha_next = a.alpha_next;
    p.coef = a.coef;
    p.err = a.err;
    p.pdl = a.pdl;
    const bool inl = a.noise == nullptr;  // no slice: Philox in the epilogue
    if (!split && inl && a.zc32 == nullptr && a.staged) {
        // in-epilogue noise with BF16 W X: the TMA-staged epilogue
        CUtensorMap stg[3];
        if ((e = make_map_stage(ctx, &stg[0], a.z, 4, a.d, a.n)) != cudaSuccess) return e;
        if ((e = make_map_stage(ctx, &stg[1], a.zb_hi, 2, a.d, a.n)) != cudaSuccess) return e;
        if ((e = make_map_stage(ctx, &stg[2], a.zb_lo, 2, a.d, a.n)) != cudaSuccess) return e;
        const int planes = a.zb_hi ? (a.zb_lo ? 2 : 1) : 0;
        const int sel = (BN == 256 ? 0 : BN == 128 ? 1 : 2) * 6 + a.coef.obs_op * 3 + planes;
        switch (sel) {
#define ENSF_STAGED(bn, st, i)                                                                   \
    case i * 6 + 0: return run_wx_staged<bn, st, 0, 0>(maps[0], maps[2], stg, p, sms, s);        \
    case i * 6 + 1: return run_wx_staged<bn, st, 0, 1>(maps[0], maps[2], stg, p, sms, s);        \
    case i * 6 + 2: return run_wx_staged<bn, st, 0, 2>(maps[0], maps[2], stg, p, sms, s);        \
    case i * 6 + 3: return run_wx_staged<bn, st, 1, 0>(maps[0], maps[2], stg, p, sms, s);        \
    case i * 6 + 4: return run_wx_staged<bn, st, 1, 1>(maps[0], maps[2], stg, p, sms, s);        \
    case i * 6 + 5: return run_wx_staged<bn, st, 1, 2>(maps[0], maps[2], stg, p, sms, s);
            ENSF_STAGED(256, 2, 0)
            ENSF_STAGED(128, 3, 1)
            ENSF_STAGED(64, 4, 2)
#undef ENSF_STAGED
            default: return cudaErrorInvalidValue;
        }
    }
    if (split) {
        if (BN == 256) return inl ? run_wx<256, 2, true, true>(maps, p, sms, s) : run_wx<256, 2, true, false>(maps, p, sms, s);
        if (BN == 128) return inl ? run_wx<128, 3, true, true>(maps, p, sms, s) : run_wx<128, 3, true, false>(maps, p, sms, s);
        return inl ? run_wx<64, 4, true, true>(maps, p, sms, s) : run_wx<64, 4, true, false>(maps, p, sms, s);
    }
    if (BN == 256) return inl ? run_wx<256, 4, false, true>(maps, p, sms, s) : run_wx<256, 4, false, false>(maps, p, sms, s);
    if (BN == 128) return inl ? run_wx<128, 6, false, true>(maps, p, sms, s) : run_wx<128, 6, false, false>(maps, p, sms, s);
    return inl ? run_wx<64, 8, false, true>(maps, p, sms, s) : run_wx<64, 8, false, false>(maps, p, sms, s);
}

cudaError_t tc_set_tuning(TcContext *ctx, int n, int n_x, int64_t d, bool split3, const GramChoice &g, int wx_bn,
                          bool wx_split, bool tf32) {
    if (!ctx) return cudaErrorInvalidValue;
    const int bk = g.bk ? g.bk : BK;
    bool ok;
    if (tf32)
        ok = (bk == 32 || g.bk == 0) &&
             (g.pair ? (g.bn == kPairTile && g.stages == kPairStagesTf32 && n % kPairTile == 0 &&
                        n_x % kPairTile == 0 && !g.a_fp32)
                     : ((g.bn == 128 && g.stages == 6) || (g.bn == 256 && g.stages == 4)));
    else if (g.pair)
        ok = split3 && g.bn == kPairTile && g.stages == kPairStages && bk == BK && n % kPairTile == 0 &&
             n_x % kPairTile == 0;
    else if (split3)
        ok = (bk == 64 && ((g.bn == 128 && g.stages == 3) || (g.bn == 256 && g.stages == 2))) ||
             (bk == 32 && ((g.bn == 128 && g.stages == 6) || (g.bn == 256 && (g.stages == 4 || g.stages == 3))));
    else
        ok = (bk == 64 && ((g.bn == 128 && g.stages == 6) || (g.bn == 256 && g.stages == 4))) ||
             (bk == 32 && ((g.bn == 128 && g.stages == 12) || (g.bn == 256 && g.stages == 8)));
    if (!ok || g.splits < 0 || (wx_bn != 0 && wx_bn != 64 && wx_bn != 128 && wx_bn != 256))
        return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (g.noise_warps != 0 && g.noise_warps != 4 && g.noise_warps != 8) return cudaErrorInvalidValue;
    if (g.a_fp32 && !g.pair) return cudaErrorInvalidValue;
    if (g.fused_softmax && (!g.pair || g.a_fp32)) return cudaErrorInvalidValue;
    GramChoice c = g;
    c.bk = tf32 ? 32 : bk;
    ctx->gram_tuned[std::make_tuple(n, n_x, d, split3)] = c;
    if (wx_bn) ctx->wx_tuned[std::make_tuple(n, d, wx_split)] = wx_bn;
    return cudaSuccess;
}

bool tc_gram_reads_fp32(TcContext *ctx, int n, int n_x, int64_t d, bool split3) {
    if (!ctx || !split3 || n % kPairTile != 0 || n_x % kPairTile != 0) return false;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->gram_tuned.find(std::make_tuple(n, n_x, d, split3));
    return it != ctx->gram_tuned.end() && it->second.pair && it->second.a_fp32;
}

namespace {
// One thread waits on an mbarrier that nothing completes, through the same
// bounded wait as every pipeline wait of the tensor-core kernels.
__global__ void k_selftest_mbar_wait(int *err) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, &abort_flag, err)) return;  // records ENSF_ETIMEOUT after kTimeoutNs
    atomicExch(err, -1);                                 // unreachable: the phase cannot complete
}
}  // namespace

cudaError_t launch_selftest_mbar_wait(int *err, cudaStream_t s) {
    k_selftest_mbar_wait<<<1, 1, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t tc_encode_map(TcContext *ctx, void *out128, const void *base, int64_t cols, int64_t rows, int64_t pitch,
                          int box_rows) {
    if (!ctx) return cudaErrorInvalidValue;
    return make_map(ctx, static_cast<CUtensorMap *>(out128), base, cols, rows, pitch, box_rows);
}

cudaError_t launch_gram_tc_batched(const void *maps, const BGramItem *items, int n_items, const BInst *insts,
                                   bool split3, int *err, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const CUtensorMap *m = static_cast<const CUtensorMap *>(maps);
    if (split3) {
        using P = Plan<kBatchTileN, 3, true>;
        auto kern = k_gram_tc_batched<kBatchTileN, 3, true>;
        cudaError_t e = set_smem(kern, P::kBytes);
        if (e != cudaSuccess) return e;
        kern<<<n_items, 192, P::kBytes, s>>>(m, items, insts, err);
    } else {
        using P = Plan<kBatchTileN, 6, false>;
        auto kern = k_gram_tc_batched<kBatchTileN, 6, false>;
        cudaError_t e = set_smem(kern, P::kBytes);
        if (e != cudaSuccess) return e;
        kern<<<n_items, 192, P::kBytes, s>>>(m, items, insts, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_softmax_batched(const BRow *rows, int n_rows, const BInst *insts, int max_n, double alpha,
                                   double inv_2beta2, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const size_t smem = sizeof(double) * static_cast<size_t>(max_n);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_softmax_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_softmax_batched<<<n_rows, 256, smem, s>>>(rows, insts, alpha, inv_2beta2);
    return cudaGetLastError();
}

cudaError_t launch_wx_em_tc_batched(const void *maps, const BWxItem *items, int n_items, const BInst *insts,
                                    bool split, const StepCoef &cf, float alpha_next, int *err, int sms,
                                    cudaStream_t s, bool staged) {
    if (n_items <= 0) return cudaSuccess;
    const CUtensorMap *m = static_cast<const CUtensorMap *>(maps);
    const int grid = n_items < sms ? n_items : sms;
    if (staged && !split) {
        using P = WxStagedPlan<kBatchTileN, 3>;
        cudaError_t e = set_smem(k_wx_em_staged_batched, P::kBytes);
        if (e != cudaSuccess) return e;
        k_wx_em_staged_batched<<<grid, kWxThreads, P::kBytes, s>>>(m, items, n_items, insts, cf, alpha_next, err);
        return cudaGetLastError();
    }
    if (split) {
        using P = WxPlan<kBatchTileN, 3, true>;
        auto kern = k_wx_em_tc_batched<kBatchTileN, 3, true>;
        cudaError_t e = set_smem(kern, P::kBytes);
        if (e != cudaSuccess) return e;
        kern<<<grid, kWxThreads, P::kBytes, s>>>(m, items, n_items, insts, cf, alpha_next, err);
    } else {
        using P = WxPlan<kBatchTileN, 6, false>;
        auto kern = k_wx_em_tc_batched<kBatchTileN, 6, false>;
        cudaError_t e = set_smem(kern, P::kBytes);
        if (e != cudaSuccess) return e;
        kern<<<grid, kWxThreads, P::kBytes, s>>>(m, items, n_items, insts, cf, alpha_next, err);
    }
    return cudaGetLastError();
}

// Time `launch` (reps launches after one warm-up) with events on stream s; ms per launch.
template <class F>
static cudaError_t time_launches(F launch, int reps, cudaStream_t s, float *ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e == cudaSuccess) *ms /= reps;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

cudaError_t tc_autotune(TcContext *ctx, const TcGramArgs *g, const TcWxArgs *w, int sms, cudaStream_t s,
                        TcTuneReport *rep, AfterGram after_gram, void *after_ctx) {
    if (!ctx) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    float wx_saving = 0.f;
    if (w) {
        const bool split = w->wb_lo != nullptr && w->xt_lo != nullptr;
        int best_bn = 0;
        float best_ms = 1e30f;
        for (int bn : {64, 128, 256}) {
            TcWxArgs a = *w;
            a.force_bn = bn;
            float ms = 0.f;
            e = time_launches([&] { return launch_wx_em_tc(ctx, a, sms, s); }, 3, s, &ms);
            if (e != cudaSuccess) return e;
            if (ms < best_ms) {
                best_ms = ms;
                best_bn = bn;
            }
        }
        {
            std::lock_guard<std::mutex> lock(ctx->mu);
            ctx->wx_tuned[std::make_tuple(w->n, w->d, split)] = best_bn;
        }
        if (rep) {
            rep->wx_bn = best_bn;
            rep->wx_ms = best_ms;
        }
        // what W X saves when it need not write the BF16 particle planes (the
        // Gram form that splits the FP32 particles itself)
        if (w->zb_hi) {
            TcWxArgs a = *w;  // without the planes
            a.force_bn = best_bn;
            a.zb_hi = a.zb_lo = nullptr;
            TcWxArgs b = *w;  // with them
            b.force_bn = best_bn;
            float with = 0.f, without = 0.f;
            for (int pass = 0; pass < 2; ++pass) {
                float t1 = 0.f, t2 = 0.f;
                if ((e = time_launches([&] { return launch_wx_em_tc(ctx, b, sms, s); }, 5, s, &t1)) != cudaSuccess)
                    return e;
                if ((e = time_launches([&] { return launch_wx_em_tc(ctx, a, sms, s); }, 5, s, &t2)) != cudaSuccess)
                    return e;
                with = pass ? std::min(with, t1) : t1;
                without = pass ? std::min(without, t2) : t2;
            }
            wx_saving = std::max(0.f, with - without);
        }
    }

    if (g) {
        // One timed launch of the Gram (with the softmax that consumes its partials).
        auto time_choice = [&](const GramChoice &ch, int reps, float *ms, int *splits_out) {
            int splits = 0, ldp = 0;
            int64_t ps = 0;
            cudaError_t r = time_launches(
                [&] {
                    cudaError_t q = gram_launch(ctx, *g, sms, ch, &splits, &ps, &ldp, s);
                    if (q == cudaSuccess && after_gram) q = after_gram(after_ctx, splits, ps, ldp, s, false);
                    return q;
                },
                reps, s, ms);
            *splits_out = splits;
            return r;
        };
        // Round 1: (tile width, ring depth, k-block width, CTA pair) x split
        // counts around the cost model's choice, three launches each.
        struct Cand {
            GramChoice ch;
            float ms;
        };
        std::vector<Cand> cands;
        // (tile width, ring depth, k-block width, CTA pair, FP32 particle operand)
        const int shapes[][5] = {{128, 3, 64, 0, 0}, {256, 2, 64, 0, 0}, {256, 3, 64, 1, 0}, {256, 3, 64, 1, 1}};
        const int shapes_tf32[][5] = {{128, 6, 32, 0, 0}, {256, 4, 32, 0, 0}, {256, 6, 32, 1, 0}};
        const int n_shapes = g->tf32 ? 3 : 4;
        for (int si = 0; si < n_shapes; ++si) {
            const int *sh = g->tf32 ? shapes_tf32[si] : shapes[si];
            const int bn = sh[0], kbw = sh[2], pr = sh[3], f32 = sh[4];
            if (f32 && !(g->z32 && w && w->zb_hi)) continue;
            if (pr && !((g->split3 || g->tf32) && g->n % kPairTile == 0 && g->n_x % kPairTile == 0)) continue;
            if (bn == 256 && g->n_x <= 128) continue;
            const int stages = (g->split3 || g->tf32) ? sh[1] : (bn == 256 ? 4 : 6);
            const int mt = (g->n + BM - 1) / BM, nt = (g->n_x + bn - 1) / bn;
            const int kblocks = static_cast<int>((g->d + kbw - 1) / kbw);
            const int s0 = choose_splits(mt * nt, kblocks, sms, static_cast<int64_t>(g->n) * g->n_x, g->partial_cap);
            std::vector<int> sps = {s0, std::max(1, s0 / 2), s0 * 2, std::max(1, (s0 * 3) / 4), (s0 * 3) / 2,
                                    std::max(1, s0 / 4), std::max(1, s0 / 8)};
            // and the split counts whose CTAs fill whole waves of the SMs
            // (the grid is tiles x splits CTAs, one resident per SM)
            for (int w = 1; w <= 8; ++w) {
                const int sp = (w * sms) / (mt * nt);
                if (sp >= 1 && std::find(sps.begin(), sps.end(), sp) == sps.end()) sps.push_back(sp);
            }
            for (int sp : sps) {
                GramChoice ch{bn, stages, sp, kbw, pr};
                ch.a_fp32 = f32;
                float ms = 0.f;
                int splits = 0;
                if ((e = time_choice(ch, 3, &ms, &splits)) != cudaSuccess) return e;
                if (f32) ms -= wx_saving;  // credited with the W X planes it makes unnecessary
                ch.splits = splits;
                bool dup = false;
                for (const Cand &c : cands)
                    dup |= c.ch.bn == ch.bn && c.ch.pair == ch.pair && c.ch.splits == ch.splits &&
                           c.ch.a_fp32 == ch.a_fp32;
                if (!dup) cands.push_back({ch, ms});
            }
        }
        std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.ms < b.ms; });
        if (cands.size() > 4) cands.resize(4);
        if (g->noise && !cands.empty()) {  // noise shared by 8 warps, or left to the 4 noise-only warps
            Cand c = cands.front();
            c.ch.noise_warps = 4;
            cands.push_back(c);
        }
        // Round 2: the leaders again, ten launches each, in two interleaved
        // passes (best of the two), so that clock drift does not decide.
        for (Cand &c : cands) c.ms = 1e30f;
        for (int pass = 0; pass < 2; ++pass)
            for (Cand &c : cands) {
                float ms = 0.f;
                int splits = 0;
                if ((e = time_choice(c.ch, 10, &ms, &splits)) != cudaSuccess) return e;
                if (c.ch.a_fp32) ms -= wx_saving;
                c.ms = std::min(c.ms, ms);
            }
        GramChoice best = default_gram_choice(*g);
        float best_ms = 1e30f;
        for (const Cand &c : cands) best_ms = std::min(best_ms, c.ms);
        // within 1 % of the fastest (timing noise), the fewest split-K slices:
        // fewer partial Grams written, read by the softmax and held in L2
        float chosen_ms = 1e30f;
        int chosen_splits = 1 << 30;
        for (const Cand &c : cands)
            if (c.ms <= best_ms * 1.01f &&
                (c.ch.splits < chosen_splits || (c.ch.splits == chosen_splits && c.ms < chosen_ms))) {
                chosen_splits = c.ch.splits;
                chosen_ms = c.ms;
                best = c.ch;
            }
        best_ms = chosen_ms;
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->gram_tuned[std::make_tuple(g->n, g->n_x, g->d, g->split3)] = best;
        if (rep) {
            rep->gram_bn = best.bn;
            rep->gram_stages = best.stages;
            rep->gram_splits = best.splits;
            rep->gram_bk = best.bk ? best.bk : BK;
            rep->gram_pair = best.pair;
            rep->gram_noise_warps = best.a_fp32 ? 4 : (best.noise_warps ? best.noise_warps : 8);
            rep->gram_a_fp32 = best.a_fp32;
            rep->gram_ms = best_ms;
        }
    }
    if (g && w && after_gram) {
        // Whole steps (Gram + softmax + W X, three in a row) with the recorded
        // shapes, launched the ordinary way and with programmatic dependent
        // launch; two interleaved passes, best of each.
        float t[2] = {1e30f, 1e30f};
        for (int pass = 0; pass < 2; ++pass)
            for (int pdl = 0; pdl < 2; ++pdl) {
                TcGramArgs ga = *g;
                ga.pdl = pdl != 0;
                TcWxArgs wa = *w;
                wa.pdl = pdl != 0;
                wa.force_bn = 0;
                float ms = 0.f;
                e = time_launches(
                    [&] {
                        cudaError_t q = cudaSuccess;
                        for (int st = 0; st < 3 && q == cudaSuccess; ++st) {
                            int splits = 0, ldp = 0;
                            int64_t ps = 0;
                            q = launch_gram_tc(ctx, ga, sms, &splits, &ps, &ldp, s);
                            if (q == cudaSuccess) q = after_gram(after_ctx, splits, ps, ldp, s, pdl != 0);
                            if (q == cudaSuccess) q = launch_wx_em_tc(ctx, wa, sms, s);
                        }
                        return q;
                    },
                    5, s, &ms);
                if (e != cudaSuccess) return e;
                t[pdl] = std::min(t[pdl], ms / 3);
            }
        if (rep) {
            rep->pdl = t[1] < t[0] ? 1 : 0;
            rep->step_ms = std::min(t[0], t[1]);
        }
    }
    return cudaSuccess;
}

}  // namespace ensf
