// ensf_small.cu -- the whole analysis of a small filter in one cooperative launch.
//
// With N <= 128 members and an L2-resident state, the three kernels of an
// Euler-Maruyama step cost more in launch and ramp latency than in work
// (the 2 x 64 x 64 case: about 8 us per kernel around a microsecond of
// arithmetic).  Here one grid of one block per SM, co-resident by cooperative
// launch, runs all K steps of Sec. III-A.2 with three grid barriers per step:
//   A  Gram partials  P_b[i][j] = sum over this block's slice of the state of
//      (z_i - alpha m)(x_j - m)                                   (Eq. 12)
//   B  rows of the softmax of the logits (2 alpha G_ij - alpha^2 |x_j - m|^2)
//      / (2 beta^2), G = sum_b P_b in FP64 in a fixed order        (Eq. 14, 16)
//   C  u = W X on this block's columns, the posterior score and the
//      Euler-Maruyama update with the step's noise                 (Eq. 7, 15, 17)
// in FP32 on the CUDA cores (the comparator precision).  Data written by
// other blocks within the launch (particles, partials, weights) is read with
// L2-only loads, never from a possibly stale L1 line.  The barrier is an
// arrival counter and a generation word in the handle's error block; every
// wait is bounded by %globaltimer: on expiry a block records ENSF_ETIMEOUT
// and every block leaves at its next barrier.
#include <cmath>

#include "ensf_internal.h"

namespace ensf {
namespace {

constexpr int kSmallThreads = 256;
constexpr int kChunk = 32;                         // state columns per shared-memory chunk
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;
constexpr int kStatusTimeout = 5;                  // ENSF_ETIMEOUT

struct SmallArgs {
    const float *x;        // forecast ensemble [n][d]
    const double *norms;   // |x_j - m|^2 [n]
    const float *centre;   // m [d]
    float *z;              // particles [n][d], xi_0 on entry, the analysis on exit
    const float *y;
    const uint8_t *mask;
    const float *noise_buf;  // [K+1][n][d] or NULL: Philox
    uint64_t seed;
    uint32_t offset;
    float *partial;        // [gram_blocks][n][n]
    float *w;              // [n][n]
    int gram_blocks;
    int64_t gram_slice;    // state columns per Gram block (multiple of kChunk)
    int64_t col_slice;     // state columns per W X block (multiple of kChunk)
    int n;
    int64_t d;
    int K;
    double eps;
    float inv_r;
    int obs_op;
    unsigned *bar;         // [0] arrivals, [1] generation
    int *err;
};

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of all blocks.  False when the analysis must stop (an error
// was recorded, here or elsewhere).
__device__ bool grid_barrier(unsigned *bar, int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = now_ns();
            while (*gen == g) {
                if (*reinterpret_cast<volatile int *>(err) != 0) {
                    ok = 0;
                    break;
                }
                if (now_ns() - t0 > kBarrierTimeoutNs) {
                    atomicCAS(err, 0, kStatusTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*reinterpret_cast<volatile int *>(err) != 0) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// The step coefficients of Eq. 9 and Eq. 11 at t_k = 1 - k/K, computed in
// double with every operation rounded as the host computes them.
__device__ StepCoef step_coef_dev(int k, int K, double eps, float inv_r, int obs_op) {
    const double t = __dsub_rn(1.0, __ddiv_rn((double)k, (double)K));
    const double alpha = __dsub_rn(1.0, __dmul_rn(t, __dsub_rn(1.0, eps)));
    const double b = __ddiv_rn(-__dsub_rn(1.0, eps), alpha);
    const double beta2 = t;
    const double sigma2 = __dsub_rn(1.0, __dmul_rn(__dmul_rn(2.0, b), beta2));
    const double dt = __ddiv_rn(1.0, (double)K);
    StepCoef c;
    c.alpha = (float)alpha;
    c.inv_beta2 = (float)__ddiv_rn(1.0, beta2);
    c.b = (float)b;
    c.sigma2 = (float)sigma2;
    c.h = (float)__dsub_rn(1.0, t);
    c.dt = (float)dt;
    c.noise_scale = (float)__dsqrt_rn(__dmul_rn(sigma2, dt));
    c.inv_r = inv_r;
    c.alpha_d = alpha;
    c.inv_2beta2_d = __ddiv_rn(1.0, __dmul_rn(2.0, beta2));
    c.k = k;
    c.obs_op = obs_op;
    c.col0 = 0;
    return c;
}

__global__ void __launch_bounds__(kSmallThreads, 1) k_analysis_small(SmallArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double lg[128];
    __shared__ double red[256];
    const int tid = threadIdx.x;
    const int n = a.n;
    for (int k = 0; k < a.K; ++k) {
        const StepCoef c = step_coef_dev(k, a.K, a.eps, a.inv_r, a.obs_op);

        // ---- A: Gram partials over this block's slice ----
        if ((int)blockIdx.x < a.gram_blocks) {
            float *Zs = sm;                 // [kChunk][128]: column-major chunk of z - alpha m
            float *Xs = sm + kChunk * 128;  // [kChunk][128]: chunk of x - m
            const int ty = tid >> 4, tx = tid & 15;  // 8 x 8 register tile at rows 8 ty, columns 8 tx
            float acc[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
            const int64_t c0 = (int64_t)blockIdx.x * a.gram_slice;
            const int64_t c1 = c0 + a.gram_slice < a.d ? c0 + a.gram_slice : a.d;
            for (int64_t cc = c0; cc < c1; cc += kChunk) {
                for (int e = tid; e < kChunk * n; e += kSmallThreads) {
                    const int row = e / kChunk, col = e % kChunk;
                    const int64_t cg = cc + col;
                    float zv = 0.f, xv = 0.f;
                    if (cg < c1) {
                        const float m = a.centre[cg];
                        zv = __fsub_rn(__ldcg(a.z + (int64_t)row * a.d + cg), __fmul_rn(c.alpha, m));
                        xv = __fsub_rn(a.x[(int64_t)row * a.d + cg], m);
                    }
                    Zs[col * 128 + row] = zv;
                    Xs[col * 128 + row] = xv;
                }
                __syncthreads();
                if (ty * 8 < n && tx * 8 < n) {
#pragma unroll 4
                    for (int col = 0; col < kChunk; ++col) {
                        float zr[8], xr[8];
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            zr[r] = Zs[col * 128 + ty * 8 + r];
                            xr[r] = Xs[col * 128 + tx * 8 + r];
                        }
#pragma unroll
                        for (int r = 0; r < 8; ++r)
#pragma unroll
                            for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(zr[r], xr[q], acc[r][q]);
                    }
                }
                __syncthreads();
            }
            float *P = a.partial + (int64_t)blockIdx.x * n * n;
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = ty * 8 + r, j = tx * 8 + q;
                    if (i < n && j < n) P[i * n + j] = acc[r][q];
                }
        }
        if (!grid_barrier(a.bar, a.err)) return;

        // ---- B: softmax rows ----
        for (int i = blockIdx.x; i < n; i += gridDim.x) {
            softmax_row<256>(i, a.partial, a.gram_blocks, (int64_t)n * n, n, n, a.norms, c.alpha_d,
                             c.inv_2beta2_d, a.w, n, nullptr, nullptr, 0, lg, red);
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.err)) return;
        float *Ws = sm;  // [n][n], the weights in shared memory for phase C
        for (int e = tid; e < n * n; e += kSmallThreads) Ws[e] = __ldcg(a.w + e);

        // ---- C: u = W X, score and Euler-Maruyama update on this block's columns ----
        {
            float *Xc = sm + 128 * 128;      // [n][kChunk]
            const int tx = tid & 31, ty = tid >> 5;  // column tx of the chunk; particle quads ty, ty + 8, ...
            const int quads = (n + 3) / 4;
            const int64_t c0 = (int64_t)blockIdx.x * a.col_slice;
            const int64_t c1 = c0 + a.col_slice < a.d ? c0 + a.col_slice : a.d;
            const float *nb = a.noise_buf ? a.noise_buf + (size_t)(k + 1) * n * a.d : nullptr;
            for (int64_t cc = c0; cc < c1; cc += kChunk) {
                __syncthreads();
                for (int e = tid; e < n * kChunk; e += kSmallThreads) {
                    const int row = e / kChunk, col = e % kChunk;
                    const int64_t cg = cc + col;
                    Xc[row * kChunk + col] = cg < c1 ? a.x[(int64_t)row * a.d + cg] : 0.f;
                }
                __syncthreads();
                const int64_t cg = cc + tx;
                if (cg >= c1) continue;
                const float yc = a.y[cg];
                const bool obs = a.mask == nullptr || a.mask[cg] != 0;
                for (int qd = ty; qd < quads; qd += kSmallThreads / 32) {
                    // the quad's four particles: loads first (independent), then the arithmetic
                    float zv[4], xi[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int i = qd * 4 + r;
                        zv[r] = i < n ? __ldcg(a.z + (int64_t)i * a.d + cg) : 0.f;
                        xi[r] = (nb && i < n) ? nb[(int64_t)i * a.d + cg] : 0.f;
                    }
                    if (!nb) {
                        const float4 v = noise4(a.seed, a.offset, k + 1, cg, qd);
                        xi[0] = v.x;
                        xi[1] = v.y;
                        xi[2] = v.z;
                        xi[3] = v.w;
                    }
                    float u[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int j = 0; j < n; ++j) {
                        const float xj = Xc[j * kChunk + tx];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int i = qd * 4 + r < n ? qd * 4 + r : n - 1;
                            u[r] = fmaf(Ws[i * n + j], xj, u[r]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int i = qd * 4 + r;
                        if (i >= n) break;
                        const float g = obs ? lik_score(c.obs_op, zv[r], yc, c.inv_r) : 0.f;
                        a.z[(int64_t)i * a.d + cg] = em_update(c, zv[r], u[r], g, xi[r]);
                    }
                }
            }
        }
        if (!grid_barrier(a.bar, a.err)) return;
    }
}

// Two blocks meet at the grid barrier, but block 1 leaves without arriving:
// block 0's bounded wait must run out and record ENSF_ETIMEOUT.
__global__ void k_selftest_grid_barrier(unsigned *bar, int *err) {
    if (blockIdx.x == 1) return;
    grid_barrier(bar, err);
}

}  // namespace

cudaError_t launch_selftest_grid_barrier(unsigned *bar, int *err, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_selftest_grid_barrier<<<2, 32, 0, s>>>(bar, err);
    return cudaGetLastError();
}

size_t small_smem_bytes() { return sizeof(float) * (size_t)(128 * 128 + 128 * kChunk); }

cudaError_t launch_analysis_small(const float *x, const double *norms, const float *centre, float *z, const float *y,
                                  const uint8_t *mask, int n, int64_t d, int K, double eps, float inv_r, int obs_op,
                                  const float *noise_buf, uint64_t seed, uint32_t offset, float *partial,
                                  int64_t partial_floats, float *w, unsigned *bar, int *err, int sms,
                                  cudaStream_t s) {
    if (n < 1 || n > 128 || d < 1 || K < 1) return cudaErrorInvalidValue;
    const size_t smem = small_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_analysis_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_analysis_small, kSmallThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = sms;  // one block per SM (all co-resident: per_sm >= 1)
    SmallArgs a;
    a.x = x;
    a.norms = norms;
    a.centre = centre;
    a.z = z;
    a.y = y;
    a.mask = mask;
    a.noise_buf = noise_buf;
    a.seed = seed;
    a.offset = offset;
    a.partial = partial;
    a.w = w;
    // Gram slices: whole chunks, at most as many partials as the scratch holds
    const int64_t chunks = (d + kChunk - 1) / kChunk;
    // Gram blocks: one per SM (each phase is latency bound: the fewer state
    // chunks a block walks through, the shorter the step)
    int64_t gb = (int64_t)blocks;
    if (chunks < gb) gb = chunks;
    if (partial_floats / ((int64_t)n * n) < gb) gb = partial_floats / ((int64_t)n * n);
    if (gb < 1) return cudaErrorInvalidValue;
    a.gram_slice = ((chunks + gb - 1) / gb) * kChunk;
    a.gram_blocks = (int)((d + a.gram_slice - 1) / a.gram_slice);
    a.col_slice = ((chunks + blocks - 1) / blocks) * kChunk;
    a.n = n;
    a.d = d;
    a.K = K;
    a.eps = eps;
    a.inv_r = inv_r;
    a.obs_op = obs_op;
    a.bar = bar;
    a.err = err;
    e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_analysis_small), dim3(blocks),
                                       dim3(kSmallThreads), args, smem, s);
}

}  // namespace ensf
