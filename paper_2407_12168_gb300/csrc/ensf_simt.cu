// ensf_simt.cu -- CUDA-core kernels of the EnSF analysis step:
//   * squared row norms |x_j - m|^2 to FP64 accuracy (the expanded logit)
//   * the counter-based Gaussian noise stream (Philox4x32-10 + Box-Muller)
//   * the plain FP32 path: Gram Z X^T, row softmax, W X with the fused
//     Euler-Maruyama epilogue
//   * FP32 -> BF16 hi/lo splits feeding the tensor-core path
//   * finite-value scan and FP64 ensemble mean / RMSE
#include <cfloat>
#include <cmath>

#include "ensf_internal.h"

namespace ensf {
namespace {

constexpr int kTile = 64;    // output tile edge of the CUDA-core GEMMs
constexpr int kTileK = 16;   // reduction depth per shared-memory stage

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// ---------------------------------------------------------------------------
// |x_j - m|^2 to FP64 accuracy (m = the centre vector, or 0): one block per
// row, float4 loads, the difference rounded to FP32 as the Gram operands are.
// Each thread keeps a double-float (unevaluated FP32 pair) sum: squares are
// split exactly into p + e with an FMA (Dekker's product), the running sum
// is updated with Knuth's error-free two-sum, so the per-thread sums carry
// about 48 bits at FP32 speed (GB300 issues FP64 at a small fraction of the
// FP32 rate); the 256 thread sums are combined in FP64 in a fixed order.
__device__ __forceinline__ void df_add_square(float &hi, float &lo, float v) {
    const float p = __fmul_rn(v, v);
    const float e = fmaf(v, v, -p);  // v*v - p exactly
    df_add(hi, lo, p);
    lo = __fadd_rn(lo, e);
}

__global__ void __launch_bounds__(256) k_row_norms(const float *__restrict__ x, int64_t d,
                                                   const float *__restrict__ centre, const int *__restrict__ rows,
                                                   double *__restrict__ out) {
    const float *row = x + (int64_t)(rows ? rows[blockIdx.x] : blockIdx.x) * d;
    float hi = 0.f, lo = 0.f;
    for (int64_t c = (int64_t)threadIdx.x * 4; c < d; c += 256 * 4) {
        float4 v = ld4(row + c);
        if (centre) {
            const float4 m = ld4(centre + c);
            v.x -= m.x; v.y -= m.y; v.z -= m.z; v.w -= m.w;
        }
        df_add_square(hi, lo, v.x);
        df_add_square(hi, lo, v.y);
        df_add_square(hi, lo, v.z);
        df_add_square(hi, lo, v.w);
    }
    __shared__ double red[256];
    red[threadIdx.x] = (double)hi + (double)lo;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Column means m[c] = (1/n) sum_j x[j][c] in FP32.  m only centres the Gram
// operands: |(z - alpha m) - alpha (x_j - m)|^2 = |z - alpha x_j|^2 for any m,
// so its rounding does not enter the result; the sum runs over four
// interleaved partial sums for memory-level parallelism.
__global__ void __launch_bounds__(256) k_col_mean(const float *__restrict__ x, int n, int64_t d,
                                                  float *__restrict__ m) {
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (c >= d) return;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int j = 0;
    for (; j + 4 <= n; j += 4) {
        a0 += x[(int64_t)j * d + c];
        a1 += x[(int64_t)(j + 1) * d + c];
        a2 += x[(int64_t)(j + 2) * d + c];
        a3 += x[(int64_t)(j + 3) * d + c];
    }
    for (; j < n; ++j) a0 += x[(int64_t)j * d + c];
    m[c] = ((a0 + a1) + (a2 + a3)) / (float)n;
}

// ---------------------------------------------------------------------------
// out[kk][i][c] = xi[k0 + kk][i][c]; one thread per (column c, particle quad).
__global__ void k_philox_normal(uint64_t seed, uint32_t offset, int k0, int n, int64_t d,
                                float *__restrict__ out) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int qd = blockIdx.y;
    int kk = blockIdx.z;
    if (c >= d) return;
    float4 v = noise4(seed, offset, k0 + kk, c, qd);
    float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int i = qd * 4 + r;
        if (i < n) out[((int64_t)kk * n + i) * d + c] = vv[r];
    }
}

// One noise slice out[i][c] = xi[k][i][c] with a bounded grid (grid-stride
// over (particle quad, column) pairs) so that it can share the SMs with a
// concurrently running Gram without crowding out its blocks.
__global__ void __launch_bounds__(256) k_noise_slice(uint64_t seed, uint32_t offset, int k, int n, int64_t d,
                                                     float *__restrict__ out, int64_t col0) {
    const int64_t quads = (n + 3) / 4;
    const int64_t total = quads * d;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int qd = (int)(idx / d);
        const int64_t c = idx - (int64_t)qd * d;
        float4 v = noise4(seed, offset, k, c + col0, qd);
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = qd * 4 + r;
            if (i < n) out[(int64_t)i * d + c] = vv[r];
        }
    }
}

// z[i][c] <- xi[0][i][c]; one thread per (column c, particle quad).
__global__ void k_init_particles(float *__restrict__ z, int n, int64_t d,
                                 const float *__restrict__ noise_buf, uint64_t seed,
                                 uint32_t offset, int64_t col0) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int qd = blockIdx.y;
    if (c >= d) return;
    float vv[4];
    if (noise_buf) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int i = qd * 4 + r;
            vv[r] = i < n ? noise_buf[(int64_t)i * d + c] : 0.f;
        }
    } else {
        float4 v = noise4(seed, offset, 0, c + col0, qd);
        vv[0] = v.x; vv[1] = v.y; vv[2] = v.z; vv[3] = v.w;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int i = qd * 4 + r;
        if (i < n) z[(int64_t)i * d + c] = vv[r];
    }
}

// ---------------------------------------------------------------------------
// partial[s][i][j] = sum_{c in slice s} z[i][c] x[j][c], FP32 FMA.
// 64x64 output tile per block, 4x4 per thread, reduction staged 16 deep.
__global__ void __launch_bounds__(256)
k_gram_fp32(const float *__restrict__ z, int n, const float *__restrict__ x, int n_x, int64_t d,
            int64_t slice_len, const float *__restrict__ centre, float alpha, float *__restrict__ partial) {
    __shared__ __align__(16) float As[kTileK][kTile + 4];
    __shared__ __align__(16) float Bs[kTileK][kTile + 4];
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    const int64_t c_begin = (int64_t)blockIdx.z * slice_len;
    const int64_t c_end = min(d, c_begin + slice_len);
    const int tx = tid & 15, ty = tid >> 4;
    const int lr = tid >> 2, lk = (tid & 3) * 4;
    float acc[4][4] = {};
    for (int64_t c0 = c_begin; c0 < c_end; c0 += kTileK) {
        const int64_t c = c0 + lk;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (i0 + lr < n && c < c_end) a = ld4(z + (int64_t)(i0 + lr) * d + c);
        if (j0 + lr < n_x && c < c_end) b = ld4(x + (int64_t)(j0 + lr) * d + c);
        if (centre && c < c_end) {  // z - alpha m and x - m: the distance is unchanged
            const float4 m = ld4(centre + c);
            a.x -= alpha * m.x; a.y -= alpha * m.y; a.z -= alpha * m.z; a.w -= alpha * m.w;
            b.x -= m.x; b.y -= m.y; b.z -= m.z; b.w -= m.w;
        }
        As[lk + 0][lr] = a.x; As[lk + 1][lr] = a.y; As[lk + 2][lr] = a.z; As[lk + 3][lr] = a.w;
        Bs[lk + 0][lr] = b.x; Bs[lk + 1][lr] = b.y; Bs[lk + 2][lr] = b.z; Bs[lk + 3][lr] = b.w;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTileK; ++kk) {
            float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(ar[r], br[q], acc[r][q]);
        }
        __syncthreads();
    }
    float *out = partial + (int64_t)blockIdx.z * n * n_x;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int i = i0 + ty * 4 + r;
        if (i >= n) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int j = j0 + tx * 4 + q;
            if (j < n_x) out[(int64_t)i * n_x + j] = acc[r][q];
        }
    }
}

// ---------------------------------------------------------------------------
// Row softmax of the logits  l_ij = (2 alpha G_ij - alpha^2 |x_j|^2) / (2 beta^2)
// (Eq. 12 expanded; the row constant -|z_i|^2/(2 beta^2) cancels in Eq. 16).
// NT threads per row.
template <int NT>
__global__ void __launch_bounds__(NT)
k_softmax_rows(const float *__restrict__ partial, int splits, int64_t part_stride, int ldp,
               int n_x, const double *__restrict__ norms, double alpha, double inv_2beta2,
               float *__restrict__ w, int ldw, __nv_bfloat16 *__restrict__ w_hi,
               __nv_bfloat16 *__restrict__ w_lo, int ldwb) {
    pdl_wait();
    pdl_launch_dependents();
    extern __shared__ double lg[];
    __shared__ double red[NT];
    softmax_row<NT>(blockIdx.x, partial, splits, part_stride, ldp, n_x, norms, alpha, inv_2beta2, w, ldw, w_hi,
                    w_lo, ldwb, lg, red);
}

// Row softmax in 256-column tiles: one warp per (row, tile) forms the tile's
// log-kernels and statistics; the last warp to finish a row (arrival counter,
// reset by that warp) normalises it.  No warp waits for another.
__global__ void __launch_bounds__(256)
k_softmax_tiled(const float *__restrict__ partial, int splits, int64_t part_stride, int ldp, int n, int n_x,
                const double *__restrict__ norms, double alpha, double inv_2beta2, DF *L, float4 *stats,
                int *rowcnt, float *__restrict__ w, int ldw, __nv_bfloat16 *__restrict__ w_hi,
                __nv_bfloat16 *__restrict__ w_lo, int ldwb) {
    pdl_wait();
    pdl_launch_dependents();
    const int nt = (n_x + kSoftTile - 1) / kSoftTile;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= (int64_t)n * nt) return;
    const int i = (int)(gw / nt), t = (int)(gw % nt);
    const int lane = threadIdx.x & 31;
    const LogitCoef kc = logit_coef(alpha, inv_2beta2);
    softmax_tile_stats(i, t, partial, splits, part_stride, ldp, n_x, norms, kc, L, n_x, stats, nt);
    __threadfence();
    int last = 0;
    if (lane == 0) last = atomicAdd(&rowcnt[i], 1) == nt - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    if (lane == 0) rowcnt[i] = 0;
    __threadfence();
    softmax_finalize_row(i, n_x, nt, L, n_x, stats, w, ldw, w_hi, w_lo, ldwb);
}

// ---------------------------------------------------------------------------
// u = W X on FP32 CUDA cores (64 particles x 64 state columns per block),
// fused with the score and the Euler-Maruyama update of Eq. 7 / Eq. 17.
__global__ void __launch_bounds__(256)
k_wx_em_fp32(const float *__restrict__ w, int ldw, const float *__restrict__ x, int n, int n_x,
             int64_t d, float *__restrict__ z, const float *__restrict__ y,
             const uint8_t *__restrict__ mask, const float *__restrict__ noise_buf, uint64_t seed,
             uint32_t offset, StepCoef cf) {
    __shared__ __align__(16) float Ws[kTileK][kTile + 4];  // Ws[j][i]
    __shared__ __align__(16) float Xs[kTileK][kTile + 4];  // Xs[j][c]
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * kTile;
    const int64_t c0 = (int64_t)blockIdx.x * kTile;
    const int tx = tid & 15, ty = tid >> 4;
    const int wr = tid >> 2, wk = (tid & 3) * 4;    // W loader: row, 4 consecutive j
    const int xr = tid >> 4, xc = (tid & 15) * 4;   // X loader: j row, 4 consecutive c
    float acc[4][4] = {};
    for (int j0 = 0; j0 < n_x; j0 += kTileK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int j = j0 + wk + q;
            Ws[wk + q][wr] = (i0 + wr < n && j < n_x) ? w[(int64_t)(i0 + wr) * ldw + j] : 0.f;
        }
        float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j0 + xr < n_x && c0 + xc < d) xv = ld4(x + (int64_t)(j0 + xr) * d + c0 + xc);
        *reinterpret_cast<float4 *>(&Xs[xr][xc]) = xv;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTileK; ++kk) {
            float4 av = *reinterpret_cast<const float4 *>(&Ws[kk][ty * 4]);
            float4 bv = *reinterpret_cast<const float4 *>(&Xs[kk][tx * 4]);
            float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(ar[r], br[q], acc[r][q]);
        }
        __syncthreads();
    }
    const int64_t c = c0 + tx * 4;
    if (c >= d) return;
    const float4 yv = ld4(y + c);
    uchar4 mv = make_uchar4(1, 1, 1, 1);
    if (mask) mv = *reinterpret_cast<const uchar4 *>(mask + c);
    const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
    const unsigned char mm[4] = {mv.x, mv.y, mv.z, mv.w};
    // noise xi[k+1][i][c]: one Philox block per column covers this thread's 4 particles
    const int ib = i0 + ty * 4;
    float xi[4][4];  // [row][column]
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (noise_buf) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                xi[r][q] = (ib + r < n) ? noise_buf[((int64_t)(cf.k + 1) * n + ib + r) * d + c + q] : 0.f;
        } else {
            float4 v = noise4(seed, offset, cf.k + 1, c + q + cf.col0, ib >> 2);
            xi[0][q] = v.x; xi[1][q] = v.y; xi[2][q] = v.z; xi[3][q] = v.w;
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = ib + r;
        if (i >= n) continue;
        float *zp = z + (int64_t)i * d + c;
        float4 zv = ld4(zp);
        float zz[4] = {zv.x, zv.y, zv.z, zv.w};
        float o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float g = mm[q] ? lik_score(cf.obs_op, zz[q], yy[q], cf.inv_r) : 0.f;
            o[q] = em_update(cf, zz[q], acc[r][q], g, xi[r][q]);
        }
        *reinterpret_cast<float4 *>(zp) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// ---------------------------------------------------------------------------
// x = hi + lo with hi = bf16(x), lo = bf16(x - hi); row-major, out stride ldo.
__global__ void k_split_bf16(const float *__restrict__ x, int64_t cols, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo, int64_t ldo, const float *__restrict__ centre,
                             float scale, const int *__restrict__ rows) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (q * 4 >= cols) return;
    float4 v = ld4(x + (int64_t)(rows ? rows[r] : r) * cols + q * 4);
    if (centre) {  // split x - scale * m (product and difference each rounded, as in the W X epilogue)
        const float4 m = ld4(centre + q * 4);
        v.x = __fsub_rn(v.x, __fmul_rn(scale, m.x));
        v.y = __fsub_rn(v.y, __fmul_rn(scale, m.y));
        v.z = __fsub_rn(v.z, __fmul_rn(scale, m.z));
        v.w = __fsub_rn(v.w, __fmul_rn(scale, m.w));
    }
    float vv[4] = {v.x, v.y, v.z, v.w};
    __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        h[e] = __float2bfloat16_rn(vv[e]);
        l[e] = __float2bfloat16_rn(vv[e] - __bfloat162float(h[e]));
    }
    *reinterpret_cast<uint2 *>(hi + (int64_t)r * ldo + q * 4) = *reinterpret_cast<uint2 *>(h);
    if (lo) *reinterpret_cast<uint2 *>(lo + (int64_t)r * ldo + q * 4) = *reinterpret_cast<uint2 *>(l);
}

// The FP32 centred copy out[r][c] = x[row(r)][c] - scale * m[c] (the TF32
// Gram's operand), rounded as the splits round it.
__global__ void k_centre_copy(const float *__restrict__ x, int64_t cols, float *__restrict__ out,
                              const float *__restrict__ centre, float scale, const int *__restrict__ rows) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (q * 4 >= cols) return;
    float4 v = ld4(x + (int64_t)(rows ? rows[r] : r) * cols + q * 4);
    if (centre) {
        const float4 m = ld4(centre + q * 4);
        v.x = __fsub_rn(v.x, __fmul_rn(scale, m.x));
        v.y = __fsub_rn(v.y, __fmul_rn(scale, m.y));
        v.z = __fsub_rn(v.z, __fmul_rn(scale, m.z));
        v.w = __fsub_rn(v.w, __fmul_rn(scale, m.w));
    }
    *reinterpret_cast<float4 *>(out + (int64_t)r * cols + q * 4) = v;
}

// Transposed split through a 32x32 shared tile: xT[c][j] from x[j][c].
__global__ void k_split_bf16_t(const float *__restrict__ x, int rows, int64_t cols,
                               __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                               int64_t ldo, const int *__restrict__ rowmap) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int j = j0 + r;
        int64_t c = c0 + tx;
        tile[r][tx] = (j < rows && c < cols) ? x[(int64_t)(rowmap ? rowmap[j] : j) * cols + c] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int64_t c = c0 + r;
        int j = j0 + tx;
        if (c < cols && j < rows) {
            float v = tile[tx][r];
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[c * ldo + j] = h;
            if (lo) lo[c * ldo + j] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void k_check_finite(const float *__restrict__ z, int64_t count, int *err_word) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < count; i += stride) bad |= !isfinite(z[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(err_word, 0, 4 /*ENSF_ENUMERIC*/);
}

// FP64 column means over the n rows and per-block partial sums of (mean - truth)^2.
__global__ void __launch_bounds__(256)
k_stats_mean(const float *__restrict__ z, int n, int64_t d, const float *__restrict__ truth,
             double *__restrict__ mean, double *__restrict__ block_sq) {
    int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double sq = 0.0;
    if (c < d) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += (double)z[(int64_t)i * d + c];
        double m = acc / (double)n;
        if (mean) mean[c] = m;
        if (truth) {
            double e = m - (double)truth[c];
            sq = e * e;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = sq;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sq[blockIdx.x] = red[0];
}

__global__ void k_stats_rmse(const double *__restrict__ block_sq, int blocks, int64_t d,
                             double *__restrict__ rmse) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < blocks; b += 256) acc += block_sq[b];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *rmse = sqrt(red[0] / (double)d);
}

// Relaxation of the analysis spread to the prior (forecast) spread, per
// state variable c: with means m_f, m_a and standard deviations s_f, s_a over
// the n members,  z_i <- m_a + (z_i - m_a) ((1 - a) + a s_f / s_a).
// mode 1 relaxes the perturbations instead:  z_i <- m_a + (1 - a)(z_i - m_a) + a (x_i - m_f).
__global__ void k_relax_spread(const float *__restrict__ prior, float *__restrict__ z, int n, int64_t d, float a,
                               int mode) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d) return;
    double sf = 0.0, sf2 = 0.0, sa = 0.0, sa2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double xf = prior[(int64_t)i * d + c], xa = z[(int64_t)i * d + c];
        sf += xf;
        sf2 += xf * xf;
        sa += xa;
        sa2 += xa * xa;
    }
    const double mf = sf / n, ma = sa / n;
    const double vf = fmax(sf2 / n - mf * mf, 0.0), va = fmax(sa2 / n - ma * ma, 0.0);
    const double ratio = va > 0.0 ? sqrt(vf / va) : 1.0;
    const double f = (1.0 - a) + a * ratio;
    for (int i = 0; i < n; ++i) {
        const int64_t o = (int64_t)i * d + c;
        if (mode == 1)
            z[o] = (float)(ma + (1.0 - a) * (z[o] - ma) + a * (prior[o] - mf));
        else
            z[o] = (float)(ma + (z[o] - ma) * f);
    }
}

}  // namespace

// Model error of the twin experiment: one thread per (particle quad, column),
// the four particles of a quad share one Philox block per process (the same
// counter layout as the analysis noise), grid-stride over the columns.
struct ModelErrorCoef {
    float c[8];
    int n;
};

__global__ void __launch_bounds__(256) k_model_error(float *__restrict__ state, int batch, int64_t d,
                                                     ModelErrorCoef coef, uint64_t seed, uint32_t cycle) {
    const int qd = blockIdx.y;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < d; c += (int64_t)gridDim.x * blockDim.x) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int p = 0; p < coef.n; ++p) {
            if (coef.c[p] == 0.0f) continue;
            const float4 v = noise4(seed, cycle, p, c, qd);
            acc[0] += coef.c[p] * v.x;
            acc[1] += coef.c[p] * v.y;
            acc[2] += coef.c[p] * v.z;
            acc[3] += coef.c[p] * v.w;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int b = qd * 4 + r;
            if (b < batch) state[(int64_t)b * d + c] += acc[r];
        }
    }
}

cudaError_t launch_model_error(float *state, int batch, int64_t d, const float *coef, int nproc, uint64_t seed,
                               uint32_t cycle, cudaStream_t s) {
    ModelErrorCoef mc{};
    mc.n = nproc;
    for (int p = 0; p < nproc; ++p) mc.c[p] = coef[p];
    int64_t bx = (d + 255) / 256;
    if (bx > 152 * 8) bx = 152 * 8;
    dim3 grid((unsigned)bx, (unsigned)((batch + 3) / 4));
    k_model_error<<<grid, 256, 0, s>>>(state, batch, d, mc, seed, cycle);
    return cudaGetLastError();
}

cudaError_t launch_relax_spread(const float *prior, float *z, int n, int64_t d, float a, int mode, cudaStream_t s) {
    k_relax_spread<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(prior, z, n, d, a, mode);
    return cudaGetLastError();
}

// ===========================================================================
cudaError_t launch_init_particles(float *z, int n, int64_t d, const float *noise_buf,
                                  uint64_t seed, uint32_t offset, cudaStream_t s, int64_t col0) {
    dim3 grid((unsigned)((d + 255) / 256), (unsigned)((n + 3) / 4));
    k_init_particles<<<grid, 256, 0, s>>>(z, n, d, noise_buf, seed, offset, col0);
    return cudaGetLastError();
}

cudaError_t launch_philox_normal(uint64_t seed, uint32_t offset, int k0, int count, int n,
                                 int64_t d, float *out, cudaStream_t s) {
    dim3 grid((unsigned)((d + 255) / 256), (unsigned)((n + 3) / 4), (unsigned)count);
    k_philox_normal<<<grid, 256, 0, s>>>(seed, offset, k0, n, d, out);
    return cudaGetLastError();
}

cudaError_t launch_noise_slice(uint64_t seed, uint32_t offset, int k, int n, int64_t d, float *out,
                               int max_blocks, cudaStream_t s, int64_t col0) {
    const int64_t total = (int64_t)((n + 3) / 4) * d;
    int64_t blocks = (total + 255) / 256;
    if (blocks > max_blocks) blocks = max_blocks;
    k_noise_slice<<<(unsigned)blocks, 256, 0, s>>>(seed, offset, k, n, d, out, col0);
    return cudaGetLastError();
}

cudaError_t launch_row_norms(const float *x, int n, int64_t d, double *out, cudaStream_t s, const float *centre,
                             const int *rows) {
    k_row_norms<<<n, 256, 0, s>>>(x, d, centre, rows, out);
    return cudaGetLastError();
}

cudaError_t launch_gram_fp32(const float *z, int n, const float *x, int n_x, int64_t d, int splits,
                             float *partial, cudaStream_t s, const float *centre, float alpha) {
    int64_t slice = (d + splits - 1) / splits;
    slice = (slice + kTileK - 1) / kTileK * kTileK;
    dim3 grid((unsigned)((n_x + kTile - 1) / kTile), (unsigned)((n + kTile - 1) / kTile), (unsigned)splits);
    k_gram_fp32<<<grid, 256, 0, s>>>(z, n, x, n_x, d, slice, centre, alpha, partial);
    return cudaGetLastError();
}

cudaError_t launch_softmax_rows(const float *partial, int splits, int64_t part_stride, int ldp, int n,
                                int n_x, const double *norms, double alpha, double inv_2beta2,
                                float *w, int ldw, __nv_bfloat16 *w_hi, __nv_bfloat16 *w_lo, int ldwb,
                                cudaStream_t s, bool pdl) {
    size_t smem = sizeof(double) * (size_t)n_x;
    if (smem > 46 * 1024) {  // (beside the static 2 KB reduction buffer)
        cudaError_t e = cudaFuncSetAttribute(k_softmax_rows<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    // (1024-thread rows, which spread short rows' partials over more threads,
    // measured slower: 16 against 10 us per launch on 20- and 128-member rows)
    return launch_k(k_softmax_rows<256>, dim3(n), dim3(256), smem, s, pdl, partial, splits, part_stride, ldp, n_x,
                    norms, alpha, inv_2beta2, w, ldw, w_hi, w_lo, ldwb);
}

cudaError_t launch_softmax_tiled(const float *partial, int splits, int64_t part_stride, int ldp, int n, int n_x,
                                 const double *norms, double alpha, double inv_2beta2, void *L, float4 *stats,
                                 int *rowcnt, float *w, int ldw, __nv_bfloat16 *w_hi, __nv_bfloat16 *w_lo, int ldwb,
                                 cudaStream_t s, bool pdl) {
    const int64_t warps = (int64_t)n * ((n_x + kSoftTile - 1) / kSoftTile);
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    return launch_k(k_softmax_tiled, dim3(blocks), dim3(256), 0, s, pdl, partial, splits, part_stride, ldp, n, n_x,
                    norms, alpha, inv_2beta2, static_cast<DF *>(L), stats, rowcnt, w, ldw, w_hi, w_lo, ldwb);
}

cudaError_t launch_wx_em_fp32(const float *w, int ldw, const float *x, int n, int n_x, int64_t d,
                              float *z, const float *y, const uint8_t *mask, const float *noise_buf,
                              uint64_t seed, uint32_t offset, const StepCoef &c, cudaStream_t s) {
    dim3 grid((unsigned)((d + kTile - 1) / kTile), (unsigned)((n + kTile - 1) / kTile));
    k_wx_em_fp32<<<grid, 256, 0, s>>>(w, ldw, x, n, n_x, d, z, y, mask, noise_buf, seed, offset, c);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float *x, int rows, int64_t cols, __nv_bfloat16 *hi,
                              __nv_bfloat16 *lo, int64_t ldo, cudaStream_t s, const float *centre, float scale,
                              const int *rowmap) {
    dim3 grid((unsigned)((cols / 4 + 255) / 256), (unsigned)rows);
    k_split_bf16<<<grid, 256, 0, s>>>(x, cols, hi, lo, ldo, centre, scale, rowmap);
    return cudaGetLastError();
}

cudaError_t launch_centre_copy(const float *x, int rows, int64_t cols, float *out, const float *centre, float scale,
                               const int *rowmap, cudaStream_t s) {
    dim3 grid((unsigned)((cols / 4 + 255) / 256), (unsigned)rows);
    k_centre_copy<<<grid, 256, 0, s>>>(x, cols, out, centre, scale, rowmap);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16_transpose(const float *x, int rows, int64_t cols, __nv_bfloat16 *hi,
                                        __nv_bfloat16 *lo, int64_t ldo, cudaStream_t s, const int *rowmap) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_split_bf16_t<<<grid, dim3(32, 8), 0, s>>>(x, rows, cols, hi, lo, ldo, rowmap);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *z, int64_t count, int *err_word, cudaStream_t s) {
    k_check_finite<<<1024, 256, 0, s>>>(z, count, err_word);
    return cudaGetLastError();
}

int stats_blocks(int64_t d) { return (int)((d + 255) / 256); }

cudaError_t launch_col_mean(const float *x, int n, int64_t d, float *m, cudaStream_t s) {
    k_col_mean<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(x, n, d, m);
    return cudaGetLastError();
}

cudaError_t launch_ensemble_stats(const float *z, int n, int64_t d, const float *truth, double *mean,
                                  double *rmse, double *scratch, cudaStream_t s) {
    int blocks = stats_blocks(d);
    k_stats_mean<<<blocks, 256, 0, s>>>(z, n, d, truth, mean, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !truth || !rmse) return e;
    k_stats_rmse<<<1, 256, 0, s>>>(scratch, blocks, d, rmse);
    return cudaGetLastError();
}

}  // namespace ensf
