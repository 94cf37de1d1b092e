// ensf_unet.cu -- the learned forecast surrogate: a small convolutional U-Net
// x_{t+Delta} = x_t + net(x_t) over the two-level SQG state, trained and run
// in BF16 with FP32 accumulation on this library's own kernels.
//
// Architecture (widths c1..c4): enc1 conv(2->c1), conv(c1->c1); 2x2 mean
// pool; enc2 (c1->c2, c2->c2); pool; enc3 (c2->c3, c3->c3); pool; mid
// (c3->c4, c4->c4); x2 nearest upsample + concat [up, skip] then two convs per
// decoder level back to c3, c2, c1; 1x1 head c1->2, no activation; residual
// output.  conv = 3x3 with circular padding (the SQG domain is periodic) +
// bias + SiLU.  Loss: mean squared error.  Optimiser: AdamW on FP32 master
// weights; BF16 copies feed the tensor cores.
//
// The 3x3 convolutions run on the tensor cores (ensf_conv.cu) wherever the
// shapes allow (channel counts multiples of 32, whole image rows per
// 128-pixel tile):
//   forward        implicit GEMM over TMA boxes of the haloed input, bias and
//                  SiLU in the epilogue                        -> z, y [P][Cout]
//   data gradient  the same kernel on the haloed dZ with tap-mirrored weights
//   weight grad.   nine GEMMs over the pixels: dZ^T [Cout][P] against the
//                  input's column-shifted transposed copies   -> dW [Cout][9][Cin]
// The 2-channel input convolution runs as direct SIMT kernels; other shapes
// (the 16 x 16 level's weight gradients, channel counts that are not
// multiples of 32) as im2col + the tcgen05 GEMM of ensf_tc.cu
// (C[M][N] = A[M][K] B[N][K]^T, FP32 accumulation, split-K partials):
//   forward        col [P][Kp]  x  W  [Cout][Kp]   -> [P][Cout]
//   data gradient  dZ  [P][Cout] x W^T [Kp][Cout]  -> dcol [P][Kp] -> col2im
//   weight grad.   dZ^T [Cout][P] x col^T [Kp][P]   -> dW [Cout][Kp]
// with P = batch * H * W pixels, Kp = 9 Cin rounded up to 8 (zero padded).
// Layouts: activations NHWC (pixel-major), weights [Cout][3][3][Cin].
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ensf.h"
#include "ensf_internal.h"
#include "ensf_tc.h"

namespace {

using bf16 = __nv_bfloat16;
constexpr int kLevels = 3;
constexpr int kConvs = 14;
constexpr int kColsumBlocks = 1024;  // row blocks of the column sums (bias and head gradients)
constexpr int kLossBlocks = 296;     // blocks of the loss reduction (two per SM)
constexpr int64_t kSiluTransposeSmem = 32 * 1024;  // dz rows a SiLU-backward block transposes in shared memory

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + __expf(-z)); }

unsigned nb(int64_t count, int t = 256) { return (unsigned)((count + t - 1) / t); }

// ------------------------------------------------------------- kernels
__global__ void k_nchw_to_nhwc(const float *__restrict__ x, int B, int C, int H, int W, float *__restrict__ f32,
                               bf16 *__restrict__ b16) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // NHWC index
    const int64_t total = (int64_t)B * H * W * C;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int xx = (int)(p % W), yy = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    const float v = x[(((int64_t)b * C + c) * H + yy) * W + xx];
    if (f32) f32[i] = v;
    if (b16) b16[i] = __float2bfloat16_rn(v);
}

// col[p][k], k = (dy*3 + dx)*C + c, circular neighbours; zero for k >= 9C.
__global__ void k_im2col(const bf16 *__restrict__ x, int B, int H, int W, int C, int Kp, bf16 *__restrict__ col) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)B * H * W * Kp;
    if (i >= total) return;
    const int k = (int)(i % Kp);
    const int64_t p = i / Kp;
    bf16 v = __float2bfloat16_rn(0.f);
    if (k < 9 * C) {
        const int c = k % C, tap = k / C, dy = tap / 3, dx = tap % 3;
        const int xx = (int)(p % W), yy = (int)((p / W) % H);
        const int64_t b = p / ((int64_t)W * H);
        const int sy = (yy + dy - 1 + H) % H, sx = (xx + dx - 1 + W) % W;
        v = x[((b * H + sy) * W + sx) * C + c];
    }
    col[i] = v;
}

// Adjoint of k_im2col: dx[b][y][x][c] (+)= sum over taps of dcol at the pixel
// that read (y, x) through that tap.
__global__ void k_col2im(const float *__restrict__ dcol, int B, int H, int W, int C, int Kp, float *__restrict__ dx,
                         int accumulate) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)B * H * W * C;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const int64_t b = p / ((int64_t)W * H);
    float acc = 0.f;
    for (int dy = 0; dy < 3; ++dy)
        for (int dxx = 0; dxx < 3; ++dxx) {
            const int oy = (yy - dy + 1 + H) % H, ox = (xx - dxx + 1 + W) % W;
            acc += dcol[((b * H + oy) * W + ox) * Kp + (dy * 3 + dxx) * C + c];
        }
    dx[i] = accumulate ? dx[i] + acc : acc;
}

// xp[b][yy][xx][c] = x[b][(yy - 1) mod h][(xx - 1) mod w][c]: the input of an
// implicit-GEMM convolution with its one-pixel circular halo; 8 channels per thread.
// I: the index type (32-bit where the element count allows: its divisions
// are several times cheaper than 64-bit ones).
template <class I>
__global__ void k_pad_circ(const bf16 *__restrict__ x, int B, int h, int w, int C, bf16 *__restrict__ xp) {
    const I i = (I)blockIdx.x * blockDim.x + threadIdx.x;  // over B (h + 2) (w + 2) C / 8
    const I c8 = C / 8;
    const I total = (I)B * (h + 2) * (w + 2) * c8;
    if (i >= total) return;
    const I cv = i % c8;
    const I pp = i / c8;
    const I xx = pp % (I)(w + 2), yy = (pp / (I)(w + 2)) % (I)(h + 2);
    const I b = pp / ((I)(w + 2) * (h + 2));
    const I sy = yy == 0 ? h - 1 : (yy == (I)h + 1 ? 0 : yy - 1);
    const I sx = xx == 0 ? w - 1 : (xx == (I)w + 1 ? 0 : xx - 1);
    reinterpret_cast<uint4 *>(xp)[i] = reinterpret_cast<const uint4 *>(x)[((b * h + sy) * w + sx) * c8 + cv];
}

// The haloed copy of x for the implicit convolutions.
void pad_circ(const bf16 *x, int B, int h, int w, int C, bf16 *xp, cudaStream_t s) {
    const int64_t total = (int64_t)B * (h + 2) * (w + 2) * (C / 8);
    if (total < ((int64_t)1 << 31))
        k_pad_circ<uint32_t><<<nb(total), 256, 0, s>>>(x, B, h, w, C, xp);
    else
        k_pad_circ<int64_t><<<nb(total), 256, 0, s>>>(x, B, h, w, C, xp);
}


__global__ void k_reduce_splits(const float *__restrict__ part, int S, int64_t count, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += part[(int64_t)s * count + i];
    out[i] = acc;
}

__global__ void k_bias_silu(const float *__restrict__ c, const float *__restrict__ bias, int64_t P, int Co,
                            float *__restrict__ z, bf16 *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * Co) return;
    const float zz = c[i] + bias[i % Co];
    z[i] = zz;
    y[i] = __float2bfloat16_rn(zz * sigmoidf_(zz));
}

// dz = dy * SiLU'(z) as BF16 for the GEMMs and, per block of rows, the
// column sums of dz (the bias gradient) in FP32: block (bx, by) covers rows
// [bx * rows_per_blk, ...) and the columns [by * 256, by * 256 + Cg); thread t
// takes column t % Cg of every (256 / Cg)-th row, and partial[bx][c] sums the
// threads of a column in thread order (fixed order; k_colsum_final ends it).
__global__ void __launch_bounds__(256) k_silu_back_colsum(const float *__restrict__ dy, const float *__restrict__ z,
                                                          int64_t P, int C, int64_t rows_per_blk,
                                                          bf16 *__restrict__ dz16, float *__restrict__ partial,
                                                          bf16 *__restrict__ dzT) {
    __shared__ float red[256];
    extern __shared__ bf16 tsm[];  // with dzT: the block's dz rows [rows_per_blk][Cg + 2] (padded: no bank conflicts)
    const int tld = min(256, C - (int)blockIdx.y * 256) + 2;
    const int cb = blockIdx.y * 256;
    const int Cg = min(256, C - cb);
    const int R = 256 / Cg;
    const int t = threadIdx.x, cl = t % Cg, j = t / Cg;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
    const int64_t r1 = r0 + rows_per_blk < P ? r0 + rows_per_blk : P;
    float acc = 0.f;
    if (j < R) {
        int64_t r = r0 + j;
        // eight rows' loads in flight before their arithmetic and stores
        for (; r + 7 * R < r1; r += 8 * R) {
            float zv[8], dv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int64_t i = (r + k * R) * C + cb + cl;
                zv[k] = z[i];
                dv[k] = dy[i];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float sg = sigmoidf_(zv[k]);
                const float g = dv[k] * sg * (1.f + zv[k] * (1.f - sg));
                const bf16 gb = __float2bfloat16_rn(g);
                dz16[(r + k * R) * C + cb + cl] = gb;
                if (dzT) tsm[(r + k * R - r0) * tld + cl] = gb;
                acc += g;
            }
        }
        for (; r < r1; r += R) {
            const int64_t i = r * C + cb + cl;
            const float zz = z[i];
            const float sg = sigmoidf_(zz);
            const float g = dy[i] * sg * (1.f + zz * (1.f - sg));
            const bf16 gb = __float2bfloat16_rn(g);
            dz16[i] = gb;
            if (dzT) tsm[(r - r0) * tld + cl] = gb;
            acc += g;
        }
    }
    red[t] = acc;
    __syncthreads();
    if (t < Cg) {
        float sum = 0.f;
        for (int k = 0; k < R; ++k) sum += red[k * Cg + t];
        partial[(int64_t)blockIdx.x * C + cb + t] = sum;
    }
    if (dzT) {
        // dzT[c][r] for the block's rows: runs of consecutive rows per channel
        const int nrows = (int)(r1 - r0);
        for (int idx = t; idx < Cg * nrows; idx += blockDim.x) {
            const int c = idx / nrows, rr = idx - c * nrows;
            dzT[(int64_t)(cb + c) * P + r0 + rr] = tsm[rr * tld + c];
        }
    }
}

// out[c] = sum over blocks of partial[blk][c]: one warp per column, lane l
// summing blocks l, l + 32, ..., then a fixed butterfly across the lanes.
__global__ void k_colsum_final(const float *__restrict__ partial, int blocks, int C, float *__restrict__ out) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= C) return;  // whole warps
    float acc = 0.f;
    for (int b = lane; b < blocks; b += 32) acc += partial[(int64_t)b * C + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[c] = acc;
}

__global__ void k_transpose_bf16(const bf16 *__restrict__ in, int64_t R, int C, bf16 *__restrict__ out) {
    __shared__ bf16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32;
    const int c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t r = r0 + k;
        const int c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < R && c < C) ? in[r * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (c < C && r < R) out[(int64_t)c * R + r] = tile[threadIdx.x][k];
    }
}

__global__ void k_pool_fwd(const bf16 *__restrict__ x, int B, int H, int W, int C, bf16 *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int h = H / 2, w = W / 2;
    if (i >= (int64_t)B * h * w * C) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int xx = (int)(p % w), yy = (int)((p / w) % h);
    const int64_t b = p / ((int64_t)w * h);
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int e = 0; e < 2; ++e) s += __bfloat162float(x[((b * H + 2 * yy + a) * W + 2 * xx + e) * C + c]);
    y[i] = __float2bfloat16_rn(0.25f * s);
}

// dx (+)= dy / 4 spread back over each 2 x 2 window, four channels
// (16 bytes) per thread; C a multiple of 4; I: the index type.
template <class I>
__global__ void k_pool_bwd(const float *__restrict__ dy, int B, int H, int W, int C, float *__restrict__ dx,
                           int accumulate) {
    const I i = (I)blockIdx.x * blockDim.x + threadIdx.x;  // over the fine grid, C / 4 per pixel
    const I c4 = C / 4;
    if (i >= (I)B * H * W * c4) return;
    const I cv = i % c4, p = i / c4;
    const I xx = p % (I)W, yy = (p / (I)W) % (I)H, b = p / ((I)W * H);
    float4 g = reinterpret_cast<const float4 *>(dy)[((b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * c4 + cv];
    g.x *= 0.25f;
    g.y *= 0.25f;
    g.z *= 0.25f;
    g.w *= 0.25f;
    float4 *d4 = reinterpret_cast<float4 *>(dx) + i;
    if (accumulate) {
        const float4 o = *d4;
        g.x += o.x;
        g.y += o.y;
        g.z += o.z;
        g.w += o.w;
    }
    *d4 = g;
}

// out[p] = [nearest-upsampled low (Cl channels), skip (Cs channels)], eight
// channels (16 bytes) per thread; Cl and Cs are multiples of 8.
__global__ void k_up_concat_fwd(const bf16 *__restrict__ low, const bf16 *__restrict__ skip, int B, int H, int W,
                                int Cl, int Cs, bf16 *__restrict__ out) {
    const int Ct8 = (Cl + Cs) / 8, Cl8 = Cl / 8, Cs8 = Cs / 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * H * W * Ct8) return;
    const int c8 = (int)(i % Ct8);
    const int64_t p = i / Ct8;
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const int64_t b = p / ((int64_t)W * H);
    reinterpret_cast<uint4 *>(out)[i] =
        c8 < Cl8 ? reinterpret_cast<const uint4 *>(low)[((b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * Cl8 + c8]
                 : reinterpret_cast<const uint4 *>(skip)[p * Cs8 + (c8 - Cl8)];
}

// Gradient of k_up_concat_fwd: dlow (coarse, the sum of its 4 fine pixels'
// first Cl channels), four channels per thread; I: the index type.
template <class I>
__global__ void k_up_bwd(const float *__restrict__ dout, int B, int H, int W, int Cl, int Cs,
                         float *__restrict__ dlow) {
    const I Ct4 = (Cl + Cs) / 4, Cl4 = Cl / 4;
    const I h = H / 2, w = W / 2;
    const I i = (I)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (I)B * h * w * Cl4) return;
    const I c = i % Cl4, p = i / Cl4;
    const I xx = p % w, yy = (p / w) % h, b = p / (w * h);
    const float4 *d4 = reinterpret_cast<const float4 *>(dout);
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int a = 0; a < 2; ++a)
        for (int e = 0; e < 2; ++e) {
            const float4 v = d4[((b * H + 2 * yy + a) * W + 2 * xx + e) * Ct4 + c];
            sum.x += v.x;
            sum.y += v.y;
            sum.z += v.z;
            sum.w += v.w;
        }
    reinterpret_cast<float4 *>(dlow)[i] = sum;
}

// dskip (+)= the skip channels of dout [P][Cl + Cs], four per thread.
template <class I>
__global__ void k_skip_bwd(const float *__restrict__ dout, int64_t P, int Cl, int Cs, float *__restrict__ dskip) {
    const I i = (I)blockIdx.x * blockDim.x + threadIdx.x;
    const I Cs4 = Cs / 4, Ct4 = (Cl + Cs) / 4, Cl4 = Cl / 4;
    if (i >= (I)P * Cs4) return;
    const I p = i / Cs4, c = i % Cs4;
    const float4 v = reinterpret_cast<const float4 *>(dout)[p * Ct4 + Cl4 + c];
    float4 *o = reinterpret_cast<float4 *>(dskip) + i;
    float4 r = *o;
    r.x += v.x;
    r.y += v.y;
    r.z += v.z;
    r.w += v.w;
    *o = r;
}

// Head: out_nchw[b][o][y][x] = x_in + sum_c d1[p][c] Wh[o][c] + bh[o].
__global__ void k_head_fwd(const bf16 *__restrict__ d1, const float *__restrict__ xin, const float *__restrict__ Wh,
                           const float *__restrict__ bh, int B, int H, int W, int C, int O, float *__restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)B * H * W) return;
    const int xx = (int)(p % W), yy = (int)((p / W) % H);
    const int64_t b = p / ((int64_t)W * H);
    for (int o = 0; o < O; ++o) {
        float acc = bh[o] + xin[p * O + o];
        for (int c = 0; c < C; ++c) acc += __bfloat162float(d1[p * C + c]) * Wh[o * C + c];
        out[((b * O + o) * H + yy) * W + xx] = acc;
    }
}

// Loss gradient and the loss's block partials: dout (NHWC) = 2 (out - tgt) /
// count, and part[blk] = sum of the squared errors of the elements blk,
// blk + gridDim.x * 256, ... taken by this block (FP32 squares summed in FP64,
// thread partials then combined in thread order).
__global__ void __launch_bounds__(256) k_mse_grad(const float *__restrict__ out, const float *__restrict__ tgt, int B,
                                                  int O, int H, int W, float *__restrict__ dout,
                                                  double *__restrict__ part) {
    __shared__ double red[256];
    const int64_t total = (int64_t)B * O * H * W;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W), yy = (int)((i / W) % H), o = (int)((i / ((int64_t)W * H)) % O);
        const int64_t b = i / ((int64_t)W * H * O);
        const float d = out[i] - tgt[i];
        const float q = d * d;
        acc += (double)q;
        dout[((b * H + yy) * W + xx) * O + o] = 2.f * d / (float)total;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int k = 0; k < 256; ++k) sum += red[k];
        part[blockIdx.x] = sum;
    }
}

// loss = (sum of the block partials) / count: one warp, lane l summing
// blocks l, l + 32, ..., then a fixed butterfly across the lanes.
__global__ void k_loss_final(const double *__restrict__ part, int blocks, int64_t count, double *__restrict__ loss) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double sum = 0.0;
    for (int b = threadIdx.x; b < blocks; b += 32) sum += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (threadIdx.x == 0) *loss = sum / (double)count;
}

// The 2-channel input convolution, direct: a warp takes 8 consecutive
// pixels of an image row, lane = output channel n0 + lane (coalesced
// stores); the 3 x 10 input neighbourhood of the 8 pixels is read once per
// warp (broadcast loads), the BF16 weights [k][n] sit in shared memory as
// floats; per pixel 18 products accumulated in FP32 in (tap, c) order, then
// the bias, z (FP32, if kept) and y = SiLU(z) (BF16).  Grid: x over 64-pixel
// blocks of an image row, y over image rows (b, y) with a stride loop, z over
// groups of 32 output channels.
constexpr int kInCh = 2;
constexpr int kInK = 9 * kInCh;
constexpr int kInPx = 8;  // pixels per warp
__global__ void __launch_bounds__(256) k_conv_in_fwd(const bf16 *__restrict__ x, int B, int H, int W,
                                                     const bf16 *__restrict__ wb, int Co, int Kp,
                                                     const float *__restrict__ bias, float *__restrict__ z,
                                                     bf16 *__restrict__ y) {
    __shared__ float wsm[kInK][32];
    const int n0 = blockIdx.z * 32, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kInK * 32; t += blockDim.x) {
        const int k = t / 32, n = n0 + t % 32;
        wsm[k][t % 32] = n < Co ? __bfloat162float(wb[(int64_t)n * Kp + k]) : 0.f;
    }
    __syncthreads();
    const int x0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kInPx;
    if (x0 >= W) return;
    const int n = n0 + lane;
    float wr[kInK];
#pragma unroll
    for (int k = 0; k < kInK; ++k) wr[k] = wsm[k][lane];
    const float bn = n < Co ? bias[n] : 0.f;
    for (int row = blockIdx.y; row < B * H; row += gridDim.y) {
        const int b = row / H, yy = row - b * H;
        float nb[3][kInPx + 2][kInCh];  // the neighbourhood, columns x0 - 1 .. x0 + 8
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            int sy = yy + dy - 1;
            sy = sy < 0 ? sy + H : (sy >= H ? sy - H : sy);
            const bf16 *rowp = x + ((int64_t)b * H + sy) * W * kInCh;
#pragma unroll
            for (int q = 0; q < kInPx + 2; ++q) {
                int sx = x0 + q - 1;
                sx = sx < 0 ? sx + W : (sx >= W ? sx - W : sx);
                const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(rowp + sx * kInCh);
                nb[dy][q][0] = __low2float(v);
                nb[dy][q][1] = __high2float(v);
            }
        }
#pragma unroll
        for (int px = 0; px < kInPx; ++px) {
            if (x0 + px >= W) break;
            float acc = 0.f;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                acc = __fmaf_rn(nb[tap / 3][px + tap % 3][0], wr[tap * kInCh], acc);
                acc = __fmaf_rn(nb[tap / 3][px + tap % 3][1], wr[tap * kInCh + 1], acc);
            }
            if (n < Co) {
                const int64_t p = (int64_t)row * W + x0 + px;
                const float zz = acc + bn;
                if (z) z[p * Co + n] = zz;
                y[p * Co + n] = __float2bfloat16_rn(zz * sigmoidf_(zz));
            }
        }
    }
}

// Weight gradient of the input convolution, block partials:
// partial[blk][n * 18 + k] = sum over the block's image rows and their pixels
// of dz[p][n] x[p shifted by tap k / 2][k % 2].  Per image row the block
// stages the three source rows with their circular halo (FP32) and the row's
// dz for its 32 output channels (FP32) in shared memory; thread t takes
// channel n0 + t % 32 and k = t / 32, t / 32 + 8, t / 32 + 16 (< 18) and runs
// over the row's pixels in order.  k_colsum_final sums the blocks.
__global__ void __launch_bounds__(256) k_conv_in_wgrad(const bf16 *__restrict__ dz, const bf16 *__restrict__ x, int B,
                                                       int H, int W, int Co, int rows_per_blk,
                                                       float *__restrict__ partial) {
    extern __shared__ float sm_in[];
    float *xs = sm_in;                          // [3][W + 2][2]
    float *dzs = sm_in + 3 * (W + 2) * kInCh;   // [W][32]
    const int nl = threadIdx.x & 31, kg = threadIdx.x >> 5;
    const int n0 = blockIdx.y * 32, n = n0 + nl;
    float acc[3] = {0.f, 0.f, 0.f};
    int off[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int k = kg + 8 * j < kInK ? kg + 8 * j : 0;
        const int tap = k / kInCh;
        off[j] = ((tap / 3) * (W + 2) + tap % 3) * kInCh + k % kInCh;  // + px * kInCh
    }
    const int r0 = blockIdx.x * rows_per_blk;
    const int r1 = min(B * H, r0 + rows_per_blk);
    for (int r = r0; r < r1; ++r) {
        const int b = r / H, yy = r % H;
        __syncthreads();  // the previous row's reads are done
        for (int i = threadIdx.x; i < 3 * (W + 2) * kInCh; i += blockDim.x) {
            const int c = i % kInCh, col = (i / kInCh) % (W + 2), dy = i / (kInCh * (W + 2));
            const int sy = (yy + dy - 1 + H) % H, sx = (col - 1 + W) % W;
            xs[i] = __bfloat162float(x[(((int64_t)b * H + sy) * W + sx) * kInCh + c]);
        }
        for (int i = threadIdx.x; i < W * 32; i += blockDim.x) {
            const int px = i / 32, c = n0 + i % 32;
            dzs[i] = c < Co ? __bfloat162float(dz[(((int64_t)b * H + yy) * W + px) * Co + c]) : 0.f;
        }
        __syncthreads();
        for (int px = 0; px < W; ++px) {
            const float d = dzs[px * 32 + nl];
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[j] = __fmaf_rn(d, xs[off[j] + px * kInCh], acc[j]);
        }
    }
    if (n >= Co) return;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (kg + 8 * j < kInK) partial[(int64_t)blockIdx.x * Co * kInK + n * kInK + kg + 8 * j] = acc[j];
}

// dd1[p][c] = sum_o dout[p][o] Wh[o][c]
__global__ void k_head_dx(const float *__restrict__ dout, const float *__restrict__ Wh, int64_t P, int C, int O,
                          float *__restrict__ dd1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    const int64_t p = i / C;
    const int c = (int)(i % C);
    float acc = 0.f;
    for (int o = 0; o < O; ++o) acc += dout[p * O + o] * Wh[o * C + c];
    dd1[i] = acc;
}

// per-block partial sums of dout[p][o] * d1[p][c] (o-major, then dout[p][o]) for the head gradients
__global__ void k_head_dw_partial(const float *__restrict__ dout, const bf16 *__restrict__ d1, int64_t P, int C, int O,
                                  int64_t rows_per_blk, float *__restrict__ partial) {
    const int j = threadIdx.x + blockIdx.y * blockDim.x;  // 0 .. O*C + O - 1
    const int nj = O * C + O;
    if (j >= nj) return;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
    const int64_t r1 = r0 + rows_per_blk < P ? r0 + rows_per_blk : P;
    float acc = 0.f;
    if (j < O * C) {
        const int o = j / C, c = j % C;
        for (int64_t r = r0; r < r1; ++r) acc += dout[r * O + o] * __bfloat162float(d1[r * C + c]);
    } else {
        const int o = j - O * C;
        for (int64_t r = r0; r < r1; ++r) acc += dout[r * O + o];
    }
    partial[(int64_t)blockIdx.x * nj + j] = acc;
}


__global__ void k_unpad_grad(const float *__restrict__ c, int Co, int K9, int Kp, float *__restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)Co * K9) return;
    g[i] = c[(i / K9) * Kp + i % K9];
}

// AdamW on the FP32 master weights.  The coefficients arrive from the host,
// where 1 - beta and the bias corrections 1 - beta^t are formed in double and
// rounded once (1 - fl32(0.999) would be 1.3e-5 away from 0.001).
__global__ void k_adamw(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, int64_t count, float lr, float b1, float b2, float omb1, float omb2,
                        float eps, float wd, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
}

}  // namespace

// ================================================================ host
struct ensf_unet {
    ensf_unet_config cfg;
    ensf::TcContext *tc = nullptr;
    int sms = 0;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    int64_t nparams = 0;
    int64_t step = 0;
    struct Conv {
        int ci, co, kp, res;  // res: resolution level 0..3
        int64_t w_off, b_off; // offsets in the flat parameter vector
        bf16 *wb, *wt;        // BF16 weights [co][kp] and [kp][co]
        bf16 *wf;             // BF16 weights of the data gradient [ci][9][co], taps mirrored
        float *z;             // pre-activation [P][co]
        bf16 *y;              // activation [P][co]
        const bf16 *in;       // input activation [P][ci]
    } conv[kConvs];
    int64_t head_w_off, head_b_off;
    float *params, *grads, *adam_m, *adam_v;
    float *xin32;              // input NHWC FP32 [P0][2]
    bf16 *xin16;               // input NHWC BF16
    bf16 *pool[kLevels];       // pooled activations at levels 1..3
    bf16 *cat[kLevels];        // decoder concat buffers (levels 2, 1, 0)
    float *out;                // prediction NCHW
    float *dout;               // loss gradient NHWC [P0][2]
    double *loss;              // device scalar
    int *err;                  // device error word of the GEMM launches (ENSF_ETIMEOUT on an expired wait)
    // scratch
    bf16 *col, *colT, *dz16, *dzT;
    bf16 *xpad;                // a convolution's input with its circular halo (implicit GEMM)
    float *gemm_c, *partial, *ga, *gb, *colsum_part;
    double *loss_part;         // block partials of the loss
    float *gskip[kLevels];     // gradients of the encoder outputs (skips), levels 0..2
    int64_t partial_cap = 0;
};

namespace {

struct Arena {
    char *base;
    size_t off = 0;
    template <class T> T *take(int64_t count) {
        size_t o = off;
        off = (off + sizeof(T) * (size_t)count + 255) / 256 * 256;
        return base ? reinterpret_cast<T *>(base + o) : nullptr;
    }
};

bool unet_cfg_ok(const ensf_unet_config *c) {
    if (!c || c->in_ch != 2 || c->out_ch != 2 || c->max_batch < 1) return false;
    if (c->height < 16 || c->width < 16 || c->height % 8 || c->width % 8) return false;
    for (int w : {c->widths[0], c->widths[1], c->widths[2], c->widths[3]})
        if (w < 8 || w % 8 || w > 1024) return false;
    return true;
}

int64_t round8(int64_t v) { return (v + 7) / 8 * 8; }

// Lays out every buffer; with a null base only measures.
size_t unet_layout(ensf_unet *u, const ensf_unet_config *c, char *base) {
    Arena a{base};
    const int w1 = c->widths[0], w2 = c->widths[1], w3 = c->widths[2], w4 = c->widths[3];
    const int cin_[kConvs] = {2, w1, w1, w2, w2, w3, w3, w4, w4 + w3, w3, w3 + w2, w2, w2 + w1, w1};
    const int cout_[kConvs] = {w1, w1, w2, w2, w3, w3, w4, w4, w3, w3, w2, w2, w1, w1};
    const int res_[kConvs] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
    const int64_t P0 = (int64_t)c->max_batch * c->height * c->width;
    auto P = [&](int r) { return P0 >> (2 * r); };
    int64_t off = 0, max_colk = 0, max_c = 0, max_chan = 0;
    for (int l = 0; l < kConvs; ++l) {
        ensf_unet::Conv &cv = u->conv[l];
        cv.ci = cin_[l];
        cv.co = cout_[l];
        cv.kp = (int)round8(9 * cv.ci);
        cv.res = res_[l];
        cv.w_off = off;
        off += 9 * (int64_t)cv.ci * cv.co;
        cv.b_off = off;
        off += cv.co;
        max_colk = std::max<int64_t>(max_colk, P(cv.res) * cv.kp);
        max_c = std::max<int64_t>(max_c, std::max<int64_t>(P(cv.res) * cv.co, P(cv.res) * cv.kp));
        max_chan = std::max<int64_t>(max_chan, P(cv.res) * std::max(cv.ci, cv.co));
    }
    u->head_w_off = off;
    off += 2 * (int64_t)w1;
    u->head_b_off = off;
    off += 2;
    u->nparams = off;
    u->params = a.take<float>(off);
    u->grads = a.take<float>(off);
    u->adam_m = a.take<float>(off);
    u->adam_v = a.take<float>(off);
    for (int l = 0; l < kConvs; ++l) {
        ensf_unet::Conv &cv = u->conv[l];
        cv.wb = a.take<bf16>((int64_t)cv.co * cv.kp);
        cv.wt = a.take<bf16>((int64_t)cv.co * cv.kp);
        cv.wf = a.take<bf16>((int64_t)cv.co * 9 * cv.ci);
        cv.z = a.take<float>(P(cv.res) * cv.co);
        cv.y = a.take<bf16>(P(cv.res) * cv.co);
    }
    u->xin32 = a.take<float>(P0 * 2);
    u->xin16 = a.take<bf16>(P0 * 2);
    u->pool[0] = a.take<bf16>(P(1) * w1);
    u->pool[1] = a.take<bf16>(P(2) * w2);
    u->pool[2] = a.take<bf16>(P(3) * w3);
    u->cat[0] = a.take<bf16>(P(2) * (w4 + w3));
    u->cat[1] = a.take<bf16>(P(1) * (w3 + w2));
    u->cat[2] = a.take<bf16>(P(0) * (w2 + w1));
    u->out = a.take<float>(P0 * 2);
    u->dout = a.take<float>(P0 * 2);
    u->loss = a.take<double>(1);
    u->loss_part = a.take<double>(kLossBlocks);
    u->err = a.take<int>(4);
    {
        int64_t mx = 0;
        for (int l = 0; l < kConvs; ++l) {
            const ensf_unet::Conv &cv = u->conv[l];
            const int64_t hp = (c->height >> cv.res) + 2, wp = (c->width >> cv.res) + 2;
            mx = std::max<int64_t>(mx, (int64_t)c->max_batch * hp * wp * std::max(cv.ci, cv.co));
        }
        u->xpad = a.take<bf16>(mx);
    }
    u->col = a.take<bf16>(max_colk);
    u->colT = a.take<bf16>(max_colk);
    u->dz16 = a.take<bf16>(max_chan);
    u->dzT = a.take<bf16>(max_chan);
    u->gemm_c = a.take<float>(max_c);
    u->ga = a.take<float>(max_chan);
    u->gb = a.take<float>(max_chan);
    u->gskip[0] = a.take<float>(P(0) * w1);
    u->gskip[1] = a.take<float>(P(1) * w2);
    u->gskip[2] = a.take<float>(P(2) * w3);
    // block partials: bias sums (<= 1024 channels), head weights (2 w1 + 2),
    // the input convolution's weights (18 w1)
    u->colsum_part = a.take<float>((int64_t)kColsumBlocks * std::max(std::max(1024, 2 * w1 + 2), kInK * w1));
    u->partial_cap = std::max<int64_t>(max_c, (int64_t)64 << 20);
    u->partial = a.take<float>(u->partial_cap);
    // inputs of the convolutions
    if (base) {
        u->conv[0].in = u->xin16;
        for (int l = 1; l < kConvs; ++l) u->conv[l].in = u->conv[l - 1].y;
        u->conv[2].in = u->pool[0];
        u->conv[4].in = u->pool[1];
        u->conv[6].in = u->pool[2];
        u->conv[8].in = u->cat[0];
        u->conv[10].in = u->cat[1];
        u->conv[12].in = u->cat[2];
    }
    return a.off;
}

ensf_status unet_fail(ensf_status s, const char *m) {
    ensf::set_last_error(m);
    return s;
}

#define UNET_CUDA(call)                                                       \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return unet_fail(ENSF_ECUDA, #call);           \
    } while (0)
#define UNET_LAUNCH()                                                         \
    do {                                                                      \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) return unet_fail(ENSF_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

// C[M][N] (FP32) = A[M][K] B[N][K]^T on the tcgen05 GEMM (split-K partials summed in order).
ensf_status gemm(ensf_unet *u, const bf16 *A, const bf16 *B, int64_t M, int64_t N, int64_t K, float *C,
                 cudaStream_t s) {
    ensf::TcGramArgs g;
    g.zb_hi = A;
    g.zb_lo = nullptr;
    g.xb_hi = B;
    g.xb_lo = nullptr;
    g.n = (int)M;
    g.n_x = (int)N;
    g.d = K;
    g.split3 = false;
    g.partial = u->partial;
    g.partial_cap = u->partial_cap;
    g.err = u->err;
    g.noise = nullptr;
    g.seed = 0;
    g.offset = 0;
    g.noise_k = 0;
    int splits = 0, ldp = 0;
    int64_t ps = 0;
    cudaError_t e = ensf::launch_gram_tc(u->tc, g, u->sms, &splits, &ps, &ldp, s);
    if (e != cudaSuccess) return unet_fail(ENSF_ECUDA, "unet gemm launch");
    k_reduce_splits<<<nb(M * N), 256, 0, s>>>(u->partial, splits, M * N, C);
    UNET_LAUNCH();
    return ENSF_OK;
}

// keep_z: store the FP32 pre-activations the backward pass reads (an
// inference forward of the implicit-GEMM convolutions skips them).
ensf_status forward(ensf_unet *u, const float *x_nchw, int B, bool keep_z, cudaStream_t s) {
    const int H = u->cfg.height, W = u->cfg.width;
    const int w1 = u->cfg.widths[0], w2 = u->cfg.widths[1], w3 = u->cfg.widths[2], w4 = u->cfg.widths[3];
    const int64_t P0 = (int64_t)B * H * W;
    k_nchw_to_nhwc<<<nb(P0 * 2), 256, 0, s>>>(x_nchw, B, 2, H, W, u->xin32, u->xin16);
    UNET_LAUNCH();
    auto conv = [&](int l) -> ensf_status {
        ensf_unet::Conv &cv = u->conv[l];
        const int h = H >> cv.res, w = W >> cv.res;
        const int64_t P = (int64_t)B * h * w;
        if (ensf::conv3x3_supported(cv.ci, cv.co, h, w, (int)P)) {
            // implicit GEMM: the haloed input, then one kernel with bias + SiLU in its epilogue
            pad_circ(cv.in, B, h, w, cv.ci, u->xpad, s);
            UNET_LAUNCH();
            if (ensf::launch_conv3x3(u->tc, u->xpad, cv.ci, B, h, w, cv.wb, cv.co, u->params + cv.b_off, 1,
                                     keep_z ? cv.z : nullptr, cv.y, u->err, s) != cudaSuccess)
                return unet_fail(ENSF_ECUDA, "unet implicit convolution launch");
            return ENSF_OK;
        }
        if (cv.ci == kInCh) {
            // the 2-channel input convolution: 18 products per output, direct
            k_conv_in_fwd<<<dim3(nb(w, 8 * kInPx), (unsigned)std::min(B * h, 65535), (cv.co + 31) / 32), 256, 0,
                            s>>>(
                cv.in, B, h, w, cv.wb, cv.co, cv.kp, u->params + cv.b_off, keep_z ? cv.z : nullptr, cv.y);
            UNET_LAUNCH();
            return ENSF_OK;
        }
        k_im2col<<<nb(P * cv.kp), 256, 0, s>>>(cv.in, B, h, w, cv.ci, cv.kp, u->col);
        UNET_LAUNCH();
        ensf_status st = gemm(u, u->col, cv.wb, P, cv.co, cv.kp, u->gemm_c, s);
        if (st != ENSF_OK) return st;
        k_bias_silu<<<nb(P * cv.co), 256, 0, s>>>(u->gemm_c, u->params + cv.b_off, P, cv.co, cv.z, cv.y);
        UNET_LAUNCH();
        return ENSF_OK;
    };
    auto pool = [&](const bf16 *x, int res, int C, bf16 *y) -> ensf_status {
        k_pool_fwd<<<nb((int64_t)B * (H >> (res + 1)) * (W >> (res + 1)) * C), 256, 0, s>>>(x, B, H >> res, W >> res,
                                                                                            C, y);
        UNET_LAUNCH();
        return ENSF_OK;
    };
    auto upcat = [&](const bf16 *low, const bf16 *skip, int res, int Cl, int Cs, bf16 *out) -> ensf_status {
        k_up_concat_fwd<<<nb((int64_t)B * (H >> res) * (W >> res) * ((Cl + Cs) / 8)), 256, 0, s>>>(
            low, skip, B, H >> res, W >> res, Cl, Cs, out);
        UNET_LAUNCH();
        return ENSF_OK;
    };
    ensf_status st;
#define STEP(x)                 \
    if ((st = (x)) != ENSF_OK) \
        return st;
    STEP(conv(0)) STEP(conv(1)) STEP(pool(u->conv[1].y, 0, w1, u->pool[0]))
    STEP(conv(2)) STEP(conv(3)) STEP(pool(u->conv[3].y, 1, w2, u->pool[1]))
    STEP(conv(4)) STEP(conv(5)) STEP(pool(u->conv[5].y, 2, w3, u->pool[2]))
    STEP(conv(6)) STEP(conv(7)) STEP(upcat(u->conv[7].y, u->conv[5].y, 2, w4, w3, u->cat[0]))
    STEP(conv(8)) STEP(conv(9)) STEP(upcat(u->conv[9].y, u->conv[3].y, 1, w3, w2, u->cat[1]))
    STEP(conv(10)) STEP(conv(11)) STEP(upcat(u->conv[11].y, u->conv[1].y, 0, w2, w1, u->cat[2]))
    STEP(conv(12)) STEP(conv(13))
#undef STEP
    k_head_fwd<<<nb(P0), 256, 0, s>>>(u->conv[13].y, u->xin32, u->params + u->head_w_off, u->params + u->head_b_off, B,
                                      H, W, w1, 2, u->out);
    UNET_LAUNCH();
    return ENSF_OK;
}

// Backward pass of one convolution: dy [P][co] -> gradients of W, b and (+)= dx [P][ci].
ensf_status conv_back(ensf_unet *u, int l, int B, const float *dy, float *dx, int accumulate, cudaStream_t s) {
    ensf_unet::Conv &cv = u->conv[l];
    const int h = u->cfg.height >> cv.res, w = u->cfg.width >> cv.res;
    const int64_t P = (int64_t)B * h * w;
    {
        // dZ and the bias gradient (column sums of dZ) in one pass
        // dZ, its transpose for the weight-gradient GEMMs (when a block's rows
        // fit in shared memory) and the bias gradient (column sums) in one pass
        const int blocks = (int)std::min<int64_t>(kColsumBlocks, P);  // enough blocks at every level
        const int64_t rows = (P + blocks - 1) / blocks;
        const int64_t tbytes = rows * (std::min(cv.co, 256) + 2) * (int64_t)sizeof(bf16);
        const bool fused_t = tbytes <= kSiluTransposeSmem;
        k_silu_back_colsum<<<dim3(blocks, (cv.co + 255) / 256), 256, fused_t ? (size_t)tbytes : 0, s>>>(
            dy, cv.z, P, cv.co, rows, u->dz16, u->colsum_part, fused_t ? u->dzT : nullptr);
        k_colsum_final<<<(cv.co + 3) / 4, 128, 0, s>>>(u->colsum_part, blocks, cv.co, u->grads + cv.b_off);
        UNET_LAUNCH();
        if (!fused_t) {
            k_transpose_bf16<<<dim3((cv.co + 31) / 32, (unsigned)((P + 31) / 32)), dim3(32, 8), 0, s>>>(
                u->dz16, P, cv.co, u->dzT);
            UNET_LAUNCH();
        }
    }
    ensf_status st;
    if (cv.ci == kInCh) {
        // the input convolution's 18 x co weight gradient: block partials of the
        // pixel sums, then a fixed-order sum over the blocks
        const int rows = (B * h + kColsumBlocks - 1) / kColsumBlocks;  // image rows per block
        const int blocks = (B * h + rows - 1) / rows;
        const int smem = (3 * (w + 2) * kInCh + w * 32) * (int)sizeof(float);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k_conv_in_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return unet_fail(ENSF_ECUDA, "unet input-convolution weight gradient: shared memory");
        k_conv_in_wgrad<<<dim3(blocks, (cv.co + 31) / 32), 256, smem, s>>>(u->dz16, cv.in, B, h, w, cv.co, rows,
                                                                           u->colsum_part);
        k_colsum_final<<<(cv.co * kInK + 3) / 4, 128, 0, s>>>(u->colsum_part, blocks, cv.co * kInK,
                                                              u->grads + cv.w_off);
        UNET_LAUNCH();
    } else if (ensf::conv3x3_wgrad_supported(cv.ci, cv.co, h, w, (int)P)) {
        // weight gradient as nine implicit GEMMs over the pixels: dZ^T against
        // the input's column-shifted, transposed copies (held in the im2col
        // scratch, which is 9 * P * ci >= 3 * B * (h + 2) * w * ci long)
        if (ensf::launch_shift3_transpose(cv.in, B, h, w, cv.ci, u->col, s) != cudaSuccess ||
            ensf::launch_conv3x3_wgrad(u->tc, u->dzT, u->col, B, h, w, cv.ci, cv.co, u->partial, u->partial_cap,
                                       u->grads + cv.w_off, u->err, s) != cudaSuccess)
            return unet_fail(ENSF_ECUDA, "unet implicit weight-gradient launch");
    } else {
        // weight gradient: dZ^T [co][P] x col^T [kp][P]
        k_im2col<<<nb(P * cv.kp), 256, 0, s>>>(cv.in, B, h, w, cv.ci, cv.kp, u->col);
        UNET_LAUNCH();
        k_transpose_bf16<<<dim3((cv.kp + 31) / 32, (unsigned)((P + 31) / 32)), dim3(32, 8), 0, s>>>(u->col, P, cv.kp,
                                                                                                  u->colT);
        UNET_LAUNCH();
        st = gemm(u, u->dzT, u->colT, cv.co, cv.kp, P, u->gemm_c, s);
        if (st != ENSF_OK) return st;
        k_unpad_grad<<<nb((int64_t)cv.co * 9 * cv.ci), 256, 0, s>>>(u->gemm_c, cv.co, 9 * cv.ci, cv.kp,
                                                                   u->grads + cv.w_off);
        UNET_LAUNCH();
    }
    if (!dx) return ENSF_OK;
    if (!accumulate && ensf::conv3x3_supported(cv.co, cv.ci, h, w, (int)P)) {
        // the data gradient as the same implicit-GEMM convolution of the haloed dZ with mirrored taps
        pad_circ(u->dz16, B, h, w, cv.co, u->xpad, s);
        UNET_LAUNCH();
        if (ensf::launch_conv3x3(u->tc, u->xpad, cv.co, B, h, w, cv.wf, cv.ci, nullptr, 0, dx, nullptr, u->err, s) !=
            cudaSuccess)
            return unet_fail(ENSF_ECUDA, "unet implicit convolution launch (data gradient)");
        return ENSF_OK;
    }
    // data gradient: dZ [P][co] x W^T [kp][co] -> dcol [P][kp] -> col2im
    st = gemm(u, u->dz16, cv.wt, P, cv.kp, cv.co, u->gemm_c, s);
    if (st != ENSF_OK) return st;
    k_col2im<<<nb(P * cv.ci), 256, 0, s>>>(u->gemm_c, B, h, w, cv.ci, cv.kp, dx, accumulate);
    UNET_LAUNCH();
    return ENSF_OK;
}

// Launches one of a kernel's two index-type forms over `count` elements:
// 32-bit indices where they suffice (their divisions are cheaper).
template <class K32, class K64, class... A>
void launch_vec(int64_t count, cudaStream_t s, K32 k32, K64 k64, A... args) {
    if (count < ((int64_t)1 << 31))
        k32<<<nb(count), 256, 0, s>>>(args...);
    else
        k64<<<nb(count), 256, 0, s>>>(args...);
}

ensf_status backward(ensf_unet *u, const float *target, int B, cudaStream_t s) {
    const int H = u->cfg.height, W = u->cfg.width;
    const int w1 = u->cfg.widths[0], w2 = u->cfg.widths[1], w3 = u->cfg.widths[2], w4 = u->cfg.widths[3];
    const int64_t P0 = (int64_t)B * H * W;
    auto P = [&](int r) { return P0 >> (2 * r); };
    k_mse_grad<<<kLossBlocks, 256, 0, s>>>(u->out, target, B, 2, H, W, u->dout, u->loss_part);
    k_loss_final<<<1, 32, 0, s>>>(u->loss_part, kLossBlocks, P0 * 2, u->loss);
    UNET_LAUNCH();
    // head
    {
        const int nj = 2 * w1 + 2;
        const int blocks = (int)std::min<int64_t>(1024, (P0 + 255) / 256);
        const int64_t rows = (P0 + blocks - 1) / blocks;
        k_head_dw_partial<<<dim3(blocks, (nj + 127) / 128), 128, 0, s>>>(u->dout, u->conv[13].y, P0, w1, 2, rows,
                                                                         u->colsum_part);
        k_colsum_final<<<(nj + 3) / 4, 128, 0, s>>>(u->colsum_part, blocks, nj, u->grads + u->head_w_off);
        k_head_dx<<<nb(P0 * w1), 256, 0, s>>>(u->dout, u->params + u->head_w_off, P0, w1, 2, u->ga);
        UNET_LAUNCH();
    }
    ensf_status st;
#define STEP(x)                 \
    if ((st = (x)) != ENSF_OK) \
        return st;
    // decoder level 0: convs 13, 12 (input = cat[2] = [up(d2) w2, e1 w1])
    STEP(conv_back(u, 13, B, u->ga, u->gb, 0, s))
    STEP(conv_back(u, 12, B, u->gb, u->ga, 0, s))   // ga = d cat[2] [P0][w2+w1]
    UNET_CUDA(cudaMemsetAsync(u->gskip[0], 0, sizeof(float) * P(0) * w1, s));
    launch_vec(P(0) * w1 / 4, s, k_skip_bwd<uint32_t>, k_skip_bwd<int64_t>, u->ga, P(0), w2, w1, u->gskip[0]);
    launch_vec(P(1) * w2 / 4, s, k_up_bwd<uint32_t>, k_up_bwd<int64_t>, u->ga, B, H, W, w2, w1, u->gb);  // gb = d d2 [P1][w2]
    UNET_LAUNCH();
    // decoder level 1: convs 11, 10 (input = cat[1] = [up(d3) w3, e2 w2])
    STEP(conv_back(u, 11, B, u->gb, u->ga, 0, s))
    STEP(conv_back(u, 10, B, u->ga, u->gb, 0, s))   // gb = d cat[1] [P1][w3+w2]
    UNET_CUDA(cudaMemsetAsync(u->gskip[1], 0, sizeof(float) * P(1) * w2, s));
    launch_vec(P(1) * w2 / 4, s, k_skip_bwd<uint32_t>, k_skip_bwd<int64_t>, u->gb, P(1), w3, w2, u->gskip[1]);
    launch_vec(P(2) * w3 / 4, s, k_up_bwd<uint32_t>, k_up_bwd<int64_t>, u->gb, B, H >> 1, W >> 1, w3, w2, u->ga);  // ga = d d3 [P2][w3]
    UNET_LAUNCH();
    // decoder level 2: convs 9, 8 (input = cat[0] = [up(m) w4, e3 w3])
    STEP(conv_back(u, 9, B, u->ga, u->gb, 0, s))
    STEP(conv_back(u, 8, B, u->gb, u->ga, 0, s))    // ga = d cat[0] [P2][w4+w3]
    UNET_CUDA(cudaMemsetAsync(u->gskip[2], 0, sizeof(float) * P(2) * w3, s));
    launch_vec(P(2) * w3 / 4, s, k_skip_bwd<uint32_t>, k_skip_bwd<int64_t>, u->ga, P(2), w4, w3, u->gskip[2]);
    launch_vec(P(3) * w4 / 4, s, k_up_bwd<uint32_t>, k_up_bwd<int64_t>, u->ga, B, H >> 2, W >> 2, w4, w3, u->gb);  // gb = d m [P3][w4]
    UNET_LAUNCH();
    // middle: convs 7, 6; then back through the pool into e3
    STEP(conv_back(u, 7, B, u->gb, u->ga, 0, s))
    STEP(conv_back(u, 6, B, u->ga, u->gb, 0, s))    // gb = d pool[2] [P3][w3]
    launch_vec(P(2) * w3 / 4, s, k_pool_bwd<uint32_t>, k_pool_bwd<int64_t>, u->gb, B, H >> 2, W >> 2, w3, u->gskip[2], 1);
    UNET_LAUNCH();
    STEP(conv_back(u, 5, B, u->gskip[2], u->ga, 0, s))
    STEP(conv_back(u, 4, B, u->ga, u->gb, 0, s))    // gb = d pool[1] [P2][w2]
    launch_vec(P(1) * w2 / 4, s, k_pool_bwd<uint32_t>, k_pool_bwd<int64_t>, u->gb, B, H >> 1, W >> 1, w2, u->gskip[1], 1);
    UNET_LAUNCH();
    STEP(conv_back(u, 3, B, u->gskip[1], u->ga, 0, s))
    STEP(conv_back(u, 2, B, u->ga, u->gb, 0, s))    // gb = d pool[0] [P1][w1]
    launch_vec(P(0) * w1 / 4, s, k_pool_bwd<uint32_t>, k_pool_bwd<int64_t>, u->gb, B, H, W, w1, u->gskip[0], 1);
    UNET_LAUNCH();
    STEP(conv_back(u, 1, B, u->gskip[0], u->ga, 0, s))
    STEP(conv_back(u, 0, B, u->ga, nullptr, 0, s))
#undef STEP
    return ENSF_OK;
}

// Every convolution's BF16 weight copies from the FP32 master weights
// W [co][9 ci] in one launch (a layer table passed by value): the elements
// [0, total_b) are Wb [co][kp] (zero padded past 9 ci) and its transpose
// Wt [kp][co], layer after layer; [total_b, total) the weights of the data
// gradient, wf[c][tap'][n] = W[n][8 - tap'][c] (taps mirrored, so that the
// gradient is the same implicit-GEMM convolution).
struct RepackTable {
    const float *w[kConvs];
    bf16 *wb[kConvs], *wt[kConvs], *wf[kConvs];
    int co[kConvs], ci[kConvs], kp[kConvs];
    int64_t end_b[kConvs], end_f[kConvs];  // running element ends of the two parts
};

__global__ void __launch_bounds__(256) k_repack_all(RepackTable t) {
    const int64_t total_b = t.end_b[kConvs - 1], total = total_b + t.end_f[kConvs - 1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < total_b) {
            int l = 0;
            while (i >= t.end_b[l]) ++l;
            const int64_t e = i - (l ? t.end_b[l - 1] : 0);
            const int Kp = t.kp[l], K9 = 9 * t.ci[l], Co = t.co[l];
            const int o = (int)(e / Kp), k = (int)(e % Kp);
            const bf16 v = __float2bfloat16_rn(k < K9 ? t.w[l][(int64_t)o * K9 + k] : 0.f);
            t.wb[l][e] = v;
            t.wt[l][(int64_t)k * Co + o] = v;
        } else {
            const int64_t j = i - total_b;
            int l = 0;
            while (j >= t.end_f[l]) ++l;
            const int64_t e = j - (l ? t.end_f[l - 1] : 0);
            const int Co = t.co[l], Ci = t.ci[l];
            const int n = (int)(e % Co), tap = (int)((e / Co) % 9), c = (int)(e / ((int64_t)9 * Co));
            t.wf[l][e] = __float2bfloat16_rn(t.w[l][((int64_t)n * 9 + (8 - tap)) * Ci + c]);
        }
    }
}

ensf_status repack(ensf_unet *u, cudaStream_t s) {
    RepackTable t;
    int64_t eb = 0, ef = 0;
    for (int l = 0; l < kConvs; ++l) {
        const ensf_unet::Conv &cv = u->conv[l];
        t.w[l] = u->params + cv.w_off;
        t.wb[l] = cv.wb;
        t.wt[l] = cv.wt;
        t.wf[l] = cv.wf;
        t.co[l] = cv.co;
        t.ci[l] = cv.ci;
        t.kp[l] = cv.kp;
        eb += (int64_t)cv.co * cv.kp;
        ef += (int64_t)cv.co * 9 * cv.ci;
        t.end_b[l] = eb;
        t.end_f[l] = ef;
    }
    k_repack_all<<<(unsigned)std::min<int64_t>(nb(eb + ef), 152 * 8), 256, 0, s>>>(t);
    UNET_LAUNCH();
    return ENSF_OK;
}

}  // namespace

extern "C" {

int64_t ensf_unet_param_count(const ensf_unet_config *cfg) {
    if (!unet_cfg_ok(cfg)) return 0;
    ensf_unet tmp;
    unet_layout(&tmp, cfg, nullptr);
    return tmp.nparams;
}

size_t ensf_unet_workspace_bytes(const ensf_unet_config *cfg) {
    if (!unet_cfg_ok(cfg)) return 0;
    ensf_unet tmp;
    return unet_layout(&tmp, cfg, nullptr);
}

ensf_status ensf_unet_create(const ensf_unet_config *cfg, void *workspace, size_t ws_bytes, ensf_unet **out) {
    if (!out) return unet_fail(ENSF_EINVAL, "ensf_unet_create: out is NULL");
    *out = nullptr;
    if (!unet_cfg_ok(cfg)) return unet_fail(ENSF_EINVAL, "ensf_unet_create: invalid configuration");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return unet_fail(ENSF_EINVAL, "ensf_unet_create: workspace must be 256-byte aligned");
    ensf_unet *u = new (std::nothrow) ensf_unet;
    if (!u) return unet_fail(ENSF_ENOMEM, "ensf_unet_create: host allocation failed");
    u->cfg = *cfg;
    const size_t need = unet_layout(u, cfg, static_cast<char *>(workspace));
    if (ws_bytes < need) {
        delete u;
        return unet_fail(ENSF_ENOMEM, "ensf_unet_create: workspace too small");
    }
    u->ws = static_cast<char *>(workspace);
    u->ws_bytes = ws_bytes;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        delete u;
        return unet_fail(ENSF_ECUDA, "ensf_unet_create: device query failed");
    }
    if (!(prop.major == 10 && prop.minor == 3)) {
        delete u;
        return unet_fail(ENSF_EUNSUPPORTED, "ensf_unet_create: needs an sm_103 device");
    }
    u->sms = prop.multiProcessorCount;
    if (ensf::tc_context_create(&u->tc) != cudaSuccess) {
        delete u;
        return unet_fail(ENSF_ECUDA, "ensf_unet_create: tensor-map encoder unavailable");
    }
    if (cudaMemset(u->adam_m, 0, sizeof(float) * u->nparams) != cudaSuccess ||
        cudaMemset(u->adam_v, 0, sizeof(float) * u->nparams) != cudaSuccess ||
        cudaMemset(u->loss, 0, sizeof(double)) != cudaSuccess || cudaMemset(u->err, 0, 4 * sizeof(int)) != cudaSuccess) {
        ensf::tc_context_destroy(u->tc);
        delete u;
        return unet_fail(ENSF_ECUDA, "ensf_unet_create: cudaMemset failed");
    }
    *out = u;
    return ENSF_OK;
}

ensf_status ensf_unet_set_params(ensf_unet *u, const float *params, void *stream) {
    if (!u || !params) return unet_fail(ENSF_EINVAL, "ensf_unet_set_params: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    UNET_CUDA(cudaMemcpyAsync(u->params, params, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice, s));
    UNET_CUDA(cudaMemsetAsync(u->adam_m, 0, sizeof(float) * u->nparams, s));
    UNET_CUDA(cudaMemsetAsync(u->adam_v, 0, sizeof(float) * u->nparams, s));
    u->step = 0;
    return repack(u, s);
}

ensf_status ensf_unet_get_params(ensf_unet *u, float *params, void *stream) {
    if (!u || !params) return unet_fail(ENSF_EINVAL, "ensf_unet_get_params: bad arguments");
    UNET_CUDA(cudaMemcpyAsync(params, u->params, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice,
                              static_cast<cudaStream_t>(stream)));
    return ENSF_OK;
}

ensf_status ensf_unet_get_moments(ensf_unet *u, float *m, float *v, int64_t *step, void *stream) {
    if (!u || !m || !v) return unet_fail(ENSF_EINVAL, "ensf_unet_get_moments: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    UNET_CUDA(cudaMemcpyAsync(m, u->adam_m, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice, s));
    UNET_CUDA(cudaMemcpyAsync(v, u->adam_v, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice, s));
    if (step) *step = u->step;
    return ENSF_OK;
}

ensf_status ensf_unet_forward(ensf_unet *u, const float *x, int batch, float *y, void *stream) {
    if (!u || !x || !y || batch < 1 || batch > u->cfg.max_batch)
        return unet_fail(ENSF_EINVAL, "ensf_unet_forward: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensf_status st = forward(u, x, batch, false, s);
    if (st != ENSF_OK) return st;
    UNET_CUDA(cudaMemcpyAsync(y, u->out, sizeof(float) * (size_t)batch * 2 * u->cfg.height * u->cfg.width,
                              cudaMemcpyDeviceToDevice, s));
    return ENSF_OK;
}

ensf_status ensf_unet_gradients(ensf_unet *u, const float *x, const float *target, int batch, float *grads,
                                double *loss, void *stream) {
    if (!u || !x || !target || batch < 1 || batch > u->cfg.max_batch)
        return unet_fail(ENSF_EINVAL, "ensf_unet_gradients: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensf_status st = forward(u, x, batch, true, s);
    if (st == ENSF_OK) st = backward(u, target, batch, s);
    if (st != ENSF_OK) return st;
    if (grads)
        UNET_CUDA(cudaMemcpyAsync(grads, u->grads, sizeof(float) * u->nparams, cudaMemcpyDeviceToDevice, s));
    if (loss) UNET_CUDA(cudaMemcpyAsync(loss, u->loss, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return ENSF_OK;
}

ensf_status ensf_unet_train_step(ensf_unet *u, const float *x, const float *target, int batch, float lr,
                                 float weight_decay, double *loss, void *stream) {
    ensf_status st = ensf_unet_gradients(u, x, target, batch, nullptr, loss, stream);
    if (st != ENSF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    u->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)u->step)), c2 = (float)(1.0 - std::pow(b2, (double)u->step));
    k_adamw<<<nb(u->nparams), 256, 0, s>>>(u->params, u->grads, u->adam_m, u->adam_v, u->nparams, lr, (float)b1,
                                          (float)b2, (float)(1.0 - b1), (float)(1.0 - b2), 1e-8f, weight_decay, c1,
                                          c2);
    UNET_LAUNCH();
    return repack(u, s);
}

ensf_status ensf_unet_destroy(ensf_unet *u) {
    if (!u) return ENSF_EINVAL;
    ensf::tc_context_destroy(u->tc);
    delete u;
    return ENSF_OK;
}

}  // extern "C"
