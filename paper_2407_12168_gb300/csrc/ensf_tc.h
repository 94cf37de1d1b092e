// ensf_tc.h -- tensor-core (tcgen05 + TMA + TMEM) stages of the analysis
// step on sm_103a.  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "ensf_device.cuh"

namespace ensf {

struct TcContext;  // tensor-map encoder and per-shape launch choices

struct GramChoice {
    int bn = 0;      // output tile width (128 or 256 forecast members)
    int stages = 0;  // shared-memory ring depth
    int splits = 0;  // split-K slices over d (0: cost model)
    int bk = 0;      // k-block width: 64 (128-byte swizzle) or 32 (64-byte swizzle); 0 = 64
    int pair = 0;    // 1: a cluster of two CTAs per 256 x 256 tile (tcgen05 cta_group::2)
    int noise_warps = 0;  // warps generating the next step's noise: 8 (default) or 4
    int a_fp32 = 0;       // pair form only: read the FP32 particles and split them in the kernel
    int fused_softmax = 0;  // pair form only: the row softmax in the Gram's epilogue (last arrivers)
};

struct TcTuneReport {
    int gram_bn = 0, gram_stages = 0, gram_splits = 0, gram_bk = 0, gram_pair = 0, gram_noise_warps = 0;
    int gram_a_fp32 = 0;
    float gram_ms = 0.f;
    int wx_bn = 0;
    float wx_ms = 0.f;
    int pdl = -1;        // 1/0: whether programmatic dependent launch made a step faster (-1: not timed)
    float step_ms = 0.f; // one Gram + softmax + W X step with that choice
};

cudaError_t tc_context_create(TcContext **out);
void tc_context_destroy(TcContext *ctx);

// Floats of split-K partial scratch the Gram needs at most for n <= max_n.
int64_t tc_partial_floats(int max_n, int sms);

struct TcGramArgs {
    const __nv_bfloat16 *zb_hi, *zb_lo;  // particles  [n][d]   (lo NULL for plain BF16)
    const __nv_bfloat16 *xb_hi, *xb_lo;  // forecast   [n_x][d]
    int n, n_x;
    int64_t d;
    bool split3;                         // hi*hi + hi*lo + lo*hi
    float *partial;                      // [splits][n][ldp]
    int64_t partial_cap;                 // capacity in floats
    int *err;
    // optional: write the noise slice xi[noise_k] [n][d] of the next step
    // with the otherwise idle epilogue warps (noise NULL: skip)
    float *noise;
    uint64_t seed;
    uint32_t offset;
    int noise_k;
    int64_t noise_col0 = 0;              // global column of column 0 (noise counters are global)
    // the row softmax, fused into the pair Gram's epilogue when the shape
    // uses pair tiles and the tuning asks for it (sm_L NULL: never)
    void *sm_L = nullptr;                // [n][n_x] pairs of floats
    float4 *sm_stats = nullptr;          // [n][ceil(n_x / 256)]
    int *sm_cnt = nullptr;               // zeroed arrival counters
    const double *sm_norms = nullptr;
    double sm_alpha = 0.0, sm_inv_2beta2 = 0.0;
    float *sm_w = nullptr;
    int sm_ldw = 0;
    __nv_bfloat16 *sm_w_hi = nullptr, *sm_w_lo = nullptr;
    int sm_ldwb = 0;
    bool *sm_done = nullptr;             // out: true if this launch also computed the weights
    // the FP32 particles [n][d] and the centre, for the form that splits
    // z - alpha * centre itself (NULL: only the BF16 planes are available)
    const float *z32 = nullptr;
    const float *centre = nullptr;
    float alpha = 0.f;
    // TF32 Gram (kind::tf32): FP32 centred operands z - alpha m [n][d] and
    // x - m [n_x][d] instead of BF16 planes
    bool tf32 = false;
    const float *zc32 = nullptr, *xc32 = nullptr;
    bool pdl = false;                    // launch with programmatic stream serialization
};

struct TcWxArgs {
    const __nv_bfloat16 *wb_hi, *wb_lo;  // weights   [n][ldw]  (lo NULL for plain BF16)
    const __nv_bfloat16 *xt_hi, *xt_lo;  // forecast transposed [d][ldw]
    int ldw;                             // row pitch (elements) of X^T, >= n_x, multiple of 8
    int ldwb;                            // row pitch of W (0: same as ldw)
    int n;
    int n_x;                             // members in the contraction (0: n)
    int64_t d;
    float *z;                            // particles [n][d], updated in place
    __nv_bfloat16 *zb_hi, *zb_lo;        // split copies of the updated particles (NULL: skip)
    float *zc32 = nullptr;               // or the FP32 centred particles (TF32 Gram), NULL: skip
    bool staged = true;                  // in-epilogue noise, BF16: the TMA-staged epilogue
    const float *y;
    const uint8_t *mask;
    const float *noise;                  // xi[k+1] as a [n][d] slice (pre-generated), or NULL:
    uint64_t seed;                       //   Philox stream (seed, offset) evaluated in the epilogue
    uint32_t offset;
    const float *centre;                 // [d] Gram centre m (NULL: none); z_hi/z_lo split z - alpha_next m
    float alpha_next;                    // alpha of the next step's Gram
    StepCoef coef;
    int *err;
    int force_bn = 0;                    // autotuner: particle tile width to use (0: tuned/default)
    bool pdl = false;                    // launch with programmatic stream serialization
};

// ------------------------------------------------------------- batched
// Many independent filters in one launch per stage.  Per-instance tensor
// maps and parameters live in device memory (the batch workspace); the work
// is a list of tiles over all instances.
constexpr int kBatchTileN = 128;   // Gram member tile and W X particle tile of the batched kernels
constexpr int kBatchKbChunk = 32;     // default k-blocks (of 64 state columns) per batched Gram work item
constexpr int kBatchKbChunkMin = 8;   // smallest such k-range the batched autotuner tries

struct BInst {
    int n;                           // particles = forecast members of this filter
    int ldw;                         // row pitch (elements) of the W and X^T planes: n rounded up to 8
    int64_t d;                       // state dimension
    int splits;                      // split-K slices of this instance's Gram
    int kb_chunk;                    // k-blocks per slice (the Gram work item's k-range)
    float *partial;                  // [splits][n][n]
    const double *norms;             // [n] |x_j - m|^2
    __nv_bfloat16 *wb_hi, *wb_lo;    // [n][ldw] weights (lo NULL for plain BF16)
    float *z;                        // [n][d] particles, updated in place
    __nv_bfloat16 *zb_hi, *zb_lo;    // [n][d] split copies for the next Gram
    const float *y;                  // [d]
    const uint8_t *mask;             // [d] or NULL
    const float *centre;             // [d] forecast mean m
    const float *noise_buf;          // [K+1][n][d] caller noise, or NULL: Philox in the kernel
    uint64_t seed;
    uint32_t offset;
    float inv_r;                     // 1 / sigma_obs^2
    int obs_op;
};
struct BGramItem { int inst, m0, n0, split; };  // one 128 x 128 Gram tile over one k-range
struct BWxItem { int inst, m0, n0; };           // 128 state columns x 128 particles
struct BRow { int inst, row; };                 // one softmax row

// Host: encode one 2-D BF16 tensor map (cols contiguous, row pitch `pitch`
// elements, box 64 x box_rows, 128-byte swizzle) into `out` (NULL base: zeroed).
cudaError_t tc_encode_map(TcContext *ctx, void *out128, const void *base, int64_t cols, int64_t rows,
                          int64_t pitch, int box_rows);
cudaError_t launch_gram_tc_batched(const void *maps, const BGramItem *items, int n_items, const BInst *insts,
                                   bool split3, int *err, cudaStream_t s);
cudaError_t launch_softmax_batched(const BRow *rows, int n_rows, const BInst *insts, int max_n, double alpha,
                                   double inv_2beta2, cudaStream_t s);
// staged: BF16 W X with the TMA-staged epilogue (maps: 8 per filter, the
// staging maps of z and its planes at 4, 5, 6; Philox noise only)
cudaError_t launch_wx_em_tc_batched(const void *maps, const BWxItem *items, int n_items, const BInst *insts,
                                    bool split, const StepCoef &cf, float alpha_next, int *err, int sms,
                                    cudaStream_t s, bool staged = false);
// 3x3 convolution with circular padding as an implicit GEMM on the tensor
// cores: out[p][n] = sum_{dy, dx, c} xpad[b][y + dy][x + dx][c] wt[n][(dy * 3 + dx) * C + c]
// (xpad: the BF16 NHWC input with a one-pixel circular halo, B x (h + 2) x (w + 2) x C;
// wt: [N][9 C] BF16).  act = 1: out32 = sum + bias (the pre-activation),
// out16 = SiLU of it; act = 0: out32 = the sum.  Either output may be NULL
// (an inference forward keeps no pre-activation), not both.  conv3x3_supported tells
// which shapes it takes (C a multiple of 32; N a multiple of 32 up to 256, or
// of 64 up to 512; whole image rows per 128-pixel tile).
bool conv3x3_supported(int C, int N, int h, int w, int P);
cudaError_t launch_conv3x3(TcContext *ctx, const __nv_bfloat16 *xpad, int C, int B, int h, int w,
                           const __nv_bfloat16 *wt, int N, const float *bias, int act, float *out32,
                           __nv_bfloat16 *out16, int *err, cudaStream_t s);
// The weight gradient of that convolution, dw[n][tap][c] (FP32, the flat
// parameter layout [N][3][3][C]) = sum_p dZ[p][n] x[p shifted by the tap][c]:
// dzT = dZ^T [N][P] BF16, xs = the input's three column-shifted, transposed,
// row-haloed copies written by launch_shift3_transpose ([3][C][B (h + 2)][w]
// BF16); split-K over the pixels into `partial` (at most partial_cap floats),
// summed in a fixed order.
bool conv3x3_wgrad_supported(int C, int N, int h, int w, int P);
cudaError_t launch_shift3_transpose(const __nv_bfloat16 *x, int B, int h, int w, int C, __nv_bfloat16 *xs,
                                    cudaStream_t s);
cudaError_t launch_conv3x3_wgrad(TcContext *ctx, const __nv_bfloat16 *dzT, const __nv_bfloat16 *xs, int B, int h,
                                 int w, int C, int N, float *partial, int64_t partial_cap, float *dw, int *err,
                                 cudaStream_t s);
// Host: the staging tensor map of the staged W X epilogue (rows x cols of
// esize-byte elements, 128 x 16 boxes, no swizzle) into `out` (NULL base: zeroed).
cudaError_t tc_encode_stage_map(TcContext *ctx, void *out128, const void *base, int esize, int64_t cols,
                                int64_t rows);

cudaError_t launch_gram_tc(TcContext *ctx, const TcGramArgs &a, int sms, int *splits,
                           int64_t *part_stride, int *ldp, cudaStream_t s);
cudaError_t launch_wx_em_tc(TcContext *ctx, const TcWxArgs &a, int sms, cudaStream_t s);

// Times the candidate launch shapes of the Gram (tile width, ring depth,
// split count) and of W X (particle tile width) on these very operands and
// records the fastest per problem shape; later launches of that shape use it.
// Synchronises `s`; either argument may be NULL.
// `after_gram(splits, part_stride, ldp, pdl)` enqueues whatever consumes the
// partials (the row softmax), so that a shape is judged by Gram + reduction.
// With both stages, it also times whole steps with and without programmatic
// dependent launch and reports which was faster (rep->pdl).
using AfterGram = cudaError_t (*)(void *ctx, int splits, int64_t part_stride, int ldp, cudaStream_t s, bool pdl);
// Records a launch shape for (n, n_x, d) as if the autotuner had chosen it
// (wx_bn 0 leaves W X alone).  cudaErrorInvalidValue for a shape that has no
// compiled kernel.
cudaError_t tc_set_tuning(TcContext *ctx, int n, int n_x, int64_t d, bool split3, const GramChoice &g, int wx_bn,
                          bool wx_split, bool tf32 = false);
// Failure-detection self-test: a bounded mbarrier wait that must run out.
cudaError_t launch_selftest_mbar_wait(int *err, cudaStream_t s);
// True when the tuned Gram for this shape reads the FP32 particles (the W X
// epilogue then need not write the BF16 particle planes).
bool tc_gram_reads_fp32(TcContext *ctx, int n, int n_x, int64_t d, bool split3);
// Number of split-K partial Grams launch_gram_tc writes for these arguments
// (with the shape recorded for them, or the default one).
int tc_gram_split_count(TcContext *ctx, const TcGramArgs &a, int sms);
cudaError_t tc_autotune(TcContext *ctx, const TcGramArgs *g, const TcWxArgs *w, int sms, cudaStream_t s,
                        TcTuneReport *rep, AfterGram after_gram = nullptr, void *after_ctx = nullptr);

}  // namespace ensf
