// ensf_internal.h -- launchers shared between the host runtime and the
// kernel translation units.  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "ensf_device.cuh"

namespace ensf {

// Launch `kern`; with `pdl`, with programmatic stream serialization (the
// kernel must begin with pdl_wait(); see ensf_device.cuh).
template <class... KArgs, class... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                     Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

// ---- CUDA-core kernels (ensf_simt.cu) ----------------------------------
// z[i][c] <- xi[0][i][c] (noise buffer or Philox stream; the stream is drawn at
// global column col0 + c)
cudaError_t launch_init_particles(float *z, int n, int64_t d, const float *noise_buf,
                                  uint64_t seed, uint32_t offset, cudaStream_t s, int64_t col0 = 0);
cudaError_t launch_philox_normal(uint64_t seed, uint32_t offset, int k0, int count, int n,
                                 int64_t d, float *out, cudaStream_t s);
// out[i][c] = xi[k][i][col0 + c] (one slice), at most max_blocks blocks of 256 threads
cudaError_t launch_noise_slice(uint64_t seed, uint32_t offset, int k, int n, int64_t d, float *out,
                               int max_blocks, cudaStream_t s, int64_t col0 = 0);
// out[j] = |x_j - centre|^2 in FP64 (centre may be NULL)
// (rows: optional row map, row r of the result reads row rows[r] of x)
cudaError_t launch_row_norms(const float *x, int n, int64_t d, double *out, cudaStream_t s,
                             const float *centre = nullptr, const int *rows = nullptr);
// m[c] = mean over the n rows of x[.][c]
cudaError_t launch_col_mean(const float *x, int n, int64_t d, float *m, cudaStream_t s);
// partial[s][i][j] = sum over slice s of (z[i][c] - alpha m[c]) (x[j][c] - m[c])
// (FP32 CUDA cores; m = centre, NULL for none)
cudaError_t launch_gram_fp32(const float *z, int n, const float *x, int n_x, int64_t d,
                             int splits, float *partial, cudaStream_t s, const float *centre = nullptr,
                             float alpha = 0.0f);
// logits from `splits` partial Grams (row stride ldp) + FP64 norms, row softmax;
// writes W FP32 [n][ldw] and, if w_hi != NULL, BF16 W_hi/W_lo [n][ldwb].
cudaError_t launch_softmax_rows(const float *partial, int splits, int64_t part_stride, int ldp,
                                int n, int n_x, const double *norms, double alpha,
                                double inv_2beta2, float *w, int ldw, __nv_bfloat16 *w_hi,
                                __nv_bfloat16 *w_lo, int ldwb, cudaStream_t s, bool pdl = false);
// The same row softmax in 256-column tiles, one warp per (row, tile): the
// log-kernels go to L ([n][n_x] pairs of floats), the tile statistics to
// stats ([n][ceil(n_x / 256)] float4), rowcnt [n] (zero between launches) counts
// finished tiles per row.  Bit-identical to the softmax fused into the pair Gram.
cudaError_t launch_softmax_tiled(const float *partial, int splits, int64_t part_stride, int ldp, int n, int n_x,
                                 const double *norms, double alpha, double inv_2beta2, void *L, float4 *stats,
                                 int *rowcnt, float *w, int ldw, __nv_bfloat16 *w_hi, __nv_bfloat16 *w_lo, int ldwb,
                                 cudaStream_t s, bool pdl = false);
// z <- EM step with u = W X computed on FP32 CUDA cores, fused epilogue.
cudaError_t launch_wx_em_fp32(const float *w, int ldw, const float *x, int n, int n_x, int64_t d,
                              float *z, const float *y, const uint8_t *mask,
                              const float *noise_buf, uint64_t seed, uint32_t offset,
                              const StepCoef &c, cudaStream_t s);
// FP32 -> (hi, lo) BF16 split of x - scale * centre (centre may be NULL),
// row-major copy with output row stride ldo
cudaError_t launch_split_bf16(const float *x, int rows, int64_t cols, __nv_bfloat16 *hi,
                              __nv_bfloat16 *lo, int64_t ldo, cudaStream_t s,
                              const float *centre = nullptr, float scale = 0.0f, const int *rowmap = nullptr);
// Transposed split: xT_hi[c][j] = bf16(x[j][c]), xT_lo likewise (ldo = row stride of xT)
cudaError_t launch_split_bf16_transpose(const float *x, int rows, int64_t cols,
                                        __nv_bfloat16 *hi, __nv_bfloat16 *lo, int64_t ldo,
                                        cudaStream_t s, const int *rowmap = nullptr);
cudaError_t launch_check_finite(const float *z, int64_t count, int *err_word, cudaStream_t s);
cudaError_t launch_ensemble_stats(const float *z, int n, int64_t d, const float *truth,
                                  double *mean, double *rmse, double *scratch, cudaStream_t s);
int stats_blocks(int64_t d);

// The whole analysis of a small filter (n <= 128, FP32) in one cooperative
// launch; z holds xi_0 on entry.  bar: two zeroed-per-launch words.
cudaError_t launch_analysis_small(const float *x, const double *norms, const float *centre, float *z, const float *y,
                                  const uint8_t *mask, int n, int64_t d, int K, double eps, float inv_r, int obs_op,
                                  const float *noise_buf, uint64_t seed, uint32_t offset, float *partial,
                                  int64_t partial_floats, float *w, unsigned *bar, int *err, int sms,
                                  cudaStream_t s);
cudaError_t launch_selftest_grid_barrier(unsigned *bar, int *err, cudaStream_t s);
cudaError_t launch_centre_copy(const float *x, int rows, int64_t cols, float *out, const float *centre, float scale,
                               const int *rowmap, cudaStream_t s);
cudaError_t launch_model_error(float *state, int batch, int64_t d, const float *coef, int nproc, uint64_t seed,
                               uint32_t cycle, cudaStream_t s);
cudaError_t launch_relax_spread(const float *prior, float *z, int n, int64_t d, float a, int mode, cudaStream_t s);

// Host-side message returned by ensf_last_error() on this thread.
void set_last_error(const char *msg);

}  // namespace ensf
