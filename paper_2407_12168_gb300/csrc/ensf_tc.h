// ensf_tc.h -- tensor-core (tcgen05 + TMA + TMEM) stages of the analysis
// step on sm_103a.  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "ensf_device.cuh"

namespace ensf {

struct TcContext;  // tensor-map encoder and per-shape launch choices

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
};

struct TcWxArgs {
    const __nv_bfloat16 *wb_hi, *wb_lo;  // weights   [n][ldw]  (lo NULL for plain BF16)
    const __nv_bfloat16 *xt_hi, *xt_lo;  // forecast transposed [d][ldw]
    int ldw;                             // row pitch (elements) of W and X^T, >= n, multiple of 8
    int n;
    int64_t d;
    float *z;                            // particles [n][d], updated in place
    __nv_bfloat16 *zb_hi, *zb_lo;        // split copies of the updated particles (NULL: skip)
    const float *y;
    const uint8_t *mask;
    const float *noise_buf;
    uint64_t seed;
    uint32_t offset;
    StepCoef coef;
    int *err;
};

cudaError_t launch_gram_tc(TcContext *ctx, const TcGramArgs &a, int sms, int *splits,
                           int64_t *part_stride, int *ldp, cudaStream_t s);
cudaError_t launch_wx_em_tc(TcContext *ctx, const TcWxArgs &a, int sms, cudaStream_t s);

}  // namespace ensf
