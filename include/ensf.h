/*
 * ensf.h -- C ABI of the GB300-native EnSF analysis step.
 *
 * The ensemble score filter (EnSF) analysis of Bao et al., "A Scalable
 * Real-Time Data Assimilation Framework for Predicting Turbulent Atmosphere
 * Dynamics" (Sec. III-A): every particle z_i starts from N(0, I) at pseudo-time
 * t = 1 and runs K Euler-Maruyama steps of the reverse-time SDE (Eq. 7),
 *
 *   z <- z - dt (b(t) z - sigma^2(t) s(z, t)) + sqrt(sigma^2(t) dt) xi,
 *
 * with the posterior score of Eq. 17, s = s_prior + h(t) grad log P(y | z):
 *
 *   s_prior(z_i) = -sum_j w_ij (z_i - alpha_t x_j) / beta_t^2        (Eq. 15)
 *   w_ij = softmax_j(-|z_i - alpha_t x_j|^2 / (2 beta_t^2))          (Eq. 12, 16)
 *   grad log P(y | z) = mask * H'(z) (y - H(z)) / sigma_obs^2         (Eq. 5)
 *
 * Schedule (Eq. 9): alpha_t = 1 - t(1 - eps), beta_t^2 = t,
 * b = d log(alpha)/dt, sigma^2 = d(beta^2)/dt - 2 b beta^2; damping
 * h(t) = 1 - t (Eq. 11); grid t_k = 1 - k/K, k = 0..K-1, dt = 1/K.
 *
 * Conventions shared by every entry point:
 *  - All array pointers are DEVICE pointers unless stated otherwise; the
 *    caller owns them.  Arrays are row-major and densely packed.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; no entry point synchronises the host
 *    except ensf_status_sync.
 *  - Argument errors are reported before anything is enqueued.  Device-side
 *    errors are recorded in an error word inside the workspace and returned
 *    (and cleared) by ensf_status_sync.
 *  - The library never allocates device memory: scratch lives in the
 *    caller-provided workspace.
 */
#ifndef ENSF_H
#define ENSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ENSF_OK = 0,
    ENSF_EINVAL = 1,        /* bad argument (NULL/misaligned pointer, size out of range) */
    ENSF_ENOMEM = 2,        /* workspace smaller than ensf_workspace_bytes() */
    ENSF_ECUDA = 3,         /* a CUDA runtime call failed */
    ENSF_ENUMERIC = 4,      /* a non-finite value was produced (when checking is on) */
    ENSF_ETIMEOUT = 5,      /* a bounded device-side wait expired */
    ENSF_EUNSUPPORTED = 6   /* configuration not supported on this device */
} ensf_status;

/* Observation operator H of Eq. 2, applied elementwise. */
typedef enum {
    ENSF_OBS_IDENTITY = 0,  /* H(z) = z,         H'(z) = 1           */
    ENSF_OBS_ARCTAN = 1     /* H(z) = arctan(z), H'(z) = 1/(1 + z^2) */
} ensf_obs_op;

/* Arithmetic of the two contractions of each Euler-Maruyama step. */
typedef enum {
    ENSF_PREC_FP32 = 0,        /* CUDA-core FP32 for the Gram Z X^T and for W X */
    ENSF_PREC_SPLIT_BF16X3 = 1 /* tensor cores: each operand split a = a_hi + a_lo in BF16,
                                  products a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32 accumulate */,
    ENSF_PREC_BF16 = 2,        /* tensor cores: one BF16 product, FP32 accumulate */
    ENSF_PREC_TF32 = 3         /* Gram only: tensor cores (kind::tf32) on the FP32 centred operands
                                  read directly (the MMA uses their TF32 part), FP32 accumulate */
} ensf_precision;

#define ENSF_FLAG_CHECK_FINITE 1u  /* scan the final particles for NaN/Inf */
#define ENSF_FLAG_INLINE_NOISE 4u  /* tensor-core W X: evaluate the Philox noise inside its epilogue
                                      instead of reading a slice pre-generated during the Gram */
#define ENSF_FLAG_CUDA_GRAPH 2u    /* ensf_analysis captures its whole launch sequence (all K
                                      Euler-Maruyama steps) into one CUDA graph and launches that;
                                      the instantiated graph is kept in the handle and updated in
                                      place when only scalars or pointers change.  Ignored on the
                                      legacy default stream and inside a caller's own capture. */
#define ENSF_FLAG_WX_UNSTAGED 16u  /* tensor-core BF16 W X with the noise evaluated in its epilogue:
                                      use the epilogue that reads and writes the particles with
                                      per-thread global accesses instead of the TMA-staged one (the
                                      same arithmetic and results; kept for comparison) */
#define ENSF_FLAG_PERSISTENT 8u    /* FP32 precisions and n <= 128: the K Euler-Maruyama steps run in
                                      one cooperative launch (one block per SM, three bounded grid
                                      barriers per step) instead of three launches per step; for
                                      small filters, whose step costs less than a kernel launch.
                                      Other configurations ignore the flag. */

typedef struct {
    int max_n;        /* largest ensemble size N this handle will run (>= 1)          */
    int64_t max_d;    /* largest state dimension d (>= 8, multiple of 8)               */
    int gram;         /* ensf_precision of the Gram cross term Z X^T (Eq. 12, 16)     */
    int wx;           /* ensf_precision of the weighted sum W X (Eq. 15)              */
    unsigned flags;   /* ENSF_FLAG_* */
} ensf_config;

/* Gaussian noise xi[k][i][j], k = 0..K (slice 0 = the initial particles,
 * slice k+1 = the noise of Euler-Maruyama step k). */
typedef struct {
    const float *buf;   /* [K+1][n][d] FP32 device buffer, or NULL: use the
                           counter-based stream below, computed inside the kernels */
    uint64_t seed;      /* Philox4x32-10 key (Salmon et al., SC'11)                */
    uint32_t offset;    /* fourth counter word (e.g. the assimilation cycle)       */
} ensf_noise;

typedef struct ensf_handle ensf_handle;

/* Bytes of device workspace a handle with this configuration needs. Returns 0
 * for an invalid configuration. */
size_t ensf_workspace_bytes(const ensf_config *cfg);

/* Create a handle over a caller-owned device workspace (256-byte aligned, at
 * least ensf_workspace_bytes(cfg) bytes, kept alive until ensf_destroy).
 * Host memory for the handle itself is allocated here.  Returns ENSF_ENOMEM
 * if ws_bytes is too small, ENSF_EUNSUPPORTED if a tensor-core precision is
 * requested on a device that is not sm_103. */
ensf_status ensf_create(const ensf_config *cfg, void *workspace, size_t ws_bytes,
                        ensf_handle **out);

/* The analysis step (Sec. III-A.2, Eq. 7 and 15-17).
 *   prior     [n][d] FP32  forecast ensemble x_j (read only; must not alias out)
 *   y         [d]    FP32  observations (entries where mask = 0 are ignored)
 *   obs_mask  [d]    uint8 1 = observed, or NULL = every point observed
 *   obs_op    ensf_obs_op
 *   sigma_obs > 0          R = sigma_obs^2 I
 *   K >= 1                 Euler-Maruyama steps on the grid t_k = 1 - k/K
 *   eps in (0, 1)          alpha_t = 1 - t(1 - eps)
 *   noise                  see ensf_noise (host struct; may not be NULL)
 *   out       [n][d] FP32  the analysis ensemble (particles after K steps)
 * Pointers must be 16-byte aligned; 1 <= n <= max_n; 8 <= d <= max_d and
 * d % 8 == 0.  Enqueued on `stream`. */
ensf_status ensf_analysis(ensf_handle *h, const float *prior, int n, int64_t d, const float *y,
                          const uint8_t *obs_mask, int obs_op, float sigma_obs, int K, float eps,
                          const ensf_noise *noise, float *out, void *stream);

/* Launch shapes chosen by ensf_autotune. */
typedef struct {
    int gram_tile_n;   /* Gram output tile width (forecast members per tile)          */
    int gram_stages;   /* shared-memory ring depth of the Gram                        */
    int gram_splits;   /* split-K slices over the state dimension                     */
    float gram_ms;     /* measured time of one Gram launch with that shape            */
    int wx_tile_n;     /* W X tile width (particles per tile)                         */
    float wx_ms;       /* measured time of one W X launch with that shape            */
    int gram_k_block;  /* Gram k-block width in elements (64 or 32)                   */
    int gram_cta_pair; /* 1: Gram tiles of 256 x 256 on a cluster of two CTAs         */
    int gram_noise_warps; /* warps of a Gram CTA generating the next step's noise (8 or 4) */
    int gram_fp32_particles; /* 1 (pair tiles only): the Gram reads the FP32 particles and splits
                                them itself, so the W X step writes no BF16 particle planes */
    int noise_inline;  /* where the counter-based draws are made when both stages run on the tensor
                          cores: 0 = written to a slice by the Gram's spare warps while its MMAs
                          run, 1 = evaluated in the W X epilogue, 2 = written to the slice by a
                          kernel on a low-priority side stream that runs beside the Gram and the
                          softmax (the draws are the same in all three) */
    int pdl;           /* 1: the per-step kernels (Gram, row softmax, W X) are launched with
                          programmatic dependent launch (each may start while its predecessor
                          finishes, and waits for it on the device), 0: ordinary launches.
                          Untuned shapes use it while n * d <= 2^24.  For ensf_set_tuning,
                          -1 keeps the current choice. */
    int gram_fused_softmax; /* 1 (pair tiles only): the row softmax runs in the Gram's epilogue -- the
                               last of a block's split-K CTAs sums the partials and forms the block's
                               log-kernels, the last block of a 128-row band normalises the band --
                               instead of a separate launch; the weights are bit-identical. */
} ensf_tuning;

/* Autotuner for the tensor-core stages: times the candidate launch shapes of
 * the Gram (tile width, ring depth, split count) and of W X (tile width) on
 * these operands (same arguments as ensf_analysis, without K) and records the
 * fastest for this (n, d) in the handle; later analyses of that shape use it.
 * When both stages run on the tensor cores with counter-based noise (no noise
 * buffer, no ENSF_FLAG_INLINE_NOISE), it tunes the shapes with the draws in
 * the Gram and in the W X epilogue, keeps the one with the smaller Gram +
 * softmax + W X time, and then compares it with the side-stream placement on
 * short whole analyses (noise_inline).
 * It then times whole steps with and without programmatic dependent launch
 * (pdl) and keeps the faster.
 * Overwrites `out` and the workspace, synchronises `stream`, and must not be
 * called while the stream is being captured.  `report` may be NULL.  A handle
 * with only CUDA-core precisions returns ENSF_OK with a zeroed report. */
ensf_status ensf_autotune(ensf_handle *h, const float *prior, int n, int64_t d, const float *y,
                          const uint8_t *obs_mask, int obs_op, float sigma_obs, float eps,
                          const ensf_noise *noise, float *out, ensf_tuning *report, void *stream);

/* Records launch shapes for analyses of this (n, d) without timing them,
 * e.g. a report saved from ensf_autotune in another process.  Uses the
 * gram_tile_n, gram_stages, gram_splits (0: the cost model), gram_k_block,
 * gram_cta_pair, gram_noise_warps, gram_fp32_particles, wx_tile_n
 * (0: unchanged), noise_inline (0, 1 or 2) and pdl (-1: unchanged) fields
 * of `t`.  Valid Gram shapes (tile width, ring depth, k-block) for the
 * split-BF16x3 Gram: (128, 3, 64), (256, 2, 64), (128, 6, 32), (256, 4, 32),
 * (256, 3, 32), and with gram_cta_pair = 1 (256, 3, 64) when n is a multiple
 * of 256 (optionally with gram_fp32_particles = 1); for the BF16 Gram:
 * (128, 6, 64), (256, 4, 64), (128, 12, 32), (256, 8, 32); for the TF32
 * Gram: (128, 6, 32), (256, 4, 32), and with gram_cta_pair = 1 (256, 6, 32)
 * when n is a multiple of 256.  EINVAL for any other shape or placement, for
 * n or d outside the handle's limits, or for a handle whose Gram runs on
 * CUDA cores. */
ensf_status ensf_set_tuning(ensf_handle *h, int n, int64_t d, const ensf_tuning *t);

/* One filter of a batched analysis. */
typedef struct {
    const float *prior;        /* [n][d] forecast ensemble (device)                 */
    int n;                     /* ensemble size, 1 <= n <= 8192                     */
    int64_t d;                 /* state dimension, multiple of 8                    */
    const float *y;            /* [d] observations                                  */
    const uint8_t *obs_mask;   /* [d] or NULL                                       */
    int obs_op;                /* ensf_obs_op                                       */
    float sigma_obs;           /* > 0                                               */
    ensf_noise noise;          /* per-filter noise (buffer [K+1][n][d] or Philox)   */
    float *out;                /* [n][d] analysis ensemble (device)                 */
} ensf_instance;

/* Device workspace a batched analysis of these instances needs with the
 * handle configuration `cfg` (0 if a precision is not a tensor-core one). */
size_t ensf_batch_workspace_bytes(const ensf_config *cfg, const ensf_instance *inst, int count);

/* Independent analyses (Sec. III-A.2) of `count` filters with uneven n and d
 * in one launch per stage: each Euler-Maruyama step is one batched Gram over
 * the tiles of all filters, one batched row softmax and one persistent batched
 * W X + score + update; all filters share K and eps.  Tensor-core precisions
 * only (ENSF_EUNSUPPORTED otherwise).  `workspace` (256-byte aligned, at least
 * ensf_batch_workspace_bytes) holds the per-filter scratch and the tile and
 * descriptor tables; the tables are uploaded from a page-locked host buffer
 * owned by the handle (allocated on the first batched call; the call waits
 * for the previous batched call's upload before reusing it).  With
 * ENSF_FLAG_CUDA_GRAPH the whole batched analysis is one CUDA graph. */
ensf_status ensf_analysis_batched(ensf_handle *h, const ensf_instance *inst, int count, int K, float eps,
                                  void *workspace, size_t ws_bytes, void *stream);

/* Autotuner of the batched analysis: times short batched analyses (K = 8,
 * same arguments otherwise; overwrites each instance's `out`) with 8, 16, 32
 * and 64 k-blocks of 64 state columns per Gram work item (the split-K range
 * of one 128 x 128 tile) and keeps the fastest in the handle for later
 * batched analyses.  *kb_chunk and *ms (either may be NULL) receive the
 * choice and the time of its K = 8 analysis.  Synchronises `stream`; not
 * while it is being captured (EINVAL).  The workspace must be sized by
 * ensf_batch_workspace_bytes (which covers every candidate). */
ensf_status ensf_autotune_batched(ensf_handle *h, const ensf_instance *inst, int count, float eps, void *workspace,
                                  size_t ws_bytes, int *kb_chunk, float *ms, void *stream);

/* Records the k-range per batched Gram work item without timing (8, 16, 32
 * or 64 k-blocks; the default is 32).  EINVAL otherwise. */
ensf_status ensf_set_batch_tuning(ensf_handle *h, int kb_chunk);

/* The analysis with the mini-batch prior score of Eq. 15-16 (J < N members
 * per evaluation): `perm` (device int32 [n]) is a permutation of the forecast
 * members, drawn by the caller; Euler-Maruyama step k uses the J members
 * perm[w J .. w J + J - 1], w = k mod (n / J), for every particle, with the
 * weights normalised over those J.  The Gram and W X cost drop by n / J.
 * J must divide n and be a multiple of 8 (or equal n).  Tensor-core
 * precisions only; other arguments as ensf_analysis. */
ensf_status ensf_analysis_minibatch(ensf_handle *h, const float *prior, int n, int64_t d, const float *y,
                                    const uint8_t *obs_mask, int obs_op, float sigma_obs, int K, float eps,
                                    const ensf_noise *noise, const int *perm, int J, float *out, void *stream);

/* ---- d-sharded analysis -------------------------------------------------
 * One filter whose state is split along d across ranks (the paper runs the
 * EnSF of one large state on many GPUs, Sec. III-A.3 and the weak-scaling
 * study of Sec. IV-B).  Every term of an Euler-Maruyama step but one is local
 * to a block of state columns: H is elementwise and R diagonal, so the
 * likelihood score, W X and the update (Eq. 7, 15, 17) need only this rank's
 * columns.  The exception is the Gram cross term z_i . x_j of the log-kernel
 * (Eq. 12, 16) and the squared norms |x_j - m|^2, sums over all of d: each
 * rank computes its columns' share, the ranks exchange them, and every rank
 * then forms the same weights.  The library holds no communicator: the
 * caller moves the shares between the calls below (e.g. an all-reduce of the
 * norms once per analysis and an all-gather of the split-K partial Grams once
 * per step), and the library never waits for another rank.
 *
 * Per analysis, on each rank:
 *   ensf_shard_prep(h, sh, norms)            this slice's norm shares -> norms [n] FP64
 *   (caller: norms <- sum over ranks of norms)
 *   for k = 0 .. K-1:
 *     ensf_shard_gram(h, sh, k, partial)     this slice's S split-K partial Grams
 *                                            -> partial [S][n][n] FP32
 *     (caller: gathered [R*S][n][n] <- the R ranks' partials in rank order)
 *     ensf_shard_update(h, sh, k, gathered, R*S, norms)
 *                                            softmax over all R*S partials (fixed order),
 *                                            then W X + score + update of this slice
 * The counter-based noise is drawn at global state columns col0 + c, so the
 * sharded analysis draws exactly the numbers of the unsharded one; with equal
 * split boundaries (each slice a whole number of the unsharded analysis's
 * split-K ranges) its Gram partials are the unsharded ones, bit for bit.
 * The handle's max_d bounds d_local; the other ensf_analysis argument rules
 * apply to the slice (16-byte alignment, d_local % 8 == 0).  The persistent
 * small-filter mode does not apply (ENSF_EUNSUPPORTED). */
typedef struct {
    const float *prior;        /* [n][d_local] this rank's columns of the forecast ensemble */
    int n;                     /* ensemble size (the same on every rank)                     */
    int64_t d_local;           /* columns held by this rank                                  */
    int64_t col0;              /* global index of the first of them                          */
    const float *y;            /* [d_local] observations of these columns                    */
    const uint8_t *obs_mask;   /* [d_local], or NULL = all observed                          */
    int obs_op;                /* ensf_obs_op                                                */
    float sigma_obs;           /* > 0                                                        */
    int K;                     /* Euler-Maruyama steps                                       */
    float eps;                 /* in (0, 1)                                                  */
    ensf_noise noise;          /* buf: [K+1][n][d_local] these columns' draws, or NULL: Philox */
    float *out;                /* [n][d_local] these columns of the particles                */
} ensf_shard;

/* Number S of split-K partial Grams ensf_shard_gram writes for (n, d_local)
 * with the handle's current shape for that size (set with ensf_set_tuning to
 * line the slices up with another run's split boundaries). */
ensf_status ensf_shard_splits(ensf_handle *h, int n, int64_t d_local, int *splits);

/* Preparation of one analysis on this slice: centre, split planes, the
 * initial particles (out) and this slice's shares of the FP64 squared norms
 * |x_j - m|^2, written to norms (device, n doubles, caller-owned). */
ensf_status ensf_shard_prep(ensf_handle *h, const ensf_shard *sh, double *norms, void *stream);

/* Step k, first half: this slice's split-K partial Grams (z_i - alpha m) .
 * (x_j - m) to partial (device, [S][n][n] FP32, S from ensf_shard_splits,
 * 16-byte aligned); also draws the step's noise where the tuning puts it. */
ensf_status ensf_shard_gram(ensf_handle *h, const ensf_shard *sh, int k, float *partial, void *stream);

/* Step k, second half: weights from all ranks' partials (partials: device
 * [splits_total][n][n] FP32, summed in index order) and the all-reduced norms
 * (device, n doubles), then W X, score and update of this slice's particles.
 * After step K-1, `out` holds this slice of the analysis ensemble. */
ensf_status ensf_shard_update(ensf_handle *h, const ensf_shard *sh, int k, const float *partials, int splits_total,
                              const double *norms, void *stream);

/* Normalised weights w_ij of Eq. 16 for given particles z [n][d] at pseudo-
 * time t, against the forecast ensemble prior [n_x][d], written to
 * w [n][n_x] FP32.  Uses the handle's Gram precision; this is the Gram +
 * log-sum-exp stage of one analysis step exposed on its own. */
ensf_status ensf_weights(ensf_handle *h, const float *z, int n, const float *prior, int n_x,
                         int64_t d, float t, float eps, float *w, void *stream);

/* Allocation-free variant of ensf_weights (FP32 Gram), for callers that may
 * not allocate device memory: applications whose own memory pool owns every
 * device allocation, and loops that must never reach an allocation that could
 * synchronise the device.  The paper has no counterpart; this is a property
 * of the library, not of the method.  It needs no handle and no workspace:
 * its scratch (the forecast mean that centres the Gram operands, the row
 * norms and the split-K partial Grams) is one static device array of
 * 4 MiB + 4 KiB that every device loading the library keeps until the
 * process exits.  The Gram runs on the centred operands z - alpha m and
 * x_j - m, as in ensf_weights.  Limits: 1 <= n, n_x <= 256 and d a multiple
 * of 8 in [8, 524288] (else ENSF_EINVAL with a message in ensf_last_error);
 * t in (0, 1].  The first call on a device looks up the array's device
 * address (with that device current), so make that first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.  Each call writes every scratch word it reads, so no state
 * carries between calls. */
ensf_status ensf_weights_static(const float *z, int n, const float *prior, int n_x, int64_t d, float t,
                                float eps, float *w, void *stream);

/* Standalone counter-based noise: out[k - k0][i][j] = xi[k][i][j] for
 * k = k0..k0+count-1, i < n, j < d (the stream used when ensf_noise.buf is
 * NULL). */
ensf_status ensf_philox_normal(uint64_t seed, uint32_t offset, int k0, int count, int n,
                               int64_t d, float *out, void *stream);

/* FP64 squared row norms  out[j] = sum_c x[j][c]^2  of x [n][d]. */
ensf_status ensf_row_norms(const float *x, int n, int64_t d, double *out, void *stream);

/* FP64 ensemble statistics of z [n][d]: mean[c] = (1/n) sum_i z[i][c]
 * (device [d], may be NULL) and, when truth != NULL, the RMSE of that mean
 * against truth [d] written to rmse (device, one double).  Uses `scratch`
 * (device, at least ensf_stats_scratch_bytes(d) bytes). */
size_t ensf_stats_scratch_bytes(int64_t d);
ensf_status ensf_ensemble_stats(const float *z, int n, int64_t d, const float *truth,
                                double *mean, double *rmse, void *scratch, void *stream);

/* Relaxation to the prior used when cycling (Sec. IV-A: the analysis spread
 * is relaxed to the prior (forecast) values), per state variable over the n
 * members (FP64 accumulation), in place on the analysis z [n][d]:
 *   mode 0 (spread):        anomalies rescaled by (1 - factor) + factor s_prior / s_analysis;
 *   mode 1 (perturbations): anomalies (1 - factor) z' + factor x'_prior.
 * factor in [0, 1]; 1 restores the forecast spread (mode 0) or perturbations (mode 1). */
ensf_status ensf_relax_spread(const float *prior, float *z, int n, int64_t d, float factor, int mode,
                              void *stream);

/* Imperfect-model error of the twin experiment (Sec. IV-A: additive
 * Gaussian model errors, uncorrelated in space and white in time, made of
 * several stochastic processes each realised with its own probability and
 * amplitude), in place on state [batch][d] (device FP32):
 *   state[b][j] += sum_{p < nproc} coef[p] * xi_p[b][j],
 * xi_p[b][j] the standard normal of the analysis noise stream (Philox4x32-10
 * + Box-Muller) at (seed, offset = cycle, step index p, particle b, element j).
 * coef: host array of nproc (1..8) floats; the caller folds each process's
 * realisation in this interval (0 or 1), its amplitude and the model's mean
 * value into coef[p].  Errors: EINVAL for NULL pointers, batch < 1, d < 1 or
 * nproc outside 1..8; ECUDA if the launch fails. */
ensf_status ensf_model_error(float *state, int batch, int64_t d, const float *coef, int nproc, uint64_t seed,
                             uint32_t cycle, void *stream);

/* Failure-detection self-test (no counterpart in the paper): runs the two
 * kinds of bounded waits of the library against conditions that never occur
 * and reports how they ended, without faulting or hanging the GPU.
 *   words[0]: a tensor-core pipeline wait on an mbarrier that nothing completes;
 *   words[1]: a grid barrier of the persistent small-filter kernel that one
 *             block leaves without arriving at.
 * words: device, 4 ints, caller-owned (words[2..3] are the barrier's scratch);
 * words[0..1] are zeroed, the two kernels run (about two seconds each), and
 * both should hold ENSF_ETIMEOUT after the stream completes.  The context
 * stays usable.  EINVAL for NULL; ECUDA if a launch fails. */
ensf_status ensf_selftest_timeouts(int *words, void *stream);

/* Launch accounting of a handle.  Every kernel launch is counted by kind
 * ("row_norms", "init_particles", "split_bf16", "gram", "softmax_rows",
 * "wx_em", "check_finite", "noise").  While profiling is on, each launch is also
 * bracketed by a CUDA event pair recorded on the launching stream (at most
 * 16384 pairs; later launches are counted but not timed).  Enabling or
 * disabling clears the counters; the first enable creates the events. */
typedef struct {
    char name[32];
    int64_t launches;        /* launches of this kind since the last enable */
    int64_t timed_launches;  /* of which bracketed by events */
    double total_ms;         /* summed event time of the timed launches */
} ensf_profile_entry;

ensf_status ensf_profile_enable(ensf_handle *h, int on);

/* Waits for the recorded events; writes up to max_entries kinds with at least
 * one launch and sets *count to the number of such kinds. */
ensf_status ensf_profile_read(ensf_handle *h, ensf_profile_entry *out, int max_entries, int *count);

/* ---- Forecast-model companion: the two-level SQG integrator --------------
 * The paper's forecast model (Sec. II-B): nonlinear Eady model on an f-plane
 * with uniform stratification and shear, zero interior PV, the boundary
 * potential temperatures theta (scaled so that d(psi)/dz = theta) advected on
 * the two lids; doubly periodic pseudo-spectral discretisation (cuFFT), RK4,
 * 2/3 dealiasing, hyperdiffusion del^8 applied implicitly after each step.
 * Nondimensional: f = 1, lengths in units of N H / f when N_over_f = H = 1. */
typedef struct {
    int n;            /* grid points per side (even, >= 8)                         */
    double L;         /* domain side                                                */
    double H;         /* depth between the lids                                     */
    double N_over_f;  /* buoyancy frequency / Coriolis parameter                    */
    double shear;     /* Lambda = dU/dz of the mean flow U(z) = Lambda (z - H/2)    */
    double dt;        /* RK4 time step                                              */
    double tau_diss;  /* e-folding time of the hyperdiffusion at the largest wavenumber */
    int diffusion;    /* 0 disables the hyperdiffusion                              */
    double tau_relax; /* Newtonian relaxation time of theta, a large-scale sink (0: none) */
} ensf_sqg_params;

typedef struct ensf_sqg ensf_sqg;

/* Device workspace for `batch` members (0 for invalid parameters).  The cuFFT
 * plans keep their own small plan data; their work area is in the workspace. */
size_t ensf_sqg_workspace_bytes(const ensf_sqg_params *p, int batch);
ensf_status ensf_sqg_create(const ensf_sqg_params *p, int batch, void *workspace, size_t ws_bytes,
                            ensf_sqg **out);
/* Advances theta [batch][2][n][n] FP32 (device; level 0 = bottom) by nsteps
 * RK4 steps, in place, on `stream`. */
ensf_status ensf_sqg_run(ensf_sqg *s, float *theta, int nsteps, void *stream);
ensf_status ensf_sqg_destroy(ensf_sqg *s);

/* ---- Learned forecast surrogate: a conv U-Net trained in BF16 -------------
 * x_{t+Delta} = x_t + net(x_t) on the two-level SQG state [B][2][H][W] (FP32
 * NCHW at the interface).  net: encoder 2->w0->w1->w2->w3 (two 3x3 convs per
 * level, circular padding, SiLU, 2x2 mean pooling), decoder with nearest x2
 * upsampling and skip concatenation back to w0, 1x1 head to 2 channels.  The
 * convolutions run as BF16 GEMMs on the tensor cores (FP32 accumulation);
 * FP32 master weights, AdamW.  Stands in for the paper's ViT (Sec. III-B).
 * Flat parameter order: per conv W [Cout][3][3][Cin] then b [Cout] (encoder,
 * middle, decoder), then head W [2][w0], b [2]. */
typedef struct {
    int in_ch;        /* 2 */
    int out_ch;       /* 2 */
    int widths[4];    /* channel widths per level, multiples of 8            */
    int height, width;/* multiples of 8, >= 16                                */
    int max_batch;
} ensf_unet_config;

typedef struct ensf_unet ensf_unet;

int64_t ensf_unet_param_count(const ensf_unet_config *cfg);
size_t ensf_unet_workspace_bytes(const ensf_unet_config *cfg);
ensf_status ensf_unet_create(const ensf_unet_config *cfg, void *workspace, size_t ws_bytes, ensf_unet **out);
/* Load / read the flat FP32 parameter vector (device); loading resets AdamW. */
ensf_status ensf_unet_set_params(ensf_unet *u, const float *params, void *stream);
ensf_status ensf_unet_get_params(ensf_unet *u, float *params, void *stream);
/* y [B][2][H][W] = surrogate forecast of x [B][2][H][W] (device FP32). */
ensf_status ensf_unet_forward(ensf_unet *u, const float *x, int batch, float *y, void *stream);
/* Mean-squared-error loss against target and its gradient w.r.t. the flat
 * parameters (device FP32 [param_count]; grads or loss may be NULL). */
ensf_status ensf_unet_gradients(ensf_unet *u, const float *x, const float *target, int batch, float *grads,
                                double *loss, void *stream);
/* One AdamW step on that loss (Loshchilov and Hutter, ICLR 2019, Algorithm 2
 * with step size 1 and schedule multiplier lr; beta1 0.9, beta2 0.999,
 * eps 1e-8; t counts the steps since the last ensf_unet_set_params):
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   w -= lr (m / (1 - beta1^t) / (sqrt(v / (1 - beta2^t)) + eps) + weight_decay w),
 * on the FP32 master weights, then the BF16 copies are refreshed; loss
 * (device) may be NULL. */
ensf_status ensf_unet_train_step(ensf_unet *u, const float *x, const float *target, int batch, float lr,
                                 float weight_decay, double *loss, void *stream);
/* Read the AdamW state: first and second moments m, v (device FP32
 * [param_count], same order as the parameters) and, when step != NULL (host),
 * the number of AdamW steps since the last ensf_unet_set_params. */
ensf_status ensf_unet_get_moments(ensf_unet *u, float *m, float *v, int64_t *step, void *stream);
ensf_status ensf_unet_destroy(ensf_unet *u);

/* ---- Page-locked host buffers for the copies of inputs and results -------
 * The analysis's inputs (the forecast ensemble, observations) and its result
 * move between host and device once per analysis.  On a GPU coupled to its
 * host CPU by a coherent link the copy engines reach host memory through
 * address translation; measured on GB300, a 2 GiB buffer pinned page by page
 * (64 KiB pages) was copied at 35-70 GB/s right after an analysis, against
 * about 200 GB/s from a buffer made of huge pages.  ensf_host_alloc returns
 * `bytes` (rounded up to whole huge pages) of page-locked host memory, an
 * anonymous mapping aligned to the transparent-huge-page size and advised and
 * collapsed into huge pages before registration with the CUDA driver (each
 * best effort: where the kernel offers no huge pages the buffer is still
 * page-locked).  Its pages are placed, before the first touch, with a
 * preference for the host NUMA node closest to the current device
 * (cudaDevAttrHostNumaId; on a two-socket host the far socket's memory is
 * reached over the inter-socket link too); a full node falls back to others.
 * flags: 0, or ENSF_HOST_SMALL_PAGES to skip the huge-page advice and
 * ENSF_HOST_ANY_NODE to skip the node preference (for comparisons).  The
 * memory is zeroed.  Release with ensf_host_free.  ENSF_EINVAL (bytes 0, out
 * NULL), ENSF_ENOMEM (mmap), ENSF_ECUDA (registration). */
#define ENSF_HOST_SMALL_PAGES 1u
#define ENSF_HOST_ANY_NODE 2u
ensf_status ensf_host_alloc(size_t bytes, unsigned flags, void **out);
/* Unregister and unmap a buffer of ensf_host_alloc (NULL: no-op). */
ensf_status ensf_host_free(void *ptr);
/* dst <- src (bytes, a multiple of 16; both 16-byte aligned) copied by a
 * kernel of `blocks` blocks on `stream` instead of a copy engine: either side
 * may be device memory or page-locked host memory, which the SMs then read or
 * write over the host link. */
ensf_status ensf_copy_sm(void *dst, const void *src, size_t bytes, int blocks, void *stream);
/* *registered = 1 if ptr lies in host memory page-locked with the CUDA driver
 * (cudaHostRegister or cudaHostAlloc), else 0. */
ensf_status ensf_host_registered(const void *ptr, int *registered);
/* Share of [ptr, ptr + bytes) that the kernel backs with huge pages right
 * now (from /proc/self/smaps; ENSF_EUNSUPPORTED where that is unreadable). */
ensf_status ensf_host_huge_fraction(const void *ptr, size_t bytes, double *fraction);
/* *node = the NUMA node holding the page at ptr (-1 when unknown or not yet
 * touched); *device_node = the host NUMA node closest to the current device
 * (-1 when the system reports none). */
ensf_status ensf_host_numa(const void *ptr, int *node, int *device_node);

/* Wait for `stream` and return the handle's recorded device error, clearing it. */
ensf_status ensf_status_sync(ensf_handle *h, void *stream);

/* Static description of a status code. */
const char *ensf_status_string(ensf_status s);

/* Host-side message of the most recent failing call on this thread ("" if none). */
const char *ensf_last_error(void);

/* Release the handle (the workspace stays the caller's). */
ensf_status ensf_destroy(ensf_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* ENSF_H */
