/*
 * ensf_oracle.c -- plain FP64 CPU oracle of the ensemble score filter (EnSF)
 * analysis step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the package's smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library; the two meet only at the seeded input generators.
 *
 * Every function follows the paper's notation (Bao et al., "A Scalable
 * Real-Time Data Assimilation Framework for Predicting Turbulent Atmosphere
 * Dynamics", Sec. III-A) and is written for obviousness, not speed: the
 * distance in the Gaussian kernel is the direct sum of squared differences,
 * sums run sequentially in double precision, and no term is skipped.
 *
 * Readings taken where the paper is silent or garbled (each also pinned by a
 * test that does not reuse this code):
 *   - schedule  alpha_t = 1 - t(1-eps), beta_t^2 = t (Eq. 9 with the paper's
 *     alpha_t = 1 - t moved off the singular end point t = 1);
 *   - terminal time T = 1, uniform grid t_k = 1 - k/K, k = 0..K-1, explicit
 *     Euler-Maruyama evaluated at t_k, step dt = 1/K;
 *   - damping h(t) = T - t = 1 - t (Eq. 11);
 *   - likelihood  exp(-1/2 (y-H(x))^T R^-1 (y-H(x))), R = sigma_obs^2 I, i.e.
 *     Eq. 5 with the usual one half; unobserved points carry no term;
 *   - weights  w_ij = softmax_j(-|z_i - alpha x_j|^2 / (2 beta^2)) over the
 *     whole forecast ensemble (Eq. 15-16 with the mini-batch J = N);
 *   - particles start at z_i = xi_0,i ~ N(0, I) (Sec. III-A.2, the standard
 *     Gaussian sample at the terminal pseudo-time);
 *   - noise: either a caller buffer xi[K+1][N][d] or Philox4x32-10 (Salmon
 *     et al., SC'11) with Box-Muller, counter (j, i/4, k, offset), evaluated
 *     here in double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Schedule, Eq. 9 and the damping h(t) of Eq. 11.                           */
/* out = {alpha, beta^2, b, sigma^2, h}.                                     */
/* b(t) = d log(alpha_t)/dt, sigma^2(t) = d(beta_t^2)/dt - 2 b(t) beta_t^2.  */
/* ------------------------------------------------------------------------ */
void ensf_oracle_schedule(double t, double eps, double *out)
{
    double alpha = 1.0 - t * (1.0 - eps);
    double dalpha_dt = -(1.0 - eps);
    double beta2 = t;
    double dbeta2_dt = 1.0;
    double b = dalpha_dt / alpha;
    double sigma2 = dbeta2_dt - 2.0 * b * beta2;
    out[0] = alpha;
    out[1] = beta2;
    out[2] = b;
    out[3] = sigma2;
    out[4] = 1.0 - t;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw (SC'11,       */
/* "Parallel random numbers: as easy as 1, 2, 3"): ten rounds of two 32x32   */
/* -> 64-bit multiplies with the Weyl key schedule.                          */
/* ------------------------------------------------------------------------ */
void ensf_oracle_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Standard normal xi[k][i][j] of the counter-based noise stream.
 * Counter = (j, i / 4, k, offset), key = (seed low word, seed high word): one
 * Philox block serves particles 4q..4q+3 of state column j.  Output words
 * (w0, w1) feed one Box-Muller pair for i % 4 in {0, 1} and (w2, w3) the pair
 * for i % 4 in {2, 3}:
 *   u1 = ((w_a >> 8) + 1) 2^-24 in (0, 1],  u2 = (w_b >> 8) 2^-24 in [0, 1),
 *   first  = sqrt(-2 ln u1) cos(2 pi u2),  second = sqrt(-2 ln u1) sin(2 pi u2).
 */
double ensf_oracle_noise(uint64_t seed, uint32_t offset, int k, int i, int64_t j)
{
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(i >> 2), (uint32_t)k, offset};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    ensf_oracle_philox4x32_10(ctr, key, w);
    int lane = i & 3;
    uint32_t wa = (lane < 2) ? w[0] : w[2];
    uint32_t wb = (lane < 2) ? w[1] : w[3];
    double u1 = ((double)(wa >> 8) + 1.0) * (1.0 / 16777216.0);
    double u2 = (double)(wb >> 8) * (1.0 / 16777216.0);
    double radius = sqrt(-2.0 * log(u1));
    double angle = 2.0 * ORACLE_PI * u2;
    return (lane & 1) ? radius * sin(angle) : radius * cos(angle);
}

void ensf_oracle_noise_fill(uint64_t seed, uint32_t offset, int k, int i, int64_t d, double *out)
{
    for (int64_t j = 0; j < d; ++j)
        out[j] = ensf_oracle_noise(seed, offset, k, i, j);
}

/* ------------------------------------------------------------------------ */
/* Observation operator of Eq. 2, elementwise: 0 = identity, 1 = arctan.    */
/* ------------------------------------------------------------------------ */
static double obs_h(int op, double z) { return op == 1 ? atan(z) : z; }
static double obs_dh(int op, double z) { return op == 1 ? 1.0 / (1.0 + z * z) : 1.0; }

/*
 * Likelihood score, the gradient of log P(y | z) of Eq. 5 with the one half
 * and R = sigma_obs^2 I:  g = H'(z) (y - H(z)) / sigma_obs^2 on observed
 * points, 0 elsewhere.  mask == NULL means every point is observed.
 */
void ensf_oracle_lik_score(const double *z, const float *y, const uint8_t *mask, int64_t d,
                           double sigma_obs, int obs_op, double *g)
{
    double inv_r = 1.0 / (sigma_obs * sigma_obs);
    for (int64_t j = 0; j < d; ++j) {
        if (mask && !mask[j]) { g[j] = 0.0; continue; }
        g[j] = obs_dh(obs_op, z[j]) * ((double)y[j] - obs_h(obs_op, z[j])) * inv_r;
    }
}

/*
 * Monte-Carlo weights of Eq. 16 for one particle z against the forecast
 * ensemble X[n][d]:  w_j = Q(z | x_j) / sum_l Q(z | x_l) with the Gaussian
 * kernel of Eq. 12,  log Q(z | x_j) = -|z - alpha x_j|^2 / (2 beta^2) + const.
 * The row maximum is subtracted before exponentiating.  Also returns the
 * log-kernel values in logit[] when logit != NULL.
 */
void ensf_oracle_weights(const float *X, int n, int64_t d, const double *z, double alpha,
                         double beta2, double *w, double *logit)
{
    double *l = logit ? logit : (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
        const float *xj = X + (size_t)j * (size_t)d;
        double dist2 = 0.0;
        for (int64_t c = 0; c < d; ++c) {
            double diff = z[c] - alpha * (double)xj[c];
            dist2 += diff * diff;
        }
        l[j] = -dist2 / (2.0 * beta2);
    }
    double lmax = l[0];
    for (int j = 1; j < n; ++j)
        if (l[j] > lmax) lmax = l[j];
    double total = 0.0;
    for (int j = 0; j < n; ++j) {
        w[j] = exp(l[j] - lmax);
        total += w[j];
    }
    for (int j = 0; j < n; ++j)
        w[j] /= total;
    if (!logit) free(l);
}

/*
 * Monte-Carlo prior score of Eq. 15 with the weights of Eq. 16:
 *   s(z, t) = sum_j -(z - alpha x_j) / beta^2 * w_j.
 * Uses sum_j w_j = 1 only implicitly: the sum is taken term by term.
 */
void ensf_oracle_prior_score(const float *X, int n, int64_t d, const double *z, double alpha,
                             double beta2, double *s)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    ensf_oracle_weights(X, n, d, z, alpha, beta2, w, NULL);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < d; ++c) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j)
            acc += -(z[c] - alpha * (double)X[(size_t)j * (size_t)d + c]) / beta2 * w[j];
        s[c] = acc;
    }
    free(w);
}

/*
 * The analysis step: each selected particle row runs the Euler-Maruyama
 * discretisation of the reverse-time SDE (Eq. 7) with the approximate
 * posterior score of Eq. 17 = prior score (Eq. 15) + h(t) * likelihood score.
 *
 *   X     forecast ensemble [n][d] (the prior sample x_{k|k-1}^j)
 *   y     observations [d];  mask [d] (NULL = all observed)
 *   noise xi[K+1][n][d] FP32 buffer, or NULL to use the Philox stream
 *         ensf_oracle_noise(seed, offset, k, i, j)
 *   rows  particle indices to run (NULL = all n); rows are independent given
 *         (X, y, xi), so any subset is computed exactly
 *   k_stop run steps k = 0..k_stop-1 of the K-step grid (k_stop = K for the
 *         full analysis; fewer only to time a bounded sample)
 *   out   [nrows][d] final particles;  traj optional [k_stop+1][nrows][d]
 *         with the particles before step 0 and after every step.
 *   perm, J mini-batch prior score (Eq. 15-16 with J < N): perm is a
 *         permutation of the n members; Euler-Maruyama step k uses the J
 *         members perm[w J .. w J + J - 1], w = k mod (n / J), for every
 *         particle, with the weights normalised over those J.  perm = NULL
 *         (or J = n with the identity) is the full ensemble.
 *   logit_perturb, perturb_seed
 *         0 for the analysis itself.  A test of how well a result is
 *         determined by its inputs sets logit_perturb > 0: every log-kernel
 *         l_ij at every step then gets  +/- logit_perturb * alpha |z_i| |x_j| / beta^2
 *         (sign from the Philox stream keyed by perturb_seed), the size of the
 *         rounding error that a dot product z_i . x_j with relative accuracy
 *         logit_perturb leaves in the expanded logit (2 alpha z.x - alpha^2
 *         |x|^2) / (2 beta^2).
 *   diag  optional [k_stop][nrows][2]: per step and row, the gap between the
 *         largest and second-largest log-kernel (how close the weights are to
 *         a tie) and the scale alpha |z| max_j |x_j| / beta^2 that bounds how
 *         much a relative error in z . x_j moves a log-kernel.
 * Returns 0, or -1 on an invalid argument.
 */
int ensf_oracle_analysis(const float *X, int n, int64_t d, const float *y, const uint8_t *mask,
                         double sigma_obs, int K, double eps, int obs_op, const float *noise,
                         uint64_t seed, uint32_t offset, const int *rows, int nrows, int k_stop,
                         const int *perm, int J, double logit_perturb, uint64_t perturb_seed, double *out,
                         double *traj, double *diag)
{
    if (n < 1 || d < 1 || K < 1 || !(eps > 0.0 && eps < 1.0) || !(sigma_obs > 0.0))
        return -1;
    if (!rows) nrows = n;
    if (nrows < 1 || k_stop < 0 || k_stop > K) return -1;
    if (!perm) J = n;
    if (J < 1 || J > n || n % J != 0) return -1;
    if (perm)
        for (int j = 0; j < n; ++j)
            if (perm[j] < 0 || perm[j] >= n) return -1;
    for (int r = 0; r < nrows; ++r) {
        int i = rows ? rows[r] : r;
        if (i < 0 || i >= n) return -1;
    }
    const double dt = 1.0 / (double)K;
    double *w = (double *)malloc(sizeof(double) * (size_t)nrows * (size_t)n);
    double *l = (double *)malloc(sizeof(double) * (size_t)nrows * (size_t)n);
    double *g = (double *)malloc(sizeof(double) * (size_t)d);
    double xmax = 0.0;
    double *xnorm = (double *)malloc(sizeof(double) * (size_t)n);
    double *znorm = (double *)malloc(sizeof(double) * (size_t)nrows);
    for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t c = 0; c < d; ++c) acc += (double)X[(size_t)j * d + c] * X[(size_t)j * d + c];
        xnorm[j] = sqrt(acc);
        if (xnorm[j] > xmax) xmax = xnorm[j];
    }

    /* z_i <- xi_0,i : the standard Gaussian sample at pseudo-time T = 1. */
    for (int r = 0; r < nrows; ++r) {
        int i = rows ? rows[r] : r;
        double *z = out + (size_t)r * (size_t)d;
        for (int64_t c = 0; c < d; ++c)
            z[c] = noise ? (double)noise[((size_t)0 * n + i) * (size_t)d + c]
                         : ensf_oracle_noise(seed, offset, 0, i, c);
    }
    if (traj) memcpy(traj, out, sizeof(double) * (size_t)nrows * (size_t)d);

    for (int k = 0; k < k_stop; ++k) {
        double t = 1.0 - (double)k * dt;
        double sch[5];
        ensf_oracle_schedule(t, eps, sch);
        double alpha = sch[0], beta2 = sch[1], b = sch[2], sigma2 = sch[3], h = sch[4];

        /* the members of this step: the whole ensemble, or the mini-batch window */
        const int w0 = perm ? (k % (n / J)) * J : 0;
        const int nm = perm ? J : n;
#define MEMBER(jj) (perm ? perm[w0 + (jj)] : (jj))
        /* log-kernels -|z_i - alpha x_j|^2 / (2 beta^2), direct form (Eq. 12) */
#pragma omp parallel for schedule(static)
        for (int j = 0; j < nm; ++j) {
            const float *xj = X + (size_t)MEMBER(j) * (size_t)d;
            for (int r = 0; r < nrows; ++r) {
                const double *z = out + (size_t)r * (size_t)d;
                double dist2 = 0.0;
                for (int64_t c = 0; c < d; ++c) {
                    double diff = z[c] - alpha * (double)xj[c];
                    dist2 += diff * diff;
                }
                l[(size_t)r * n + j] = -dist2 / (2.0 * beta2);
            }
        }
        if (logit_perturb > 0.0) {
            for (int r = 0; r < nrows; ++r) {
                const double *z = out + (size_t)r * (size_t)d;
                double zn = 0.0;
                for (int64_t c = 0; c < d; ++c) zn += z[c] * z[c];
                znorm[r] = sqrt(zn);
            }
            for (int r = 0; r < nrows; ++r) {
                int i = rows ? rows[r] : r;
                for (int j = 0; j < nm; ++j) {
                    uint32_t ctr[4] = {(uint32_t)MEMBER(j), (uint32_t)i, (uint32_t)k, 0x51EDu};
                    uint32_t key[2] = {(uint32_t)perturb_seed, (uint32_t)(perturb_seed >> 32)};
                    uint32_t bits[4];
                    ensf_oracle_philox4x32_10(ctr, key, bits);
                    double sign = (bits[0] & 1u) ? 1.0 : -1.0;
                    l[(size_t)r * n + j] += sign * logit_perturb * alpha * znorm[r] * xnorm[MEMBER(j)] / beta2;
                }
            }
        }
        /* normalised weights (Eq. 16) */
        for (int r = 0; r < nrows; ++r) {
            double *lr = l + (size_t)r * n, *wr = w + (size_t)r * n;
            double lmax = lr[0];
            for (int j = 1; j < nm; ++j)
                if (lr[j] > lmax) lmax = lr[j];
            if (diag) {
                double second = -HUGE_VAL;
                int top = 0;
                for (int j = 1; j < nm; ++j)
                    if (lr[j] > lr[top]) top = j;
                for (int j = 0; j < nm; ++j)
                    if (j != top && lr[j] > second) second = lr[j];
                const double *z = out + (size_t)r * (size_t)d;
                double zn = 0.0;
                for (int64_t c = 0; c < d; ++c) zn += z[c] * z[c];
                diag[((size_t)k * nrows + r) * 2 + 0] = (nm > 1) ? lmax - second : HUGE_VAL;
                diag[((size_t)k * nrows + r) * 2 + 1] = alpha * sqrt(zn) * xmax / beta2;
            }
            double total = 0.0;
            for (int j = 0; j < nm; ++j) {
                wr[j] = exp(lr[j] - lmax);
                total += wr[j];
            }
            for (int j = 0; j < nm; ++j)
                wr[j] /= total;
        }
        for (int r = 0; r < nrows; ++r) {
            int i = rows ? rows[r] : r;
            double *z = out + (size_t)r * (size_t)d;
            const double *wr = w + (size_t)r * n;
            ensf_oracle_lik_score(z, y, mask, d, sigma_obs, obs_op, g);
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < d; ++c) {
                /* prior score, Eq. 15 */
                double s_prior = 0.0;
                for (int j = 0; j < nm; ++j)
                    s_prior += -(z[c] - alpha * (double)X[(size_t)MEMBER(j) * (size_t)d + c]) / beta2 * wr[j];
                /* posterior score, Eq. 17 */
                double s = s_prior + h * g[c];
                double xi = noise ? (double)noise[((size_t)(k + 1) * n + i) * (size_t)d + c]
                                  : ensf_oracle_noise(seed, offset, k + 1, i, c);
                /* one backward Euler-Maruyama step of Eq. 7 from t to t - dt */
                z[c] = z[c] - dt * (b * z[c] - sigma2 * s) + sqrt(sigma2 * dt) * xi;
            }
        }
        if (traj)
            memcpy(traj + (size_t)(k + 1) * nrows * (size_t)d, out,
                   sizeof(double) * (size_t)nrows * (size_t)d);
#undef MEMBER
    }
    free(w);
    free(l);
    free(g);
    free(xnorm);
    free(znorm);
    return 0;
}

/* Ensemble mean over rows (FP64) and the RMSE of that mean against truth. */
double ensf_oracle_mean_rmse(const double *Z, int n, int64_t d, const float *truth, double *mean)
{
    double sq = 0.0;
    for (int64_t c = 0; c < d; ++c) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i)
            acc += Z[(size_t)i * (size_t)d + c];
        double m = acc / (double)n;
        if (mean) mean[c] = m;
        double e = m - (double)truth[c];
        sq += e * e;
    }
    return sqrt(sq / (double)d);
}

int ensf_oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
