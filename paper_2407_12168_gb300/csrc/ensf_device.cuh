// ensf_device.cuh -- device-side helpers shared by the EnSF kernels:
// the counter-based noise stream, the observation operator, and the per-step
// coefficient block.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ensf {

// Coefficients of one Euler-Maruyama step at pseudo-time t (Eq. 9, Eq. 11).
// Computed on the host in double precision from t and eps.
struct StepCoef {
    float alpha;        // alpha_t = 1 - t(1 - eps)
    float inv_beta2;    // 1 / beta_t^2 = 1 / t
    float b;            // d log(alpha_t) / dt
    float sigma2;       // d(beta_t^2)/dt - 2 b beta_t^2
    float h;            // damping h(t) = 1 - t
    float dt;           // 1 / K
    float noise_scale;  // sqrt(sigma^2 dt)
    float inv_r;        // 1 / sigma_obs^2
    double alpha_d;     // alpha_t (double, for the logits)
    double inv_2beta2_d;// 1 / (2 beta_t^2) (double, for the logits)
    int k;              // step index; the step consumes noise slice k + 1
    int obs_op;         // 0 identity, 1 arctan
    int64_t col0;       // global index of state column 0 of the kernel's operands (the
                        // noise counter uses global columns: a slice of the state draws
                        // what the whole state draws there); 0 for a whole state
};

// Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11): ten
// rounds of two 32x32->64-bit multiplies, Weyl-sequence key schedule.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Four standard normals xi[k][4q .. 4q+3][j] of the noise stream (four
// consecutive particles of state column j): counter (j, q, k, offset), key
// (seed low, seed high); words (x, y) and (z, w) each feed one Box-Muller pair
// with u1 = ((a >> 8) + 1) 2^-24 in (0, 1] and u2 = (b >> 8) 2^-24 in [0, 1):
// xi = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
//
// Evaluated with the SFU approximations (lg2, sqrt, sin, cos), which cost a
// few instructions where the correctly rounded library functions cost tens;
// the draws are consumed inside the W X epilogue, whose issue slots they
// share.  Accuracy against the exact transform: ln u1 comes from a short
// series of ln(1 - v), v = 1 - u1 (exact), where v < 2^-7 (error < 1e-11) and
// from lg2 elsewhere (absolute error < 4e-7, relative < 3 ulp); the angle is
// shifted into [-pi, pi), where sin and cos carry absolute errors < 4e-7.
// Each normal is then within about 3e-6 (absolute) of the exact value.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 box_muller(uint32_t a24, uint32_t b24) {
    const float two_m24 = 5.9604644775390625e-8f;  // 2^-24
    const float u1 = __fmul_rn(__uint2float_rn(a24 + 1u), two_m24);
    const float v1 = __fmul_rn(__uint2float_rn(0xFFFFFFu - a24), two_m24);  // 1 - u1, exact
    // ln(1 - v) = -v (1 + v/2 + v^2/3 + v^3/4 + ...), truncated after v^3/4
    const float ser = -__fmul_rn(v1, __fmaf_rn(v1, __fmaf_rn(v1, __fmaf_rn(v1, 0.25f, 0.333333343f), 0.5f), 1.0f));
    const float ln_u1 = v1 < 0.0078125f ? ser : __logf(u1);
    const float r = sqrt_approx(__fmul_rn(-2.0f, ln_u1));
    // 2 pi u2 = pi + theta, theta = 2 pi (u2 - 1/2) in [-pi, pi): cos, sin change sign
    const float theta = __fmul_rn(__int2float_rn(static_cast<int>(b24) - 8388608), 3.74507028e-7f);  // 2 pi 2^-24
    float sn, cs;
    __sincosf(theta, &sn, &cs);
    return make_float2(-__fmul_rn(r, cs), -__fmul_rn(r, sn));
}

__device__ __forceinline__ float4 noise4(uint64_t seed, uint32_t offset, int k, int64_t j, int q) {
    U4 c{(uint32_t)j, (uint32_t)q, (uint32_t)k, offset};
    U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float2 a = box_muller(r.x >> 8, r.y >> 8);
    const float2 b = box_muller(r.z >> 8, r.w >> 8);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Likelihood score term mask * H'(z) (y - H(z)) / sigma_obs^2 (Eq. 5).
// Every rounding is spelled out (no contraction left to the compiler), so
// all kernels that share these functions compute bit-identical particles.
__device__ __forceinline__ float lik_score(int op, float z, float y, float inv_r) {
    if (op == 1) {
        const float dh = __fdiv_rn(1.0f, __fmaf_rn(z, z, 1.0f));
        return __fmul_rn(__fmul_rn(dh, __fsub_rn(y, atanf(z))), inv_r);
    }
    return __fmul_rn(__fsub_rn(y, z), inv_r);
}

// One Euler-Maruyama step of the reverse-time SDE (Eq. 7) with the posterior
// score of Eq. 17, given u = sum_j w_ij x_j (the weighted forecast mean),
// g = the likelihood score (0 where unobserved) and the noise draw xi.
__device__ __forceinline__ float em_update(const StepCoef &c, float z, float u, float g, float xi) {
    const float s_prior = __fmul_rn(__fmaf_rn(c.alpha, u, -z), c.inv_beta2);  // -(z - alpha u) / beta^2, Eq. 15
    const float s = __fmaf_rn(c.h, g, s_prior);                                // Eq. 17
    const float drift = __fmaf_rn(c.b, z, -__fmul_rn(c.sigma2, s));            // b z - sigma^2 s
    return __fmaf_rn(c.noise_scale, xi, __fmaf_rn(-c.dt, drift, z));          // Eq. 7
}


// Programmatic dependent launch.  The per-step kernels (Gram, row softmax,
// W X) are launched with programmatic stream serialization: a kernel may be
// launched while its predecessor in the stream still runs, so every thread
// first waits until that predecessor has completed and its writes are
// visible (pdl_wait), and then lets the next kernel be launched
// (pdl_launch_dependents), whose blocks in turn wait at their own pdl_wait.
// Both are no-ops in a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Knuth's TwoSum: (hi, lo) += v with the rounding error of hi + v carried
// into lo, so hi + lo keeps about twice FP32's precision.  Explicit _rn
// intrinsics keep the compiler from contracting or reordering the steps.
__device__ __forceinline__ void df_add(float &hi, float &lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// Double-float arithmetic: a value carried as an unevaluated FP32 sum hi + lo
// (about 48 significant bits; Dekker 1971, Knuth's TwoSum).  The _rn
// intrinsics keep the compiler from contracting or reordering the steps.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_norm(float hi, float lo) {  // |hi| >= |lo| not required
    const float s = __fadd_rn(hi, lo);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(lo, bb));
    return DF{s, err};
}

// a + b (TwoSum of the high parts, low parts added to the error term)
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = df_norm(a.hi, b.hi);
    return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// a * b (exact product of the high parts by FMA, cross terms added)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

// A double input (the FP64 norms, the host's coefficients) split into two
// floats as it is read; everything after this runs in FP32.
__device__ __forceinline__ DF df_from(double v) {
    const float h = __double2float_rn(v);
    return DF{h, __double2float_rn(v - static_cast<double>(h))};
}

// sum_{s0 <= s < s1} p[s * stride], ascending s, as a compensated FP32 sum
// (error of order (s1 - s0)^2 2^-48 relative to sum |p|; FP64 units are few
// on this part, FP32 ones are not).  The loads go out eight at a time, also
// for a short tail: the partials sit in L2 and each load waits on it.
__device__ __forceinline__ DF sum_partials(const float *__restrict__ p, int64_t stride, int s0, int s1) {
    float hi = 0.f, lo = 0.f;
    for (int s = s0; s < s1; s += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (s + q < s1) ? __ldcg(p + (int64_t)(s + q) * stride) : 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (s + q < s1) df_add(hi, lo, v[q]);
    }
    return df_norm(hi, lo);
}

// Log-kernel of Eq. 12 in its expanded form, l = (2 alpha G - alpha^2 |x|^2) / (2 beta^2)
// (the row constant -|z|^2 / (2 beta^2) cancels in the softmax), in double-float.
struct LogitCoef {
    DF two_alpha, alpha_sq, inv_2beta2;
};

__device__ __forceinline__ LogitCoef logit_coef(double alpha, double inv_2beta2) {
    const DF a = df_from(alpha);
    return LogitCoef{DF{2.f * a.hi, 2.f * a.lo}, df_mul(a, a), df_from(inv_2beta2)};
}

__device__ __forceinline__ DF logit(const LogitCoef &k, DF g, double norm) {
    const DF t = df_add(df_mul(k.two_alpha, g), df_neg(df_mul(k.alpha_sq, df_from(norm))));
    return df_mul(t, k.inv_2beta2);
}

// One row i of the softmax of Eq. 16 from split-K partial Grams (read through
// L2 only: they may come from other blocks of the same launch; block of NT
// threads; lg = n_x doubles of shared memory, red = NT doubles, both used as
// pairs of floats):
//   G_ij = sum_s partial[s][i][j]  (fixed order: deterministic),
//   l_ij = (2 alpha G_ij - alpha^2 |x_j|^2) / (2 beta^2), w_ij = softmax_j(l_ij),
// all in FP32, the sums and the logits compensated (double-float).
// Writes FP32 w and/or the BF16 split w = w_hi + w_lo.  When the row is short,
// `groups` threads share a column j, each summing a fixed range of splits
// (the group sums are then added in group order: deterministic).
template <int NT>
__device__ __forceinline__ void softmax_row(int i, const float *__restrict__ partial, int splits,
                                            int64_t part_stride, int ldp, int n_x,
                                            const double *__restrict__ norms, double alpha,
                                            double inv_2beta2, float *__restrict__ w, int ldw,
                                            __nv_bfloat16 *__restrict__ w_hi,
                                            __nv_bfloat16 *__restrict__ w_lo, int ldwb, double *lg_raw,
                                            double *red_raw) {
    DF *lg = reinterpret_cast<DF *>(lg_raw);
    DF *red = reinterpret_cast<DF *>(red_raw);
    float *redf = reinterpret_cast<float *>(red_raw);
    const int tid = threadIdx.x;
    const LogitCoef kc = logit_coef(alpha, inv_2beta2);
    const int groups = n_x >= NT ? 1 : min(NT / n_x, splits);
    const int per = (splits + groups - 1) / groups;
    float lmax = -FLT_MAX;
    if (groups == 1) {
        for (int j = tid; j < n_x; j += NT) {
            const DF l = logit(kc, sum_partials(partial + (int64_t)i * ldp + j, part_stride, 0, splits), norms[j]);
            lg[j] = l;
            lmax = fmaxf(lmax, l.hi);
        }
    } else {
        const int j = tid % n_x, grp = tid / n_x;
        if (grp < groups) {
            const int s0 = grp * per, s1 = min(splits, s0 + per);
            red[grp * n_x + j] = sum_partials(partial + (int64_t)i * ldp + j, part_stride, s0, s1);
        }
        __syncthreads();
        if (tid < n_x) {
            DF g = red[tid];
            for (int q = 1; q < groups; ++q) g = df_add(g, red[q * n_x + tid]);
            const DF l = logit(kc, g, norms[tid]);
            lg[tid] = l;
            lmax = l.hi;
        }
        __syncthreads();
    }
    redf[tid] = lmax;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (tid < s) redf[tid] = fmaxf(redf[tid], redf[tid + s]);
        __syncthreads();
    }
    const float m = redf[0];
    __syncthreads();
    float sh = 0.f, sl = 0.f;
    for (int j = tid; j < n_x; j += NT) {
        const DF l = lg[j];
        const DF dl = df_norm(__fsub_rn(l.hi, m), l.lo);  // l.hi - m is exact where it matters (near the max)
        const float e = expf(__fadd_rn(dl.hi, dl.lo));
        lg[j].hi = e;
        df_add(sh, sl, e);
    }
    red[tid] = df_norm(sh, sl);
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = df_add(red[tid], red[tid + s]);
        __syncthreads();
    }
    const float inv = __frcp_rn(__fadd_rn(red[0].hi, red[0].lo));
    for (int j = tid; j < n_x; j += NT) {
        const float wv = __fmul_rn(lg[j].hi, inv);
        if (w) w[(int64_t)i * ldw + j] = wv;
        if (w_hi) {
            __nv_bfloat16 hi = __float2bfloat16_rn(wv);
            w_hi[(int64_t)i * ldwb + j] = hi;
            if (w_lo) w_lo[(int64_t)i * ldwb + j] = __float2bfloat16_rn(wv - __bfloat162float(hi));
        }
    }
}

// ---- Row softmax of Eq. 16 in tiles of 256 columns, one warp per (row, tile)
// The form shared by the separate softmax launch and the softmax fused into
// the pair Gram's epilogue (bit-identical results).  Per row i and column
// tile t, a warp forms the log-kernels l_ij of its 256 columns (written to L
// as double-float pairs), their maximum m_t and s_t = sum_j exp(l_ij - m_t);
// once every tile of the row is done, the row is normalised with
// M = max_t m_t and S = sum_t s_t exp(m_t - M):  w_ij = exp(l_ij - M) / S.
// Column j of tile t is handled by lane j % 32 in both phases; every sum runs
// in a fixed order.  L, stats and the partials are read through L2 (other
// blocks may have written them).
constexpr int kSoftTile = 256;

__device__ __forceinline__ void softmax_tile_stats(int i, int t, const float *__restrict__ partial, int splits,
                                                   int64_t part_stride, int ldp, int n_x,
                                                   const double *__restrict__ norms, const LogitCoef &kc, DF *L,
                                                   int ldl, float4 *stats, int nt) {
    const int lane = threadIdx.x & 31;
    DF l[8];
    float mx = -FLT_MAX;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int j = t * kSoftTile + e * 32 + lane;
        if (j < n_x) {
            l[e] = logit(kc, sum_partials(partial + (int64_t)i * ldp + j, part_stride, 0, splits), norms[j]);
            L[(int64_t)i * ldl + j] = l[e];
            mx = fmaxf(mx, l[e].hi);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int j = t * kSoftTile + e * 32 + lane;
        if (j < n_x) {
            const DF dl = df_norm(__fsub_rn(l[e].hi, mx), l[e].lo);
            df_add(sh, sl, expf(__fadd_rn(dl.hi, dl.lo)));
        }
    }
    DF s = df_norm(sh, sl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {  // lane 0 ends with the fixed-order total
        const DF x{__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o)};
        if (lane < o) s = df_add(s, x);
    }
    if (lane == 0) stats[(int64_t)i * nt + t] = make_float4(mx, s.hi, s.lo, 0.f);
}

__device__ __forceinline__ void softmax_finalize_row(int i, int n_x, int nt, const DF *L, int ldl,
                                                     const float4 *stats, float *__restrict__ w, int ldw,
                                                     __nv_bfloat16 *__restrict__ w_hi,
                                                     __nv_bfloat16 *__restrict__ w_lo, int ldwb) {
    const int lane = threadIdx.x & 31;
    float M = -FLT_MAX;
    for (int t = 0; t < nt; ++t) M = fmaxf(M, __ldcg(&stats[(int64_t)i * nt + t].x));
    DF S{0.f, 0.f};
    for (int t = 0; t < nt; ++t) {
        const float4 st = __ldcg(&stats[(int64_t)i * nt + t]);
        S = df_add(S, df_mul(DF{st.y, st.z}, DF{expf(__fsub_rn(st.x, M)), 0.f}));
    }
    const float inv = __frcp_rn(__fadd_rn(S.hi, S.lo));
    const float2 *Lf = reinterpret_cast<const float2 *>(L);
    for (int j = lane; j < n_x; j += 32) {
        const float2 lv = __ldcg(&Lf[(int64_t)i * ldl + j]);
        const DF dl = df_norm(__fsub_rn(lv.x, M), lv.y);
        const float wv = __fmul_rn(expf(__fadd_rn(dl.hi, dl.lo)), inv);
        if (w) w[(int64_t)i * ldw + j] = wv;
        if (w_hi) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(wv);
            w_hi[(int64_t)i * ldwb + j] = hi;
            if (w_lo) w_lo[(int64_t)i * ldwb + j] = __float2bfloat16_rn(wv - __bfloat162float(hi));
        }
    }
}

}  // namespace ensf
