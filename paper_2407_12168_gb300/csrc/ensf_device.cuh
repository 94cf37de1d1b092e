// ensf_device.cuh -- device-side helpers shared by the EnSF kernels:
// the counter-based noise stream, the observation operator, and the per-step
// coefficient block.
#pragma once

#include <cstdint>
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
// with u1 = ((a >> 8) + 1) 2^-24 in (0, 1] and u2 = (b >> 8) 2^-24 in [0, 1).
__device__ __forceinline__ float4 noise4(uint64_t seed, uint32_t offset, int k, int64_t j, int q) {
    U4 c{(uint32_t)j, (uint32_t)q, (uint32_t)k, offset};
    U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float two_m24 = 5.9604644775390625e-8f;  // 2^-24
    float u1a = (float)((r.x >> 8) + 1u) * two_m24;
    float u2a = (float)(r.y >> 8) * two_m24;
    float u1b = (float)((r.z >> 8) + 1u) * two_m24;
    float u2b = (float)(r.w >> 8) * two_m24;
    float ra = sqrtf(-2.0f * logf(u1a));
    float rb = sqrtf(-2.0f * logf(u1b));
    float sa, ca, sb, cb;
    sincospif(2.0f * u2a, &sa, &ca);
    sincospif(2.0f * u2b, &sb, &cb);
    return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// Likelihood score term mask * H'(z) (y - H(z)) / sigma_obs^2 (Eq. 5).
__device__ __forceinline__ float lik_score(int op, float z, float y, float inv_r) {
    if (op == 1) {
        float dh = 1.0f / (1.0f + z * z);
        return dh * (y - atanf(z)) * inv_r;
    }
    return (y - z) * inv_r;
}

// One Euler-Maruyama step of the reverse-time SDE (Eq. 7) with the posterior
// score of Eq. 17, given u = sum_j w_ij x_j (the weighted forecast mean),
// g = the likelihood score (0 where unobserved) and the noise draw xi.
__device__ __forceinline__ float em_update(const StepCoef &c, float z, float u, float g, float xi) {
    float s_prior = -(z - c.alpha * u) * c.inv_beta2;   // Eq. 15 with sum_j w_ij = 1
    float s = s_prior + c.h * g;                       // Eq. 17
    return z - c.dt * (c.b * z - c.sigma2 * s) + c.noise_scale * xi;
}

}  // namespace ensf
