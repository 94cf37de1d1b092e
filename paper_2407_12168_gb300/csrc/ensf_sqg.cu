// ensf_sqg.cu -- GPU integrator of the two-level SQG forecast model
// (the paper's forecast model, Sec. II-B: nonlinear Eady model, f-plane,
// uniform stratification and shear, pseudo-spectral in x and y, RK4 in
// time, 2/3 dealiasing, implicit hyperdiffusion), batched over ensemble
// members.  theta is scaled so that d(psi)/dz = theta on each boundary; the
// zero-PV interior gives, for horizontal wavenumber K, m = (N/f) K, mu = m H:
//   psi_0 = (theta_1 - theta_0 cosh mu) / (m sinh mu),
//   psi_H = (theta_1 cosh mu - theta_0) / (m sinh mu);
// on each boundary, with the mean flow U(z) = Lambda (z - H/2):
//   d theta/dt = -(U_l + u) theta_x - v theta_y + Lambda v,  u = -psi_y, v = psi_x,
// hyperdiffusion nu del^8 applied after each RK4 step as 1/(1 + dt nu K^8),
// and (optionally) Newtonian relaxation -theta / tau_relax as a large-scale sink.
// Transforms are cuFFT (R2C / C2R, FP32); everything else is in the kernels
// below.  The state is kept spectral during a run.
#include <cufft.h>

#include <cmath>
#include <cstdio>
#include <new>

#include "../../include/ensf.h"
#include "ensf_internal.h"

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Geo {
    int n, nh;        // grid side, n/2 + 1 retained x modes
    float dk;         // 2 pi / L
    float kcut;       // 2/3 of the largest wavenumber
    float inv_n2;     // 1 / n^2 (cuFFT transforms are unnormalised)
    float n_over_f, H, shear, dt, nu;
    float inv_relax;  // 1 / tau_relax (0: no relaxation)
};

__device__ __forceinline__ void wavenumber(const Geo &g, int iy, int ix, float &kx, float &ky) {
    kx = g.dk * ix;
    ky = g.dk * (iy <= g.n / 2 ? iy : iy - g.n);
}

// From theta_hat [B][2][n][nh] the four spectral fields per level, scaled by
// 1/n^2 for the inverse transform: theta_x, theta_y, u = -psi_y, v = psi_x.
__global__ void k_sqg_fields(const cufftComplex *__restrict__ th, cufftComplex *__restrict__ f, Geo g, int batch) {
    const int64_t plane = (int64_t)g.n * g.nh;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)batch * plane) return;
    const int b = (int)(idx / plane);
    const int64_t r = idx - (int64_t)b * plane;
    const int iy = (int)(r / g.nh), ix = (int)(r - (int64_t)iy * g.nh);
    float kx, ky;
    wavenumber(g, iy, ix, kx, ky);
    const float K = sqrtf(kx * kx + ky * ky);
    const cufftComplex t0 = th[((int64_t)b * 2 + 0) * plane + r];
    const cufftComplex t1 = th[((int64_t)b * 2 + 1) * plane + r];
    cufftComplex p0 = make_cuComplex(0.f, 0.f), p1 = p0;
    if (K > 0.f) {
        const float m = g.n_over_f * K, mu = m * g.H;
        // cosh/sinh of large mu overflow FP32: use the ratios, which stay finite
        float coth_mu, csch_mu;
        if (mu > 20.f) {
            coth_mu = 1.f;
            csch_mu = 2.f * expf(-mu);
        } else {
            const float s = sinhf(mu), c = coshf(mu);
            coth_mu = c / s;
            csch_mu = 1.f / s;
        }
        const float inv_m = 1.f / m;
        p0 = make_cuComplex((t1.x * csch_mu - t0.x * coth_mu) * inv_m, (t1.y * csch_mu - t0.y * coth_mu) * inv_m);
        p1 = make_cuComplex((t1.x * coth_mu - t0.x * csch_mu) * inv_m, (t1.y * coth_mu - t0.y * csch_mu) * inv_m);
    }
    // odd derivatives have no Nyquist component
    const bool nyq = (iy == g.n / 2) || (ix == g.n / 2);
    const cufftComplex tl[2] = {t0, t1}, pl[2] = {p0, p1};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const cufftComplex t = tl[l], p = pl[l];
        cufftComplex *base = f + (((int64_t)b * 2 + l) * 4) * plane + r;
        if (nyq) {
            const cufftComplex zero = make_cuComplex(0.f, 0.f);
            base[0] = zero;
            base[plane] = zero;
            base[2 * plane] = zero;
            base[3 * plane] = zero;
            continue;
        }
        // i k z = (-k z.y, k z.x)
        base[0 * plane] = make_cuComplex(-kx * t.y * g.inv_n2, kx * t.x * g.inv_n2);   // theta_x
        base[1 * plane] = make_cuComplex(-ky * t.y * g.inv_n2, ky * t.x * g.inv_n2);   // theta_y
        base[2 * plane] = make_cuComplex(ky * p.y * g.inv_n2, -ky * p.x * g.inv_n2);   // u = -psi_y
        base[3 * plane] = make_cuComplex(-kx * p.y * g.inv_n2, kx * p.x * g.inv_n2);   // v = psi_x
    }
}

// Grid-point right-hand side of each level from the four grid fields.
__global__ void k_sqg_rhs(const float *__restrict__ f, float *__restrict__ rhs, Geo g, int batch) {
    const int64_t grid = (int64_t)g.n * g.n;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)batch * 2 * grid) return;
    const int64_t bl = idx / grid, r = idx - bl * grid;
    const int l = (int)(bl & 1);
    const float *base = f + bl * 4 * grid + r;
    const float tx = base[0], ty = base[grid], u = base[2 * grid], v = base[3 * grid];
    const float U = g.shear * ((l == 0 ? 0.f : g.H) - 0.5f * g.H);
    rhs[idx] = -(U + u) * tx - v * ty + g.shear * v;
}

// RK4 bookkeeping in spectral space, with the 2/3 dealiasing of the tendency
// and, after the last stage, the implicit hyperdiffusion factor.
__global__ void k_sqg_rk(int stage, cufftComplex *__restrict__ th, const cufftComplex *__restrict__ tend,
                         cufftComplex *__restrict__ acc, cufftComplex *__restrict__ next, Geo g, int batch) {
    const int64_t plane = (int64_t)g.n * g.nh;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)batch * 2 * plane) return;
    const int64_t r = idx % plane;
    const int iy = (int)(r / g.nh), ix = (int)(r - (int64_t)iy * g.nh);
    float kx, ky;
    wavenumber(g, iy, ix, kx, ky);
    const bool keep = fabsf(kx) < g.kcut && fabsf(ky) < g.kcut;
    cufftComplex t = keep ? tend[idx] : make_cuComplex(0.f, 0.f);
    const cufftComplex x = th[idx];
    if (g.inv_relax > 0.f) {  // linear relaxation at the stage input
        const cufftComplex xin = stage == 1 ? x : next[idx];
        t.x -= g.inv_relax * xin.x;
        t.y -= g.inv_relax * xin.y;
    }
    const float dt = g.dt;
    if (stage == 1) {
        acc[idx] = t;
        next[idx] = make_cuComplex(x.x + 0.5f * dt * t.x, x.y + 0.5f * dt * t.y);
    } else if (stage == 2 || stage == 3) {
        const cufftComplex a = acc[idx];
        acc[idx] = make_cuComplex(a.x + 2.f * t.x, a.y + 2.f * t.y);
        const float h = stage == 2 ? 0.5f * dt : dt;
        next[idx] = make_cuComplex(x.x + h * t.x, x.y + h * t.y);
    } else {
        const cufftComplex a = acc[idx];
        const float K2 = kx * kx + ky * ky;
        const float damp = 1.f / (1.f + dt * g.nu * K2 * K2 * K2 * K2);
        th[idx] = make_cuComplex((x.x + dt / 6.f * (a.x + t.x)) * damp, (x.y + dt / 6.f * (a.y + t.y)) * damp);
    }
}

__global__ void k_scale(float *__restrict__ x, int64_t count, float s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) x[i] *= s;
}

unsigned blocks_for(int64_t count) { return (unsigned)((count + 255) / 256); }

}  // namespace

struct ensf_sqg {
    ensf_sqg_params p;
    int batch = 0;
    Geo g;
    cufftHandle r2c_state = 0, c2r_state = 0, c2r_fields = 0, r2c_rhs = 0;
    cufftComplex *th = nullptr, *next = nullptr, *acc = nullptr, *tend = nullptr, *fhat = nullptr;
    float *fgrid = nullptr, *rhs = nullptr;
    void *work = nullptr;
};

namespace {

struct SqgSizes {
    size_t th, next, acc, tend, fhat, fgrid, rhs, work, total;
};

bool sqg_params_ok(const ensf_sqg_params *p, int batch) {
    return p && batch >= 1 && p->n >= 8 && p->n % 2 == 0 && p->L > 0 && p->H > 0 && p->N_over_f > 0 &&
           p->dt > 0 && p->tau_diss > 0;
}

// Plans over `batch` members; work sizes returned through `ws` (no work area allocated).
cufftResult make_plans(int n, int batch, cufftHandle *r2c_state, cufftHandle *c2r_state, cufftHandle *c2r_fields,
                       cufftHandle *r2c_rhs, size_t ws[4]) {
    int dims[2] = {n, n};
    cufftHandle *h[4] = {r2c_state, c2r_state, c2r_fields, r2c_rhs};
    const cufftType types[4] = {CUFFT_R2C, CUFFT_C2R, CUFFT_C2R, CUFFT_R2C};
    const int counts[4] = {2 * batch, 2 * batch, 8 * batch, 2 * batch};
    for (int i = 0; i < 4; ++i) {
        cufftResult r = cufftCreate(h[i]);
        if (r != CUFFT_SUCCESS) return r;
        r = cufftSetAutoAllocation(*h[i], 0);
        if (r != CUFFT_SUCCESS) return r;
        r = cufftMakePlanMany(*h[i], 2, dims, nullptr, 1, 0, nullptr, 1, 0, types[i], counts[i], &ws[i]);
        if (r != CUFFT_SUCCESS) return r;
    }
    return CUFFT_SUCCESS;
}

SqgSizes sqg_sizes(int n, int batch, const size_t ws[4]) {
    const size_t spec = sizeof(cufftComplex) * (size_t)n * (n / 2 + 1);
    const size_t grid = sizeof(float) * (size_t)n * n;
    SqgSizes s;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
    s.th = take(spec * 2 * batch);
    s.next = take(spec * 2 * batch);
    s.acc = take(spec * 2 * batch);
    s.tend = take(spec * 2 * batch);
    s.fhat = take(spec * 8 * batch);
    s.fgrid = take(grid * 8 * batch);
    s.rhs = take(grid * 2 * batch);
    size_t w = 0;
    for (int i = 0; i < 4; ++i) w = ws[i] > w ? ws[i] : w;
    s.work = take(w > 0 ? w : 1);
    s.total = off;
    return s;
}

ensf_status sqg_fail(ensf_status st, const char *msg) {
    ensf::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" {

size_t ensf_sqg_workspace_bytes(const ensf_sqg_params *p, int batch) {
    if (!sqg_params_ok(p, batch)) return 0;
    cufftHandle h[4] = {0, 0, 0, 0};
    size_t ws[4] = {0, 0, 0, 0};
    cufftResult r = make_plans(p->n, batch, &h[0], &h[1], &h[2], &h[3], ws);
    for (int i = 0; i < 4; ++i)
        if (h[i]) cufftDestroy(h[i]);
    if (r != CUFFT_SUCCESS) return 0;
    return sqg_sizes(p->n, batch, ws).total;
}

ensf_status ensf_sqg_create(const ensf_sqg_params *p, int batch, void *workspace, size_t ws_bytes, ensf_sqg **out) {
    if (!out) return sqg_fail(ENSF_EINVAL, "ensf_sqg_create: out is NULL");
    *out = nullptr;
    if (!sqg_params_ok(p, batch)) return sqg_fail(ENSF_EINVAL, "ensf_sqg_create: bad parameters");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
        return sqg_fail(ENSF_EINVAL, "ensf_sqg_create: workspace must be 256-byte aligned");
    ensf_sqg *s = new (std::nothrow) ensf_sqg;
    if (!s) return sqg_fail(ENSF_ENOMEM, "ensf_sqg_create: host allocation failed");
    size_t ws[4] = {0, 0, 0, 0};
    if (make_plans(p->n, batch, &s->r2c_state, &s->c2r_state, &s->c2r_fields, &s->r2c_rhs, ws) != CUFFT_SUCCESS) {
        ensf_sqg_destroy(s);
        return sqg_fail(ENSF_ECUDA, "ensf_sqg_create: cuFFT plan creation failed");
    }
    const SqgSizes z = sqg_sizes(p->n, batch, ws);
    if (ws_bytes < z.total) {
        ensf_sqg_destroy(s);
        return sqg_fail(ENSF_ENOMEM, "ensf_sqg_create: workspace too small");
    }
    char *w = static_cast<char *>(workspace);
    s->p = *p;
    s->batch = batch;
    s->th = reinterpret_cast<cufftComplex *>(w + z.th);
    s->next = reinterpret_cast<cufftComplex *>(w + z.next);
    s->acc = reinterpret_cast<cufftComplex *>(w + z.acc);
    s->tend = reinterpret_cast<cufftComplex *>(w + z.tend);
    s->fhat = reinterpret_cast<cufftComplex *>(w + z.fhat);
    s->fgrid = reinterpret_cast<float *>(w + z.fgrid);
    s->rhs = reinterpret_cast<float *>(w + z.rhs);
    s->work = w + z.work;
    cufftHandle hs[4] = {s->r2c_state, s->c2r_state, s->c2r_fields, s->r2c_rhs};
    for (cufftHandle h : hs)
        if (cufftSetWorkArea(h, s->work) != CUFFT_SUCCESS) {
            ensf_sqg_destroy(s);
            return sqg_fail(ENSF_ECUDA, "ensf_sqg_create: cufftSetWorkArea failed");
        }
    Geo &g = s->g;
    g.n = p->n;
    g.nh = p->n / 2 + 1;
    g.dk = (float)(2.0 * M_PI / p->L);
    const double kmax = 2.0 * M_PI / p->L * (p->n / 2);
    g.kcut = (float)(2.0 / 3.0 * kmax);
    g.inv_n2 = (float)(1.0 / ((double)p->n * p->n));
    g.n_over_f = (float)p->N_over_f;
    g.H = (float)p->H;
    g.shear = (float)p->shear;
    g.dt = (float)p->dt;
    g.nu = p->diffusion ? (float)(1.0 / (p->tau_diss * std::pow(kmax, 8))) : 0.f;
    g.inv_relax = p->tau_relax > 0 ? (float)(1.0 / p->tau_relax) : 0.f;
    *out = s;
    return ENSF_OK;
}

ensf_status ensf_sqg_run(ensf_sqg *s, float *theta, int nsteps, void *stream) {
    if (!s || !theta || nsteps < 0) return sqg_fail(ENSF_EINVAL, "ensf_sqg_run: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cufftHandle hs[4] = {s->r2c_state, s->c2r_state, s->c2r_fields, s->r2c_rhs};
    for (cufftHandle h : hs)
        if (cufftSetStream(h, st) != CUFFT_SUCCESS) return sqg_fail(ENSF_ECUDA, "ensf_sqg_run: cufftSetStream");
    const Geo &g = s->g;
    const int B = s->batch;
    const int64_t spec_all = (int64_t)B * 2 * g.n * g.nh;
    if (cufftExecR2C(s->r2c_state, theta, s->th) != CUFFT_SUCCESS)
        return sqg_fail(ENSF_ECUDA, "ensf_sqg_run: forward transform failed");
    for (int step = 0; step < nsteps; ++step) {
        for (int stage = 1; stage <= 4; ++stage) {
            const cufftComplex *in = stage == 1 ? s->th : s->next;
            k_sqg_fields<<<blocks_for((int64_t)B * g.n * g.nh), 256, 0, st>>>(in, s->fhat, g, B);
            if (cufftExecC2R(s->c2r_fields, s->fhat, s->fgrid) != CUFFT_SUCCESS)
                return sqg_fail(ENSF_ECUDA, "ensf_sqg_run: inverse transform failed");
            k_sqg_rhs<<<blocks_for((int64_t)B * 2 * g.n * g.n), 256, 0, st>>>(s->fgrid, s->rhs, g, B);
            if (cufftExecR2C(s->r2c_rhs, s->rhs, s->tend) != CUFFT_SUCCESS)
                return sqg_fail(ENSF_ECUDA, "ensf_sqg_run: forward transform failed");
            k_sqg_rk<<<blocks_for(spec_all), 256, 0, st>>>(stage, s->th, s->tend, s->acc, s->next, g, B);
        }
    }
    if (cufftExecC2R(s->c2r_state, s->th, theta) != CUFFT_SUCCESS)
        return sqg_fail(ENSF_ECUDA, "ensf_sqg_run: inverse transform failed");
    k_scale<<<blocks_for((int64_t)B * 2 * g.n * g.n), 256, 0, st>>>(theta, (int64_t)B * 2 * g.n * g.n, g.inv_n2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sqg_fail(ENSF_ECUDA, cudaGetErrorString(e));
    return ENSF_OK;
}

ensf_status ensf_sqg_destroy(ensf_sqg *s) {
    if (!s) return ENSF_EINVAL;
    cufftHandle hs[4] = {s->r2c_state, s->c2r_state, s->c2r_fields, s->r2c_rhs};
    for (cufftHandle h : hs)
        if (h) cufftDestroy(h);
    delete s;
    return ENSF_OK;
}

}  // extern "C"
