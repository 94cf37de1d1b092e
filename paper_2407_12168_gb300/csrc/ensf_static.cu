// ensf_static.cu -- the allocation-free variant of the weights stage.
//
// ensf_weights_static() computes the normalised weights of ensf_weights()
// with the FP32 Gram -- on the same centred operands (z - alpha m and x_j - m,
// m the forecast mean over the members), so the expanded log-kernel keeps its
// accuracy down to small pseudo-times -- but takes its scratch (the centre,
// the FP64 row norms and the split-K partial Grams) from one file-scope device
// array instead of a caller workspace.  It exists for callers that may not
// allocate device memory at all -- applications whose own pool owns every
// device allocation, or loops that must never hit an allocation that could
// synchronise the device -- and so cannot size and hand over a workspace.
//
// Limits: n <= 256 particles, n_x <= 256 forecast members, d <= 524288 state
// entries, at most 8 split-K slices; the array holds 4 MiB + 4 KiB and stays
// resident on every device that loads the library until the process exits.
// All calls share the array: calls that overlap on the GPU (two streams, or
// two host threads) race on it.  Every word a call reads is first written by
// that same call, so nothing needs clearing between calls.
#include <cstdio>
#include <mutex>

#include "../../include/ensf.h"
#include "ensf_internal.h"

namespace {

constexpr int kStaticMaxN = 256;
constexpr int64_t kStaticMaxD = 524288;
constexpr int kStaticMaxSplits = 8;
constexpr size_t kNormBytes = 4096;  // room for kStaticMaxN doubles, 256-byte aligned
constexpr size_t kCentreBytes = sizeof(float) * kStaticMaxD;
constexpr size_t kPartialBytes = sizeof(float) * kStaticMaxSplits * kStaticMaxN * kStaticMaxN;
constexpr size_t kStaticScratchBytes = kNormBytes + kCentreBytes + kPartialBytes;
constexpr int kMaxDevices = 64;

// The scratch array.  Host code must not use its name as an address: the
// device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

ensf_status static_fail(ensf_status s, const char *msg) {
    ensf::set_last_error(msg);  // reported by ensf_last_error()
    return s;
}

}  // namespace

extern "C" {

ensf_status ensf_weights_static(const float *z, int n, const float *prior, int n_x, int64_t d, float t, float eps,
                                float *w, void *stream) {
    auto aligned16 = [](const void *p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!aligned16(z) || !aligned16(prior) || !aligned16(w))
        return static_fail(ENSF_EINVAL, "ensf_weights_static: z, prior and w must be non-NULL and 16-byte aligned");
    if (n < 1 || n > kStaticMaxN || n_x < 1 || n_x > kStaticMaxN)
        return static_fail(ENSF_EINVAL,
                           "ensf_weights_static: n and n_x must lie in [1, 256] (the static scratch holds no more)");
    if (d < 8 || d % 8 != 0 || d > kStaticMaxD)
        return static_fail(ENSF_EINVAL,
                           "ensf_weights_static: d must be a multiple of 8 in [8, 524288] (the static scratch "
                           "holds no more)");
    if (!(t > 0.0f && t <= 1.0f) || !(eps > 0.0f && eps < 1.0f))
        return static_fail(ENSF_EINVAL, "ensf_weights_static: need t in (0, 1] and eps in (0, 1)");
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess)
        return static_fail(ENSF_ECUDA, "ensf_weights_static: cudaGetSymbolAddress of the scratch array failed");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return static_fail(ENSF_ECUDA, "ensf_weights_static: device query failed");
    double *norms = static_cast<double *>(scratch);
    float *centre = reinterpret_cast<float *>(static_cast<unsigned char *>(scratch) + kNormBytes);
    float *partial = reinterpret_cast<float *>(static_cast<unsigned char *>(scratch) + kNormBytes + kCentreBytes);
    // split-K slices: about two CTAs per SM, at most kStaticMaxSplits, at least 512 columns each
    const int tiles = ((n + 63) / 64) * ((n_x + 63) / 64);
    int splits = (2 * sms + tiles - 1) / tiles;
    splits = splits > kStaticMaxSplits ? kStaticMaxSplits : splits;
    const int64_t by_d = d / 512 > 0 ? d / 512 : 1;
    if (splits > by_d) splits = static_cast<int>(by_d);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double td = t, alpha = 1.0 - td * (1.0 - static_cast<double>(eps));
    // centre m = forecast mean; |z - alpha x_j|^2 = |(z - alpha m) - alpha (x_j - m)|^2
    if (ensf::launch_col_mean(prior, n_x, d, centre, s) != cudaSuccess ||
        ensf::launch_row_norms(prior, n_x, d, norms, s, centre) != cudaSuccess ||
        ensf::launch_gram_fp32(z, n, prior, n_x, d, splits, partial, s, centre, static_cast<float>(alpha)) !=
            cudaSuccess ||
        ensf::launch_softmax_rows(partial, splits, static_cast<int64_t>(n) * n_x, n_x, n, n_x, norms, alpha,
                                  1.0 / (2.0 * td), w, n_x, nullptr, nullptr, 0, s) != cudaSuccess)
        return static_fail(ENSF_ECUDA, "ensf_weights_static: kernel launch failed");
    return ENSF_OK;
}

}  // extern "C"
