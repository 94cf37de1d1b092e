// ensf_host.cu -- page-locked host buffers backed by huge pages, for the
// host <-> device copies of an analysis's inputs and results.
//
// On a GPU coupled to its host CPU by a coherent link, the copy engines read
// and write host memory through address translation.  Measured on GB300:
// after a few minutes of other host work, a 2 GiB buffer pinned page by page
// (64 KiB pages) was copied at 35-70 GB/s right after an analysis had swept
// the GPU's working set, against ~200 GB/s back to back; the same copy from a
// buffer made of transparent huge pages ran at ~200 GB/s in both cases.  So
// these buffers are anonymous mappings aligned to the huge-page size, advised
// as huge pages (and collapsed into them where the kernel supports it) before
// they are registered with the CUDA driver as page-locked memory.
//
// On a host with several NUMA nodes (two Grace sockets, each with its own
// memory and GPUs) a buffer whose pages sit on the far socket is reached over
// the inter-socket link as well: the pages are placed, before the first
// touch, with a preference (MPOL_PREFERRED, so a full node falls back to the
// others instead of failing) for the host node the CUDA driver reports as the
// device's closest.
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include <sys/mman.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <cuda_runtime.h>

#include "../../include/ensf.h"
#include "ensf_internal.h"

#ifndef MADV_HUGEPAGE
#define MADV_HUGEPAGE 14
#endif
#ifndef MADV_COLLAPSE
#define MADV_COLLAPSE 25
#endif

namespace {

struct Mapping {
    void *raw;         // what mmap returned
    size_t raw_bytes;  // its length
    size_t bytes;      // the caller's size
};

std::mutex g_host_mutex;
std::unordered_map<void *, Mapping> g_host_maps;

// Size of a transparent huge page (PMD mapping) on this kernel: 2 MiB with
// 4 KiB base pages, 512 MiB with 64 KiB ones.
size_t huge_page_bytes() {
    size_t hp = 0;
    if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (fscanf(f, "%llu", &v) == 1) hp = static_cast<size_t>(v);
        fclose(f);
    }
    return hp ? hp : (size_t(2) << 20);
}

// Memory-policy constants of the Linux system calls (linux/mempolicy.h).
constexpr int kMpolPreferred = 1;
constexpr unsigned long kMpolFNode = 1, kMpolFAddr = 2;
constexpr int kMaxNodes = 1024;
constexpr int kMaskWords = kMaxNodes / (8 * static_cast<int>(sizeof(unsigned long)));

// Host NUMA node closest to the current device, or -1 (no NUMA, or unknown).
int device_host_node() {
    int dev = 0, id = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&id, cudaDevAttrHostNumaId, dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return id;
}

// Prefer `node` for the not yet touched pages of [addr, addr + len).
bool prefer_node(void *addr, size_t len, int node) {
    if (node < 0 || node >= kMaxNodes) return false;
    unsigned long mask[kMaskWords] = {0};
    const int bits = 8 * static_cast<int>(sizeof(unsigned long));
    mask[node / bits] |= 1UL << (node % bits);
    return syscall(SYS_mbind, addr, len, kMpolPreferred, mask, static_cast<unsigned long>(kMaxNodes) + 1, 0UL) == 0;
}

ensf_status host_fail(ensf_status s, const char *msg) {
    ensf::set_last_error(msg);
    return s;
}

// dst[i] = src[i] for n 16-byte words, grid-stride, four words in flight per
// thread; either side may be device memory or page-locked host memory (the
// loads and stores then travel over the host link, issued by the SMs instead
// of a copy engine).
__global__ void __launch_bounds__(256) k_copy16(uint4 *__restrict__ dst, const uint4 *__restrict__ src, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

}  // namespace

extern "C" {

ensf_status ensf_host_alloc(size_t bytes, unsigned flags, void **out) {
    if (!out || bytes == 0) return host_fail(ENSF_EINVAL, "ensf_host_alloc: need bytes > 0 and out != NULL");
    *out = nullptr;
    const size_t hp = huge_page_bytes();
    const size_t len = (bytes + hp - 1) / hp * hp;
    const size_t raw_len = len + hp;  // room to align the start to a huge page
    void *raw = mmap(nullptr, raw_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (raw == MAP_FAILED) return host_fail(ENSF_ENOMEM, "ensf_host_alloc: mmap failed");
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(raw) + hp - 1) / hp * hp);
    if (!(flags & ENSF_HOST_SMALL_PAGES)) {
        madvise(base, len, MADV_HUGEPAGE);  // best effort: the kernel may not offer huge pages
    }
    if (!(flags & ENSF_HOST_ANY_NODE)) prefer_node(base, len, device_host_node());  // best effort
    // touch every page now (with huge pages advised, each first touch of a
    // huge-page range faults in a whole huge page)
    const long pg = sysconf(_SC_PAGESIZE) > 0 ? sysconf(_SC_PAGESIZE) : 4096;
    for (size_t off = 0; off < len; off += static_cast<size_t>(pg)) base[off] = 0;
    if (!(flags & ENSF_HOST_SMALL_PAGES)) {
        madvise(base, len, MADV_COLLAPSE);  // best effort: gather small pages left by a failed fault
    }
    cudaError_t e = cudaHostRegister(base, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        munmap(raw, raw_len);
        return host_fail(ENSF_ECUDA, "ensf_host_alloc: cudaHostRegister failed");
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mutex);
        g_host_maps[base] = Mapping{raw, raw_len, bytes};
    }
    *out = base;
    return ENSF_OK;
}

ensf_status ensf_host_free(void *ptr) {
    if (!ptr) return ENSF_OK;
    Mapping m;
    {
        std::lock_guard<std::mutex> lock(g_host_mutex);
        auto it = g_host_maps.find(ptr);
        if (it == g_host_maps.end()) return host_fail(ENSF_EINVAL, "ensf_host_free: not a buffer of ensf_host_alloc");
        m = it->second;
        g_host_maps.erase(it);
    }
    cudaError_t e = cudaHostUnregister(ptr);
    munmap(m.raw, m.raw_bytes);
    return e == cudaSuccess ? ENSF_OK : host_fail(ENSF_ECUDA, "ensf_host_free: cudaHostUnregister failed");
}

ensf_status ensf_copy_sm(void *dst, const void *src, size_t bytes, int blocks, void *stream) {
    if (!dst || !src || (reinterpret_cast<uintptr_t>(dst) & 15u) || (reinterpret_cast<uintptr_t>(src) & 15u) ||
        bytes % 16 != 0 || blocks < 1)
        return host_fail(ENSF_EINVAL, "ensf_copy_sm: 16-byte aligned pointers, a multiple of 16 bytes, blocks >= 1");
    if (bytes == 0) return ENSF_OK;
    // device-side addresses of page-locked host memory (the same address under
    // unified addressing; device memory passes through)
    void *d_dst = dst;
    const void *d_src = src;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, dst) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer)
        d_dst = a.devicePointer;
    else
        cudaGetLastError();
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer)
        d_src = a.devicePointer;
    else
        cudaGetLastError();
    k_copy16<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<uint4 *>(d_dst),
                                                                      static_cast<const uint4 *>(d_src),
                                                                      static_cast<int64_t>(bytes / 16));
    return cudaGetLastError() == cudaSuccess ? ENSF_OK : host_fail(ENSF_ECUDA, "ensf_copy_sm: launch failed");
}

ensf_status ensf_host_registered(const void *ptr, int *registered) {
    if (!ptr || !registered) return host_fail(ENSF_EINVAL, "ensf_host_registered: NULL argument");
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *registered = 0;
        return ENSF_OK;
    }
    *registered = attr.type == cudaMemoryTypeHost ? 1 : 0;
    return ENSF_OK;
}

ensf_status ensf_host_numa(const void *ptr, int *node, int *device_node) {
    if (!ptr || !node || !device_node) return host_fail(ENSF_EINVAL, "ensf_host_numa: NULL argument");
    *device_node = device_host_node();
    int nd = -1;
    if (syscall(SYS_get_mempolicy, &nd, nullptr, 0UL, const_cast<void *>(ptr), kMpolFNode | kMpolFAddr) != 0) nd = -1;
    *node = nd;
    return ENSF_OK;
}

ensf_status ensf_host_huge_fraction(const void *ptr, size_t bytes, double *fraction) {
    if (!ptr || !fraction) return host_fail(ENSF_EINVAL, "ensf_host_huge_fraction: NULL argument");
    *fraction = 0.0;
    FILE *f = fopen("/proc/self/smaps", "r");
    if (!f) return host_fail(ENSF_EUNSUPPORTED, "ensf_host_huge_fraction: /proc/self/smaps unreadable");
    const uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    char line[512];
    bool inside = false;
    unsigned long long huge_kb = 0;
    while (fgets(line, sizeof line, f)) {
        unsigned long long lo = 0, hi = 0;
        char c0 = line[0];
        const bool header = ((c0 >= '0' && c0 <= '9') || (c0 >= 'a' && c0 <= 'f')) &&
                            sscanf(line, "%llx-%llx", &lo, &hi) == 2 && strchr(line, '-') != nullptr &&
                            strncmp(line, "AnonHugePages", 13) != 0;
        if (header) {
            inside = (a < hi) && (a + bytes > lo);
            continue;
        }
        unsigned long long kb = 0;
        if (inside && sscanf(line, "AnonHugePages: %llu kB", &kb) == 1) huge_kb += kb;
    }
    fclose(f);
    const double frac = static_cast<double>(huge_kb) * 1024.0 / static_cast<double>(bytes);
    *fraction = frac > 1.0 ? 1.0 : frac;
    return ENSF_OK;
}

}  // extern "C"
