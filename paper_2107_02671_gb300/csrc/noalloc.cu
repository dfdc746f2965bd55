// noalloc.cu -- nnfft_exec_host_noalloc: the host-buffer forward transform for
// callers that cannot allocate device memory when they call us.
//
// nnfft_exec_host copies the caller's host arrays through device staging buffers
// that the plan allocates (cudaMalloc) on first use.  Some callers cannot allow
// that allocation: their GPU memory is owned by another allocator (a framework's
// caching allocator that has reserved nearly all of the device, so a cudaMalloc
// would fail or fragment it), or they run a latency-bound serving loop in which
// an allocation stall inside the call is not acceptable.  This variant stages f
// and y in one file-scope static device array instead, so it allocates nothing.
//
// Limits and sharing rules:
//   * The array is NOALLOC_BYTES = 4 MiB on every GPU that loads the library, held
//     until the process exits.  f's part is rounded up to 256 bytes; M1 and M2
//     complex values of the plan's type must fit (complex128: (M1+M2)*16 bytes,
//     about 262,000 points in total; complex64: half the bytes).  Larger plans get
//     NNFFT_EINVAL.
//   * Every call on a device shares the same array and leaves its contents behind;
//     f and y are fully overwritten by each call, so nothing needs clearing.
//     Calls whose GPU work overlaps (two host threads, or two plans on different
//     streams) race on the array: serialise them.
//   * The call runs on the plan's device (the device that was current when the plan
//     was made): if another device is current, it switches to the plan's device for
//     the call and back before returning, so the staging array used is always the
//     copy on the GPU that holds the plan's buffers and streams.
//   * The first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that
//     first call before any stream capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "nnfft.h"

namespace {

constexpr size_t NOALLOC_BYTES = size_t(4) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on device dev, which must be current (set up
// once per device).
int scratch_address(int dev, void **out) {
    cudaError_t e = cudaSuccess;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return nnfft::report_error(NNFFT_ECUDA, "device index beyond the no-alloc table");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return nnfft::report_error(NNFFT_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                                        cudaGetErrorString(e));
        }
        g_noalloc_addr[dev] = ptr;
    }
    *out = g_noalloc_addr[dev];
    return NNFFT_OK;
}

// The transform itself, with the plan's device current.
int exec_noalloc_on_device(nnfft_plan_t p, int dev, const void *f_host, void *y_host);

}  // namespace

extern "C" int nnfft_exec_host_noalloc(nnfft_plan_t p, const void *f_host, void *y_host) {
    if (!p) return nnfft::report_error(NNFFT_EINVAL, "null plan");
    const int dev = nnfft::plan_device(p);
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nnfft::report_error(NNFFT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    if (cur == dev) return exec_noalloc_on_device(p, dev, f_host, y_host);
    if ((e = cudaSetDevice(dev)) != cudaSuccess) {
        cudaGetLastError();
        return nnfft::report_error(NNFFT_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    const int rc = exec_noalloc_on_device(p, dev, f_host, y_host);
    if ((e = cudaSetDevice(cur)) != cudaSuccess && rc == NNFFT_OK) {
        cudaGetLastError();
        return nnfft::report_error(NNFFT_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    return rc;
}

namespace {

int exec_noalloc_on_device(nnfft_plan_t p, int dev, const void *f_host, void *y_host) {
    nnfft_info info;
    int rc = nnfft_plan_info(p, &info);
    if (rc) return rc;
    if ((info.M1 > 0 && !f_host) || (info.M2 > 0 && !y_host))
        return nnfft::report_error(NNFFT_EINVAL, "null data pointer");
    const size_t cs = info.dtype == NNFFT_C128 ? 2 * sizeof(double) : 2 * sizeof(float);
    const size_t f_bytes = (size_t)info.M1 * cs, y_bytes = (size_t)info.M2 * cs;
    const size_t y_off = (f_bytes + 255) & ~size_t(255);
    if (y_off + y_bytes > NOALLOC_BYTES)
        return nnfft::report_error(
            NNFFT_EINVAL, "nnfft_exec_host_noalloc: M1 + M2 values exceed the 4 MiB static "
                          "staging array; use nnfft_exec_host");
    void *base = nullptr;
    if ((rc = scratch_address(dev, &base))) return rc;
    unsigned char *f_dev = static_cast<unsigned char *>(base);
    unsigned char *y_dev = f_dev + y_off;
    cudaStream_t st = nnfft::plan_stream(p);
    cudaError_t e = cudaSuccess;
    if (f_bytes) e = cudaMemcpyAsync(f_dev, f_host, f_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nnfft::report_error(NNFFT_ECUDA, std::string("copy f: ") + cudaGetErrorString(e));
    }
    if ((rc = nnfft_exec(p, f_dev, y_dev))) return rc;
    if (y_bytes) e = cudaMemcpyAsync(y_host, y_dev, y_bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nnfft::report_error(NNFFT_ECUDA, std::string("copy y: ") + cudaGetErrorString(e));
    }
    return nnfft_sync(p);
}

}  // namespace
