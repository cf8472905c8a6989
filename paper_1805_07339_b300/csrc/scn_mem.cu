// Device memory of library objects: videos' shot tables, sequences' scratch,
// plans' jobs and items.
//
// Mapping new device memory (a cudaMalloc that needs fresh pages, or a memory
// pool that grows) waits for the kernels in flight on every stream.  Objects
// are created while earlier work still runs (a stream runner creates the next
// video's sequences while the current one is generated and counted), so each
// of them would stall the host behind the GPU.  Instead, object memory comes
// from one stream-ordered pool per device that keeps everything it maps and is
// grown ahead in large steps (at least doubling), so only the rare growth
// waits.  Objects are filled on a library stream that waits for no other
// stream, and obj_finish() returns once that fill is complete, so a kernel
// launched afterwards on any stream sees the data.  Fills are copies (the copy
// engine), never kernels, so they complete even while other grids fill the SMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "scn_internal.h"

namespace scn {
namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kGrowMin = size_t(64) << 20;  // first reservation and smallest growth step

struct DeviceMem {
    cudaStream_t fill = nullptr;
    cudaMemPool_t pool = nullptr;
};

std::mutex g_mu;
DeviceMem g_dev[kMaxDevices];

// The calling device's fill stream and pool, created on first use.
cudaError_t device_mem(DeviceMem** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    DeviceMem& d = g_dev[dev];
    if (!d.fill) {
        e = cudaStreamCreateWithFlags(&d.fill, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            d.fill = nullptr;
            return e;
        }
    }
    if (!d.pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&d.pool, &props);
        if (e != cudaSuccess) {
            d.pool = nullptr;
            return e;
        }
        uint64_t keep_all = ~uint64_t(0);  // never give mapped memory back while the process runs
        e = cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
        if (e != cudaSuccess) return e;
    }
    *out = &d;
    return cudaSuccess;
}

}  // namespace

cudaError_t obj_stream(cudaStream_t* s) {
    std::lock_guard<std::mutex> g(g_mu);
    DeviceMem* d = nullptr;
    const cudaError_t e = device_mem(&d);
    if (e == cudaSuccess) *s = d->fill;
    return e;
}

cudaError_t obj_alloc(void** p, size_t bytes) {
    *p = nullptr;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceMem* d = nullptr;
    cudaError_t e = device_mem(&d);
    if (e != cudaSuccess) return e;
    bytes = std::max<size_t>(bytes, 256);
    uint64_t reserved = 0, used = 0;
    e = cudaMemPoolGetAttribute(d->pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(d->pool, cudaMemPoolAttrUsedMemCurrent, &used);
    if (e != cudaSuccess) return e;
    if (used + bytes > reserved) {
        // grow once by a large step: map it with one block and hand it back to the pool,
        // which keeps it for the allocations that follow (same stream, stream order)
        const size_t grow = std::max({bytes, static_cast<size_t>(reserved), kGrowMin});
        void* big = nullptr;
        if (cudaMallocFromPoolAsync(&big, grow, d->pool, d->fill) == cudaSuccess) {
            e = cudaFreeAsync(big, d->fill);
            if (e != cudaSuccess) return e;
        } else {
            cudaGetLastError();  // a step too large to map: let the exact request decide
        }
    }
    return cudaMallocFromPoolAsync(p, bytes, d->pool, d->fill);
}

cudaError_t obj_upload(void* dst, const void* src, size_t bytes) {
    cudaStream_t s = nullptr;
    const cudaError_t e = obj_stream(&s);
    return e != cudaSuccess ? e : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

cudaError_t obj_zero(void* dst, size_t bytes) {
    // zeros uploaded by the copy engine, not a memset: a memset is a kernel, and a
    // kernel queued behind a grid that fills the GPU waits for that grid to drain
    static const std::vector<uint8_t> zeros(size_t(1) << 20, 0);
    cudaStream_t s = nullptr;
    cudaError_t e = obj_stream(&s);
    for (size_t off = 0; e == cudaSuccess && off < bytes; off += zeros.size())
        e = cudaMemcpyAsync(static_cast<char*>(dst) + off, zeros.data(), std::min(zeros.size(), bytes - off),
                            cudaMemcpyHostToDevice, s);
    return e;
}

cudaError_t obj_finish() {
    cudaStream_t s = nullptr;
    const cudaError_t e = obj_stream(&s);
    return e != cudaSuccess ? e : cudaStreamSynchronize(s);
}

void obj_free(void* p) {
    if (!p) return;
    // the block's own device, which need not be the current one when the object is destroyed
    int cur = 0, dev = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return;
    cudaPointerAttributes at = {};
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeDevice) dev = at.device;
    cudaGetLastError();
    if (dev < 0) dev = cur;
    if (dev != cur && cudaSetDevice(dev) != cudaSuccess) return;
    // as cudaFree would: no launch on any stream may still use the block
    cudaDeviceSynchronize();
    cudaStream_t s = nullptr;
    if (obj_stream(&s) == cudaSuccess) cudaFreeAsync(p, s);
    if (dev != cur) cudaSetDevice(cur);
}

}  // namespace scn
