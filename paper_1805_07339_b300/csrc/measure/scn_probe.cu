// Measured ceiling of the unit that binds the fused histogram kernel: shared-
// memory reductions.  The fused kernel counts every pixel with three
// red.shared.add.u32 (one per channel) into lane-private table columns, so
// each warp-wide reduction is one conflict-free shared-memory wavefront; its
// throughput, not HBM, sets that kernel's pace.  This probe issues the same
// reductions in the same table layout (lane column, two warps per 128-byte half
// of a 256-byte row, two warps per 16-bit counter half, one region of rows per
// four warps) from the same counting warps of a CTA of the same size, with
// nothing else to do, and times them with the SM's own cycle counter, so the
// rate it returns (warp reductions per SM clock) is the ceiling the fused
// kernel's own rate is compared with.
//
// Measurement only: built into its own library (libscn_probe.so), outside the
// C ABI of libscn.so; the benchmark and its test load it.  The paper has no
// counterpart.
//
//   int scn_probe_shared_reductions(int32_t iters, int32_t grid,
//                                   unsigned long long* d_cycles, void* stream)
// launches `grid` CTAs of the hist kernel's shape (its threads and its counter
// table) in which each counting warp issues 8 * iters red.shared.add.u32 in the
// kernel's table layout and nothing else; d_cycles[b] (device, 8-byte aligned,
// `grid` entries) receives CTA b's elapsed SM clock cycles over that loop, so
// warps * 8 * iters / d_cycles[b] is the warp reductions per SM clock.
// Returns 0 (launched, asynchronous on `stream`), 1 for iters outside
// [1, 2^20], grid outside [1, 65535] or a null / misaligned d_cycles, 4 for a
// CUDA error (the status numbering of scn.h).
//
//   void scn_probe_geometry(int32_t* warps, int32_t* reductions_per_pixel)
// reports the counting warps per CTA and the kernel's shared-memory reductions
// per pixel.
#include <cuda_runtime.h>

#include "../scn_internal.h"
#include "../scn_ptx.cuh"

namespace scn {
namespace {

constexpr int kProbeAddrs = 8;  // rows a warp cycles through

__global__ void __launch_bounds__(kHistThreads, 1) red_probe_kernel(int32_t iters, unsigned long long* cycles) {
    extern __shared__ __align__(1024) uint8_t tab[];
    for (int i = threadIdx.x; i < kTabBytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(tab)[i] = make_uint4(0, 0, 0, 0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t col = ptx::smem_u32(tab) + static_cast<uint32_t>((warp / kGroupWarps) * kTabRowsPerRegion * 256 +
                                                                    (warp & 1) * 128 + lane * 4);
    const uint32_t inc = (warp & 2) ? 65536u : 1u;
    uint32_t addr[kProbeAddrs];
#pragma unroll
    for (int k = 0; k < kProbeAddrs; ++k)
        addr[k] = col + static_cast<uint32_t>(((k * 17 + warp * 5) % kTabRowsPerRegion) * 256);
    __syncthreads();
    const long long t0 = clock64();
    if (warp < kConsumerWarps) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeAddrs; ++k) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr[k]), "r"(inc));
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(t1 - t0);
}

}  // namespace
}  // namespace scn

extern "C" {

void scn_probe_geometry(int32_t* warps, int32_t* reductions_per_pixel) {
    if (warps) *warps = scn::kConsumerWarps;
    if (reductions_per_pixel) *reductions_per_pixel = scn::kReductionsPerPixel;
}

int scn_probe_shared_reductions(int32_t iters, int32_t grid, unsigned long long* d_cycles, void* stream) {
    if (iters < 1 || iters > (1 << 20) || grid < 1 || grid > 65535 || !d_cycles) return SCN_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_cycles) & 7u) return SCN_EINVAL;
    const size_t smem = static_cast<size_t>(scn::kTabBytes);
    if (cudaFuncSetAttribute(scn::red_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return SCN_ECUDA;
    scn::red_probe_kernel<<<static_cast<unsigned>(grid), scn::kHistThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        iters, d_cycles);
    return cudaGetLastError() == cudaSuccess ? SCN_OK : SCN_ECUDA;
}

}  // extern "C"
