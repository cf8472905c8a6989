// Measured ceiling of the unit that binds the fused histogram kernel: shared-
// memory reductions.  The fused kernel counts every pixel with three
// red.shared.add.u32 (one per channel) into lane-private table columns, so
// each warp-wide reduction is one conflict-free shared-memory wavefront; its
// throughput, not HBM, sets that kernel's pace.  This probe issues the same
// reductions in the same table layout (lane column, two warps per 128-byte half
// of a 256-byte row, two warps per 16-bit counter half, 136 rows per region of
// four warps) from the same 20 counting warps of a 672-thread CTA, with
// nothing else to do, and times them with the SM's own cycle counter, so the
// rate it returns (warp reductions per SM clock) is the ceiling the fused
// kernel's own rate is compared with.
#include <cuda_runtime.h>

#include "scn_internal.h"
#include "scn_ptx.cuh"

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

scn_status scn_probe_shared_reductions(int32_t iters, int32_t grid, unsigned long long* d_cycles, void* stream) {
    if (iters < 1 || iters > (1 << 20) || grid < 1 || grid > 65535 || !d_cycles) return SCN_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_cycles) & 7u) return SCN_EINVAL;
    const size_t smem = static_cast<size_t>(scn::kTabBytes);
    SCN_CUDA_TRY(cudaFuncSetAttribute(scn::red_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    scn::red_probe_kernel<<<static_cast<unsigned>(grid), scn::kHistThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        iters, d_cycles);
    SCN_CUDA_TRY(cudaGetLastError());
    return SCN_OK;
}

}  // extern "C"
