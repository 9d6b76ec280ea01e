// Measurement helper behind the histogram's roofline: the rate at which this
// GPU retires 32-bit shared-memory atomic adds. The paper has no counterpart;
// the kernel does none of the method's arithmetic. Every thread of one full
// wave of CTAs adds 1 to `iters` counters; the 32 lanes of a warp always hit
// 32 distinct banks (the pattern of the histogram's interleaved walk when its
// lanes land in distinct bins), and the counter addresses are compile-time
// offsets from one register, so each atomic is one instruction with no
// address arithmetic around it.

#include "hlf_internal.cuh"

namespace hlf {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) smem_atomic_probe_kernel(uint32_t iters,
                                                                          unsigned long long* sum)
{
    __shared__ uint32_t bins[4 * kProbeUnroll * 32];
    for (int i = threadIdx.x; i < 4 * kProbeUnroll * 32; i += kProbeThreads) bins[i] = 0;
    __syncthreads();
    uint32_t* my = bins + (threadIdx.x & 31) + kProbeUnroll * 32 * ((threadIdx.x >> 5) & 3);
    for (uint32_t i = 0; i < iters; i += kProbeUnroll) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k) atomicAdd(my + 32 * k, 1u);
    }
    __syncthreads();
    unsigned long long part = 0;
    for (int i = threadIdx.x; i < 4 * kProbeUnroll * 32; i += kProbeThreads) part += bins[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, part);
}

}  // namespace
}  // namespace hlf

extern "C" hlf_status hlf_probe_smem_atomics(uint32_t iters, uint64_t* sum_dev, uint64_t* atomics, void* stream)
{
    if (!sum_dev || !atomics || iters == 0 || iters % hlf::kProbeUnroll) return HLF_ERR_ARG;
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, hlf::smem_atomic_probe_kernel, hlf::kProbeThreads, 0) !=
            cudaSuccess ||
        fit < 1)
        return HLF_ERR_CUDA;
    const unsigned grid = (unsigned)(hlf::sm_count() * fit);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(sum_dev, 0, sizeof(uint64_t), s) != cudaSuccess) return HLF_ERR_CUDA;
    hlf::smem_atomic_probe_kernel<<<grid, hlf::kProbeThreads, 0, s>>>(iters,
                                                                       reinterpret_cast<unsigned long long*>(sum_dev));
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    *atomics = (uint64_t)grid * hlf::kProbeThreads * iters;
    return HLF_OK;
}
