// Stage 1 for one matrix: one CTA runs factor_block (factor_impl.cuh) with
// the rows of A in registers: one row per thread up to n = 512, two rows per
// thread above (at most 512 threads, so up to 128 registers each and no
// spilling of the 16-word rows of n = 1024).

#include "factor_impl.cuh"

namespace hlf {
namespace {

template <int W>
constexpr int rows_per_thread() { return W <= 8 ? 1 : 2; }

template <int W>
__global__ void __launch_bounds__(512, 1) factor_kernel(const uint64_t* __restrict__ A, int n, FactorOut o)
{
    extern __shared__ __align__(16) unsigned char smem[];
    factor_block<W, rows_per_thread<W>(), HLF_MAX_N>(A, n, o, smem);
}

template <int W>
hlf_status launch_factor_w(const uint64_t* A, int n, const FactorOut& o, cudaStream_t s)
{
    constexpr int R = rows_per_thread<W>();
    const int threads = ((n + R - 1) / R + 31) / 32 * 32;
    const size_t smem = factor_smem_bytes<W, HLF_MAX_N>(n);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(factor_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)factor_smem_bytes<W, HLF_MAX_N>(HLF_MAX_N)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    factor_kernel<W><<<1, threads, smem, s>>>(A, n, o);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_factor(const uint64_t* A, int n, int W, const FactorOut& o, cudaStream_t s)
{
    switch (W) {
    case 1: return launch_factor_w<1>(A, n, o, s);
    case 2: return launch_factor_w<2>(A, n, o, s);
    case 3: return launch_factor_w<3>(A, n, o, s);
    case 4: return launch_factor_w<4>(A, n, o, s);
    case 5: return launch_factor_w<5>(A, n, o, s);
    case 6: return launch_factor_w<6>(A, n, o, s);
    case 7: return launch_factor_w<7>(A, n, o, s);
    case 8: return launch_factor_w<8>(A, n, o, s);
    case 9: return launch_factor_w<9>(A, n, o, s);
    case 10: return launch_factor_w<10>(A, n, o, s);
    case 11: return launch_factor_w<11>(A, n, o, s);
    case 12: return launch_factor_w<12>(A, n, o, s);
    case 13: return launch_factor_w<13>(A, n, o, s);
    case 14: return launch_factor_w<14>(A, n, o, s);
    case 15: return launch_factor_w<15>(A, n, o, s);
    case 16: return launch_factor_w<16>(A, n, o, s);
    default: return HLF_ERR_SIZE;
    }
}

}  // namespace hlf
