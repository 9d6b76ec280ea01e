// Stage 2 for small instances without the rank on the host: the kernel reads
// r from the status word the factor kernel wrote, and stores z(i) =
// z0 ^ XOR_{k in g(i)} B_k (Eq. 3 with the Gray-code basis order) for every
// i < min(2^r, cap), each straight from the definition. Meant for instances
// of up to a few million solutions, where the time is the launch and the
// host round trip it saves; hlf_enumerate_store walks large windows.

#include "enum_impl.cuh"
#include "upto.cuh"

namespace hlf {
namespace {

template <int W>
__global__ void __launch_bounds__(kThreads) store_upto_kernel(const uint64_t* __restrict__ table,
                                                              const int32_t* info, uint64_t cap,
                                                              uint64_t* __restrict__ out)
{
    __shared__ Table<W> t;
    __shared__ uint64_t s_count;
    load_table<W>(t, table);
    if (threadIdx.x == 0) {
        const int32_t r = *reinterpret_cast<const volatile int32_t*>(info + 1);  // -1 after a fault
        s_count = r < 0 ? 0ull : (r >= 64 ? cap : (cap < (1ull << r) ? cap : (1ull << r)));
    }
    __syncthreads();
    const uint64_t count = s_count;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t z[W];
        seed<W>(t, i, z);
#pragma unroll
        for (int w = 0; w < W; ++w) out[i * W + w] = z[w];
    }
}

template <int W>
hlf_status launch_store_upto_w(const uint64_t* table, const int32_t* info, uint64_t cap, uint64_t* out,
                               cudaStream_t s)
{
    const uint64_t most = (uint64_t)sm_count() * 4;
    uint64_t blocks = (cap + kThreads - 1) / kThreads;
    if (blocks > most) blocks = most;
    if (blocks == 0) blocks = 1;
    store_upto_kernel<W><<<(unsigned)blocks, kThreads, 0, s>>>(table, info, cap, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_store_upto(const uint64_t* table, int W, const int32_t* info, uint64_t cap, uint64_t* out,
                             cudaStream_t s)
{
    switch (W) {
    case 1: return launch_store_upto_w<1>(table, info, cap, out, s);
    case 2: return launch_store_upto_w<2>(table, info, cap, out, s);
    case 3: return launch_store_upto_w<3>(table, info, cap, out, s);
    case 4: return launch_store_upto_w<4>(table, info, cap, out, s);
    case 5: return launch_store_upto_w<5>(table, info, cap, out, s);
    case 6: return launch_store_upto_w<6>(table, info, cap, out, s);
    case 7: return launch_store_upto_w<7>(table, info, cap, out, s);
    case 8: return launch_store_upto_w<8>(table, info, cap, out, s);
    case 9: return launch_store_upto_w<9>(table, info, cap, out, s);
    case 10: return launch_store_upto_w<10>(table, info, cap, out, s);
    case 11: return launch_store_upto_w<11>(table, info, cap, out, s);
    case 12: return launch_store_upto_w<12>(table, info, cap, out, s);
    case 13: return launch_store_upto_w<13>(table, info, cap, out, s);
    case 14: return launch_store_upto_w<14>(table, info, cap, out, s);
    case 15: return launch_store_upto_w<15>(table, info, cap, out, s);
    case 16: return launch_store_upto_w<16>(table, info, cap, out, s);
    default: return HLF_ERR_SIZE;
    }
}

}  // namespace hlf
