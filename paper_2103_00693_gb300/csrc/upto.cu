// Stage 2 for small instances without the rank on the host: the kernels read
// r from the status word the factor kernel wrote.
//   store_upto_kernel   stores z(i) = z0 ^ XOR_{k in g(i)} B_k (Eq. 3 with
//                       the Gray-code basis order) for every i < min(2^r, cap),
//                       each straight from the definition. Meant for
//                       instances of up to a few million solutions, where the
//                       time is the launch and the host round trip it saves;
//                       hlf_enumerate_store walks large windows.
//   reduce_upto_kernel  the reduce of [0, min(2^r, cap)) with the walk of the
//                       single-instance reduce; the run per thread is cut on
//                       the device from the actual count.

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
        if (HLF_IN_BOUNDS(i, cap, kSiteUptoStore)) {
#pragma unroll
            for (int w = 0; w < W; ++w) out[i * W + w] = z[w];
        }
    }
}

template <int W, int U>
__global__ void __launch_bounds__(kThreads) reduce_upto_kernel(const uint64_t* __restrict__ table,
                                                               const int32_t* info, uint64_t cap,
                                                               hlf_reduce* __restrict__ out)
{
    __shared__ Table<W> t;
    __shared__ uint64_t s_count;
    load_table_hash_domain<W>(t, table);
    if (threadIdx.x == 0) {
        const int32_t r = *reinterpret_cast<const volatile int32_t*>(info + 1);  // -1 after a fault
        s_count = r < 0 ? 0ull : (r >= 64 ? cap : (cap < (1ull << r) ? cap : (1ull << r)));
    }
    __syncthreads();
    const uint64_t count = s_count;
    const uint64_t threads = (uint64_t)gridDim.x * blockDim.x;
    uint64_t per = (count + threads - 1) / threads;
    per = (per + (1ull << U) - 1) & ~((1ull << U) - 1);  // runs stay aligned to the Gray blocks
    if (per == 0) per = 1ull << U;
    const uint64_t a = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * per;
    Acc<W> acc;
    acc.zero();
    uint64_t cnt = 0;
    if (a < count) {
        cnt = min(per, count - a);
        reduce_run<W, U>(t, a, cnt, acc);
    }
    block_reduce<W>(cnt, acc);
    if (threadIdx.x == 0 && cnt) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&out->count), (unsigned long long)cnt);
        atomicAdd(reinterpret_cast<unsigned long long*>(&out->hsum), (unsigned long long)acc.hs);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t f = acc.fold_word(w);
            if (f) atomicXor(reinterpret_cast<unsigned long long*>(&out->xor_fold[w]), (unsigned long long)f);
        }
    }
}

template <int W>
hlf_status launch_reduce_upto_w(const uint64_t* table, const int32_t* info, uint64_t cap, hlf_reduce* out,
                                cudaStream_t s)
{
    constexpr int U = reduce_unroll(W);
    // one wave at most (8 CTAs of 256 threads per SM), and runs of at least
    // 256 solutions (enough to amortise a seed of <= 64 row XORs) when the
    // whole cap is enumerated: small instances spread over many SMs
    const uint64_t most = (uint64_t)sm_count() * 8;
    uint64_t blocks = (cap + 256 * kThreads - 1) / (256 * kThreads);
    if (blocks > most) blocks = most;
    if (blocks == 0) blocks = 1;
    reduce_upto_kernel<W, U><<<(unsigned)blocks, kThreads, 0, s>>>(table, info, cap, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
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

hlf_status launch_reduce_upto(const uint64_t* table, int W, const int32_t* info, uint64_t cap, hlf_reduce* out,
                              cudaStream_t s)
{
    switch (W) {
    case 1: return launch_reduce_upto_w<1>(table, info, cap, out, s);
    case 2: return launch_reduce_upto_w<2>(table, info, cap, out, s);
    case 3: return launch_reduce_upto_w<3>(table, info, cap, out, s);
    case 4: return launch_reduce_upto_w<4>(table, info, cap, out, s);
    case 5: return launch_reduce_upto_w<5>(table, info, cap, out, s);
    case 6: return launch_reduce_upto_w<6>(table, info, cap, out, s);
    case 7: return launch_reduce_upto_w<7>(table, info, cap, out, s);
    case 8: return launch_reduce_upto_w<8>(table, info, cap, out, s);
    case 9: return launch_reduce_upto_w<9>(table, info, cap, out, s);
    case 10: return launch_reduce_upto_w<10>(table, info, cap, out, s);
    case 11: return launch_reduce_upto_w<11>(table, info, cap, out, s);
    case 12: return launch_reduce_upto_w<12>(table, info, cap, out, s);
    case 13: return launch_reduce_upto_w<13>(table, info, cap, out, s);
    case 14: return launch_reduce_upto_w<14>(table, info, cap, out, s);
    case 15: return launch_reduce_upto_w<15>(table, info, cap, out, s);
    case 16: return launch_reduce_upto_w<16>(table, info, cap, out, s);
    default: return HLF_ERR_SIZE;
    }
}

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

HLF_DEBUG_TAKE(upto)

}  // namespace hlf
