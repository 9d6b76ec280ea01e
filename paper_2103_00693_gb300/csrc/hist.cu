// Histogram of a bit field of every solution in a window, computed on the
// device while enumerating (no solution is stored): the counts behind the
// paper's output distributions of Figs. 3, 6 and 7, where each square shows
// how often one bit pattern of the first or last bits occurs.
//
// The walk is the reduce's (enum_impl.cuh, raw table: no hash); each
// solution's bits [lo, lo + nbits) select a bin. Up to 2^14 bins live in
// shared memory per CTA (32-bit counters, flushed to the global 64-bit bins
// with one atomic per nonzero bin); wider fields count straight into global
// memory.

#include "enum_impl.cuh"

namespace hlf {
namespace {

constexpr int kHistSmemBits = 14;
constexpr uint64_t kHistMaxPerThread = 1ull << 23;  // keeps a CTA's counts below 2^32

template <int W>
struct HistSink {
    uint32_t* s_bins;               // shared, when nbits <= kHistSmemBits
    unsigned long long* g_bins;     // global, otherwise
    int word, shift, nbits;
    uint64_t mask;
    __device__ __forceinline__ void consume(const uint64_t (&z)[W])
    {
        uint64_t a = 0, b = 0;  // words `word` and `word + 1`, selected without indexing registers
#pragma unroll
        for (int k = 0; k < W; ++k) {
            if (k == word) a = z[k];
            if (k == word + 1) b = z[k];
        }
        uint64_t v = a >> shift;
        if (shift) v |= b << (64 - shift);
        v &= mask;
        if (nbits <= kHistSmemBits) atomicAdd(&s_bins[v], 1u);
        else atomicAdd(&g_bins[v], 1ull);
    }
};

template <int W, int U>
__global__ void __launch_bounds__(kThreads) hist_kernel(const uint64_t* __restrict__ table, uint64_t offset,
                                                        uint64_t count, uint64_t per_thread, uint64_t used,
                                                        int lo, int nbits, unsigned long long* __restrict__ out)
{
    extern __shared__ uint32_t s_bins[];
    __shared__ Table<W> t;
    load_table<W>(t, table);
    const bool in_smem = nbits <= kHistSmemBits;
    const uint32_t nb = 1u << nbits;
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    HistSink<W> sink{s_bins, out, lo >> 6, lo & 63, nbits, nbits == 64 ? ~0ull : ((1ull << nbits) - 1)};
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < used) {
        const uint64_t a = g * per_thread;
        if (a < count) walk_run<W, U, HistSink<W>>(t, offset + a, min(per_thread, count - a), sink);
    }
    __syncthreads();
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
            if (s_bins[i]) atomicAdd(&out[i], (unsigned long long)s_bins[i]);
}

template <int W>
hlf_status launch_hist_w(const uint64_t* table, uint64_t offset, uint64_t count, int lo, int nbits,
                         uint64_t* out, cudaStream_t s)
{
    constexpr int U = unroll_for(W);
    const size_t smem = nbits <= kHistSmemBits ? (sizeof(uint32_t) << nbits) : 0;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(hist_kernel<W, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(uint32_t) << kHistSmemBits)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hist_kernel<W, U>, kThreads, smem) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    const uint64_t max_threads = (uint64_t)sm_count() * per_sm * kThreads;
    uint64_t threads = (count + 2047) / 2048;
    if (threads > max_threads) threads = max_threads;
    if (threads == 0) threads = 1;
    uint64_t per_thread = (count + threads - 1) / threads;
    per_thread = (per_thread + (1ull << U) - 1) & ~((1ull << U) - 1);
    if (per_thread > kHistMaxPerThread) per_thread = kHistMaxPerThread;
    const uint64_t used = (count + per_thread - 1) / per_thread;
    const uint64_t blocks = (used + kThreads - 1) / kThreads;
    if (blocks > 0x7fffffffull) return HLF_ERR_RANGE;
    hist_kernel<W, U><<<(unsigned)blocks, kThreads, smem, s>>>(table, offset, count, per_thread, used, lo, nbits,
                                                               reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_histogram(const uint64_t* table, int W, uint64_t offset, uint64_t count, int lo, int nbits,
                            uint64_t* out, cudaStream_t s)
{
    switch (W) {
    case 1: return launch_hist_w<1>(table, offset, count, lo, nbits, out, s);
    case 2: return launch_hist_w<2>(table, offset, count, lo, nbits, out, s);
    case 3: return launch_hist_w<3>(table, offset, count, lo, nbits, out, s);
    case 4: return launch_hist_w<4>(table, offset, count, lo, nbits, out, s);
    case 5: return launch_hist_w<5>(table, offset, count, lo, nbits, out, s);
    case 6: return launch_hist_w<6>(table, offset, count, lo, nbits, out, s);
    case 7: return launch_hist_w<7>(table, offset, count, lo, nbits, out, s);
    case 8: return launch_hist_w<8>(table, offset, count, lo, nbits, out, s);
    case 9: return launch_hist_w<9>(table, offset, count, lo, nbits, out, s);
    case 10: return launch_hist_w<10>(table, offset, count, lo, nbits, out, s);
    case 11: return launch_hist_w<11>(table, offset, count, lo, nbits, out, s);
    case 12: return launch_hist_w<12>(table, offset, count, lo, nbits, out, s);
    case 13: return launch_hist_w<13>(table, offset, count, lo, nbits, out, s);
    case 14: return launch_hist_w<14>(table, offset, count, lo, nbits, out, s);
    case 15: return launch_hist_w<15>(table, offset, count, lo, nbits, out, s);
    case 16: return launch_hist_w<16>(table, offset, count, lo, nbits, out, s);
    default: return HLF_ERR_SIZE;
    }
}

}  // namespace hlf
