// Batched stage 1 + stage 2 in one persistent launch: thousands of
// instances of uneven n (<= 256) are factored (CLA module of Section 2) and
// the first min(2^r, cap) solutions of each are reduced on the device.
//
// Work queue. CTAs pull item numbers from a global atomic counter. Items
// 0 .. B-1 factor instance b (the whole CTA runs factor_block). Items B and
// above are enumeration chunks: item B + b * C + c reduces solutions
// [c * chunk, (c + 1) * chunk) of instance b, C = ceil(cap / chunk); chunks
// past min(2^r, cap) are empty. Items are handed out in order, so every factor
// item has been taken by a running CTA before any chunk item is; a chunk of
// instance b waits (bounded) for the ready flag that the CTA factoring b sets
// after its table is written, and that CTA waits on nothing. Chunk results
// are added into the instance's hlf_reduce with 64-bit atomics.
//
// Every wait is bounded: after spin_limit polls the chunk is skipped and
// HLF_ERR_TIMEOUT is recorded in the batch status word.

#include <mutex>
#include <new>

#include "enum_impl.cuh"
#include "factor_impl.cuh"

namespace hlf {
namespace {

constexpr int kBatchMaxN = 256;
constexpr int kBatchMaxW = 4;
constexpr int kTableSlot = kTableTotalRows * kBatchMaxW;  // words per instance table slot

struct BatchArgs {
    const uint64_t* A;        // packed rows of all instances
    const int64_t* word_off;  // [B] word offset of instance b in A
    const int32_t* n;         // [B]
    int32_t B;
    uint64_t cap;             // solutions reduced per instance: min(2^min(r,64), cap)
    uint64_t chunk;           // solutions per work item
    uint32_t chunks_per_inst;
    int32_t* r_out;           // [B] rank, or -status
    hlf_reduce* red_out;      // [B]
    // workspace
    uint64_t* tables;         // [B][kTableSlot]
    int32_t* info;            // [B][2]
    int32_t* ready;           // [B]
    uint32_t* counter;        // [1]
    int32_t* status;          // [1]
    uint32_t spin_limit;
    uint32_t first_item;      // 0; B only when a test skips the factor items
};

__device__ __forceinline__ int ld_acquire(const int32_t* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr size_t batch_smem_bytes()
{
    size_t m = 0;
    m = factor_smem_bytes<1, kBatchMaxN>(kBatchMaxN) > m ? factor_smem_bytes<1, kBatchMaxN>(kBatchMaxN) : m;
    m = factor_smem_bytes<2, kBatchMaxN>(kBatchMaxN) > m ? factor_smem_bytes<2, kBatchMaxN>(kBatchMaxN) : m;
    m = factor_smem_bytes<3, kBatchMaxN>(kBatchMaxN) > m ? factor_smem_bytes<3, kBatchMaxN>(kBatchMaxN) : m;
    m = factor_smem_bytes<4, kBatchMaxN>(kBatchMaxN) > m ? factor_smem_bytes<4, kBatchMaxN>(kBatchMaxN) : m;
    m = sizeof(Table<kBatchMaxW>) > m ? sizeof(Table<kBatchMaxW>) : m;
    return (m + 15) / 16 * 16;
}

template <int W>
__device__ void batch_factor(const BatchArgs& a, int b, int n, unsigned char* smem)
{
    FactorOut o{nullptr, nullptr, a.tables + (size_t)b * kTableSlot, a.info + 2 * b, nullptr};
    factor_block<W, 1, kBatchMaxN>(a.A + a.word_off[b], n, o, smem);
}

template <int W>
__device__ void batch_chunk(const BatchArgs& a, int b, uint64_t first, uint64_t len, unsigned char* smem)
{
    constexpr int U = reduce_unroll(W);
    constexpr uint64_t kBlk = 1ull << U;
    Table<W>& t = *reinterpret_cast<Table<W>*>(smem);
    load_table_hash_domain<W>(t, a.tables + (size_t)b * kTableSlot);
    __syncthreads();
    // per-thread runs of whole 2^U blocks (chunks start at multiples of 2^U)
    const uint64_t per = ((len + blockDim.x - 1) / blockDim.x + kBlk - 1) & ~(kBlk - 1);
    Acc<W> acc;
    acc.zero();
    uint64_t cnt = 0;
    const uint64_t s = threadIdx.x * per;
    if (s < len) {
        cnt = min(per, len - s);
        reduce_run<W, U>(t, first + s, cnt, acc);
    }
    block_reduce<W>(cnt, acc);
    if (threadIdx.x == 0 && cnt) {
        hlf_reduce* r = a.red_out + b;
        atomicAdd(reinterpret_cast<unsigned long long*>(&r->count), (unsigned long long)cnt);
        atomicAdd(reinterpret_cast<unsigned long long*>(&r->hsum), (unsigned long long)acc.hs);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t f = acc.fold_word(w);
            if (f) atomicXor(reinterpret_cast<unsigned long long*>(&r->xor_fold[w]), (unsigned long long)f);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 4) batch_kernel(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ int s_state;  // instance rank (>= 0), or < 0 to skip the chunk
    const uint32_t n_items = (uint32_t)a.B + (uint32_t)a.B * a.chunks_per_inst;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u) + a.first_item;
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        if (item < (uint32_t)a.B) {
            const int b = (int)item;
            const int n = a.n[b];
            if (n < 1 || n > kBatchMaxN) {
                if (threadIdx.x == 0) {
                    a.info[2 * b] = HLF_ERR_SIZE;
                    a.info[2 * b + 1] = -1;
                }
            } else {
                switch ((n + 63) >> 6) {
                case 1: batch_factor<1>(a, b, n, smem); break;
                case 2: batch_factor<2>(a, b, n, smem); break;
                case 3: batch_factor<3>(a, b, n, smem); break;
                default: batch_factor<4>(a, b, n, smem); break;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const int st = a.info[2 * b];
                a.r_out[b] = st ? -st : a.info[2 * b + 1];
                __threadfence();
                st_release(a.ready + b, 1);
            }
            continue;
        }
        const uint32_t j = item - (uint32_t)a.B;
        const int b = (int)(j / a.chunks_per_inst);
        const uint64_t c = j % a.chunks_per_inst;
        if (threadIdx.x == 0) {
            uint32_t polls = 0;
            while (ld_acquire(a.ready + b) == 0 && ++polls < a.spin_limit) __nanosleep(128);
            if (polls >= a.spin_limit) {
                atomicCAS(a.status, 0, HLF_ERR_TIMEOUT);
                s_state = -1;
            } else {
                s_state = __ldcg(a.info + 2 * b) ? -1 : __ldcg(a.info + 2 * b + 1);
            }
        }
        __syncthreads();
        const int r = s_state;
        __syncthreads();
        if (r < 0) continue;
        const int n = a.n[b];
        const uint64_t space_cap = r >= 64 ? ~0ull : (1ull << r);
        const uint64_t total = space_cap < a.cap ? space_cap : a.cap;
        const uint64_t first = c * a.chunk;
        if (first >= total) continue;
        const uint64_t len = min(a.chunk, total - first);
        switch ((n + 63) >> 6) {
        case 1: batch_chunk<1>(a, b, first, len, smem); break;
        case 2: batch_chunk<2>(a, b, first, len, smem); break;
        case 3: batch_chunk<3>(a, b, first, len, smem); break;
        default: batch_chunk<4>(a, b, first, len, smem); break;
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace hlf

// ---------------------------------------------------------------------------
// Scratch for hlf_batch_factor_reduce_noalloc: a file-scope device array, so
// that entry point never allocates. It holds the same workspace a plan holds,
// for up to HLF_BATCH_NOALLOC_MAX matrices. Host code must not use the
// array's name as a device address: the address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
namespace hlf {
namespace {

struct NoAllocScratch {
    uint64_t tables[(size_t)HLF_BATCH_NOALLOC_MAX * kTableSlot];
    int32_t info[2 * HLF_BATCH_NOALLOC_MAX];
    int32_t ready[HLF_BATCH_NOALLOC_MAX];
    uint32_t counter;
    int32_t status;
};

}  // namespace
}  // namespace hlf

static __device__ __align__(256) unsigned char g_batch_noalloc_scratch[sizeof(hlf::NoAllocScratch)];

static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_addr[64] = {nullptr};

struct hlf_batch {
    int device = 0;
    int32_t max_instances = 0;
    unsigned char* dmem = nullptr;
    uint64_t* tables = nullptr;
    int32_t* info = nullptr;
    int32_t* ready = nullptr;
    uint32_t* counter = nullptr;  // counter and status are adjacent (one memset)
    int32_t* status = nullptr;
    int32_t ctas_per_sm = 0;      // 0 = as many as fit
    uint64_t chunk = 1ull << 16;
    uint32_t spin_limit = 1u << 23;
    uint32_t debug = 0;           // HLF_BATCH_DEBUG_* fault-injection flags (tests only)
    cudaEvent_t last = nullptr;
    cudaStream_t priv = nullptr;
};

extern "C" {

hlf_status hlf_batch_create(int32_t max_instances, hlf_batch** out)
{
    if (!out) return HLF_ERR_ARG;
    *out = nullptr;
    if (max_instances < 1 || max_instances > (1 << 24)) return HLF_ERR_ARG;
    if (hlf::take_injected_alloc_failure()) return HLF_ERR_NOMEM;
    hlf_batch* b = new (std::nothrow) hlf_batch;
    if (!b) return HLF_ERR_NOMEM;
    b->max_instances = max_instances;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return HLF_ERR_CUDA;
    }
    const size_t tab = sizeof(uint64_t) * hlf::kTableSlot * (size_t)max_instances;
    const size_t info = sizeof(int32_t) * 2 * (size_t)max_instances;
    const size_t ready = sizeof(int32_t) * (size_t)max_instances;
    const size_t off_info = tab;
    const size_t off_ready = (off_info + info + 255) / 256 * 256;
    const size_t off_ctr = (off_ready + ready + 255) / 256 * 256;
    const size_t bytes = off_ctr + 256;
    if (cudaMalloc(&b->dmem, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return HLF_ERR_NOMEM;
    }
    b->tables = reinterpret_cast<uint64_t*>(b->dmem);
    b->info = reinterpret_cast<int32_t*>(b->dmem + off_info);
    b->ready = reinterpret_cast<int32_t*>(b->dmem + off_ready);
    b->counter = reinterpret_cast<uint32_t*>(b->dmem + off_ctr);
    b->status = reinterpret_cast<int32_t*>(b->dmem + off_ctr + 4);
    if (cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemset(b->status, 0, sizeof(int32_t)) != cudaSuccess) {
        hlf_batch_destroy(b);
        return HLF_ERR_CUDA;
    }
    static bool attr_set[64] = {false};
    if (b->device < 64 && !attr_set[b->device]) {
        if (cudaFuncSetAttribute(hlf::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)hlf::batch_smem_bytes()) != cudaSuccess) {
            hlf_batch_destroy(b);
            return HLF_ERR_CUDA;
        }
        attr_set[b->device] = true;
    }
    *out = b;
    return HLF_OK;
}

hlf_status hlf_batch_set_tiles(hlf_batch* b, int32_t ctas_per_sm, uint64_t chunk)
{
    if (!b || ctas_per_sm < 0 || ctas_per_sm > 64 || chunk < 256 || (chunk & (chunk - 1))) return HLF_ERR_ARG;
    b->ctas_per_sm = ctas_per_sm;
    b->chunk = chunk;
    return HLF_OK;
}

hlf_status hlf_batch_set_spin_limit(hlf_batch* b, uint32_t polls)
{
    if (!b || polls == 0) return HLF_ERR_ARG;
    b->spin_limit = polls;
    return HLF_OK;
}

hlf_status hlf_batch_set_debug(hlf_batch* b, uint32_t flags)
{
    if (!b || (flags & ~1u)) return HLF_ERR_ARG;
    b->debug = flags;
    return HLF_OK;
}

hlf_status hlf_batch_factor_reduce(hlf_batch* b, const uint64_t* A_dev, const int64_t* word_off_dev,
                                   const int32_t* n_dev, int32_t count, uint64_t cap, int32_t* r_dev,
                                   hlf_reduce* red_dev, void* stream)
{
    if (!b || count < 0 || count > b->max_instances || cap == 0) return HLF_ERR_ARG;
    if (count == 0) return HLF_OK;
    if (!A_dev || !word_off_dev || !n_dev || !r_dev || !red_dev) return HLF_ERR_ARG;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) return HLF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf::BatchArgs a{};
    a.A = A_dev;
    a.word_off = word_off_dev;
    a.n = n_dev;
    a.B = count;
    a.cap = cap;
    a.chunk = b->chunk;
    const uint64_t cpi = (cap + b->chunk - 1) / b->chunk;
    if (cpi > (1u << 20)) return HLF_ERR_RANGE;
    a.chunks_per_inst = (uint32_t)cpi;
    a.r_out = r_dev;
    a.red_out = red_dev;
    a.tables = b->tables;
    a.info = b->info;
    a.ready = b->ready;
    a.counter = b->counter;
    a.status = b->status;
    a.spin_limit = b->spin_limit;
    // With debug flag 1 the queue starts after the factor items, so no ready
    // flag is ever set and every chunk's bounded wait runs out.
    a.first_item = (b->debug & 1u) ? (uint32_t)count : 0u;
    const size_t smem = hlf::batch_smem_bytes();
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, hlf::batch_kernel, hlf::kThreads, smem) != cudaSuccess ||
        fit < 1)
        return HLF_ERR_CUDA;
    const int per_sm = (b->ctas_per_sm > 0 && b->ctas_per_sm < fit) ? b->ctas_per_sm : fit;
    const int grid = hlf::sm_count() * per_sm;
    // The 32-bit queue counter is incremented once per item and once more by
    // every CTA when it finds the queue empty; it must not wrap.
    if ((uint64_t)count * (cpi + 1) + (uint64_t)grid > 0xffffffffull) return HLF_ERR_RANGE;
    if (cudaMemsetAsync(b->counter, 0, sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(b->ready, 0, sizeof(int32_t) * (size_t)count, s) != cudaSuccess ||
        cudaMemsetAsync(red_dev, 0, sizeof(hlf_reduce) * (size_t)count, s) != cudaSuccess)
        return HLF_ERR_CUDA;
    hlf::batch_kernel<<<grid, hlf::kThreads, smem, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    // While the stream is being captured into a CUDA graph the event is not
    // recorded; after replaying such a graph, synchronise the stream before
    // hlf_batch_get_status.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return HLF_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return HLF_OK;
    return cudaEventRecord(b->last, s) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

hlf_status hlf_batch_get_status(hlf_batch* b)
{
    if (!b) return HLF_ERR_ARG;
    if (cudaEventSynchronize(b->last) != cudaSuccess) return HLF_ERR_CUDA;
    int32_t st = 0;
    if (cudaMemcpyAsync(&st, b->status, sizeof(st), cudaMemcpyDeviceToHost, b->priv) != cudaSuccess ||
        cudaStreamSynchronize(b->priv) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (st != 0) {
        if (cudaMemsetAsync(b->status, 0, sizeof(int32_t), b->priv) != cudaSuccess ||
            cudaStreamSynchronize(b->priv) != cudaSuccess)
            return HLF_ERR_CUDA;
    }
    return (hlf_status)st;
}

hlf_status hlf_batch_factor_reduce_noalloc(const uint64_t* A_dev, const int64_t* word_off_dev,
                                           const int32_t* n_dev, int32_t count, uint64_t cap, int32_t* r_dev,
                                           hlf_reduce* red_dev, void* stream)
{
    if (count < 0 || cap == 0) return HLF_ERR_ARG;
    if (count > HLF_BATCH_NOALLOC_MAX) return HLF_ERR_SIZE;
    if (count == 0) return HLF_OK;
    if (!A_dev || !word_off_dev || !n_dev || !r_dev || !red_dev) return HLF_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HLF_ERR_CUDA;
    if (dev < 0 || dev >= 64) return HLF_ERR_ARG;
    unsigned char* base = nullptr;
    {
        // First call on this device: find the scratch array's device address
        // (the device is current here) and allow the kernel its shared memory.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_batch_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return HLF_ERR_CUDA;
            }
            if (cudaFuncSetAttribute(hlf::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hlf::batch_smem_bytes()) != cudaSuccess) {
                cudaGetLastError();
                return HLF_ERR_CUDA;
            }
            g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_noalloc_addr[dev];
    }
    hlf::NoAllocScratch* sc = reinterpret_cast<hlf::NoAllocScratch*>(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf::BatchArgs a{};
    a.A = A_dev;
    a.word_off = word_off_dev;
    a.n = n_dev;
    a.B = count;
    a.cap = cap;
    a.chunk = 1ull << 16;
    const uint64_t cpi = (cap + a.chunk - 1) / a.chunk;
    if (cpi > (1u << 20) || (uint64_t)count * (cpi + 1) > 0xffffffffull) return HLF_ERR_RANGE;
    a.chunks_per_inst = (uint32_t)cpi;
    a.r_out = r_dev;
    a.red_out = red_dev;
    a.tables = sc->tables;
    a.info = sc->info;
    a.ready = sc->ready;
    a.counter = &sc->counter;
    a.status = &sc->status;
    a.spin_limit = 1u << 23;
    a.first_item = 0;
    // The array keeps the previous call's contents: clear the queue counter,
    // the status word and this call's ready flags; the results are overwritten.
    if (cudaMemsetAsync(&sc->counter, 0, sizeof(uint32_t) + sizeof(int32_t), s) != cudaSuccess ||
        cudaMemsetAsync(sc->ready, 0, sizeof(int32_t) * (size_t)count, s) != cudaSuccess ||
        cudaMemsetAsync(red_dev, 0, sizeof(hlf_reduce) * (size_t)count, s) != cudaSuccess)
        return HLF_ERR_CUDA;
    const size_t smem = hlf::batch_smem_bytes();
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, hlf::batch_kernel, hlf::kThreads, smem) != cudaSuccess ||
        fit < 1)
        return HLF_ERR_CUDA;
    hlf::batch_kernel<<<hlf::sm_count() * fit, hlf::kThreads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

hlf_status hlf_batch_destroy(hlf_batch* b)
{
    if (!b) return HLF_OK;
    hlf_status st = HLF_OK;
    if (b->last && cudaEventSynchronize(b->last) != cudaSuccess) st = HLF_ERR_CUDA;
    if (b->dmem && cudaFree(b->dmem) != cudaSuccess) st = HLF_ERR_CUDA;
    if (b->last) cudaEventDestroy(b->last);
    if (b->priv) cudaStreamDestroy(b->priv);
    delete b;
    return st;
}

}  // extern "C"
