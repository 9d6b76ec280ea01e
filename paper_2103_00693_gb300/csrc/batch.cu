// Batched stage 1 + stage 2 in persistent launches: thousands of instances
// of uneven n (<= 256) are factored (CLA module of Section 2) and the first
// min(2^r, cap) solutions of each are reduced on the device or stored.
//
// Work queue. CTAs pull item numbers from a global atomic counter. A launch
// has factor items (one per instance: the whole CTA runs factor_block) and/or
// enumeration chunks (item c of instance b covers solutions
// [c * chunk, (c + 1) * chunk); chunks past the instance's total are empty).
// The fused launch (hlf_batch_factor_reduce) has both: factor items 0 .. B-1
// first, then the chunks. Items are handed out in order, so every factor item
// has been taken by a running CTA before any chunk item is; a chunk of
// instance b waits (bounded) for the ready flag that the CTA factoring b sets
// after its table is written, and that CTA waits on nothing. The separate
// calls (hlf_factor_batched, then hlf_enumerate_batched) run the two kinds in
// two launches; the factorisations stay in the plan's workspace in between.
// Reduce chunks add into the instance's hlf_reduce with 64-bit atomics; store
// chunks write their solutions, 32 consecutive ones per warp step, with the
// lane-interleaved Gray identity of the single-instance store kernel.
//
// Launch shape. One kernel per CTA size T = 64, 128 or 256 threads (2, 4 or
// 8 warps per work item, chosen by the autotuner): every item, factorisation
// or chunk, is worked on by one CTA, and a CTA of T threads holds 256 / T
// rows of a matrix per thread. Smaller CTAs factor more instances at once
// (more CTAs per SM); larger ones walk a chunk with more threads.
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
constexpr int kInfo = 4;  // per instance: status, rank, n, unused
constexpr int kStoreM = 5;  // log2 of the 32 consecutive solutions a warp stores per step

enum : uint32_t { kModeFused = 0, kModeFactor = 1, kModeReduce = 2, kModeStore = 3 };

struct BatchArgs {
    const uint64_t* A;        // packed rows of all instances
    const int64_t* word_off;  // fused: [B] word offsets; factor: [B + 1] offsets (n from the sizes)
    const int32_t* n;         // fused: [B]; otherwise unused
    int32_t B;
    uint32_t mode;
    uint64_t cap;             // solutions per instance: min(2^min(r,64), cap)
    uint64_t chunk;           // solutions per work item
    uint32_t chunks_per_inst;
    int32_t* r_out;           // [B] rank, or -status (fused and factor launches)
    hlf_reduce* red_out;      // [B] (fused and reduce launches)
    uint64_t* out;            // store launches: solutions of instance b at out + out_off[b]
    const int64_t* out_off;   // [B + 1]; instance b stores at most (out_off[b+1] - out_off[b]) / W_b
    // workspace
    uint64_t* tables;         // [B][kTableSlot]
    int32_t* info;            // [B][kInfo]
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

template <int T>
constexpr size_t batch_smem_bytes()
{
    constexpr int NW = T / 32;
    size_t m = 0;
    m = factor_smem_bytes<1, kBatchMaxN, NW>(kBatchMaxN) > m ? factor_smem_bytes<1, kBatchMaxN, NW>(kBatchMaxN) : m;
    m = factor_smem_bytes<2, kBatchMaxN, NW>(kBatchMaxN) > m ? factor_smem_bytes<2, kBatchMaxN, NW>(kBatchMaxN) : m;
    m = factor_smem_bytes<3, kBatchMaxN, NW>(kBatchMaxN) > m ? factor_smem_bytes<3, kBatchMaxN, NW>(kBatchMaxN) : m;
    m = factor_smem_bytes<4, kBatchMaxN, NW>(kBatchMaxN) > m ? factor_smem_bytes<4, kBatchMaxN, NW>(kBatchMaxN) : m;
    // store chunks: table, step rows C_j, per-warp staging
    const size_t st = sizeof(Table<kBatchMaxW>) + sizeof(uint64_t) * (kTableRows - kStoreM) * kBatchMaxW +
                      sizeof(uint64_t) * NW * stage_words<kBatchMaxW>();
    m = st > m ? st : m;
    return (m + 15) / 16 * 16;
}
static_assert(batch_smem_bytes<256>() <= 48 * 1024, "fits the default dynamic shared-memory limit");
static_assert(batch_smem_bytes<64>() <= 48 * 1024, "fits the default dynamic shared-memory limit");

// n of a matrix given only its size in words: n * ceil(n / 64) words. The
// word counts of different W do not overlap (W = k gives (64k(k-1), 64k^2]),
// so n is unique; -1 if the size fits no n <= kBatchMaxN.
__device__ __forceinline__ int n_of_words(int64_t words)
{
#pragma unroll
    for (int W = 1; W <= kBatchMaxW; ++W) {
        if (words % W) continue;
        const int64_t n = words / W;
        if (n > 64 * (W - 1) && n <= 64 * W) return (int)n;
    }
    return -1;
}

template <int W, int T>
__device__ void batch_factor(const BatchArgs& a, int b, int n, const uint64_t* A, unsigned char* smem)
{
    FactorOut o{nullptr, nullptr, a.tables + (size_t)b * kTableSlot, a.info + kInfo * b, nullptr};
    factor_block<W, kBatchMaxN / T, kBatchMaxN, T / 32>(A, n, o, smem);
}

template <int W, int T>
__device__ void batch_reduce_chunk(const BatchArgs& a, int b, uint64_t first, uint64_t len, unsigned char* smem)
{
    constexpr int U = reduce_unroll(W);
    constexpr uint64_t kBlk = 1ull << U;
    Table<W>& t = *reinterpret_cast<Table<W>*>(smem);
    load_table_hash_domain<W>(t, a.tables + (size_t)b * kTableSlot);
    __syncthreads();
    // per-thread runs of whole 2^U blocks (chunks start at multiples of 2^U)
    const uint64_t per = ((len + T - 1) / T + kBlk - 1) & ~(kBlk - 1);
    Acc<W> acc;
    acc.zero();
    uint64_t cnt = 0;
    const uint64_t s = threadIdx.x * per;
    if (s < len) {
        cnt = min(per, len - s);
        reduce_run<W, U>(t, first + s, cnt, acc);
    }
    block_reduce<W, T>(cnt, acc);
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

// Solutions [first, first + len) of instance b to out[(i) * W ..] (first is a
// multiple of 32). Warp w takes a run of groups of 32 consecutive indices;
// lane l of group h holds z(32h + l), and with
// g(32h + l) = (g(h) << 5) ^ ((h & 1) << 4) ^ g(l) every lane steps from
// group h - 1 to h by the same row C_j = B_4 ^ B_{5+j}, j = ctz(h). The
// ragged end (< 32 indices) is seeded index by index from the definition.
template <int W, int T>
__device__ void batch_store_chunk(const BatchArgs& a, int b, uint64_t first, uint64_t len, unsigned char* smem)
{
    constexpr int NC = kTableRows - kStoreM;
    Table<W>& t = *reinterpret_cast<Table<W>*>(smem);
    uint64_t(*C)[W] = reinterpret_cast<uint64_t(*)[W]>(smem + sizeof(Table<W>));
    uint64_t* stage = reinterpret_cast<uint64_t*>(smem + sizeof(Table<W>) + sizeof(uint64_t) * NC * W);
    load_table<W>(t, a.tables + (size_t)b * kTableSlot);
    __syncthreads();
    for (int i = threadIdx.x; i < NC * W; i += T) {
        const int j = i / W, w = i % W;
        C[j][w] = t.B[kStoreM - 1][w] ^ t.B[kStoreM + j][w];
    }
    __syncthreads();
    uint64_t* out = a.out + a.out_off[b];
    const long long room = (a.out_off[b + 1] - a.out_off[b]) / W;  // solutions the instance may store
    (void)room;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t g0 = first >> kStoreM, g1 = (first + len) >> kStoreM;
    const uint64_t per = (g1 - g0 + T / 32 - 1) / (T / 32);
    const uint64_t h0 = g0 + warp * per;
    const uint64_t h1 = min(h0 + per, g1);
    if (h0 < h1) {  // uniform per warp
        uint64_t z[W];
        seed<W>(t, (h0 << kStoreM) + lane, z);
        for (uint64_t h = h0;;) {
            if constexpr (W == 1) {
                if (HLF_IN_BOUNDS((h << kStoreM) + lane, room, kSiteBatchStore)) st_cs(out + (h << kStoreM) + lane, z[0]);
            } else if (HLF_RANGE_IN_BOUNDS(h << kStoreM, 32, room, kSiteBatchStore)) {  // warp-uniform
                store_warp_coalesced<W, false>(out + (h << kStoreM) * W, z, stage + warp * stage_words<W>(), lane);
            }
            if (++h == h1) break;
            xor_row<W>(z, C[ctz64(h)]);
        }
    }
    const uint64_t tail0 = g1 << kStoreM;
    if (threadIdx.x < first + len - tail0) {
        const uint64_t i = tail0 + threadIdx.x;
        uint64_t z[W];
        seed<W>(t, i, z);
        if (HLF_IN_BOUNDS(i, room, kSiteBatchStore)) {
#pragma unroll
            for (int w = 0; w < W; ++w) out[i * W + w] = z[w];
        }
    }
}

template <int T>
__global__ void __launch_bounds__(T, 1024 / T) batch_kernel(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_item;
    __shared__ int s_state;  // instance rank (>= 0), or < 0 to skip the chunk
    __shared__ int s_n;
    const bool has_factor = a.mode == kModeFused || a.mode == kModeFactor;
    const bool has_chunks = a.mode != kModeFactor;
    const uint32_t n_factor = has_factor ? (uint32_t)a.B : 0u;
    const uint32_t n_items = n_factor + (has_chunks ? (uint32_t)a.B * a.chunks_per_inst : 0u);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u) + a.first_item;
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        if (item < n_factor) {
            const int b = (int)item;
            const uint64_t* A = a.A + a.word_off[b];
            const int n = a.mode == kModeFused ? a.n[b] : n_of_words(a.word_off[b + 1] - a.word_off[b]);
            if (n < 1 || n > kBatchMaxN) {
                if (threadIdx.x == 0) {
                    a.info[kInfo * b] = HLF_ERR_SIZE;
                    a.info[kInfo * b + 1] = -1;
                }
            } else {
                switch ((n + 63) >> 6) {
                case 1: batch_factor<1, T>(a, b, n, A, smem); break;
                case 2: batch_factor<2, T>(a, b, n, A, smem); break;
                case 3: batch_factor<3, T>(a, b, n, A, smem); break;
                default: batch_factor<4, T>(a, b, n, A, smem); break;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                a.info[kInfo * b + 2] = n;
                const int st = a.info[kInfo * b];
                a.r_out[b] = st ? -st : a.info[kInfo * b + 1];
                __threadfence();
                st_release(a.ready + b, 1);
            }
            continue;
        }
        const uint32_t j = item - n_factor;
        const int b = (int)(j / a.chunks_per_inst);
        const uint64_t c = j % a.chunks_per_inst;
        if (threadIdx.x == 0) {
            uint32_t polls = 0;
            while (ld_acquire(a.ready + b) == 0 && ++polls < a.spin_limit) __nanosleep(128);
            if (polls >= a.spin_limit) {
                atomicCAS(a.status, 0, HLF_ERR_TIMEOUT);
                s_state = -1;
            } else {
                s_state = __ldcg(a.info + kInfo * b) ? -1 : __ldcg(a.info + kInfo * b + 1);
                s_n = __ldcg(a.info + kInfo * b + 2);
            }
        }
        __syncthreads();
        const int r = s_state;
        const int n = s_n;
        __syncthreads();
        if (r < 0) continue;
        const int W = (n + 63) >> 6;
        const uint64_t space_cap = r >= 64 ? ~0ull : (1ull << r);
        uint64_t total = space_cap < a.cap ? space_cap : a.cap;
        if (a.mode == kModeStore) {
            const uint64_t room = (uint64_t)(a.out_off[b + 1] - a.out_off[b]) / (uint64_t)W;
            total = room < total ? room : total;
        }
        const uint64_t first = c * a.chunk;
        if (first >= total) continue;
        const uint64_t len = min(a.chunk, total - first);
        if (a.mode == kModeStore) {
            switch (W) {
            case 1: batch_store_chunk<1, T>(a, b, first, len, smem); break;
            case 2: batch_store_chunk<2, T>(a, b, first, len, smem); break;
            case 3: batch_store_chunk<3, T>(a, b, first, len, smem); break;
            default: batch_store_chunk<4, T>(a, b, first, len, smem); break;
            }
        } else {
            switch (W) {
            case 1: batch_reduce_chunk<1, T>(a, b, first, len, smem); break;
            case 2: batch_reduce_chunk<2, T>(a, b, first, len, smem); break;
            case 3: batch_reduce_chunk<3, T>(a, b, first, len, smem); break;
            default: batch_reduce_chunk<4, T>(a, b, first, len, smem); break;
            }
        }
        __syncthreads();
    }
}

// Launch shapes: warps per work item -> the kernel of that CTA size.
struct Shape {
    void (*kernel)(BatchArgs);
    int threads;
    size_t smem;
};

Shape shape_for(int warps)
{
    switch (warps) {
    case 2: return {batch_kernel<64>, 64, batch_smem_bytes<64>()};
    case 4: return {batch_kernel<128>, 128, batch_smem_bytes<128>()};
    default: return {batch_kernel<256>, 256, batch_smem_bytes<256>()};
    }
}

// Zero what the launch needs zeroed, size the persistent grid and launch.
// Nothing is enqueued when a host-side check fails.
hlf_status launch_batch(BatchArgs& a, int warps, int ctas_per_sm, cudaStream_t s)
{
    const Shape sh = shape_for(warps);
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, sh.kernel, sh.threads, sh.smem) != cudaSuccess ||
        fit < 1)
        return HLF_ERR_CUDA;
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < fit) ? ctas_per_sm : fit;
    const int grid = sm_count() * per_sm;
    const bool has_factor = a.mode == kModeFused || a.mode == kModeFactor;
    const bool has_chunks = a.mode != kModeFactor;
    const uint64_t items = (has_factor ? (uint64_t)a.B : 0) + (has_chunks ? (uint64_t)a.B * a.chunks_per_inst : 0);
    // The 32-bit queue counter is incremented once per item and once more by
    // every CTA when it finds the queue empty; it must not wrap.
    if (items + (uint64_t)grid > 0xffffffffull) return HLF_ERR_RANGE;
    if (cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), s) != cudaSuccess) return HLF_ERR_CUDA;
    if (has_factor && cudaMemsetAsync(a.ready, 0, sizeof(int32_t) * (size_t)a.B, s) != cudaSuccess)
        return HLF_ERR_CUDA;
    if ((a.mode == kModeFused || a.mode == kModeReduce) &&
        cudaMemsetAsync(a.red_out, 0, sizeof(hlf_reduce) * (size_t)a.B, s) != cudaSuccess)
        return HLF_ERR_CUDA;
    sh.kernel<<<grid, sh.threads, sh.smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace
HLF_DEBUG_TAKE(batch)

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
    int32_t info[kInfo * HLF_BATCH_NOALLOC_MAX];
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
    uint32_t* counter = nullptr;  // counter and status are adjacent
    int32_t* status = nullptr;
    int32_t warps = 8;            // warps per work item (CTA size / 32)
    int32_t ctas_per_sm = 0;      // 0 = as many as fit
    uint64_t chunk = 1ull << 16;
    uint32_t spin_limit = 1u << 23;
    uint32_t debug = 0;           // HLF_BATCH_DEBUG_* fault-injection flags (tests only)
    int32_t factored = 0;         // instances factored by the last factor or fused launch
    cudaEvent_t last = nullptr;
    cudaStream_t priv = nullptr;
};

namespace {

// Fills the workspace pointers and launch knobs of a plan into a.
void plan_args(const hlf_batch* b, hlf::BatchArgs& a)
{
    a.tables = b->tables;
    a.info = b->info;
    a.ready = b->ready;
    a.counter = b->counter;
    a.status = b->status;
    a.spin_limit = b->spin_limit;
    a.chunk = b->chunk;
}

hlf_status chunks_of(uint64_t cap, uint64_t chunk, uint32_t* cpi)
{
    const uint64_t c = (cap + chunk - 1) / chunk;
    if (c > (1u << 20)) return HLF_ERR_RANGE;
    *cpi = (uint32_t)c;
    return HLF_OK;
}

// Records the plan's last-launch event (not while the stream is captured into
// a CUDA graph; after replaying such a graph, synchronise the stream before
// hlf_batch_get_status).
hlf_status record_last(hlf_batch* b, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return HLF_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return HLF_OK;
    return cudaEventRecord(b->last, s) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

hlf_status check_device(const hlf_batch* b)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) return HLF_ERR_ARG;
    return HLF_OK;
}

}  // namespace

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
    const size_t info = sizeof(int32_t) * hlf::kInfo * (size_t)max_instances;
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
    *out = b;
    return HLF_OK;
}

hlf_status hlf_batch_set_tiles(hlf_batch* b, int32_t warps_per_item, int32_t ctas_per_sm, uint64_t chunk)
{
    if (!b || (warps_per_item != 2 && warps_per_item != 4 && warps_per_item != 8) || ctas_per_sm < 0 ||
        ctas_per_sm > 64 || chunk < 256 || (chunk & (chunk - 1)))
        return HLF_ERR_ARG;
    b->warps = warps_per_item;
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
    hlf::NvtxRange nvtx_range("hlf_batch_factor_reduce");
    if (!b || count < 0 || count > b->max_instances || cap == 0) return HLF_ERR_ARG;
    if (count == 0) return HLF_OK;
    if (!A_dev || !word_off_dev || !n_dev || !r_dev || !red_dev) return HLF_ERR_ARG;
    if (check_device(b) != HLF_OK) return HLF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf::BatchArgs a{};
    plan_args(b, a);
    a.A = A_dev;
    a.word_off = word_off_dev;
    a.n = n_dev;
    a.B = count;
    a.mode = hlf::kModeFused;
    a.cap = cap;
    if (chunks_of(cap, b->chunk, &a.chunks_per_inst) != HLF_OK) return HLF_ERR_RANGE;
    a.r_out = r_dev;
    a.red_out = red_dev;
    // With debug flag 1 the queue starts after the factor items, so no ready
    // flag is ever set and every chunk's bounded wait runs out.
    a.first_item = (b->debug & 1u) ? (uint32_t)count : 0u;
    const hlf_status st = hlf::launch_batch(a, b->warps, b->ctas_per_sm, s);
    if (st != HLF_OK) return st;
    b->factored = count;
    return record_last(b, s);
}

hlf_status hlf_factor_batched(hlf_batch* b, const uint64_t* A_dev, const int64_t* offsets_dev, int32_t count,
                              int32_t* r_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_factor_batched");
    if (!b || count < 0 || count > b->max_instances) return HLF_ERR_ARG;
    if (count == 0) {
        b->factored = 0;
        return HLF_OK;
    }
    if (!A_dev || !offsets_dev || !r_dev) return HLF_ERR_ARG;
    if (check_device(b) != HLF_OK) return HLF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf::BatchArgs a{};
    plan_args(b, a);
    a.A = A_dev;
    a.word_off = offsets_dev;
    a.B = count;
    a.mode = hlf::kModeFactor;
    a.r_out = r_dev;
    a.first_item = (b->debug & 1u) ? (uint32_t)count : 0u;
    const hlf_status st = hlf::launch_batch(a, b->warps, b->ctas_per_sm, s);
    if (st != HLF_OK) return st;
    b->factored = count;
    return record_last(b, s);
}

hlf_status hlf_enumerate_batched(hlf_batch* b, uint64_t cap, hlf_reduce* red_dev, uint64_t* out_dev,
                                 const int64_t* out_offsets_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_batched");
    if (!b || cap == 0 || (!red_dev) == (!out_dev) || (out_dev && !out_offsets_dev)) return HLF_ERR_ARG;
    if (b->factored < 1) return HLF_ERR_ARG;
    if (check_device(b) != HLF_OK) return HLF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf::BatchArgs a{};
    plan_args(b, a);
    a.B = b->factored;
    a.mode = out_dev ? hlf::kModeStore : hlf::kModeReduce;
    a.cap = cap;
    if (chunks_of(cap, b->chunk, &a.chunks_per_inst) != HLF_OK) return HLF_ERR_RANGE;
    a.red_out = red_dev;
    a.out = out_dev;
    a.out_off = out_offsets_dev;
    const hlf_status st = hlf::launch_batch(a, b->warps, b->ctas_per_sm, s);
    if (st != HLF_OK) return st;
    return record_last(b, s);
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
    hlf::NvtxRange nvtx_range("hlf_batch_factor_reduce_noalloc");
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
        // (the device is current here).
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_batch_noalloc_scratch) != cudaSuccess || !p) {
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
    a.mode = hlf::kModeFused;
    a.cap = cap;
    a.chunk = 1ull << 16;
    if (chunks_of(cap, a.chunk, &a.chunks_per_inst) != HLF_OK) return HLF_ERR_RANGE;
    a.r_out = r_dev;
    a.red_out = red_dev;
    a.tables = sc->tables;
    a.info = sc->info;
    a.ready = sc->ready;
    a.counter = &sc->counter;
    a.status = &sc->status;
    a.spin_limit = 1u << 23;
    a.first_item = 0;
    // The array keeps the previous call's contents: clear the status word;
    // the launch clears the queue counter and this call's ready flags and
    // results.
    if (cudaMemsetAsync(&sc->status, 0, sizeof(int32_t), s) != cudaSuccess) return HLF_ERR_CUDA;
    return hlf::launch_batch(a, 8, 0, s);
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
