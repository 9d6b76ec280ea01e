// Many enumeration windows, of different matrices and word counts, stored in
// ONE launch: the serving path's continuous batching. Each window is the
// stage-2 materialisation of hlf_enumerate_store (Section 2, Fig. 1(c)); the
// batching only schedules them together.
//
// The host cuts every window into warp tasks: task 0 of a window writes its
// ragged head and tail (the indices before the first and after the last
// multiple of G, seeded one by one from the definition), the other tasks
// cover runs of up to kTaskGroups aligned groups of G consecutive indices
// with the lane-interleaved Gray identity of enumerate.cu (one row XOR per
// solution, a warp writes G consecutive solutions per step; solutions of
// W > 1 words are restaged in shared memory so that the warp's stores are
// coalesced). Warps take tasks
// grid-stride and find their window by binary search over the task prefix
// sums. The basis rows are read through the read-only cache: every lane of a
// warp reads the same row, so each load is one broadcast.

#include <new>

#include "enum_impl.cuh"

namespace hlf {
namespace {

constexpr uint64_t kTaskGroups = 64;

struct WinDesc {
    const uint64_t* table;  // [66][W]: B_0..B_64 (zero-padded), z0
    uint64_t* out;          // [count][W]
    uint64_t offset, count;
    uint64_t n_head, tail_first, n_tail;  // ragged indices, as in StorePlan
    uint64_t h_first, h_end;              // aligned groups [h_first, h_end)
    uint64_t task_base;                   // tasks of earlier windows
    uint32_t W, ntasks;
};

template <int W>
__device__ __forceinline__ void seed_g(const uint64_t* __restrict__ tab, uint64_t i, uint64_t (&z)[W])
{
    uint64_t g = i ^ (i >> 1);
#pragma unroll
    for (int w = 0; w < W; ++w) z[w] = __ldg(tab + kTableZ0Row * W + w);
    while (g) {
        const int k = __ffsll((long long)g) - 1;
        g &= g - 1;
#pragma unroll
        for (int w = 0; w < W; ++w) z[w] ^= __ldg(tab + k * W + w);
    }
}

template <int W>
__device__ void many_task(const WinDesc& d, uint64_t u, int lane, uint64_t* stage)
{
    constexpr int S = (W == 1) ? 2 : 1;
    constexpr uint64_t G = 32 * S;
    constexpr int M = (S == 2) ? 6 : 5;
    if (u == 0 && d.n_head + d.n_tail) {
        for (uint64_t e = lane; e < d.n_head + d.n_tail; e += 32) {
            const uint64_t i = e < d.n_head ? d.offset + e : d.tail_first + (e - d.n_head);
            uint64_t z[W];
            seed_g<W>(d.table, i, z);
            if (HLF_IN_BOUNDS(i - d.offset, d.count, kSiteManyStore)) {
#pragma unroll
                for (int w = 0; w < W; ++w) d.out[(i - d.offset) * W + w] = z[w];
            }
        }
        return;
    }
    const uint64_t gt = (d.n_head + d.n_tail) ? u - 1 : u;
    const uint64_t h0 = d.h_first + gt * kTaskGroups;
    if (h0 >= d.h_end) return;
    const uint64_t h1 = min(h0 + kTaskGroups, d.h_end);
    uint64_t z[W];
    seed_g<W>(d.table, h0 * G + (uint64_t)(S * lane), z);
    const bool even = (d.offset & 1) == 0;  // outputs are 16-byte aligned (checked by the caller)
    for (uint64_t h = h0;;) {
        if constexpr (S == 2) {
            uint64_t* p = d.out + (h * G + (uint64_t)(S * lane) - d.offset) * W;
            const uint64_t z1 = z[0] ^ __ldg(d.table);  // g(2t+1) = g(2t) ^ 1
            if (HLF_RANGE_IN_BOUNDS(h * G + (uint64_t)(S * lane) - d.offset, 2, d.count, kSiteManyStore)) {
                if (even) {
                    st_cs_v2(p, z[0], z1);
                } else {
                    st_cs(p, z[0]);
                    st_cs(p + 1, z1);
                }
            }
        } else {  // the check is warp-uniform
            if (HLF_RANGE_IN_BOUNDS(h * G - d.offset, G, d.count, kSiteManyStore))
                store_warp_coalesced<W, true>(d.out + (h * G - d.offset) * W, z, stage, lane);
        }
        if (++h == h1) break;
        const int j = ctz64(h);
#pragma unroll
        for (int w = 0; w < W; ++w) z[w] ^= __ldg(d.table + (M - 1) * W + w) ^ __ldg(d.table + (M + j) * W + w);
    }
}

__global__ void __launch_bounds__(kThreads, 2) many_kernel(const WinDesc* __restrict__ d, int k, uint64_t total_tasks)
{
    extern __shared__ __align__(16) uint64_t s_stage[];  // [warps][stage_words<16>()]
    uint64_t* stage = s_stage + (threadIdx.x >> 5) * stage_words<HLF_MAX_W>();
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total_tasks; t += nwarps) {
        int lo = 0, hi = k - 1;  // last window with task_base <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].task_base <= t) lo = mid;
            else hi = mid - 1;
        }
        const WinDesc& w = d[lo];
        const uint64_t u = t - w.task_base;
        switch (w.W) {
        case 1: many_task<1>(w, u, lane, stage); break;
        case 2: many_task<2>(w, u, lane, stage); break;
        case 3: many_task<3>(w, u, lane, stage); break;
        case 4: many_task<4>(w, u, lane, stage); break;
        case 5: many_task<5>(w, u, lane, stage); break;
        case 6: many_task<6>(w, u, lane, stage); break;
        case 7: many_task<7>(w, u, lane, stage); break;
        case 8: many_task<8>(w, u, lane, stage); break;
        case 9: many_task<9>(w, u, lane, stage); break;
        case 10: many_task<10>(w, u, lane, stage); break;
        case 11: many_task<11>(w, u, lane, stage); break;
        case 12: many_task<12>(w, u, lane, stage); break;
        case 13: many_task<13>(w, u, lane, stage); break;
        case 14: many_task<14>(w, u, lane, stage); break;
        case 15: many_task<15>(w, u, lane, stage); break;
        default: many_task<16>(w, u, lane, stage); break;
        }
    }
}

// Host-side cut of one window into tasks (the same plan as the single-window
// store kernel).
void plan_window(WinDesc& d, uint32_t W)
{
    const uint64_t G = W == 1 ? 64 : 32;
    const int M = W == 1 ? 6 : 5;
    const uint64_t end = d.offset + d.count;
    const bool ends_at_2_64 = d.count != 0 && end == 0;
    const uint64_t a0 = (d.offset + (G - 1)) & ~(G - 1);
    const bool a0_wrapped = a0 < d.offset;
    const uint64_t h_first = a0 / G;
    const uint64_t h_end = ends_at_2_64 ? (1ull << (64 - M)) : end / G;
    const uint64_t groups = (!a0_wrapped && h_end > h_first) ? h_end - h_first : 0;
    if (groups == 0) {
        d.n_head = d.count;
        d.n_tail = 0;
        d.tail_first = 0;
        d.h_first = d.h_end = 0;
    } else {
        d.n_head = a0 - d.offset;
        d.h_first = h_first;
        d.h_end = h_end;
        d.tail_first = h_end * G;
        d.n_tail = d.count - d.n_head - groups * G;
    }
    d.W = W;
    d.ntasks = (uint32_t)((d.n_head + d.n_tail ? 1 : 0) + (groups + kTaskGroups - 1) / kTaskGroups);
}

}  // namespace

// The handle's enumeration table, rank and word count, and the record of a
// use of the handle on a stream (defined in hlf_api.cu).
hlf_status handle_enum_view(hlf_handle* h, const uint64_t** table, int32_t* r, int32_t* W);
hlf_status handle_record_use(hlf_handle* h, cudaStream_t s);

HLF_DEBUG_TAKE(many)

}  // namespace hlf

struct hlf_many {
    int device = 0;
    int32_t max_windows = 0;
    hlf::WinDesc* dev[2] = {nullptr, nullptr};
    hlf::WinDesc* host[2] = {nullptr, nullptr};  // pinned staging
    cudaEvent_t done[2] = {nullptr, nullptr};
    int next = 0;
};

extern "C" {

hlf_status hlf_many_create(int32_t max_windows, hlf_many** out)
{
    if (!out) return HLF_ERR_ARG;
    *out = nullptr;
    if (max_windows < 1 || max_windows > (1 << 22)) return HLF_ERR_ARG;
    if (hlf::take_injected_alloc_failure()) return HLF_ERR_NOMEM;
    hlf_many* m = new (std::nothrow) hlf_many;
    if (!m) return HLF_ERR_NOMEM;
    m->max_windows = max_windows;
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        delete m;
        return HLF_ERR_CUDA;
    }
    const size_t bytes = sizeof(hlf::WinDesc) * (size_t)max_windows;
    for (int b = 0; b < 2; ++b) {
        if (cudaMalloc(&m->dev[b], bytes) != cudaSuccess || cudaMallocHost(&m->host[b], bytes) != cudaSuccess ||
            cudaEventCreateWithFlags(&m->done[b], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            hlf_many_destroy(m);
            return HLF_ERR_NOMEM;
        }
    }
    *out = m;
    return HLF_OK;
}

hlf_status hlf_enumerate_store_many(hlf_many* m, hlf_handle* const* hs, const uint64_t* offsets,
                                    const uint64_t* counts, uint64_t* const* outs_dev, int32_t k, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_store_many");
    if (!m || k < 0 || k > m->max_windows) return HLF_ERR_ARG;
    if (k == 0) return HLF_OK;
    if (!hs || !offsets || !counts || !outs_dev) return HLF_ERR_ARG;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != m->device) return HLF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int b = m->next;
    if (cudaEventSynchronize(m->done[b]) != cudaSuccess) return HLF_ERR_CUDA;  // staging b is free again
    hlf::WinDesc* d = m->host[b];
    uint64_t tasks = 0;
    int32_t used = 0;
    for (int32_t j = 0; j < k; ++j) {
        if (!hs[j] || (counts[j] && !outs_dev[j])) return HLF_ERR_ARG;
        if (reinterpret_cast<uintptr_t>(outs_dev[j]) % 16) return HLF_ERR_ARG;
        const uint64_t* table = nullptr;
        int32_t r = 0, W = 0;
        hlf_status st = hlf::handle_enum_view(hs[j], &table, &r, &W);
        if (st != HLF_OK) return st;
        const uint64_t off = offsets[j], cnt = counts[j];
        const bool ok = r < 64 ? (off <= (1ull << r) && cnt <= (1ull << r) - off)
                               : (cnt == 0 || cnt - 1 <= ~0ull - off);
        if (!ok) return HLF_ERR_RANGE;
        if (cnt == 0) continue;
        hlf::WinDesc& w = d[used++];
        w = hlf::WinDesc{};
        w.table = table;
        w.out = outs_dev[j];
        w.offset = off;
        w.count = cnt;
        hlf::plan_window(w, (uint32_t)W);
        w.task_base = tasks;
        tasks += w.ntasks;
    }
    if (used == 0) return HLF_OK;
    if (cudaMemcpyAsync(m->dev[b], d, sizeof(hlf::WinDesc) * (size_t)used, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return HLF_ERR_CUDA;
    // Two CTAs per SM keep HBM busy for stores and leave room on every SM for
    // the factorisations a serving loop runs alongside.
    const uint64_t warps_cap = (uint64_t)hlf::sm_count() * 2 * (hlf::kThreads / 32);
    const uint64_t warps = tasks < warps_cap ? tasks : warps_cap;
    const unsigned blocks = (unsigned)((warps * 32 + hlf::kThreads - 1) / hlf::kThreads);
    constexpr size_t smem = (size_t)(hlf::kThreads / 32) * hlf::stage_words<HLF_MAX_W>() * sizeof(uint64_t);
    hlf::many_kernel<<<blocks, hlf::kThreads, smem, s>>>(m->dev[b], used, tasks);
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    if (cudaEventRecord(m->done[b], s) != cudaSuccess) return HLF_ERR_CUDA;
    // every handle read by this launch must outlive it (hlf_destroy waits)
    for (int32_t j = 0; j < k; ++j) {
        if (j > 0 && hs[j] == hs[j - 1]) continue;
        hlf_status st = hlf::handle_record_use(hs[j], s);
        if (st != HLF_OK) return st;
    }
    m->next = 1 - b;
    return HLF_OK;
}

hlf_status hlf_many_destroy(hlf_many* m)
{
    if (!m) return HLF_OK;
    hlf_status st = HLF_OK;
    for (int b = 0; b < 2; ++b) {
        if (m->done[b] && cudaEventSynchronize(m->done[b]) != cudaSuccess) st = HLF_ERR_CUDA;
        if (m->dev[b] && cudaFree(m->dev[b]) != cudaSuccess) st = HLF_ERR_CUDA;
        if (m->host[b] && cudaFreeHost(m->host[b]) != cudaSuccess) st = HLF_ERR_CUDA;
        if (m->done[b]) cudaEventDestroy(m->done[b]);
    }
    delete m;
    return st;
}

}  // extern "C"
