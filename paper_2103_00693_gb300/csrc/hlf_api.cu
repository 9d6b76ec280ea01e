// C ABI of libhlf (declared in include/hlf.h): argument checks, the handle
// and its device buffers, and the launches of the stage-1 and stage-2 kernels.

#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hlf_internal.cuh"
#include "upto.cuh"

struct hlf_handle {
    int32_t n = 0;
    int32_t W = 0;
    int device = 0;
    unsigned char* dmem = nullptr;  // one allocation: factor scratch | piv | table | ptable | basis
    int32_t* info = nullptr;         // status word: pinned host memory, device-mapped
    int32_t* info_dev = nullptr;     // the same words as the kernels address them
    int32_t* piv = nullptr;
    uint64_t* table = nullptr;
    uint64_t* ptable = nullptr;     // the paper-order table
    uint64_t* basis = nullptr;
    int32_t order = HLF_ORDER_GRAY; // which table the stage-2 calls read
    cudaEvent_t factored = nullptr;  // recorded after the factor kernel
    // one event per stream the handle has been used on, recorded after the
    // latest work on that stream (hlf_destroy and hlf_get_status wait for all)
    static constexpr int kMaxStreams = 8;
    cudaStream_t use_stream[kMaxStreams] = {};
    cudaEvent_t use_event[kMaxStreams] = {};
    int n_uses = 0;
    cudaStream_t priv = nullptr;     // private non-blocking stream, created on first need
    bool rank_known = false;
    int32_t r = -1;
};

namespace {

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Switches to the handle's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Status words live in pinned, device-mapped host memory: kernels store them
// directly and the host reads them after an event, with no copy. A copy
// would queue behind whatever large transfers the copy engines are busy
// with, which stalls a serving loop. Slabs are allocated on first need and
// kept until the process exits; slots are recycled.
constexpr int kSlotWords = 16;
constexpr int kSlotsPerSlab = 4096;
std::mutex g_slot_mu;
std::vector<int32_t*> g_free_slots;
// Slots of destroyed handles whose last work may still be in flight, each with
// an event recorded after that work (the event is owned here). Reclaimed in
// order once the event has completed.
struct PendingSlot {
    int32_t* slot;
    cudaEvent_t done;
};
std::vector<PendingSlot> g_pending_slots;
size_t g_pending_head = 0;

// Under g_slot_mu: recycle up to `max` pending slots whose work has finished.
void reclaim_pending_slots(int max)
{
    while (max-- > 0 && g_pending_head < g_pending_slots.size()) {
        PendingSlot& p = g_pending_slots[g_pending_head];
        const cudaError_t q = cudaEventQuery(p.done);
        if (q == cudaErrorNotReady) break;
        cudaGetLastError();  // a failed query leaves the slot to be recycled as well
        cudaEventDestroy(p.done);
        g_free_slots.push_back(p.slot);
        ++g_pending_head;
    }
    if (g_pending_head == g_pending_slots.size()) {
        g_pending_slots.clear();
        g_pending_head = 0;
    } else if (g_pending_head >= 1024 && 2 * g_pending_head >= g_pending_slots.size()) {
        g_pending_slots.erase(g_pending_slots.begin(), g_pending_slots.begin() + (long)g_pending_head);
        g_pending_head = 0;  // the list never outgrows twice its live entries
    }
}

int32_t* acquire_status_slot()
{
    std::lock_guard<std::mutex> lock(g_slot_mu);
    if (g_free_slots.empty()) reclaim_pending_slots(8);
    if (g_free_slots.empty()) {
        void* p = nullptr;
        if (cudaHostAlloc(&p, sizeof(int32_t) * kSlotWords * kSlotsPerSlab,
                          cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        int32_t* base = static_cast<int32_t*>(p);
        for (int i = kSlotsPerSlab - 1; i >= 0; --i) g_free_slots.push_back(base + i * kSlotWords);
    }
    int32_t* slot = g_free_slots.back();
    g_free_slots.pop_back();
    std::memset(slot, 0, sizeof(int32_t) * kSlotWords);
    return slot;
}

void release_status_slot(int32_t* slot)
{
    std::lock_guard<std::mutex> lock(g_slot_mu);
    g_free_slots.push_back(slot);
}

// Recycle a slot once `done` (recorded after the last work that may write it)
// has completed; takes ownership of the event.
void defer_slot_release(int32_t* slot, cudaEvent_t done)
{
    std::lock_guard<std::mutex> lock(g_slot_mu);
    g_pending_slots.push_back({slot, done});
}

// One non-blocking stream per device, created on first need, on which
// hlf_destroy of a handle used on several streams waits for each stream's
// last use and then frees. Nothing on the host ever waits on it.
cudaStream_t release_stream(int dev)
{
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

hlf_status ensure_priv(hlf_handle* h)
{
    if (h->priv) return HLF_OK;
    return cudaStreamCreateWithFlags(&h->priv, cudaStreamNonBlocking) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

// Host wait for every stream's latest work through h.
hlf_status wait_uses(hlf_handle* h)
{
    for (int i = 0; i < h->n_uses; ++i)
        if (cudaEventSynchronize(h->use_event[i]) != cudaSuccess) return HLF_ERR_CUDA;
    return HLF_OK;
}

hlf_status read_info(hlf_handle* h, int32_t out[2], bool all_uses)
{
    if (all_uses ? wait_uses(h) != HLF_OK : cudaEventSynchronize(h->factored) != cudaSuccess) return HLF_ERR_CUDA;
    const volatile int32_t* w = h->info;
    out[0] = w[0];
    out[1] = w[1];
    return HLF_OK;
}

hlf_status ensure_rank(hlf_handle* h)
{
    if (h->rank_known) return HLF_OK;
    int32_t info[2];
    hlf_status st = read_info(h, info, false);
    if (st != HLF_OK) return st;
    if (info[0] != HLF_OK) return (hlf_status)info[0];
    h->r = info[1];
    h->rank_known = true;
    return HLF_OK;
}

const uint64_t* enum_table(const hlf_handle* h) { return h->order == HLF_ORDER_PAPER ? h->ptable : h->table; }

// Is [offset, offset + count) inside [0, 2^min(r, 64))?
bool window_ok(int32_t r, uint64_t offset, uint64_t count)
{
    if (r < 64) {
        const uint64_t space = 1ull << r;
        return offset <= space && count <= space - offset;
    }
    return count == 0 || count - 1 <= ~0ull - offset;
}

}  // namespace

namespace hlf {

// Record that work reading or writing h's buffers was enqueued on s.
hlf_status handle_record_use(hlf_handle* h, cudaStream_t s)
{
    for (int i = 0; i < h->n_uses; ++i)
        if (h->use_stream[i] == s) return cudaEventRecord(h->use_event[i], s) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
    int slot = h->n_uses;
    if (slot == hlf_handle::kMaxStreams) {  // table full: retire the oldest stream's event
        if (cudaEventSynchronize(h->use_event[0]) != cudaSuccess) return HLF_ERR_CUDA;
        slot = 0;
    } else {
        if (cudaEventCreateWithFlags(&h->use_event[slot], cudaEventDisableTiming) != cudaSuccess)
            return HLF_ERR_CUDA;
        ++h->n_uses;
    }
    h->use_stream[slot] = s;
    return cudaEventRecord(h->use_event[slot], s) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace hlf

namespace {

hlf_status after_launch(hlf_handle* h, hlf_status st, cudaStream_t s)
{
    if (st != HLF_OK) return st;
    return hlf::handle_record_use(h, s);
}

}  // namespace

namespace hlf {

hlf_status handle_enum_view(hlf_handle* h, const uint64_t** table, int32_t* r, int32_t* W)
{
    if (!h) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    *table = enum_table(h);
    *r = h->r;
    *W = h->W;
    return HLF_OK;
}

void keep_pool_memory()
{
    // Keep freed blocks in the device's default pool instead of returning
    // them to the driver at every synchronisation (once per device).
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = 1ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}

namespace {
std::atomic<int32_t> g_fail_allocs{0};
}

bool take_injected_alloc_failure()
{
    int32_t v = g_fail_allocs.load(std::memory_order_relaxed);
    while (v > 0)
        if (g_fail_allocs.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return true;
    return false;
}

HLF_DEBUG_TAKE(api)

namespace {

// one thread, no memory access: the check itself (site kSiteProbe)
__global__ void debug_probe_kernel(long long i, long long n)
{
    (void)HLF_IN_BOUNDS(i, n, kSiteProbe);
}

}  // namespace

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64) cache[dev] = sms;
    return sms;
}

}  // namespace hlf

extern "C" {

const char* hlf_status_string(hlf_status s)
{
    switch (s) {
    case HLF_OK: return "ok";
    case HLF_ERR_ARG: return "invalid argument";
    case HLF_ERR_SIZE: return "n outside [1, 1024]";
    case HLF_ERR_NOT_SYMMETRIC: return "A is not symmetric";
    case HLF_ERR_PADDING: return "padding bit set beyond column n";
    case HLF_ERR_RANGE: return "window or index outside [0, 2^min(r,64))";
    case HLF_ERR_NOMEM: return "out of memory";
    case HLF_ERR_TIMEOUT: return "bounded device wait gave up";
    case HLF_ERR_CUDA: return "CUDA runtime error";
    case HLF_ERR_INTERNAL: return "internal invariant failed";
    }
    return "unknown status";
}

hlf_status hlf_debug_fail_allocs(int32_t count)
{
    if (count < 0) return HLF_ERR_ARG;
    hlf::g_fail_allocs.store(count, std::memory_order_relaxed);
    return HLF_OK;
}

hlf_status hlf_debug_violation(uint64_t* first, int32_t* is_debug)
{
    if (!first || !is_debug) return HLF_ERR_ARG;
    *is_debug = hlf::kDebugBuild ? 1 : 0;
    *first = 0;
    if (!hlf::kDebugBuild) return HLF_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return HLF_ERR_CUDA;
    uint64_t (*const take[])() = {hlf::debug_take_api,  hlf::debug_take_enumerate, hlf::debug_take_many,
                                   hlf::debug_take_upto, hlf::debug_take_batch,     hlf::debug_take_dense,
                                   hlf::debug_take_factor, hlf::debug_take_hist};
    for (auto f : take) {  // every word is read (and so cleared); the first record is kept
        const uint64_t v = f();
        if (v == ~0ull) return HLF_ERR_CUDA;
        if (v && !*first) *first = v;
    }
    return HLF_OK;
}

hlf_status hlf_debug_bounds_probe(int64_t i, int64_t n, void* stream)
{
    hlf::debug_probe_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(i, n);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

int32_t hlf_device_count(void)
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return -1;
    return n;
}

hlf_status hlf_factor(const uint64_t* A_dev, int32_t n, void* stream, hlf_handle** out)
{
    hlf::NvtxRange nvtx_range("hlf_factor");
    if (!out) return HLF_ERR_ARG;
    *out = nullptr;
    if (!A_dev) return HLF_ERR_ARG;
    if (n < 1 || n > HLF_MAX_N) return HLF_ERR_SIZE;
    if (hlf::take_injected_alloc_failure()) return HLF_ERR_NOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf_handle* h = new (std::nothrow) hlf_handle;
    if (!h) return HLF_ERR_NOMEM;
    h->n = n;
    h->W = (n + 63) / 64;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return HLF_ERR_CUDA;
    }
    const size_t off_piv = 256;  // [0, 256): the factor kernels' device scratch (kFactorWorkWords int32)
    const size_t off_table = round_up(off_piv + sizeof(int32_t) * n, 256);
    const size_t off_ptable = round_up(off_table + sizeof(uint64_t) * hlf::kTableTotalRows * h->W, 256);
    const size_t off_basis = round_up(off_ptable + sizeof(uint64_t) * hlf::kTableTotalRows * h->W, 256);
    const size_t bytes = off_basis + sizeof(uint64_t) * (size_t)n * h->W;
    // Stream-ordered allocation: no device-wide synchronisation, so a serving
    // loop can create and destroy handles while other work is in flight.
    hlf::keep_pool_memory();
    if (cudaMallocAsync(&h->dmem, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HLF_ERR_NOMEM;
    }
    h->info = acquire_status_slot();
    if (!h->info || cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->info_dev), h->info, 0) != cudaSuccess) {
        cudaGetLastError();
        hlf_destroy(h);
        return HLF_ERR_NOMEM;
    }
    h->piv = reinterpret_cast<int32_t*>(h->dmem + off_piv);
    h->table = reinterpret_cast<uint64_t*>(h->dmem + off_table);
    h->ptable = reinterpret_cast<uint64_t*>(h->dmem + off_ptable);
    h->basis = reinterpret_cast<uint64_t*>(h->dmem + off_basis);
    if (cudaEventCreateWithFlags(&h->factored, cudaEventDisableTiming) != cudaSuccess) {
        hlf_destroy(h);
        return HLF_ERR_CUDA;
    }
    hlf::FactorOut o{h->basis, h->piv, h->table, h->info_dev, h->ptable, reinterpret_cast<int32_t*>(h->dmem)};
    hlf_status st = hlf::launch_factor(A_dev, n, h->W, o, s);
    if (st == HLF_OK && cudaEventRecord(h->factored, s) != cudaSuccess) st = HLF_ERR_CUDA;
    st = after_launch(h, st, s);
    if (st != HLF_OK) {
        hlf_destroy(h);
        return st;
    }
    *out = h;
    return HLF_OK;
}

hlf_status hlf_get_rank(hlf_handle* h, int32_t* r)
{
    hlf::NvtxRange nvtx_range("hlf_get_rank");
    if (!h || !r) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    *r = h->r;
    return HLF_OK;
}

hlf_status hlf_set_order(hlf_handle* h, int32_t order)
{
    if (!h || (order != HLF_ORDER_GRAY && order != HLF_ORDER_PAPER)) return HLF_ERR_ARG;
    h->order = order;
    return HLF_OK;
}

hlf_status hlf_get_shape(hlf_handle* h, int32_t* n, int32_t* W)
{
    if (!h) return HLF_ERR_ARG;
    if (n) *n = h->n;
    if (W) *W = h->W;
    return HLF_OK;
}

hlf_status hlf_get_factor(hlf_handle* h, int32_t* piv_host, uint64_t* z0_host, uint64_t* basis_host)
{
    hlf::NvtxRange nvtx_range("hlf_get_factor");
    if (!h) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st == HLF_OK) st = ensure_priv(h);
    if (st != HLF_OK) return st;
    const size_t W = h->W;
    if (piv_host && h->r > 0 &&
        cudaMemcpyAsync(piv_host, h->piv, sizeof(int32_t) * h->r, cudaMemcpyDeviceToHost, h->priv) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (z0_host && cudaMemcpyAsync(z0_host, h->table + hlf::kTableZ0Row * W, sizeof(uint64_t) * W,
                                   cudaMemcpyDeviceToHost, h->priv) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (basis_host && h->r > 0 &&
        cudaMemcpyAsync(basis_host, h->basis, sizeof(uint64_t) * W * h->r, cudaMemcpyDeviceToHost, h->priv) !=
            cudaSuccess)
        return HLF_ERR_CUDA;
    return cudaStreamSynchronize(h->priv) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

hlf_status hlf_get_status(hlf_handle* h)
{
    if (!h) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    int32_t info[2];
    hlf_status st = read_info(h, info, true);
    if (st != HLF_OK) return st;
    if (info[0] != HLF_OK) *const_cast<volatile int32_t*>(h->info) = 0;  // all work through h is done
    return (hlf_status)info[0];
}

hlf_status hlf_enumerate_store(hlf_handle* h, uint64_t offset, uint64_t count, uint64_t* out_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_store");
    if (!h || (!out_dev && count)) return HLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out_dev) % 16) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (!window_ok(h->r, offset, count)) return HLF_ERR_RANGE;
    if (count == 0) return HLF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_store(enum_table(h), h->W, offset, count, out_dev, s), s);
}

hlf_status hlf_enumerate_store_upto(hlf_handle* h, uint64_t cap, uint64_t* out_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_store_upto");
    if (!h || (!out_dev && cap) || cap > HLF_STORE_UPTO_MAX) return HLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out_dev) % 8) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    if (cap == 0) return HLF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamWaitEvent(s, h->factored, 0) != cudaSuccess) return HLF_ERR_CUDA;
    return after_launch(h, hlf::launch_store_upto(enum_table(h), h->W, h->info_dev, cap, out_dev, s), s);
}

hlf_status hlf_enumerate_reduce_upto(hlf_handle* h, uint64_t cap, hlf_reduce* red_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_reduce_upto");
    if (!h || !red_dev) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamWaitEvent(s, h->factored, 0) != cudaSuccess) return HLF_ERR_CUDA;
    if (cudaMemsetAsync(red_dev, 0, sizeof(hlf_reduce), s) != cudaSuccess) return HLF_ERR_CUDA;
    if (cap == 0) return after_launch(h, HLF_OK, s);
    return after_launch(h, hlf::launch_reduce_upto(enum_table(h), h->W, h->info_dev, cap, red_dev, s), s);
}

hlf_status hlf_enumerate_store_dense(hlf_handle* h, uint64_t offset, uint64_t count, uint64_t* out_dev,
                                     void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_store_dense");
    if (!h || (!out_dev && count)) return HLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out_dev) % 8) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (!window_ok(h->r, offset, count)) return HLF_ERR_RANGE;
    if (count == 0) return HLF_OK;
    if (count > (~0ull - 63) / (uint64_t)h->n) return HLF_ERR_RANGE;  // stream length in bits
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_store_dense(enum_table(h), h->n, offset, count, out_dev, s), s);
}

hlf_status hlf_enumerate_reduce(hlf_handle* h, uint64_t offset, uint64_t count, hlf_reduce* red_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_reduce");
    if (!h || !red_dev) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (!window_ok(h->r, offset, count)) return HLF_ERR_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(red_dev, 0, sizeof(hlf_reduce), s) != cudaSuccess) return HLF_ERR_CUDA;
    if (count == 0) return after_launch(h, HLF_OK, s);
    return after_launch(h, hlf::launch_reduce(enum_table(h), h->W, offset, count, red_dev, s), s);
}

hlf_status hlf_enumerate_histogram(hlf_handle* h, uint64_t offset, uint64_t count, int32_t bit_lo, int32_t nbits,
                                   uint64_t* hist_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_histogram");
    if (!h || !hist_dev || nbits < 1 || nbits > HLF_HIST_MAX_BITS || bit_lo < 0) return HLF_ERR_ARG;
    if (bit_lo + nbits > h->n) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (!window_ok(h->r, offset, count)) return HLF_ERR_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(hist_dev, 0, sizeof(uint64_t) << nbits, s) != cudaSuccess) return HLF_ERR_CUDA;
    if (count == 0) return after_launch(h, HLF_OK, s);
    return after_launch(h, hlf::launch_histogram(h->order == HLF_ORDER_PAPER ? h->ptable : h->table, h->W, offset,
                                                 count, bit_lo, nbits, hist_dev, s), s);
}

hlf_status hlf_enumerate_reduce_chunks(hlf_handle* h, uint64_t offset, uint64_t chunk, uint64_t n_chunks,
                                       hlf_reduce* red_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_enumerate_reduce_chunks");
    if (!h || (!red_dev && n_chunks) || chunk == 0) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (n_chunks && chunk > ~0ull / n_chunks) return HLF_ERR_RANGE;
    if (!window_ok(h->r, offset, chunk * n_chunks)) return HLF_ERR_RANGE;
    if (n_chunks == 0) return HLF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_reduce_chunks(enum_table(h), h->W, offset, chunk, n_chunks, red_dev, s), s);
}

hlf_status hlf_sample(hlf_handle* h, const uint64_t* idx_dev, uint64_t m, uint64_t* out_dev, void* stream)
{
    hlf::NvtxRange nvtx_range("hlf_sample");
    if (!h || (m && (!idx_dev || !out_dev))) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (m == 0) return HLF_OK;
    const int nb = h->r < HLF_MAX_VARYING ? h->r : HLF_MAX_VARYING;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_sample(enum_table(h), h->W, nb, idx_dev, m, out_dev, h->info_dev, s), s);
}

hlf_status hlf_destroy(hlf_handle* h)
{
    hlf::NvtxRange nvtx_range("hlf_destroy");
    if (!h) return HLF_OK;
    hlf_status st = HLF_OK;
    {
        // Device memory is freed, and the status slot recycled, in stream
        // order after the latest work on every stream that used the handle:
        // the host does not wait and no device-wide synchronisation happens.
        // Used on one stream: the memory is freed on that stream and the slot
        // recycled once the stream's use event has completed. Otherwise the
        // device's release stream waits for every use event, frees, and
        // records the event that recycles the slot.
        DeviceGuard g(h->device);
        bool queued = false;
        if (h->n_uses == 1) {
            queued = !h->dmem || cudaFreeAsync(h->dmem, h->use_stream[0]) == cudaSuccess;
            if (queued) {
                h->dmem = nullptr;
                if (h->info) {
                    defer_slot_release(h->info, h->use_event[0]);
                    h->use_event[0] = nullptr;  // owned by the pending list now
                    h->info = nullptr;
                }
            }
        } else {
            cudaStream_t rs = release_stream(h->device);
            queued = rs != nullptr;
            for (int i = 0; queued && i < h->n_uses; ++i)
                queued = cudaStreamWaitEvent(rs, h->use_event[i], 0) == cudaSuccess;
            if (queued && h->dmem) queued = cudaFreeAsync(h->dmem, rs) == cudaSuccess;
            if (queued) h->dmem = nullptr;
            if (queued && h->info) {
                cudaEvent_t done = nullptr;
                queued = cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess &&
                         cudaEventRecord(done, rs) == cudaSuccess;
                if (queued) {
                    defer_slot_release(h->info, done);
                    h->info = nullptr;
                } else if (done) {
                    cudaEventDestroy(done);
                }
            }
        }
        if (!queued) {  // error paths only: wait, then release synchronously
            cudaGetLastError();
            wait_uses(h);
            if (h->dmem && cudaFree(h->dmem) != cudaSuccess) st = HLF_ERR_CUDA;
            if (h->info) release_status_slot(h->info);
        }
        for (int i = 0; i < h->n_uses; ++i)
            if (h->use_event[i]) cudaEventDestroy(h->use_event[i]);
        if (h->factored) cudaEventDestroy(h->factored);
        if (h->priv) cudaStreamDestroy(h->priv);
    }
    delete h;
    return st;
}

}  // extern "C"
