// C ABI of libhlf (declared in include/hlf.h): argument checks, the handle
// and its device buffers, and the launches of the stage-1 and stage-2 kernels.

#include <cstring>
#include <new>

#include "hlf_internal.cuh"

struct hlf_handle {
    int32_t n = 0;
    int32_t W = 0;
    int device = 0;
    unsigned char* dmem = nullptr;  // one allocation: info | piv | table | basis
    int32_t* info = nullptr;
    int32_t* piv = nullptr;
    uint64_t* table = nullptr;
    uint64_t* basis = nullptr;
    cudaEvent_t last = nullptr;     // recorded after the last work enqueued through the handle
    cudaStream_t priv = nullptr;    // private non-blocking stream for status reads
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

hlf_status read_info(hlf_handle* h, int32_t out[2])
{
    if (cudaEventSynchronize(h->last) != cudaSuccess) return HLF_ERR_CUDA;
    if (cudaMemcpyAsync(out, h->info, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, h->priv) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (cudaStreamSynchronize(h->priv) != cudaSuccess) return HLF_ERR_CUDA;
    return HLF_OK;
}

hlf_status ensure_rank(hlf_handle* h)
{
    if (h->rank_known) return HLF_OK;
    int32_t info[2];
    hlf_status st = read_info(h, info);
    if (st != HLF_OK) return st;
    if (info[0] != HLF_OK) return (hlf_status)info[0];
    h->r = info[1];
    h->rank_known = true;
    return HLF_OK;
}

// Is [offset, offset + count) inside [0, 2^min(r, 64))?
bool window_ok(int32_t r, uint64_t offset, uint64_t count)
{
    if (r < 64) {
        const uint64_t space = 1ull << r;
        return offset <= space && count <= space - offset;
    }
    return count == 0 || count - 1 <= ~0ull - offset;
}

hlf_status after_launch(hlf_handle* h, hlf_status st, cudaStream_t s)
{
    if (st != HLF_OK) return st;
    return cudaEventRecord(h->last, s) == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
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
    *table = h->table;
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

int32_t hlf_device_count(void)
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return -1;
    return n;
}

hlf_status hlf_factor(const uint64_t* A_dev, int32_t n, void* stream, hlf_handle** out)
{
    if (!out) return HLF_ERR_ARG;
    *out = nullptr;
    if (!A_dev) return HLF_ERR_ARG;
    if (n < 1 || n > HLF_MAX_N) return HLF_ERR_SIZE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hlf_handle* h = new (std::nothrow) hlf_handle;
    if (!h) return HLF_ERR_NOMEM;
    h->n = n;
    h->W = (n + 63) / 64;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return HLF_ERR_CUDA;
    }
    const size_t off_piv = 64;
    const size_t off_table = round_up(off_piv + sizeof(int32_t) * n, 256);
    const size_t off_basis = round_up(off_table + sizeof(uint64_t) * hlf::kTableTotalRows * h->W, 256);
    const size_t bytes = off_basis + sizeof(uint64_t) * (size_t)n * h->W;
    // Stream-ordered allocation: no device-wide synchronisation, so a serving
    // loop can create and destroy handles while other work is in flight.
    hlf::keep_pool_memory();
    if (cudaMallocAsync(&h->dmem, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HLF_ERR_NOMEM;
    }
    h->info = reinterpret_cast<int32_t*>(h->dmem);
    h->piv = reinterpret_cast<int32_t*>(h->dmem + off_piv);
    h->table = reinterpret_cast<uint64_t*>(h->dmem + off_table);
    h->basis = reinterpret_cast<uint64_t*>(h->dmem + off_basis);
    if (cudaEventCreateWithFlags(&h->last, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->priv, cudaStreamNonBlocking) != cudaSuccess) {
        hlf_destroy(h);
        return HLF_ERR_CUDA;
    }
    hlf::FactorOut o{h->basis, h->piv, h->table, h->info};
    hlf_status st = hlf::launch_factor(A_dev, n, h->W, o, s);
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
    if (!h || !r) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    *r = h->r;
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
    if (!h) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
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
    hlf_status st = read_info(h, info);
    if (st != HLF_OK) return st;
    if (info[0] != HLF_OK) {
        const int32_t zero = 0;
        if (cudaMemcpyAsync(h->info, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->priv) != cudaSuccess ||
            cudaStreamSynchronize(h->priv) != cudaSuccess)
            return HLF_ERR_CUDA;
    }
    return (hlf_status)info[0];
}

hlf_status hlf_enumerate_store(hlf_handle* h, uint64_t offset, uint64_t count, uint64_t* out_dev, void* stream)
{
    if (!h || (!out_dev && count)) return HLF_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out_dev) % 16) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (!window_ok(h->r, offset, count)) return HLF_ERR_RANGE;
    if (count == 0) return HLF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_store(h->table, h->W, offset, count, out_dev, s), s);
}

hlf_status hlf_enumerate_reduce(hlf_handle* h, uint64_t offset, uint64_t count, hlf_reduce* red_dev, void* stream)
{
    if (!h || !red_dev) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (!window_ok(h->r, offset, count)) return HLF_ERR_RANGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(red_dev, 0, sizeof(hlf_reduce), s) != cudaSuccess) return HLF_ERR_CUDA;
    if (count == 0) return after_launch(h, HLF_OK, s);
    return after_launch(h, hlf::launch_reduce(h->table, h->W, offset, count, red_dev, s), s);
}

hlf_status hlf_enumerate_reduce_chunks(hlf_handle* h, uint64_t offset, uint64_t chunk, uint64_t n_chunks,
                                       hlf_reduce* red_dev, void* stream)
{
    if (!h || (!red_dev && n_chunks) || chunk == 0) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (n_chunks && chunk > ~0ull / n_chunks) return HLF_ERR_RANGE;
    if (!window_ok(h->r, offset, chunk * n_chunks)) return HLF_ERR_RANGE;
    if (n_chunks == 0) return HLF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_reduce_chunks(h->table, h->W, offset, chunk, n_chunks, red_dev, s), s);
}

hlf_status hlf_sample(hlf_handle* h, const uint64_t* idx_dev, uint64_t m, uint64_t* out_dev, void* stream)
{
    if (!h || (m && (!idx_dev || !out_dev))) return HLF_ERR_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return HLF_ERR_CUDA;
    hlf_status st = ensure_rank(h);
    if (st != HLF_OK) return st;
    if (m == 0) return HLF_OK;
    const int nb = h->r < HLF_MAX_VARYING ? h->r : HLF_MAX_VARYING;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return after_launch(h, hlf::launch_sample(h->table, h->W, nb, idx_dev, m, out_dev, h->info, s), s);
}

hlf_status hlf_destroy(hlf_handle* h)
{
    if (!h) return HLF_OK;
    hlf_status st = HLF_OK;
    {
        // Freed in stream order after the handle's last work: the host does
        // not wait, and no device-wide synchronisation happens.
        DeviceGuard g(h->device);
        if (h->dmem) {
            bool freed = h->priv && h->last && cudaStreamWaitEvent(h->priv, h->last, 0) == cudaSuccess &&
                         cudaFreeAsync(h->dmem, h->priv) == cudaSuccess;
            if (!freed) {  // error paths only: a plain synchronising free
                cudaGetLastError();
                if (cudaFree(h->dmem) != cudaSuccess) st = HLF_ERR_CUDA;
            }
        }
        if (h->last) cudaEventDestroy(h->last);
        if (h->priv) cudaStreamDestroy(h->priv);
    }
    delete h;
    return st;
}

}  // extern "C"
