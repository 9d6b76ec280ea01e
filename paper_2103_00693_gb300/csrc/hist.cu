// Histogram of a bit field of every solution in a window, computed on the
// device while enumerating (no solution is stored): the counts behind the
// paper's output distributions of Figs. 3, 6 and 7, where each square shows
// how often one bit pattern of the first or last bits occurs.
//
// The field of a solution, bits [lo, lo + nbits) of z, is a GF(2)-linear
// function of z, so it commutes with the walk's XORs: with f_k the field of
// B_k and f_z the field of z0, the field of z(i) is
//     v(i) = f_z ^ XOR_{k in g(i)} f_k.
// The kernels therefore walk the table projected onto the field (one 32-bit
// value per row, whatever n is) and never form the solutions themselves:
// each solution costs one 32-bit XOR and one atomic on its bin. For bins in
// shared memory (nbits <= 15) the projected values are kept multiplied by 4,
// so a value is directly the byte offset of its 32-bit counter.
//
// Two walks, two kernels; both are launched, and each CTA of the walk the
// field does not call for returns after reading the table (every CTA comes
// to the same answer):
// - lane-interleaved (the store kernel's walk, enumerate.cu): lane t of a warp
//   holds index 32 h + t and every lane steps by the same value
//   C_j = f_4 ^ f_{5+j}, j = ctz(h+1). The 32 values a warp counts at once
//   are v(32 h) combined with the 32 combinations of f_0..f_4, so when
//   f_0..f_4 are linearly independent the 32 lanes land in 32 distinct bins,
//   and the shared-memory atomics do not collide.
// - per-thread runs (the reduce's walk), for fields the first five rows leave
//   (nearly) unchanged: there the interleaved lanes would all hit one bin,
//   while a thread's run stays in one bin for many solutions.
// Up to 2^15 bins live in shared memory per CTA (32-bit counters, flushed to
// the global 64-bit bins with one atomic per nonzero bin); wider fields count
// straight into global memory.

#include <type_traits>

#include "enum_impl.cuh"

namespace hlf {
namespace {

constexpr int kHistSmemBits = 15;  // 2^15 32-bit bins: 128 KB of shared memory
constexpr int kHistG = 32;                              // consecutive indices per warp step
constexpr uint64_t kHistMaxGroupsPerWarp = 1ull << 23;  // keeps a CTA's counts below 2^32
constexpr uint64_t kHistMaxPerThread = 1ull << 23;      // the same bound for the run walk
constexpr int kIL = 6;  // interleaved walk: 2^6 groups per unrolled Gray block
constexpr int kRU = 6;  // run walk: 2^6 solutions per unrolled Gray block

// Field values of the table rows: f[k] = field(B_k) for k < 65 (rows past
// min(r, 64) and row 64 are zero), f[65] = field(z0), each << scale.
struct FieldTable {
    uint32_t f[kTableTotalRows];
};

__device__ __forceinline__ void load_field_table(FieldTable& t, const uint64_t* __restrict__ g, int W, int lo,
                                                 int nbits, int scale)
{
    const int word = lo >> 6, sh = lo & 63;
    const uint64_t mask = (1ull << nbits) - 1;  // nbits <= 20
    for (int k = threadIdx.x; k < kTableTotalRows; k += blockDim.x) {
        const uint64_t* row = g + (size_t)k * W;
        uint64_t v = row[word] >> sh;
        if (sh && word + 1 < W) v |= row[word + 1] << (64 - sh);
        t.f[k] = (uint32_t)(v & mask) << scale;
    }
}

__device__ __forceinline__ uint32_t seed_field(const FieldTable& t, uint64_t i)
{
    uint64_t g = i ^ (i >> 1);
    uint32_t v = t.f[kTableZ0Row];
    while (g) {
        v ^= t.f[__ffsll((long long)g) - 1];
        g &= g - 1;
    }
    return v;
}

// Bins in shared memory: v is the byte offset of the counter.
struct SmemSink {
    unsigned char* base;
    uint32_t nb;  // bins
    __device__ __forceinline__ void consume(uint32_t v)
    {
        if (HLF_IN_BOUNDS(v >> 2, nb, kSiteHistBin)) atomicAdd(reinterpret_cast<uint32_t*>(base + v), 1u);
    }
    __device__ __forceinline__ void flush() {}
};

// Bins in global memory. Coalesce (the run walk): repeats of the current bin
// are counted in a register and added with one atomic when the bin changes; a
// field the first rows leave unchanged keeps one bin for long stretches of a
// thread's run, and global atomics on one address would serialise.
template <bool Coalesce>
struct GlobalSink {
    unsigned long long* bins;
    uint32_t nb;  // bins
    uint32_t cur = 0;
    uint32_t pending = 0;
    __device__ __forceinline__ void consume(uint32_t v)
    {
        if constexpr (Coalesce) {
            if (v == cur) {
                ++pending;
            } else {
                if (pending && HLF_IN_BOUNDS(cur, nb, kSiteHistBin)) atomicAdd(&bins[cur], (unsigned long long)pending);
                cur = v;
                pending = 1;
            }
        } else {
            if (HLF_IN_BOUNDS(v, nb, kSiteHistBin)) atomicAdd(&bins[v], 1ull);
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (Coalesce && pending && HLF_IN_BOUNDS(cur, nb, kSiteHistBin))
            atomicAdd(&bins[cur], (unsigned long long)pending);
        pending = 0;
    }
};

// 2^L consecutive steps of a reflected-Gray block over the register values
// R[0..L-1]: (first half, flip R[L-1], second half).
template <int L, typename Sink>
struct GrayBlock32 {
    static __device__ __forceinline__ void run(uint32_t& v, const uint32_t (&R)[kIL > kRU ? kIL : kRU], Sink& sink)
    {
        GrayBlock32<L - 1, Sink>::run(v, R, sink);
        v ^= R[L - 1];
        GrayBlock32<L - 1, Sink>::run(v, R, sink);
    }
};
template <typename Sink>
struct GrayBlock32<0, Sink> {
    static __device__ __forceinline__ void run(uint32_t& v, const uint32_t (&)[kIL > kRU ? kIL : kRU], Sink& sink)
    {
        sink.consume(v);
    }
};

struct HistPlan {
    uint64_t offset, count;
    uint64_t n_head;      // ragged indices [offset, offset + n_head)
    uint64_t tail_first;  // ragged indices [tail_first, offset + count)
    uint64_t n_tail;
    uint64_t h_first;     // groups [h_first, h_end) of 32 consecutive indices
    uint64_t h_end;
    uint64_t per_warp;    // groups per warp
    uint64_t per_thread;  // the run walk: [offset + g * per_thread, ...) for threads g < used
    uint64_t used;
    int W;                // the table's words per row
};

// True when f_0..f_4 are linearly independent over GF(2).
__device__ bool fields_independent(const FieldTable& t)
{
    uint32_t basis[5];
    int r = 0;
    for (int k = 0; k < 5; ++k) {
        uint32_t v = t.f[k];
        for (int j = 0; j < r; ++j)
            if ((v ^ basis[j]) < v) v ^= basis[j];  // reduce by the leading bit of basis[j]
        if (!v) return false;
        basis[r++] = v;
        for (int j = r - 1; j > 0 && basis[j] > basis[j - 1]; --j) {  // keep leading bits descending
            const uint32_t x = basis[j];
            basis[j] = basis[j - 1];
            basis[j - 1] = x;
        }
    }
    return true;
}

// The lane-interleaved walk.
template <bool InSmem>
__global__ void __launch_bounds__(kThreads) hist_interleaved_kernel(const uint64_t* __restrict__ table,
                                                                    HistPlan pl, int lo, int nbits,
                                                                    unsigned long long* __restrict__ out)
{
    constexpr int M = 5;  // log2 of the group
    extern __shared__ uint32_t s_bins[];
    __shared__ FieldTable t;
    __shared__ uint32_t s_C[kTableRows - M];  // C_j = f_{M-1} ^ f_{M+j}
    __shared__ bool s_skip;
    load_field_table(t, table, pl.W, lo, nbits, InSmem ? 2 : 0);
    const uint32_t nb = 1u << nbits;
    if (InSmem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) s_skip = !fields_independent(t);  // the run walk's case
    for (int j = threadIdx.x; j < kTableRows - M; j += blockDim.x) s_C[j] = t.f[M - 1] ^ t.f[M + j];
    __syncthreads();
    if (s_skip) return;  // uniform over the CTA

    using Sink = typename std::conditional<InSmem, SmemSink, GlobalSink<false>>::type;
    Sink sink;
    if constexpr (InSmem) sink.base = reinterpret_cast<unsigned char*>(s_bins);
    else sink.bins = out;
    sink.nb = nb;
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt < pl.n_head + pl.n_tail) {  // ragged head and tail, one index per thread
        const uint64_t i = gt < pl.n_head ? pl.offset + gt : pl.tail_first + (gt - pl.n_head);
        sink.consume(seed_field(t, i));
    }
    const uint64_t wg = gt >> 5;
    const int lane = threadIdx.x & 31;
    if (wg * pl.per_warp < pl.h_end - pl.h_first) {
        const uint64_t h0 = pl.h_first + wg * pl.per_warp;
        const uint64_t h1 = min(h0 + pl.per_warp, pl.h_end);
        uint32_t v = seed_field(t, h0 * kHistG + (uint64_t)lane);
        // Group h + 1 follows group h by C_ctz(h+1) (h < 2^59, so ctz <= 58).
        // Aligned blocks of 2^kIL groups run as reflected-Gray blocks over
        // C_0..C_{kIL-1} held in registers.
        uint64_t h = h0;
        while (h < h1 && (h & ((1u << kIL) - 1))) {
            sink.consume(v);
            if (++h < h1) v ^= s_C[ctz64(h)];
        }
        if (h + (1u << kIL) <= h1) {
            uint32_t R[kIL > kRU ? kIL : kRU];
#pragma unroll
            for (int k = 0; k < kIL; ++k) R[k] = s_C[k];
            do {
                GrayBlock32<kIL, Sink>::run(v, R, sink);
                h += 1u << kIL;
                if (h < h1) v ^= s_C[ctz64(h)];
            } while (h + (1u << kIL) <= h1);
        }
        while (h < h1) {
            sink.consume(v);
            if (++h < h1) v ^= s_C[ctz64(h)];
        }
    }
    __syncthreads();
    if (InSmem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
            if (s_bins[i]) atomicAdd(&out[i], (unsigned long long)s_bins[i]);
}

// The per-thread run walk.
template <bool InSmem>
__global__ void __launch_bounds__(kThreads) hist_runs_kernel(const uint64_t* __restrict__ table, HistPlan pl,
                                                             int lo, int nbits, unsigned long long* __restrict__ out)
{
    extern __shared__ uint32_t s_bins[];
    __shared__ FieldTable t;
    __shared__ bool s_skip;
    load_field_table(t, table, pl.W, lo, nbits, InSmem ? 2 : 0);
    const uint32_t nb = 1u << nbits;
    if (InSmem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) s_skip = fields_independent(t);  // the interleaved walk's case
    __syncthreads();
    if (s_skip) return;
    using Sink = typename std::conditional<InSmem, SmemSink, GlobalSink<true>>::type;
    Sink sink;
    if constexpr (InSmem) sink.base = reinterpret_cast<unsigned char*>(s_bins);
    else sink.bins = out;
    sink.nb = nb;
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < pl.used) {
        uint64_t i = pl.offset + g * pl.per_thread;
        const uint64_t a = g * pl.per_thread;
        if (a < pl.count) {
            uint64_t len = min(pl.per_thread, pl.count - a);
            uint32_t v = seed_field(t, i);
            constexpr uint64_t kBlk = 1ull << kRU;
            while (len && (i & (kBlk - 1))) {  // head up to a multiple of 2^kRU
                sink.consume(v);
                --len;
                ++i;
                if (len) v ^= t.f[ctz64(i)];
            }
            if (len >= kBlk) {
                uint32_t R[kIL > kRU ? kIL : kRU];
#pragma unroll
                for (int k = 0; k < kRU; ++k) R[k] = t.f[k];
                do {
                    GrayBlock32<kRU, Sink>::run(v, R, sink);
                    len -= kBlk;
                    i += kBlk;
                    if (len) v ^= t.f[ctz64(i)];  // ctz(i) >= kRU here
                } while (len >= kBlk);
            }
            while (len) {  // tail
                sink.consume(v);
                --len;
                ++i;
                if (len) v ^= t.f[ctz64(i)];
            }
            sink.flush();
        }
    }
    __syncthreads();
    if (InSmem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
            if (s_bins[i]) atomicAdd(&out[i], (unsigned long long)s_bins[i]);
}

template <typename K>
hlf_status hist_attrs(K kernel, size_t smem, int* per_sm)
{
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(uint32_t) << kHistSmemBits)) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, kThreads, smem) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (*per_sm < 1) *per_sm = 1;
    return HLF_OK;
}

template <bool InSmem>
hlf_status launch_hist_k(const uint64_t* table, int W, uint64_t offset, uint64_t count, int lo, int nbits,
                         uint64_t* out, cudaStream_t s)
{
    HistPlan pl{};
    pl.offset = offset;
    pl.count = count;
    pl.W = W;
    // Full groups are [h_first * 32, h_end * 32); the window's end can be 2^64
    // exactly (r >= 64), which wraps to 0 in 64 bits.
    const uint64_t G = kHistG;
    const uint64_t end = offset + count;
    const bool ends_at_2_64 = count != 0 && end == 0;
    const uint64_t a0 = (offset + (G - 1)) & ~(G - 1);
    const bool a0_wrapped = a0 < offset;
    const uint64_t h_first = a0 / G;
    const uint64_t h_end = ends_at_2_64 ? (0ull - G) / G + 1 : end / G;
    const uint64_t groups = (!a0_wrapped && h_end > h_first) ? h_end - h_first : 0;
    if (groups == 0) {
        pl.n_head = count;
        pl.h_first = pl.h_end = 0;
    } else {
        pl.n_head = a0 - offset;
        pl.h_first = h_first;
        pl.h_end = h_end;
        pl.tail_first = h_end * G;  // wraps to 0 only when the tail is empty
        pl.n_tail = count - pl.n_head - groups * G;
    }
    const size_t smem = InSmem ? (sizeof(uint32_t) << nbits) : 0;
    // CTAs per SM of each walk's kernel, per device, at the largest shared-memory size
    static int fit[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm_i = 1, per_sm_r = 1;
    if (dev < 64 && fit[dev][0] && smem == (sizeof(uint32_t) << kHistSmemBits)) {
        per_sm_i = fit[dev][0];
        per_sm_r = fit[dev][1];
    } else {
        hlf_status st = hist_attrs(hist_interleaved_kernel<InSmem>, smem, &per_sm_i);
        if (st == HLF_OK) st = hist_attrs(hist_runs_kernel<InSmem>, smem, &per_sm_r);
        if (st != HLF_OK) return st;
        if (dev < 64 && smem == (sizeof(uint32_t) << kHistSmemBits)) {
            fit[dev][0] = per_sm_i;
            fit[dev][1] = per_sm_r;
        }
    }

    // interleaved walk: at least 64 groups (2048 solutions) per warp, one wave
    const uint64_t max_warps = (uint64_t)sm_count() * per_sm_i * (kThreads / 32);
    uint64_t warps = (groups + 63) / 64;
    if (warps > max_warps) warps = max_warps;
    if (warps == 0) warps = 1;
    pl.per_warp = groups ? (groups + warps - 1) / warps : 1;
    if (pl.per_warp > kHistMaxGroupsPerWarp) pl.per_warp = kHistMaxGroupsPerWarp;
    warps = groups ? (groups + pl.per_warp - 1) / pl.per_warp : 1;
    uint64_t threads_i = warps * 32;
    if (threads_i < pl.n_head + pl.n_tail) threads_i = pl.n_head + pl.n_tail;
    // run walk: runs of whole 2^kRU blocks, at least 2048 solutions each, one wave
    const uint64_t max_threads = (uint64_t)sm_count() * per_sm_r * kThreads;
    uint64_t rthreads = (count + 2047) / 2048;
    if (rthreads > max_threads) rthreads = max_threads;
    if (rthreads == 0) rthreads = 1;
    pl.per_thread = (count + rthreads - 1) / rthreads;
    pl.per_thread = (pl.per_thread + (1ull << kRU) - 1) & ~((1ull << kRU) - 1);
    if (pl.per_thread > kHistMaxPerThread) pl.per_thread = kHistMaxPerThread;
    pl.used = (count + pl.per_thread - 1) / pl.per_thread;

    // Both are launched; the CTAs of the walk the field does not call for
    // return after reading the table.
    const uint64_t blocks_i = (threads_i + kThreads - 1) / kThreads;
    const uint64_t blocks_r = (pl.used + kThreads - 1) / kThreads;
    if (blocks_i > 0x7fffffffull || blocks_r > 0x7fffffffull) return HLF_ERR_RANGE;
    auto* o = reinterpret_cast<unsigned long long*>(out);
    hist_interleaved_kernel<InSmem><<<(unsigned)blocks_i, kThreads, smem, s>>>(table, pl, lo, nbits, o);
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    hist_runs_kernel<InSmem><<<(unsigned)blocks_r, kThreads, smem, s>>>(table, pl, lo, nbits, o);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_histogram(const uint64_t* table, int W, uint64_t offset, uint64_t count, int lo, int nbits,
                            uint64_t* out, cudaStream_t s)
{
    if (W < 1 || W > HLF_MAX_W || lo < 0 || nbits < 1 || nbits > HLF_HIST_MAX_BITS || lo + nbits > 64 * W)
        return HLF_ERR_ARG;
    if (nbits <= kHistSmemBits) return launch_hist_k<true>(table, W, offset, count, lo, nbits, out, s);
    return launch_hist_k<false>(table, W, offset, count, lo, nbits, out, s);
}

HLF_DEBUG_TAKE(hist)

}  // namespace hlf
