// Histogram of a bit field of every solution in a window, computed on the
// device while enumerating (no solution is stored): the counts behind the
// paper's output distributions of Figs. 3, 6 and 7, where each square shows
// how often one bit pattern of the first or last bits occurs.
//
// Two walks, two kernels; both are launched, and each CTA of the walk the
// field does not call for returns after reading the table (every CTA comes
// to the same answer):
// - lane-interleaved (the store kernel's walk, enumerate.cu): lane t of a warp
//   holds index 32 h + t and every lane steps by the same row
//   C_j = B_4 ^ B_{5+j}, j = ctz(h+1). The 32 solutions a warp counts at once
//   are z(32 h) combined with the 32 combinations of B_0..B_4, so when the
//   field bits of B_0..B_4 are linearly independent the 32 lanes land in 32
//   distinct bins, and the shared-memory atomics do not collide.
// - per-thread runs (the reduce's walk, enum_impl.cuh), for fields the first
//   five rows leave (nearly) unchanged: there the interleaved lanes would all
//   hit one bin, while a thread's run stays in one bin for many solutions.
// Each solution's bits [lo, lo + nbits) select a bin. They lie in at most
// two words of the solution, and XOR acts word by word, so the kernels walk
// the projection of the table onto those words (P = 1 or 2 words per row,
// whatever n is) and the field starts in the first projected word. Up to
// 2^14 bins live in shared memory per CTA (32-bit counters, flushed to the
// global 64-bit bins with one atomic per nonzero bin); wider fields count
// straight into global memory.

#include "enum_impl.cuh"

namespace hlf {
namespace {

constexpr int kHistSmemBits = 15;  // 2^15 32-bit bins: 128 KB of shared memory
constexpr int kHistG = 32;                              // consecutive indices per warp step
constexpr uint64_t kHistMaxGroupsPerWarp = 1ull << 23;  // keeps a CTA's counts below 2^32
constexpr uint64_t kHistMaxPerThread = 1ull << 23;      // the same bound for the run walk

// Coalesce (the run walk with bins in global memory): repeats of the current
// bin are counted in a register and added with one atomic when the bin
// changes, and flush() adds the last count. A field the first rows leave
// unchanged keeps one bin for long stretches of a thread's run, and global
// atomics on one address would serialise.
template <int P, bool Coalesce = false>
struct HistSink {
    uint32_t* s_bins;               // shared, when nbits <= kHistSmemBits
    unsigned long long* g_bins;     // global, otherwise
    uint32_t shift;                 // the field's first bit in projected word 0
    int nbits;
    uint64_t mask;
    uint64_t cur = 0;               // Coalesce: the current bin and its pending count
    uint32_t pending = 0;
    __device__ __forceinline__ uint64_t field(const uint64_t (&z)[P]) const
    {
        uint64_t v = z[0] >> shift;
        if constexpr (P == 2) v |= shl64(z[1], 64 - shift);  // 0 when shift == 0
        return v & mask;
    }
    __device__ __forceinline__ void add(uint64_t v, uint32_t c)
    {
        if (nbits <= kHistSmemBits) atomicAdd(&s_bins[v], c);
        else atomicAdd(&g_bins[v], (unsigned long long)c);
    }
    __device__ __forceinline__ void consume(const uint64_t (&z)[P])
    {
        const uint64_t v = field(z);
        if constexpr (Coalesce) {
            if (v == cur) {
                ++pending;
            } else {
                if (pending) add(cur, pending);
                cur = v;
                pending = 1;
            }
        } else {
            add(v, 1u);
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (Coalesce && pending) add(cur, pending);
        pending = 0;
    }
};

// The table's rows (and z0) projected onto words [word, word + P).
template <int P>
__device__ __forceinline__ void load_table_projected(Table<P>& t, const uint64_t* __restrict__ g, int Wfull,
                                                     int word)
{
    uint64_t* d = &t.B[0][0];
    for (int i = threadIdx.x; i < kTableTotalRows * P; i += blockDim.x)
        d[i] = g[(i / P) * Wfull + word + i % P];
}

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
    int Wfull, word;      // the table's words per row; the first projected word
};

// True when the field bits of B_0..B_4 are linearly independent over GF(2).
template <int W>
__device__ bool fields_independent(const Table<W>& t, const HistSink<W, false>& sink)
{
    uint64_t basis[5];
    int r = 0;
    for (int k = 0; k < 5; ++k) {
        uint64_t row[W];
#pragma unroll
        for (int w = 0; w < W; ++w) row[w] = t.B[k][w];
        uint64_t v = sink.field(row);
        for (int j = 0; j < r; ++j)
            if ((v ^ basis[j]) < v) v ^= basis[j];  // reduce by the leading bit of basis[j]
        if (!v) return false;
        basis[r++] = v;
        for (int j = r - 1; j > 0 && basis[j] > basis[j - 1]; --j) {  // keep leading bits descending
            const uint64_t x = basis[j];
            basis[j] = basis[j - 1];
            basis[j - 1] = x;
        }
    }
    return true;
}

// The lane-interleaved walk.
template <int W>
__global__ void __launch_bounds__(kThreads) hist_interleaved_kernel(const uint64_t* __restrict__ table,
                                                                    HistPlan pl, int lo, int nbits,
                                                                    unsigned long long* __restrict__ out)
{
    constexpr int M = 5;  // log2 of the group
    extern __shared__ uint32_t s_bins[];
    __shared__ Table<W> t;
    __shared__ uint64_t s_C[kTableRows - M][W];  // C_j = B_{M-1} ^ B_{M+j}
    __shared__ bool s_skip;
    load_table_projected<W>(t, table, pl.Wfull, pl.word);
    const bool in_smem = nbits <= kHistSmemBits;
    const uint32_t nb = 1u << nbits;
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    HistSink<W> sink{s_bins, out, (uint32_t)(lo & 63), nbits, nbits == 64 ? ~0ull : ((1ull << nbits) - 1)};
    if (threadIdx.x == 0) s_skip = !fields_independent<W>(t, sink);  // the run walk's case
    for (int i = threadIdx.x; i < (kTableRows - M) * W; i += blockDim.x) {
        const int j = i / W, w = i % W;
        s_C[j][w] = t.B[M - 1][w] ^ t.B[M + j][w];
    }
    __syncthreads();
    if (s_skip) return;  // uniform over the CTA

    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt < pl.n_head + pl.n_tail) {  // ragged head and tail, one index per thread
        const uint64_t i = gt < pl.n_head ? pl.offset + gt : pl.tail_first + (gt - pl.n_head);
        uint64_t z[W];
        seed<W>(t, i, z);
        sink.consume(z);
    }
    const uint64_t wg = gt >> 5;
    const int lane = threadIdx.x & 31;
    if (wg * pl.per_warp < pl.h_end - pl.h_first) {
        const uint64_t h0 = pl.h_first + wg * pl.per_warp;
        const uint64_t h1 = min(h0 + pl.per_warp, pl.h_end);
        uint64_t z[W];
        seed<W>(t, h0 * kHistG + (uint64_t)lane, z);
        // Group h + 1 follows group h by the row C_ctz(h+1) (h < 2^59, so
        // ctz <= 59). Aligned blocks of 2^L groups run as reflected-Gray
        // blocks over C_0..C_{L-1}, as the reduce's runs do over B_0..B_{U-1}
        // (shorter blocks for wide rows, which would cost registers).
        constexpr int L = W == 1 ? 4 : (W <= 4 ? 2 : 1);
        uint64_t h = h0;
        while (h < h1 && (h & ((1u << L) - 1))) {
            sink.consume(z);
            if (++h < h1) xor_row<W>(z, s_C[ctz64(h)]);
        }
        if (h + (1u << L) <= h1) {
            if constexpr (W == 1) {
                uint64_t Cr[L][1];
#pragma unroll
                for (int k = 0; k < L; ++k) Cr[k][0] = s_C[k][0];
                do {
                    GrayBlock<W, L, uint64_t[L][1], HistSink<W>>::run(z, Cr, sink);
                    h += 1u << L;
                    if (h < h1) xor_row<W>(z, s_C[ctz64(h)]);
                } while (h + (1u << L) <= h1);
            } else {
                do {
                    GrayBlock<W, L, uint64_t[kTableRows - M][W], HistSink<W>>::run(z, s_C, sink);
                    h += 1u << L;
                    if (h < h1) xor_row<W>(z, s_C[ctz64(h)]);
                } while (h + (1u << L) <= h1);
            }
        }
        while (h < h1) {
            sink.consume(z);
            if (++h < h1) xor_row<W>(z, s_C[ctz64(h)]);
        }
    }
    __syncthreads();
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
            if (s_bins[i]) atomicAdd(&out[i], (unsigned long long)s_bins[i]);
}

// The per-thread run walk.
template <int W, int U, bool Coalesce>
__global__ void __launch_bounds__(kThreads) hist_runs_kernel(const uint64_t* __restrict__ table, HistPlan pl,
                                                             int lo, int nbits, unsigned long long* __restrict__ out)
{
    extern __shared__ uint32_t s_bins[];
    __shared__ Table<W> t;
    __shared__ bool s_skip;
    load_table_projected<W>(t, table, pl.Wfull, pl.word);
    const bool in_smem = nbits <= kHistSmemBits;
    const uint32_t nb = 1u << nbits;
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    const uint64_t mask = nbits == 64 ? ~0ull : ((1ull << nbits) - 1);
    if (threadIdx.x == 0)  // the interleaved walk's case
        s_skip = fields_independent<W>(t, HistSink<W, false>{s_bins, out, (uint32_t)(lo & 63), nbits, mask});
    __syncthreads();
    if (s_skip) return;
    HistSink<W, Coalesce> sink{s_bins, out, (uint32_t)(lo & 63), nbits, mask};
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < pl.used) {
        const uint64_t a = g * pl.per_thread;
        if (a < pl.count) {
            walk_run<W, U, HistSink<W, Coalesce>>(t, pl.offset + a, min(pl.per_thread, pl.count - a), sink);
            sink.flush();
        }
    }
    __syncthreads();
    if (in_smem)
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

template <int W>
hlf_status launch_hist_w(const uint64_t* table, int Wfull, uint64_t offset, uint64_t count, int lo, int nbits,
                         uint64_t* out, cudaStream_t s)
{
    constexpr int U = reduce_unroll(W);
    HistPlan pl{};
    pl.offset = offset;
    pl.count = count;
    pl.Wfull = Wfull;
    pl.word = lo >> 6;
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
    const size_t smem = nbits <= kHistSmemBits ? (sizeof(uint32_t) << nbits) : 0;
    static int fit[64][2] = {};  // CTAs per SM of each walk's kernel, per device
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm_i = 1, per_sm_r = 1;
    if (dev < 64 && fit[dev][0] && smem == (sizeof(uint32_t) << kHistSmemBits)) {
        per_sm_i = fit[dev][0];
        per_sm_r = fit[dev][1];
    } else {
        hlf_status st = hist_attrs(hist_interleaved_kernel<W>, smem, &per_sm_i);
        if (st == HLF_OK)
            st = smem ? hist_attrs(hist_runs_kernel<W, U, false>, smem, &per_sm_r)
                      : hist_attrs(hist_runs_kernel<W, U, true>, smem, &per_sm_r);
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
    // run walk: runs of whole 2^U blocks, at least 2048 solutions each, one wave
    const uint64_t max_threads = (uint64_t)sm_count() * per_sm_r * kThreads;
    uint64_t rthreads = (count + 2047) / 2048;
    if (rthreads > max_threads) rthreads = max_threads;
    if (rthreads == 0) rthreads = 1;
    pl.per_thread = (count + rthreads - 1) / rthreads;
    pl.per_thread = (pl.per_thread + (1ull << U) - 1) & ~((1ull << U) - 1);
    if (pl.per_thread > kHistMaxPerThread) pl.per_thread = kHistMaxPerThread;
    pl.used = (count + pl.per_thread - 1) / pl.per_thread;

    // Both are launched; the CTAs of the walk the field does not call for
    // return after reading the table.
    const uint64_t blocks_i = (threads_i + kThreads - 1) / kThreads;
    const uint64_t blocks_r = (pl.used + kThreads - 1) / kThreads;
    if (blocks_i > 0x7fffffffull || blocks_r > 0x7fffffffull) return HLF_ERR_RANGE;
    auto* o = reinterpret_cast<unsigned long long*>(out);
    hist_interleaved_kernel<W><<<(unsigned)blocks_i, kThreads, smem, s>>>(table, pl, lo, nbits, o);
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    if (smem)
        hist_runs_kernel<W, U, false><<<(unsigned)blocks_r, kThreads, smem, s>>>(table, pl, lo, nbits, o);
    else  // bins in global memory: coalesce repeats
        hist_runs_kernel<W, U, true><<<(unsigned)blocks_r, kThreads, smem, s>>>(table, pl, lo, nbits, o);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_histogram(const uint64_t* table, int W, uint64_t offset, uint64_t count, int lo, int nbits,
                            uint64_t* out, cudaStream_t s)
{
    if (W < 1 || W > HLF_MAX_W || lo < 0 || nbits < 1 || lo + nbits > 64 * W) return HLF_ERR_ARG;
    // the field's words: one, or two when it crosses a word boundary
    if ((lo & 63) + nbits > 64) return launch_hist_w<2>(table, W, offset, count, lo, nbits, out, s);
    return launch_hist_w<1>(table, W, offset, count, lo, nbits, out, s);
}

}  // namespace hlf
