// Stage 2 of the two-stage scheme: the classical parallel circuit of
// Section 2 (Eqs. 1-3, Fig. 1(c)) that turns the stage-1 quantities into the
// solutions z = y ^ z^a, y in Col(A), one after another.
//
// On the GPU the paper's binary counter over R^(r) becomes the reflected Gray
// code over the RREF basis (the reading stated in hlf.h):
//     z(i) = z0 ^ XOR_{k in g(i)} B_k,  g(i) = i ^ (i >> 1),
// so consecutive solutions differ by one basis row, z(i+1) = z(i) ^ B_ctz(i+1),
// and any window can be seeded independently with <= 64 row XORs.
//
// Kernels
//   reduce_kernel        each thread seeds its own contiguous run of indices
//                        and walks it one XOR per solution; blocks of 2^U
//                        solutions are unrolled so that the first U basis
//                        rows are compile-time register operands. The
//                        per-thread (count, hash sum, XOR-fold) is reduced by
//                        warp shuffles, shared memory and one 64-bit atomic
//                        per quantity per CTA.
//   reduce_chunks_kernel the same walk, one CTA per chunk, one result per chunk.
//   store_kernel         coalesced materialisation. Lane t of a warp owns
//                        index G*h + S*t (+1), G = 32*S. With m = log2 G,
//                          g(G h + t) = (g(h) << m) ^ ((h & 1) << (m-1)) ^ g(t),
//                        so stepping h -> h+1 XORs the same row
//                        C_j = B_{m-1} ^ B_{m+j}, j = ctz(h+1), into every
//                        lane: one XOR per solution and a warp writes G
//                        consecutive solutions per step (512 B at W = 1;
//                        at W > 1 the lanes' solutions are restaged in
//                        shared memory so that the warp writes its 32*W
//                        words with consecutive lanes on consecutive words).
//   sample_kernel        z(i) at arbitrary indices, straight from the formula.

#include "enum_impl.cuh"

namespace hlf {
namespace {



template <int W, int U, int T>
__global__ void __launch_bounds__(T, min_ctas_for(W)) reduce_kernel(const uint64_t* __restrict__ table,
                                                                   uint64_t offset, uint64_t count,
                                                                   uint64_t per_thread, uint64_t threads_used,
                                                                   hlf_reduce* __restrict__ out)
{
    __shared__ Table<W> t;
    load_table_hash_domain<W>(t, table);
    __syncthreads();
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Acc<W> acc;
    acc.zero();
    uint64_t cnt = 0;
    if (g < threads_used) {
        const uint64_t a = g * per_thread;
        if (a < count) {
            const uint64_t len = min(per_thread, count - a);
            cnt = len;
            reduce_run<W, U>(t, offset + a, len, acc);
        }
    }
    block_reduce<W, T>(cnt, acc);
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

template <int W, int U>
__global__ void __launch_bounds__(kThreads) reduce_chunks_kernel(const uint64_t* __restrict__ table,
                                                                 uint64_t offset, uint64_t chunk,
                                                                 uint64_t n_chunks, hlf_reduce* __restrict__ out)
{
    __shared__ Table<W> t;
    load_table_hash_domain<W>(t, table);
    __syncthreads();
    const uint64_t per_thread = (chunk + blockDim.x - 1) / blockDim.x;
    for (uint64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        Acc<W> acc;
        acc.zero();
        uint64_t cnt = 0;
        const uint64_t a = threadIdx.x * per_thread;
        if (a < chunk) {
            const uint64_t len = min(per_thread, chunk - a);
            cnt = len;
            reduce_run<W, U>(t, offset + c * chunk + a, len, acc);
        }
        block_reduce<W>(cnt, acc);
        if (threadIdx.x == 0) {
            hlf_reduce& r = out[c];
            r.count = cnt;
            r.hsum = acc.hs;
#pragma unroll
            for (int w = 0; w < HLF_MAX_W; ++w) r.xor_fold[w] = w < W ? acc.fold_word(w) : 0ull;
        }
    }
}

struct StorePlan {
    uint64_t offset, count;
    uint64_t n_head;       // ragged indices [offset, offset + n_head)
    uint64_t tail_first;   // ragged indices [tail_first, offset + count)
    uint64_t n_tail;
    uint64_t h_first;      // groups [h_first, h_end) of G consecutive indices
    uint64_t h_end;
    uint64_t per_warp;     // groups per warp
};

// S = solutions per lane (2 for W = 1, so a lane writes one 16-byte pair).
template <int W, int S>
__global__ void __launch_bounds__(kThreads) store_kernel(const uint64_t* __restrict__ table, StorePlan pl,
                                                         uint64_t* __restrict__ out)
{
    constexpr int G = 32 * S;
    constexpr int M = (S == 2) ? 6 : 5;  // log2 G
    extern __shared__ __align__(16) uint64_t s_stage[];  // W > 1: [warps][stage_words<W>()]
    __shared__ Table<W> t;
    __shared__ uint64_t s_C[kTableRows - M][W];  // C_j = B_{M-1} ^ B_{M+j}
    load_table<W>(t, table);
    __syncthreads();
    for (int i = threadIdx.x; i < (kTableRows - M) * W; i += blockDim.x) {
        const int j = i / W, w = i % W;
        s_C[j][w] = t.B[M - 1][w] ^ t.B[M + j][w];
    }
    __syncthreads();

    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // ragged head and tail, one index per thread, from the definition
    if (gt < pl.n_head + pl.n_tail) {
        const uint64_t i = gt < pl.n_head ? pl.offset + gt : pl.tail_first + (gt - pl.n_head);
        uint64_t z[W];
        seed<W>(t, i, z);
        if (HLF_IN_BOUNDS(i - pl.offset, pl.count, kSiteStore)) {
#pragma unroll
            for (int w = 0; w < W; ++w) out[(i - pl.offset) * W + w] = z[w];
        }
    }

    const uint64_t wg = gt >> 5;
    const int lane = threadIdx.x & 31;
    const uint64_t h0 = pl.h_first + wg * pl.per_warp;
    if (wg * pl.per_warp >= pl.h_end - pl.h_first) return;
    const uint64_t h1 = min(h0 + pl.per_warp, pl.h_end);
    uint64_t z[W];
    seed<W>(t, h0 * G + (uint64_t)(S * lane), z);
    // W = 1: a lane's pair starts at word out + (even index - offset); it is
    // 16-byte aligned when the output's word index and the offset agree in parity
    const bool even = (((reinterpret_cast<uintptr_t>(out) >> 3) ^ pl.offset) & 1) == 0;
    for (uint64_t h = h0;;) {
        if constexpr (S == 2) {
            uint64_t* p = out + (h * G + (uint64_t)(S * lane) - pl.offset) * W;
            const uint64_t z1 = z[0] ^ t.B[0][0];  // g(2t+1) = g(2t) ^ 1
            if (HLF_RANGE_IN_BOUNDS(h * G + (uint64_t)(S * lane) - pl.offset, 2, pl.count, kSiteStore)) {
                if (even) {
                    st_cs_v2(p, z[0], z1);
                } else {
                    st_cs(p, z[0]);
                    st_cs(p + 1, z1);
                }
            }
        } else {  // W > 1: out is 16-byte aligned (checked by the callers); the check is warp-uniform
            if (HLF_RANGE_IN_BOUNDS(h * G - pl.offset, G, pl.count, kSiteStore))
                store_warp_coalesced<W, true>(out + (h * G - pl.offset) * W, z,
                                              s_stage + (threadIdx.x >> 5) * stage_words<W>(), lane);
        }
        if (++h == h1) break;
        xor_row<W>(z, s_C[ctz64(h)]);
    }
}

// ----------------------------------------------------------------- sample

template <int W>
__global__ void __launch_bounds__(kThreads) sample_kernel(const uint64_t* __restrict__ table, int nb,
                                                          const uint64_t* __restrict__ idx, uint64_t m,
                                                          uint64_t* __restrict__ out, int32_t* info)
{
    __shared__ Table<W> t;
    load_table<W>(t, table);
    __syncthreads();
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = idx[j];
        uint64_t z[W];
        if (nb < 64 && (i >> nb)) {
            *reinterpret_cast<volatile int32_t*>(info) = HLF_ERR_RANGE;  // host-mapped status word
#pragma unroll
            for (int w = 0; w < W; ++w) z[w] = 0;
        } else {
            seed<W>(t, i, z);
        }
        if (HLF_IN_BOUNDS(j, m, kSiteStore)) {
#pragma unroll
            for (int w = 0; w < W; ++w) out[j * W + w] = z[w];
        }
    }
}

// ------------------------------------------------------------- launchers


// CTAs of `kernel` that fit on one SM at once (at least 1): grids are sized
// to one wave, since every kernel here gives its CTAs equal work and a
// partial second wave would cost a whole extra wave.
template <typename K>
int blocks_per_sm(K kernel, size_t smem)
{
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, kThreads, smem) != cudaSuccess || fit < 1) {
        cudaGetLastError();
        return 1;
    }
    return fit;
}

template <int W>
hlf_status launch_reduce_w(const uint64_t* table, uint64_t offset, uint64_t count, hlf_reduce* out,
                           cudaStream_t s)
{
    constexpr int U = reduce_unroll(W);
    constexpr int T = reduce_threads(W);
    // one wave: as many CTAs as fit on every SM at once
    static int fit[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && fit[dev] == 0 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit[dev], reduce_kernel<W, U, T>, T, 0) != cudaSuccess)
        return HLF_ERR_CUDA;
    const int per_sm = (dev < 64 && fit[dev] > 0) ? fit[dev] : 1;
    const uint64_t max_threads = (uint64_t)sm_count() * per_sm * T;
    const uint64_t min_run = 2048;  // amortises the <= 64-row seed
    uint64_t threads = (count + min_run - 1) / min_run;
    if (threads > max_threads) threads = max_threads;
    if (threads == 0) threads = 1;
    uint64_t per_thread = (count + threads - 1) / threads;
    per_thread = (per_thread + (1ull << U) - 1) & ~((1ull << U) - 1);  // keep runs aligned
    const uint64_t used = (count + per_thread - 1) / per_thread;
    const unsigned blocks = (unsigned)((used + T - 1) / T);
    reduce_kernel<W, U, T><<<blocks, T, 0, s>>>(table, offset, count, per_thread, used, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

template <int W>
hlf_status launch_reduce_chunks_w(const uint64_t* table, uint64_t offset, uint64_t chunk, uint64_t n_chunks,
                                  hlf_reduce* out, cudaStream_t s)
{
    constexpr int U = reduce_unroll(W);
    const uint64_t cap = (uint64_t)sm_count() * blocks_per_sm(reduce_chunks_kernel<W, U>, 0);
    const unsigned blocks = (unsigned)(n_chunks < cap ? n_chunks : cap);
    reduce_chunks_kernel<W, U><<<blocks, kThreads, 0, s>>>(table, offset, chunk, n_chunks, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

template <int W>
hlf_status launch_store_w(const uint64_t* table, uint64_t offset, uint64_t count, uint64_t* out,
                          cudaStream_t s)
{
    constexpr int S = (W == 1) ? 2 : 1;
    constexpr uint64_t G = 32 * S;
    StorePlan pl{};
    pl.offset = offset;
    pl.count = count;
    // Full groups are [h_first * G, h_end * G). The window's end offset+count
    // can be 2^64 exactly (r >= 64), which wraps to 0 in 64 bits; then the
    // last group index is 2^(64 - log2 G).
    const uint64_t end = offset + count;
    const bool ends_at_2_64 = count != 0 && end == 0;
    const uint64_t a0 = (offset + (G - 1)) & ~(G - 1);
    const bool a0_wrapped = a0 < offset;
    const uint64_t h_first = a0 / G;
    const uint64_t h_end = ends_at_2_64 ? (0ull - G) / G + 1 : end / G;
    const uint64_t groups = (!a0_wrapped && h_end > h_first) ? h_end - h_first : 0;
    if (groups == 0) {
        pl.n_head = count;
        pl.n_tail = 0;
        pl.tail_first = 0;
        pl.h_first = pl.h_end = 0;
    } else {
        pl.n_head = a0 - offset;
        pl.h_first = h_first;
        pl.h_end = h_end;
        pl.tail_first = h_end * G;  // wraps to 0 only when the tail is empty
        pl.n_tail = count - pl.n_head - groups * G;
    }
    const size_t smem = S == 1 ? (size_t)(kThreads / 32) * stage_words<W>() * sizeof(uint64_t) : 0;
    if (S == 1) {
        static bool attr_set[64] = {false};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 64 && !attr_set[dev]) {
            if (cudaFuncSetAttribute(store_kernel<W, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return HLF_ERR_CUDA;
            attr_set[dev] = true;
        }
    }
    const uint64_t max_warps = (uint64_t)sm_count() * blocks_per_sm(store_kernel<W, S>, smem) * (kThreads / 32);
    const uint64_t min_groups = 64;
    uint64_t warps = (groups + min_groups - 1) / min_groups;
    if (warps > max_warps) warps = max_warps;
    if (warps == 0) warps = 1;
    pl.per_warp = groups ? (groups + warps - 1) / warps : 1;
    const uint64_t ragged = pl.n_head + pl.n_tail;
    uint64_t threads = warps * 32;
    if (threads < ragged) threads = ragged;
    const unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
    store_kernel<W, S><<<blocks, kThreads, smem, s>>>(table, pl, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

template <int W>
hlf_status launch_sample_w(const uint64_t* table, int nb, const uint64_t* idx, uint64_t m, uint64_t* out,
                           int32_t* info, cudaStream_t s)
{
    const uint64_t cap = (uint64_t)sm_count() * blocks_per_sm(sample_kernel<W>, 0);
    uint64_t blocks = (m + kThreads - 1) / kThreads;
    if (blocks > cap) blocks = cap;
    sample_kernel<W><<<(unsigned)blocks, kThreads, 0, s>>>(table, nb, idx, m, out, info);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

#define HLF_DISPATCH_W(W, CALL)                     \
    switch (W) {                                    \
    case 1: return CALL(1);                         \
    case 2: return CALL(2);                         \
    case 3: return CALL(3);                         \
    case 4: return CALL(4);                         \
    case 5: return CALL(5);                         \
    case 6: return CALL(6);                         \
    case 7: return CALL(7);                         \
    case 8: return CALL(8);                         \
    case 9: return CALL(9);                         \
    case 10: return CALL(10);                       \
    case 11: return CALL(11);                       \
    case 12: return CALL(12);                       \
    case 13: return CALL(13);                       \
    case 14: return CALL(14);                       \
    case 15: return CALL(15);                       \
    case 16: return CALL(16);                       \
    default: return HLF_ERR_SIZE;                   \
    }

}  // namespace

hlf_status launch_reduce(const uint64_t* table, int W, uint64_t offset, uint64_t count, hlf_reduce* out,
                         cudaStream_t s)
{
#define CALL(w) launch_reduce_w<w>(table, offset, count, out, s)
    HLF_DISPATCH_W(W, CALL)
#undef CALL
}

hlf_status launch_reduce_chunks(const uint64_t* table, int W, uint64_t offset, uint64_t chunk,
                                uint64_t n_chunks, hlf_reduce* out, cudaStream_t s)
{
#define CALL(w) launch_reduce_chunks_w<w>(table, offset, chunk, n_chunks, out, s)
    HLF_DISPATCH_W(W, CALL)
#undef CALL
}

hlf_status launch_store(const uint64_t* table, int W, uint64_t offset, uint64_t count, uint64_t* out,
                        cudaStream_t s)
{
#define CALL(w) launch_store_w<w>(table, offset, count, out, s)
    HLF_DISPATCH_W(W, CALL)
#undef CALL
}

hlf_status launch_sample(const uint64_t* table, int W, int nb, const uint64_t* idx, uint64_t m,
                         uint64_t* out, int32_t* info, cudaStream_t s)
{
#define CALL(w) launch_sample_w<w>(table, nb, idx, m, out, info, s)
    HLF_DISPATCH_W(W, CALL)
#undef CALL
}

HLF_DEBUG_TAKE(enumerate)

}  // namespace hlf
