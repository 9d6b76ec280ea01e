// Device helpers of stage 2 (the classical parallel circuit of Section 2,
// Eqs. 1-3, Fig. 1(c)), shared by the single-instance kernels and the batched
// persistent kernel: the shared-memory enumeration table, seeding a run from
// the definition z(i) = z0 ^ XOR_{k in g(i)} B_k, the reflected-Gray walk of a
// run with its reduce, the per-thread reduce accumulator and the block
// reduction.
#pragma once

#include "hlf_internal.cuh"

namespace hlf {

constexpr int kThreads = 256;

// Solutions unrolled per Gray block (2^U) in the per-thread walks: 2^6 at
// W = 1, 2^4 at W = 2, 2^3 at W = 3, 4, and 2^2 beyond, where each solution is
// already 24W - 4 operations and deeper unrolling only costs registers.
// Shape of the single-instance reduce: at W <= 4 one CTA of 1024 threads per
// SM with up to 64 registers each; with the deeper unroll, measured 7-10%
// faster than several 256-thread CTAs with 40-44 registers each.
constexpr int reduce_unroll(int W) { return W == 1 ? 6 : (W == 2 ? 4 : (W <= 4 ? 3 : 2)); }
constexpr int reduce_threads(int W) { return W <= 4 ? 1024 : kThreads; }
constexpr int min_ctas_for(int W) { return W <= 4 ? 1 : 2; }

template <int W>
struct Table {
    uint64_t B[kTableRows][W];  // B_0..B_63, zero rows beyond min(r,64), row 64 zero
    uint64_t z0[W];
};

template <int W>
__device__ __forceinline__ void load_table(Table<W>& t, const uint64_t* __restrict__ g)
{
    uint64_t* d = &t.B[0][0];
    for (int i = threadIdx.x; i < kTableTotalRows * W; i += blockDim.x) d[i] = g[i];
}

// The first layer of the SplitMix64 finalizer, L(x) = x ^ (x >> 30), is
// linear over GF(2), so it commutes with the walk's XORs:
// L(z(i+1)) = L(z(i)) ^ L(B_ctz(i+1)). The reduce therefore walks y = L(z) on
// word 0, with a table whose word-0 entries are L(B_k) and L(z0), and hashes
// y with the remaining layers (mix_tail). Hash values are bit-identical to
// mix64(z); the XOR-fold of word 0 is taken in the L domain and mapped back
// once with L^-1(y) = y ^ (y >> 30) ^ (y >> 60).
__device__ __forceinline__ uint64_t mix_head(uint64_t x) { return x ^ (x >> 30); }
__device__ __forceinline__ uint64_t mix_head_inv(uint64_t y) { return y ^ (y >> 30) ^ (y >> 60); }
__device__ __forceinline__ uint64_t mix_tail(uint64_t y)
{
    y *= 0xBF58476D1CE4E5B9ull;
    y ^= y >> 27;
    y *= 0x94D049BB133111EBull;
    y ^= y >> 31;
    return y;
}

// Table for the reduce: word 0 of every row (and of z0) taken through L.
template <int W>
__device__ __forceinline__ void load_table_hash_domain(Table<W>& t, const uint64_t* __restrict__ g)
{
    uint64_t* d = &t.B[0][0];
    for (int i = threadIdx.x; i < kTableTotalRows * W; i += blockDim.x) {
        const uint64_t v = __ldcg(g + i);
        d[i] = (i % W == 0) ? mix_head(v) : v;
    }
}

// 64-bit shifts with PTX semantics: amounts of 64 give 0.
__device__ __forceinline__ uint64_t shl64(uint64_t x, uint32_t s)
{
    uint64_t r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
__device__ __forceinline__ uint64_t shr64(uint64_t x, uint32_t s)
{
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
template <int W>
__device__ __forceinline__ void xor_row(uint64_t (&z)[W], const uint64_t* __restrict__ b)
{
#pragma unroll
    for (int w = 0; w < W; ++w) z[w] ^= b[w];
}

// z(i) from its definition (seed of a run).
template <int W>
__device__ __forceinline__ void seed(const Table<W>& t, uint64_t i, uint64_t (&z)[W])
{
    uint64_t g = i ^ (i >> 1);
#pragma unroll
    for (int w = 0; w < W; ++w) z[w] = t.z0[w];
    while (g) {
        const int k = __ffsll((long long)g) - 1;
        g &= g - 1;
        xor_row<W>(z, t.B[k]);
    }
}

// Per-thread accumulator of the reduce, fed with solutions whose word 0 is in
// the L domain (see load_table_hash_domain): sum of hashes and XOR-fold.
template <int W>
struct Acc {
    uint64_t hs;
    uint64_t fold[W];
    __device__ __forceinline__ void zero()
    {
        hs = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) fold[w] = 0;
    }
    __device__ __forceinline__ void consume(const uint64_t (&z)[W])
    {
        uint64_t h = mix_tail(z[0]);  // = mix64 of the solution's word 0
#pragma unroll
        for (int w = 1; w < W; ++w) h = mix64(h ^ z[w]);
        hs += h;
#pragma unroll
        for (int w = 0; w < W; ++w) fold[w] ^= z[w];
    }
    // The hash alone: for the solutions of whole aligned Gray blocks, whose
    // XOR is zero (see reduce_run).
    __device__ __forceinline__ void consume_hash(const uint64_t (&z)[W])
    {
        uint64_t h = mix_tail(z[0]);
#pragma unroll
        for (int w = 1; w < W; ++w) h = mix64(h ^ z[w]);
        hs += h;
    }
    // XOR-fold back in the solution domain (after all XOR reductions).
    __device__ __forceinline__ uint64_t fold_word(int w) const { return w == 0 ? mix_head_inv(fold[0]) : fold[w]; }
};

// The accumulator seen by whole aligned Gray blocks: hash only.
template <int W>
struct HashOnly {
    Acc<W>& acc;
    __device__ __forceinline__ void consume(const uint64_t (&z)[W]) { acc.consume_hash(z); }
};

// 2^L consecutive solutions starting at an index that is a multiple of 2^L:
// the reflected Gray code is (first half, flip bit L-1, second half), so the
// step between the halves is row L-1, at a compile-time index. `Rows` is a
// register array (W = 1) or the shared-memory table (W > 1, where register
// copies of U rows of W words would cost more occupancy than they save).
// `Sink` consumes each solution (the reduce accumulator, a histogram).
template <int W, int L, typename Rows, typename Sink>
struct GrayBlock {
    static __device__ __forceinline__ void run(uint64_t (&z)[W], const Rows& Br, Sink& sink)
    {
        GrayBlock<W, L - 1, Rows, Sink>::run(z, Br, sink);
        xor_row<W>(z, Br[L - 1]);
        GrayBlock<W, L - 1, Rows, Sink>::run(z, Br, sink);
    }
};
template <int W, typename Rows, typename Sink>
struct GrayBlock<W, 0, Rows, Sink> {
    static __device__ __forceinline__ void run(uint64_t (&z)[W], const Rows&, Sink& sink) { sink.consume(z); }
};

// The reduce of [i, i + len). The solutions of an aligned block of 2^U
// consecutive indices (U >= 2) are z_s ^ XOR_{k in S} B_k over all subsets S
// of {0..U-1}: z_s and every B_k occur an even number of times, so their
// XOR is zero (in the L domain too, L being linear). Whole blocks therefore
// feed only the hash; the head and the tail of the run (partial blocks) feed
// hash and fold. The fold is exact, and one 64-bit XOR per solution lighter.
template <int W, int U>
__device__ __forceinline__ void reduce_run(const Table<W>& t, uint64_t i, uint64_t len, Acc<W>& acc)
{
    static_assert(U >= 2, "a block of 2^U solutions XORs to zero only for U >= 2");
    if (len == 0) return;
    uint64_t z[W];
    seed<W>(t, i, z);
    constexpr uint64_t kBlk = 1ull << U;
    while (len && (i & (kBlk - 1))) {  // head up to a multiple of 2^U
        acc.consume(z);
        --len;
        ++i;
        if (len) xor_row<W>(z, t.B[ctz64(i)]);
    }
    if (len >= kBlk) {
        HashOnly<W> ho{acc};
        if constexpr (W == 1) {
            uint64_t Br[U][W];
#pragma unroll
            for (int k = 0; k < U; ++k) Br[k][0] = t.B[k][0];
            do {
                GrayBlock<W, U, uint64_t[U][W], HashOnly<W>>::run(z, Br, ho);
                len -= kBlk;
                i += kBlk;
                if (len) xor_row<W>(z, t.B[ctz64(i)]);  // ctz(i) >= U here
            } while (len >= kBlk);
        } else {
            do {
                GrayBlock<W, U, uint64_t[kTableRows][W], HashOnly<W>>::run(z, t.B, ho);
                len -= kBlk;
                i += kBlk;
                if (len) xor_row<W>(z, t.B[ctz64(i)]);
            } while (len >= kBlk);
        }
    }
    while (len) {  // tail
        acc.consume(z);
        --len;
        ++i;
        if (len) xor_row<W>(z, t.B[ctz64(i)]);
    }
}

// Block-wide (count, hsum, fold) reduction over a CTA of THREADS threads;
// the result is valid in thread 0.
template <int W, int THREADS = kThreads>
__device__ __forceinline__ void block_reduce(uint64_t& cnt, Acc<W>& acc)
{
    static_assert(THREADS % 32 == 0 && THREADS <= 1024, "one partial per warp, reduced by one warp");
    __shared__ uint64_t s_part[THREADS / 32][2 + W];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        acc.hs += __shfl_xor_sync(0xffffffffu, acc.hs, o);
#pragma unroll
        for (int w = 0; w < W; ++w) acc.fold[w] ^= __shfl_xor_sync(0xffffffffu, acc.fold[w], o);
    }
    if (lane == 0) {
        s_part[warp][0] = cnt;
        s_part[warp][1] = acc.hs;
#pragma unroll
        for (int w = 0; w < W; ++w) s_part[warp][2 + w] = acc.fold[w];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        cnt = lane < nw ? s_part[lane][0] : 0;
        acc.hs = lane < nw ? s_part[lane][1] : 0;
#pragma unroll
        for (int w = 0; w < W; ++w) acc.fold[w] = lane < nw ? s_part[lane][2 + w] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            acc.hs += __shfl_xor_sync(0xffffffffu, acc.hs, o);
#pragma unroll
            for (int w = 0; w < W; ++w) acc.fold[w] ^= __shfl_xor_sync(0xffffffffu, acc.fold[w], o);
        }
    }
    __syncthreads();  // s_part may be reused by the caller
}

// Streaming (evict-first) global stores: the solutions are written once and
// not read back by this kernel.

__device__ __forceinline__ void st_cs_v2(uint64_t* p, uint64_t a, uint64_t b)
{
    asm volatile("st.global.cs.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void st_cs(uint64_t* p, uint64_t a)
{
    asm volatile("st.global.cs.u64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}

// 32 consecutive solutions of W > 1 words, one per lane (lane l holds the
// solution whose W words start at dst + l*W), written out coalesced: each lane
// stages its words in shared memory with an odd row stride (W | 1, so the
// lane-strided writes of one word index fall in distinct banks), then
// consecutive lanes store consecutive words of the 32*W-word block. `stage`
// holds 32*(W|1) words for this warp. With W even, dst must be 16-byte
// aligned and each lane stores word pairs.
template <int W>
constexpr int stage_words()
{
    return 32 * (W | 1);
}

template <int W, bool Pairs>
__device__ __forceinline__ void store_warp_coalesced(uint64_t* dst, const uint64_t (&z)[W], uint64_t* stage,
                                                     int lane)
{
    static_assert(W > 1, "W = 1 stores pairs of solutions straight from registers");
    constexpr int SW = W | 1;
#pragma unroll
    for (int w = 0; w < W; ++w) stage[lane * SW + w] = z[w];
    __syncwarp();
    if constexpr (Pairs && W % 2 == 0) {
#pragma unroll 4
        for (int k = 0; k < W / 2; ++k) {
            const int q = 2 * (lane + 32 * k);  // even, so q % W is even and q, q + 1 share a row
            const int l = q / W, w = q - l * W;
            st_cs_v2(dst + q, stage[l * SW + w], stage[l * SW + w + 1]);
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < W; ++k) {
            const int q = lane + 32 * k;
            const int l = q / W, w = q - l * W;
            st_cs(dst + q, stage[l * SW + w]);
        }
    }
    __syncwarp();  // the stage is rewritten by the next call
}

}  // namespace hlf
