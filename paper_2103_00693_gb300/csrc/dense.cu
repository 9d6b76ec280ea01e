// Stage 2 materialised as one dense bit stream: solution t of a window takes
// bits [t*n, (t+1)*n) of the output (stream bit b = bit b % 64 of word b / 64),
// instead of W whole words. For n = 36 that is 36 bits instead of 64 per
// solution. The solutions are those of hlf_enumerate_store.
//
// n < 64 (one word per row), dense1_kernel: a lane owns a run of M
// consecutive solutions whose bits fill whole words, M*n being a multiple of
// 64 (M = max(64 / gcd(n, 64), 16)). Every run therefore starts on a word
// boundary and solution t of a run sits at bit (t*n) mod 64 of its word in
// every lane alike, so the lanes append their solutions to a two-word bit
// buffer in lockstep and stage each completed word in shared memory; after 32
// runs (one per lane, a "pass") the pass's 32*M*n/64 words leave in one TMA
// bulk store (cp.async.bulk, double-buffered staging) when the output is
// 16-byte aligned, else the warp copies them out, coalesced. Inside a run, solution t+1 is solution t XOR B_ctz(i+1);
// that row index depends only on i mod M except at the one step of a run
// where i+1 is a multiple of M, so every other step uses a row shared by all
// lanes (compile-time registers when the window offset is a multiple of M, a
// shared-memory table otherwise). From one pass to the next a lane's run
// start x advances by 32*M = 2^b, and g(x) ^ g(x + 2^b) has exactly bits b-1
// and c, c = b + (number of trailing ones of x >> b): two row XORs.
//
// n = 64 with a 16-byte aligned output is the packed store itself; otherwise
// (n >= 64), dense_kernel: a warp produces 64
// consecutive solutions per step; 64 solutions of n bits are exactly n words,
// so every group's words start on a word boundary for any n. Each lane walks
// two Gray chains (relative positions 2*lane and 2*lane+1 of the group) that
// advance by 64 in absolute index per step: with i = 64 H + l,
// z(i + 64) = z(i) ^ B_5 ^ B_{6 + ctz(H + 1)} (the lane-interleaved identity
// of enumerate.cu), so a step is one row XOR per solution whatever the
// window's offset. The group's 64 solutions are staged in shared memory;
// output word j of a group holds stream bits [64 j, 64 j + 64), which start
// at bit o of solution s, with (s, o) taken from a per-CTA table built once
// (no division in the loop). Each lane assembles whole output words with
// shifts, and the warp writes the group's n words out, coalesced.

#include "enum_impl.cuh"

namespace hlf {
namespace {

constexpr int kDenseGroup = 64;
constexpr int kDenseSteps = kTableRows - 6;  // C_j = B_5 ^ B_{6+j}, j = 0..58

struct DensePlan {
    uint64_t offset, count;
    uint64_t groups;    // ceil(count / 64)
    uint64_t per_warp;  // groups per warp
    int n;
};

// `len` (1..64) bits of a W-word solution starting at bit `pos`.
template <int W>
__device__ __forceinline__ uint64_t extract_bits(const uint64_t* sol, int pos, int len)
{
    const int w = pos >> 6;
    const int sh = pos & 63;
    uint64_t v = sol[w] >> sh;
    if (sh && sh + len > 64) v |= sol[w + 1] << (64 - sh);
    return len == 64 ? v : v & ((1ull << len) - 1);
}

template <int W>
__global__ void __launch_bounds__(kThreads) dense_kernel(const uint64_t* __restrict__ table, DensePlan pl,
                                                         uint64_t* __restrict__ out)
{
    extern __shared__ __align__(16) uint64_t s_dyn[];
    // [n] start words (s << 16 | o: output word j starts at bit o of solution s), then [warps][64][W] solutions
    uint32_t* s_start = reinterpret_cast<uint32_t*>(s_dyn);
    __shared__ Table<W> t;
    __shared__ uint64_t s_C[kDenseSteps][W];
    const int n = pl.n;
    uint64_t* s_sol = s_dyn + (n + 1) / 2;
    load_table<W>(t, table);
    __syncthreads();
    for (int i = threadIdx.x; i < kDenseSteps * W; i += blockDim.x) {
        const int j = i / W, w = i % W;
        s_C[j][w] = t.B[5][w] ^ t.B[6 + j][w];
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int s = (64 * j) / n;
        s_start[j] = ((uint32_t)s << 16) | (uint32_t)(64 * j - s * n);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint64_t* sol = s_sol + (size_t)warp * kDenseGroup * W;
    const uint64_t wg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t k0 = wg * pl.per_warp;
    if (k0 >= pl.groups) return;
    const uint64_t k1 = min(k0 + pl.per_warp, pl.groups);

    uint64_t z[2][W];
    uint64_t H[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const uint64_t i = pl.offset + (uint64_t)kDenseGroup * k0 + (uint64_t)(2 * lane + e);
        H[e] = i >> 6;
        seed<W>(t, i, z[e]);
    }
    for (uint64_t k = k0;;) {
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int w = 0; w < W; ++w) sol[(2 * lane + e) * W + w] = z[e][w];
        __syncwarp();
        const uint64_t rem = pl.count - (uint64_t)kDenseGroup * k;
        const int valid = rem < kDenseGroup ? (int)rem : kDenseGroup;
        uint64_t* dst = out + k * (uint64_t)n;
        const int nwords = (valid * n + 63) >> 6;
        for (int j = lane; j < nwords; j += 32) {
            const uint32_t st = s_start[j];
            int s = (int)(st >> 16);
            const int o = (int)(st & 0xffff);
            uint64_t v;
            int got;
            if constexpr (W == 1) {
                v = sol[s] >> o;
                got = n - o;
                for (++s; got < 64 && s < valid; ++s, got += n) v |= sol[s] << got;
            } else {
                got = min(64, n - o);
                v = extract_bits<W>(sol + s * W, o, got);
                for (++s; got < 64 && s < valid; ++s) {
                    const int take = min(n, 64 - got);
                    v |= extract_bits<W>(sol + s * W, 0, take) << got;
                    got += take;
                }
            }
            dst[j] = v;
        }
        __syncwarp();
        if (++k == k1) break;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            H[e] += 1;
            xor_row<W>(z[e], s_C[ctz64(H[e])]);
        }
    }
}

// ------------------------------------------------------------ n < 64
constexpr int kD1Threads = 256;
constexpr int kD1Warps = kD1Threads / 32;

struct Dense1Plan {
    uint64_t offset, count;
    uint64_t passes;    // ceil(count / (32 M)); a pass is 32 runs of M solutions
    uint64_t full;      // passes whose 32 runs are all inside the window
    uint64_t per_warp;  // consecutive passes per warp
    uint64_t words;     // ceil(count * n / 64), the stream's length in words
    int n, wpr;         // wpr = M * n / 64 words per run
    int nbuf;           // staging buffers per warp (2: a pass overlaps the bulk store of the last)
};

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Shifts with PTX semantics: amounts of 64 give 0 (no special case for an
// empty bit buffer).
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
// Predicated shared-memory store (no branch around it).
__device__ __forceinline__ void st_shared_if(bool p, uint64_t* a, uint64_t v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.u64 [%1], %2;\n\t}" ::"r"((uint32_t)p),
                 "r"((uint32_t)__cvta_generic_to_shared(a)), "l"(v)
                 : "memory");
}

// Step t of a lane's run (t = T, a compile-time constant, so that the
// aligned walk's row index ctz(T + 1) selects a register): append solution
// z to the bit buffer (lo, fill), stage a completed word at mine[w], then
// step z to solution T + 1. Everything that depends on the bit position is
// the same in every lane, and the word is staged by a predicated store.
template <int M, int T, bool Aligned, bool Tail>
struct Dense1Step {
    static __device__ __forceinline__ void go(uint64_t& z, uint64_t& lo, uint32_t& fill, uint32_t& w, uint64_t valid,
                                              uint32_t n, const uint64_t* s_step, const uint64_t (&Breg)[ilog2(M)],
                                              int tstar, uint64_t sp, uint64_t* mine)
    {
        const uint64_t v = (Tail && (uint64_t)T >= valid) ? 0ull : z;
        lo |= shl64(v, fill);
        const bool full = fill + n >= 64;
        st_shared_if(full, mine + w, lo);
        const uint64_t carry = shr64(v, 64 - fill);  // bits of v past the word; 0 when fill == 0
        lo = full ? carry : lo;
        w += full;
        fill = full ? fill + n - 64 : fill + n;
        if constexpr (T + 1 < M) {
            if constexpr (Aligned) {
                constexpr int k = ilog2((T + 1) & -(T + 1));  // ctz(T + 1)
                z ^= Breg[k];
            } else {
                z ^= s_step[T];
                if (T == tstar) z ^= sp;
            }
            Dense1Step<M, T + 1, Aligned, Tail>::go(z, lo, fill, w, valid, n, s_step, Breg, tstar, sp, mine);
        }
    }
};

// One lane's run of M solutions starting at absolute index i0 (solution z):
// the wpr completed words go to `mine`. Tail: solutions t >= valid are
// outside the window and contribute zero bits.
template <int M, bool Aligned, bool Tail>
__device__ __forceinline__ void dense1_run(uint64_t z, uint64_t i0, uint64_t valid, int n,
                                           const uint64_t* s_B, const uint64_t* s_step,
                                           const uint64_t (&Breg)[ilog2(M)], int tstar, uint64_t* mine)
{
    uint64_t sp = 0;  // the lane's own row at the step where i0 + t + 1 is a multiple of M
    if constexpr (!Aligned) sp = s_B[ctz64(i0 + (uint64_t)tstar + 1)];
    uint64_t lo = 0;
    uint32_t fill = 0, w = 0;
    Dense1Step<M, 0, Aligned, Tail>::go(z, lo, fill, w, valid, (uint32_t)n, s_step, Breg, tstar, sp, mine);
}

// Bulk (TMA) stores from shared to global memory: a whole pass's words leave
// in one cp.async.bulk issued by lane 0, tracked in bulk groups of that lane.
// Source and destination are 16-byte aligned and the size is a multiple of
// 16 bytes (checked by the launcher).
__device__ __forceinline__ void fence_smem_to_async_proxy()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_store(uint64_t* gdst, const uint64_t* ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait_read()  // at most N groups still reading shared memory
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Bulk: the output is 16-byte aligned, so full passes leave as bulk stores;
// otherwise (and for the last, partial pass) the warp copies its words out.
template <int M, bool Aligned, bool Bulk>
__global__ void __launch_bounds__(kD1Threads, M == 64 ? 3 : 4) dense1_kernel(const uint64_t* __restrict__ table, Dense1Plan pl,
                                                            uint64_t* __restrict__ out)
{
    constexpr int A = ilog2(M);
    constexpr int b = A + 5;  // a pass advances every run start by 32 M = 2^b
    extern __shared__ __align__(16) uint64_t s_stage[];  // [warps][nbuf][32 * wpr]
    __shared__ uint64_t s_B[kTableRows];
    __shared__ uint64_t s_step[M];
    __shared__ uint64_t s_z0;
    for (int k = threadIdx.x; k < kTableRows; k += blockDim.x) s_B[k] = table[k];
    if (threadIdx.x == 0) s_z0 = table[kTableZ0Row];
    const uint32_t off_low = (uint32_t)pl.offset & (M - 1);
    __syncthreads();
    if constexpr (!Aligned) {
        for (int t = threadIdx.x; t < M; t += blockDim.x) {
            const uint32_t u = (off_low + (uint32_t)t + 1) & (M - 1);
            s_step[t] = u ? s_B[__ffs(u) - 1] : 0ull;
        }
        __syncthreads();
    }
    const int tstar = Aligned ? M : (int)(M - 1 - off_low);
    uint64_t Breg[A];
#pragma unroll
    for (int k = 0; k < A; ++k) Breg[k] = s_B[k];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t gw = (uint64_t)blockIdx.x * kD1Warps + warp;
    const uint64_t P0 = gw * pl.per_warp;
    if (P0 >= pl.passes) return;
    const uint64_t P1 = min(P0 + pl.per_warp, pl.passes);
    const int n = pl.n;
    const uint64_t pass_words = 32ull * (uint64_t)pl.wpr;
    uint64_t* const stages = s_stage + (size_t)warp * pl.nbuf * pass_words;

    uint64_t j0 = (P0 * 32 + (uint64_t)lane) * M;  // run start, relative to the window
    uint64_t i0 = pl.offset + j0;                  // and absolute
    uint64_t zs = s_z0;
    for (uint64_t g = i0 ^ (i0 >> 1); g; g &= g - 1) zs ^= s_B[__ffsll((long long)g) - 1];

    for (uint64_t P = P0;;) {
        uint64_t* stage = stages + (size_t)((P - P0) & (uint64_t)(pl.nbuf - 1)) * pass_words;
        uint64_t* mine = stage + (size_t)lane * pl.wpr;
        if constexpr (Bulk) {  // the bulk store that last read this buffer is done reading it
            if (lane == 0) {
                if (pl.nbuf == 2) bulk_wait_read<1>();
                else bulk_wait_read<0>();
            }
            __syncwarp();
        }
        if (P < pl.full) {
            dense1_run<M, Aligned, false>(zs, i0, M, n, s_B, s_step, Breg, tstar, mine);
        } else {
            const uint64_t valid = j0 < pl.count ? min(pl.count - j0, (uint64_t)M) : 0;
            dense1_run<M, Aligned, true>(zs, i0, valid, n, s_B, s_step, Breg, tstar, mine);
        }
        const uint64_t w0 = P * pass_words;
        const int nw = (int)min(pass_words, pl.words - w0);
        if (Bulk && nw == (int)pass_words) {
            fence_smem_to_async_proxy();  // this lane's staged words, before the async proxy reads them
            __syncwarp();
            if (lane == 0) bulk_store(out + w0, stage, (uint32_t)(pass_words * sizeof(uint64_t)));
        } else {
            __syncwarp();
            for (int q = lane; q < nw; q += 32) st_cs(out + w0 + q, stage[q]);
            __syncwarp();
        }
        if (++P == P1) break;
        const int c = b + ctz64(~(i0 >> b));  // <= 64: the top b bits of i0 >> b are 0
        zs ^= s_B[b - 1] ^ s_B[c];
        i0 += 32ull * M;
        j0 += 32ull * M;
    }
    if (Bulk && lane == 0) bulk_wait_all();  // shared memory stays valid until the stores are done
}

template <int M, bool Aligned, bool Bulk>
hlf_status launch_dense1_k(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                           cudaStream_t s)
{
    constexpr uint64_t per_pass = 32ull * M;
    Dense1Plan pl{};
    pl.offset = offset;
    pl.count = count;
    pl.n = n;
    pl.wpr = M * n / 64;
    pl.full = count / per_pass;
    pl.passes = pl.full + (count % per_pass != 0);
    pl.words = (count * (uint64_t)n + 63) / 64;  // count * n <= 2^64 - 64 (checked by the caller)
    // two buffers per warp while a CTA's staging stays within 64 KB (wpr <= 16)
    pl.nbuf = (Bulk && pl.wpr <= 16) ? 2 : 1;
    const size_t smem = (size_t)kD1Warps * pl.nbuf * 32 * pl.wpr * sizeof(uint64_t);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        const int most = kD1Warps * 32 * 64 * (int)sizeof(uint64_t);  // 128 KB: wpr <= 63 with one buffer
        if (cudaFuncSetAttribute(dense1_kernel<M, Aligned, Bulk>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 most) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense1_kernel<M, Aligned, Bulk>, kD1Threads, smem) !=
        cudaSuccess)
        return HLF_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    const uint64_t max_warps = (uint64_t)sm_count() * per_sm * kD1Warps;
    const uint64_t warps = pl.passes < max_warps ? pl.passes : max_warps;
    pl.per_warp = (pl.passes + warps - 1) / warps;
    const uint64_t used = (pl.passes + pl.per_warp - 1) / pl.per_warp;
    const unsigned blocks = (unsigned)((used + kD1Warps - 1) / kD1Warps);
    dense1_kernel<M, Aligned, Bulk><<<blocks, kD1Threads, smem, s>>>(table, pl, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

template <int M, bool Aligned>
hlf_status launch_dense1(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                         cudaStream_t s)
{
    // a pass is 256 * wpr bytes, so pass starts are 16-byte aligned when out is
    if (reinterpret_cast<uintptr_t>(out) % 16 == 0) return launch_dense1_k<M, Aligned, true>(table, n, offset, count, out, s);
    return launch_dense1_k<M, Aligned, false>(table, n, offset, count, out, s);
}

// ------------------------------------------------------------ n >= 64
template <int W>
hlf_status launch_dense_w(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                          cudaStream_t s)
{
    DensePlan pl{};
    pl.offset = offset;
    pl.count = count;
    pl.n = n;
    pl.groups = (count + kDenseGroup - 1) / kDenseGroup;
    // start table (n x 4 bytes, rounded to words) + 64 solutions of W words per warp
    const size_t smem = ((size_t)(n + 1) / 2 + (size_t)(kThreads / 32) * kDenseGroup * W) * sizeof(uint64_t);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(dense_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((32 * W + (kThreads / 32) * kDenseGroup * W) * sizeof(uint64_t))) !=
            cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    // one wave: as many CTAs as fit on every SM at once (equal work per warp,
    // so a partial second wave would double the time)
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_kernel<W>, kThreads, smem) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    const uint64_t max_warps = (uint64_t)sm_count() * per_sm * (kThreads / 32);
    uint64_t warps = (pl.groups + 15) / 16;
    if (warps > max_warps) warps = max_warps;
    if (warps == 0) warps = 1;
    pl.per_warp = (pl.groups + warps - 1) / warps;
    const unsigned blocks = (unsigned)((warps * 32 + kThreads - 1) / kThreads);
    dense_kernel<W><<<blocks, kThreads, smem, s>>>(table, pl, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_store_dense(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                              cudaStream_t s)
{
    if (n < 64) {
        const int m = 64 / (n & -n);  // 64 / gcd(n, 64)
        const int M = m < 16 ? 16 : m;
        const bool aligned = (offset & (uint64_t)(M - 1)) == 0;
        switch (M) {
        case 16: return aligned ? launch_dense1<16, true>(table, n, offset, count, out, s)
                                : launch_dense1<16, false>(table, n, offset, count, out, s);
        case 32: return aligned ? launch_dense1<32, true>(table, n, offset, count, out, s)
                                : launch_dense1<32, false>(table, n, offset, count, out, s);
        default: return aligned ? launch_dense1<64, true>(table, n, offset, count, out, s)
                                : launch_dense1<64, false>(table, n, offset, count, out, s);
        }
    }
    if (n == 64 && reinterpret_cast<uintptr_t>(out) % 16 == 0)  // one whole word per solution
        return launch_store(table, 1, offset, count, out, s);
    switch ((n + 63) / 64) {
    case 1: return launch_dense_w<1>(table, n, offset, count, out, s);
    case 2: return launch_dense_w<2>(table, n, offset, count, out, s);
    case 3: return launch_dense_w<3>(table, n, offset, count, out, s);
    case 4: return launch_dense_w<4>(table, n, offset, count, out, s);
    case 5: return launch_dense_w<5>(table, n, offset, count, out, s);
    case 6: return launch_dense_w<6>(table, n, offset, count, out, s);
    case 7: return launch_dense_w<7>(table, n, offset, count, out, s);
    case 8: return launch_dense_w<8>(table, n, offset, count, out, s);
    case 9: return launch_dense_w<9>(table, n, offset, count, out, s);
    case 10: return launch_dense_w<10>(table, n, offset, count, out, s);
    case 11: return launch_dense_w<11>(table, n, offset, count, out, s);
    case 12: return launch_dense_w<12>(table, n, offset, count, out, s);
    case 13: return launch_dense_w<13>(table, n, offset, count, out, s);
    case 14: return launch_dense_w<14>(table, n, offset, count, out, s);
    case 15: return launch_dense_w<15>(table, n, offset, count, out, s);
    case 16: return launch_dense_w<16>(table, n, offset, count, out, s);
    default: return HLF_ERR_SIZE;
    }
}

}  // namespace hlf
