// Stage 2 materialised as one dense bit stream: solution t of a window takes
// bits [t*n, (t+1)*n) of the output (stream bit b = bit b % 64 of word b / 64),
// instead of W whole words. For n = 36 that is 36 bits instead of 64 per
// solution. The solutions are those of hlf_enumerate_store.
//
// n < 64, dense1_kernel: a lane owns a run of M
// consecutive solutions whose bits fill whole words, M*n being a multiple of
// 64 (M = max(64 / gcd(n, 64), 16)). Every run therefore starts on a word
// boundary and solution t of a run sits at bit (t*n) mod 64 of its word in
// every lane alike, so the lanes append their solutions to a two-word bit
// buffer in lockstep and stage each completed word in shared memory. After
// 32 runs (one per lane, a "pass") the pass's 32*M*n/64 words leave in one
// TMA bulk store (cp.async.bulk, double-buffered staging) when the output is
// 16-byte aligned; otherwise the warp copies them out, coalesced. Inside a
// run, solution t+1 is solution t XOR B_ctz(i+1); that row index depends
// only on i mod M except at the one step of a run where i+1 is a multiple of
// M, so every other step uses a row shared by all lanes (compile-time
// registers when the window offset is a multiple of M, a shared-memory table
// otherwise). From one pass to the next a lane's run start x advances by
// 32*M = 2^b, and g(x) ^ g(x + 2^b) has exactly bits b-1 and c,
// c = b + (number of trailing ones of x >> b): two row XORs.
//
// n = 64 is the packed store itself (hlf_enumerate_store's kernel, which also
// takes the 8-byte aligned outputs this entry point allows).
//
// n > 64: 64 solutions of n bits are exactly n words (a group). For n <= 256,
// dense3_kernel steps whole group blocks by one n-word XOR each (see there);
// it also serves n <= 48 at offsets the lane runs of dense1_kernel do not
// start on (blocks of 64 * 2^s solutions there). For n > 256, dense2_kernel:
// a warp produces one group per step, two solutions per lane, each placed
// with funnel shifts at its bit offset in the group.

#include "enum_impl.cuh"

namespace hlf {
namespace {

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
            if (lane == 0 && HLF_RANGE_IN_BOUNDS(w0, pass_words, pl.words, kSiteDenseStore))
                bulk_store(out + w0, stage, (uint32_t)(pass_words * sizeof(uint64_t)));
        } else {
            __syncwarp();
            for (int q = lane; q < nw; q += 32)
                if (HLF_IN_BOUNDS(w0 + q, pl.words, kSiteDenseStore)) st_cs(out + w0 + q, stage[q]);
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

// ------------------------------------------------------------ n > 64
constexpr int kD2Threads = 256;
constexpr int kD2Warps = kD2Threads / 32;
constexpr int kD2Steps = kTableRows - 6;  // C_j = B_5 ^ B_{6+j}, j = 0..58

struct Dense2Plan {
    uint64_t offset, count;
    uint64_t groups;    // ceil(count / 64); a group is 64 solutions, n words of the stream
    uint64_t full;      // groups with all 64 solutions inside the window
    uint64_t per_warp;  // consecutive groups per warp
    uint64_t words;     // ceil(count * n / 64)
    int n, nbuf;        // nbuf: staging buffers of n words per warp
};

// Solution z (W words, n > 64 bits) placed at bit c of st[0]: the words
// st[0..L], L = (c + n - 1) / 64, each written plainly, or merged (read, OR,
// write) where the first or last word is shared with a neighbour already
// placed. Tail: an invalid solution places zeros.
template <int W, bool Tail>
__device__ __forceinline__ void dense2_put(uint64_t* st, const uint64_t (&z)[W], bool valid, uint32_t c, int L,
                                           bool merge_first, bool merge_last)
{
    uint64_t prev = 0;
#pragma unroll
    for (int w = 0; w <= W; ++w) {
        const uint64_t cur = (w < W && (!Tail || valid)) ? z[w] : 0ull;
        const uint64_t v = shl64(cur, c) | shr64(prev, 64 - c);
        prev = cur;
        if (w <= L) {
            if ((w == 0 && merge_first) || (w == L && merge_last)) st[w] |= v;
            else st[w] = v;
        }
    }
}

// A warp produces one group (64 solutions, exactly n words) per step. Lane l
// walks the solutions 2l and 2l+1 of each group, which advance by 64 in
// absolute index per step: with i = 64 H + t, z(i + 64) = z(i) ^ B_5 ^
// B_{6 + ctz(H + 1)} (the lane-interleaved identity of enumerate.cu). Solution
// t starts at bit t*n of the group, word (t*n) / 64, bit (t*n) % 64, and fills
// W or W+1 words. As n > 64, a word holds bits of at most two solutions, and
// solutions t and t+2 share none: the even solutions place their words first,
// plainly, then the odd ones merge into the first and last words they share.
// P consecutive groups share a staging buffer (the launcher, which serves
// n > 256, uses P = 1). Their P*n words leave in one bulk store when the
// output is 16-byte aligned and P*n*8 bytes is a multiple of 16, else the
// warp copies them out.
template <int W, bool Bulk, int P>
__global__ void __launch_bounds__(kD2Threads) dense2_kernel(const uint64_t* __restrict__ table, Dense2Plan pl,
                                                            uint64_t* __restrict__ out)
{
    extern __shared__ __align__(16) uint64_t s_stage2[];  // [warps][nbuf][P * n]
    __shared__ Table<W> t;
    __shared__ uint64_t s_C[kD2Steps][W];
    load_table<W>(t, table);
    __syncthreads();
    for (int i = threadIdx.x; i < kD2Steps * W; i += blockDim.x) {
        const int j = i / W, w = i % W;
        s_C[j][w] = t.B[5][w] ^ t.B[6 + j][w];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t gw = (uint64_t)blockIdx.x * kD2Warps + warp;
    const uint64_t k0 = gw * pl.per_warp;
    if (k0 >= pl.groups) return;
    const uint64_t k1 = min(k0 + pl.per_warp, pl.groups);
    const int n = pl.n;
    uint64_t* const stages = s_stage2 + (size_t)warp * pl.nbuf * P * n;

    const uint32_t tA = 2 * lane, tB = 2 * lane + 1;  // this lane's solutions in every group
    const int bA = (int)((tA * n) >> 6), bB = (int)((tB * n) >> 6);
    const uint32_t cA = (tA * n) & 63, cB = (tB * n) & 63;
    const int LA = (int)((cA + n - 1) >> 6), LB = (int)((cB + n - 1) >> 6);
    const bool mfB = cB != 0;                       // B shares its first word with A
    const bool mlB = (((tB + 1) * n) & 63) != 0;    // and its last with the next lane's A

    uint64_t zA[W], zB[W];
    const uint64_t iA = pl.offset + 64 * k0 + tA;
    uint64_t HA = iA >> 6, HB = (iA + 1) >> 6;
    seed<W>(t, iA, zA);
    seed<W>(t, iA + 1, zB);

    // P consecutive groups share a staging buffer and leave in one store
    for (uint64_t k = k0;;) {
        uint64_t* st = stages + (size_t)(((k - k0) / P) & (uint64_t)(pl.nbuf - 1)) * P * n;
        if constexpr (Bulk) {  // the bulk store that last read this buffer is done reading it
            if (lane == 0) {
                if (pl.nbuf == 2) bulk_wait_read<1>();
                else bulk_wait_read<0>();
            }
            __syncwarp();
        }
        const int pg = (int)min((uint64_t)P, k1 - k);  // groups in this step (uniform)
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (p < pg) {
                uint64_t* sg = st + p * n;
                const uint64_t kk = k + p;
                if (kk < pl.full) {
                    dense2_put<W, false>(sg + bA, zA, true, cA, LA, false, false);
                    __syncwarp();
                    dense2_put<W, false>(sg + bB, zB, true, cB, LB, mfB, mlB);
                } else {
                    const uint64_t rem = pl.count - 64 * kk;
                    dense2_put<W, true>(sg + bA, zA, tA < rem, cA, LA, false, false);
                    __syncwarp();
                    dense2_put<W, true>(sg + bB, zB, tB < rem, cB, LB, mfB, mlB);
                }
                if (kk + 1 < k1) {  // on to group kk + 1
                    HA += 1;  // H < 2^58, so ctz(H + 1) <= 58
                    xor_row<W>(zA, s_C[ctz64(HA)]);
                    HB += 1;
                    xor_row<W>(zB, s_C[ctz64(HB)]);
                }
            }
        }
        const uint64_t w0 = k * (uint64_t)n;
        const int nw = (int)min((uint64_t)pg * n, pl.words - w0);
        if (Bulk && nw == P * n) {
            fence_smem_to_async_proxy();
            __syncwarp();
            if (lane == 0 && HLF_RANGE_IN_BOUNDS(w0, P * n, pl.words, kSiteDenseStore))
                bulk_store(out + w0, st, (uint32_t)(P * n * sizeof(uint64_t)));
        } else {
            __syncwarp();
            for (int q = lane; q < nw; q += 32)
                if (HLF_IN_BOUNDS(w0 + q, pl.words, kSiteDenseStore)) st_cs(out + w0 + q, st[q]);
            __syncwarp();
        }
        k += (uint64_t)pg;
        if (k == k1) break;
    }
    if (Bulk && lane == 0) bulk_wait_all();
}
template <int W, bool Bulk, int P>
hlf_status launch_dense2_k(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                           cudaStream_t s)
{
    Dense2Plan pl{};
    pl.offset = offset;
    pl.count = count;
    pl.n = n;
    pl.full = count / 64;
    pl.groups = pl.full + (count % 64 != 0);
    pl.words = (count * (uint64_t)n + 63) / 64;  // count * n <= 2^64 - 64 (checked by the caller)
    pl.nbuf = (Bulk && P * n <= 512) ? 2 : 1;
    const size_t smem = (size_t)kD2Warps * pl.nbuf * P * n * sizeof(uint64_t);  // <= 64 KB
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(dense2_kernel<W, Bulk, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kD2Warps * 1024 * (int)sizeof(uint64_t)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense2_kernel<W, Bulk, P>, kD2Threads, smem) !=
        cudaSuccess)
        return HLF_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    const uint64_t max_warps = (uint64_t)sm_count() * per_sm * kD2Warps;
    const uint64_t warps = pl.groups < max_warps ? pl.groups : max_warps;
    pl.per_warp = (pl.groups + warps - 1) / warps;
    pl.per_warp = (pl.per_warp + P - 1) / P * P;  // whole steps of P groups
    const uint64_t used = (pl.groups + pl.per_warp - 1) / pl.per_warp;
    const unsigned blocks = (unsigned)((used + kD2Warps - 1) / kD2Warps);
    dense2_kernel<W, Bulk, P><<<blocks, kD2Threads, smem, s>>>(table, pl, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

// ------------------------------------------------------------ block walk
// dense3_kernel walks whole blocks of G = 64 * 2^s consecutive solutions
// (s = 0 for 64 < n <= 256; for n < 64, s makes a block K = n * 2^s words,
// 128 < K <= 256). With m = 6 + s, block H holds the solutions G H + t,
// t < G, and their K-word dense block is
//     G(H) = S0 ^ R(D(H)).
// With g(G H + t) = (g(H) << m) ^ ((H & 1) << (m - 1)) ^ g(t), solution
// G H + t is Zc(t) ^ D(H), where Zc(t) = z0 ^ XOR_{k in g(t)} B_k
// (B_0..B_{m-1} only) and D(H) = XOR_{k in (g(H) << m) ^ ((H & 1) << (m-1))} B_k.
// Placing G solutions side by side is linear in them, so the block splits
// into S0, the placement of Zc(0..G-1) (the same for every block), and
// R(D(H)), the placement of G copies of D(H) (the tiling R). D(H + 1) =
// D(H) ^ C_j with C_j = B_{m-1} ^ B_{m+j}, j = ctz(H + 1), so
// G(H + 1) = G(H) ^ T_j with T_j = R(C_j): one K-word XOR per block.
//
// The window [offset, offset + count) starts e = (offset mod G) n bits into
// the block of its first group Hw = offset / G, so stream word p holds bits
// [64 p + e, 64 p + e + 64) of the blocks laid end to end: with e = 64 a + b,
// word p = k K + q - a comes from block Hw + k as
//     G'(H)[q] = f(G(H)[q], G(H)[q + 1]),  f(x, y) = (x >> b) | (y << (64 - b)),
// where G(H)[K] is word 0 of the next block, G(H + 1)[0]. f is linear too, so
// the step into block H is G'(H) = G'(H - 1) ^ S_H with
//     S_H[q] = f(T_j[q], T_j[q + 1]) for q < K - 1,
//     S_H[K - 1] = f(T_j[K - 1], T_j'[0]),   j = ctz(H), j' = ctz(H + 1).
// One of H, H + 1 is odd, so (j, j') is (j, 0) for even H and (0, j') for odd
// H: the rows S for j, j' < kD3J are kept in shared memory, 2 kD3J rows of K
// words (all but 1 / 2^kD3J of the steps), and formed on the fly otherwise
// (b = 0 makes f the identity). Lane l holds the words l + 32 m of G' in
// registers and stores them straight to global memory, so a warp writes 256
// consecutive bytes per store instruction and nothing is staged; per block a
// lane spends about four instructions per word it owns (load, 64-bit XOR,
// store).
constexpr int kD3J = 8;
constexpr int kD3Threads = 256;
constexpr int kD3Warps = kD3Threads / 32;
constexpr int kD3MaxK = 256;  // block words for n < 64

struct Dense3Plan {
    uint64_t Hw;        // offset / G: the window's first block
    uint64_t groups;    // blocks the window touches
    uint64_t per_warp;  // consecutive blocks per warp
    uint64_t words;     // ceil(count * n / 64), the stream's length
    uint64_t last_mask; // valid bits of the stream's last word
    uint32_t a, b;      // e = 64 a + b bits of the first block precede the window
    int n;              // bits per solution
    int m;              // log2 of the solutions per block (6 + s)
    int K;              // words per block (n * 2^s)
};

// Bits [c, c + 64) of the W-word vector x (zero past its last word); x in
// registers, selected without dynamic indexing.
template <int W>
__device__ __forceinline__ uint64_t window64_reg(const uint64_t (&x)[W], uint32_t c)
{
    const uint32_t w = c >> 6, s = c & 63;
    uint64_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        if (i == (int)w) lo = x[i];
        if (i == (int)w + 1) hi = x[i];
    }
    return shr64(lo, s) | (s ? shl64(hi, 64 - s) : 0ull);
}

// Word q of the tiling R(x): copies of the n-bit vector x (shared memory, W
// words, zero past bit n) side by side. n > 64: copy t = 64 q / n starts the
// word at its bit c = 64 q - t n; when fewer than 64 of its bits remain, the
// next copy's first bits follow (no word touches three copies). n < 64
// (W = 1): the tiling is periodic with period n, so the word is bits
// [c, c + 64) of x repeated over 128 bits, c = 64 q mod n.
template <int W>
__device__ __forceinline__ uint64_t tile_word(const uint64_t* x, int n, uint32_t q)
{
    const uint32_t c = (64u * q) % (uint32_t)n;  // q < 256: 32-bit arithmetic
    if (W == 1 && n < 64) {
        uint64_t lo = 0, hi = 0;
        for (uint32_t at = 0; at < 128; at += (uint32_t)n) {
            if (at < 64) {
                lo |= shl64(x[0], at);
                hi |= at ? shr64(x[0], 64 - at) : 0ull;
            } else {
                hi |= shl64(x[0], at - 64);
            }
        }
        return c ? (lo >> c) | (hi << (64 - c)) : lo;
    }
    const uint32_t w = c >> 6, s = c & 63;
    uint64_t v = shr64(x[w], s);
    if (s && (int)w + 1 < W) v |= shl64(x[w + 1], 64 - s);
    if ((uint32_t)n - c < 64) v |= shl64(x[0], (uint32_t)n - c);
    return v;
}

// Word q of S0: the placement of Zc(0..G-1).
template <int W>
__device__ __forceinline__ uint64_t group_base_word(const Table<W>& t, int n, int m, uint32_t q)
{
    if (W == 1 && n < 64) {
        // every solution t whose bits [t n, t n + n) meet [64 q, 64 q + 64)
        uint64_t v = 0;
        const uint32_t t0 = (64u * q) / (uint32_t)n, t1 = (64u * q + 63) / (uint32_t)n;
        for (uint32_t tt = t0; tt <= t1; ++tt) {
            const uint32_t g = tt ^ (tt >> 1);
            uint64_t z = t.z0[0];
            for (int k = 0; k < m; ++k)
                if ((g >> k) & 1u) z ^= t.B[k][0];
            const int sh = (int)(tt * (uint32_t)n) - (int)(64u * q);
            v |= sh >= 0 ? shl64(z, (uint32_t)sh) : shr64(z, (uint32_t)(-sh));
        }
        return v;
    }
    const uint32_t t1 = (64u * q) / (uint32_t)n;
    const uint32_t c = 64 * q - t1 * (uint32_t)n;
    uint64_t a[W];
    uint64_t next0 = t.z0[0];  // word 0 of Zc(t1 + 1)
#pragma unroll
    for (int w = 0; w < W; ++w) a[w] = t.z0[w];
    const uint32_t g1 = t1 ^ (t1 >> 1), g2 = (t1 + 1) ^ ((t1 + 1) >> 1);
    for (int k = 0; k < m; ++k) {  // a block of 2^m solutions: Gray bits below m
        if ((g1 >> k) & 1u) xor_row<W>(a, t.B[k]);
        if ((g2 >> k) & 1u) next0 ^= t.B[k][0];
    }
    uint64_t v = window64_reg<W>(a, c);
    if ((uint32_t)n - c < 64) v |= shl64(next0, (uint32_t)n - c);  // t1 + 1 < 2^m here
    return v;
}

__device__ __forceinline__ uint64_t funnel(uint64_t x, uint64_t y, uint32_t b)
{
    return b ? (x >> b) | (y << (64 - b)) : x;
}

// Word q of the step row S for (j, j'), formed from C_j and C_j' (the rows
// of rare steps; out of line so that the walk's loops stay unrolled).
template <int W>
__device__ __noinline__ uint64_t step_word(const uint64_t* Cj, const uint64_t* Cjn, int n, int K, uint32_t q,
                                           uint32_t b)
{
    const uint64_t x = tile_word<W>(Cj, n, q);
    return funnel(x, q + 1 < (uint32_t)K ? tile_word<W>(Cj, n, q + 1) : tile_word<W>(Cjn, n, 0), b);
}

// MW: block words per lane (2W for 64 < n <= 256, 8 for n < 64).
template <int W, int MW>
__global__ void __launch_bounds__(kD3Threads, W == 3 ? 4 : (W == 4 ? 3 : (MW > 4 ? 4 : 5))) dense3_kernel(
    const uint64_t* __restrict__ table, Dense3Plan pl, uint64_t* __restrict__ out)
{
    // S rows [2 kD3J][K] (row j: (j, 0), row kD3J + j': (0, j')), S0 [K],
    // D [warps][W]
    extern __shared__ __align__(16) uint64_t s_d3[];
    __shared__ Table<W> t;
    __shared__ uint64_t s_C[kD2Steps][W];  // C_j = B_{m-1} ^ B_{m+j} (zero past row 64)
    const int n = pl.n, K = pl.K, mb = pl.m;
    const uint32_t b = pl.b;
    uint64_t* const s_S = s_d3;
    uint64_t* const s_S0 = s_S + 2 * kD3J * K;
    uint64_t* const s_D = s_S0 + K;
    load_table<W>(t, table);
    __syncthreads();
    for (int i = threadIdx.x; i < kD2Steps * W; i += blockDim.x) {
        const int j = i / W, w = i % W;
        s_C[j][w] = mb + j < kTableRows ? t.B[mb - 1][w] ^ t.B[mb + j][w] : 0ull;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kD3J * K; i += blockDim.x) {
        const int row = i / K, q = i % K;
        const int j = row < kD3J ? row : 0, jn = row < kD3J ? 0 : row - kD3J;
        const uint64_t x = tile_word<W>(s_C[j], n, (uint32_t)q);
        const uint64_t y = q + 1 < K ? tile_word<W>(s_C[j], n, (uint32_t)q + 1) : tile_word<W>(s_C[jn], n, 0);
        s_S[i] = funnel(x, y, b);
    }
    for (int q = threadIdx.x; q < K; q += blockDim.x) s_S0[q] = group_base_word<W>(t, n, mb, (uint32_t)q);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t k0 = ((uint64_t)blockIdx.x * kD3Warps + warp) * pl.per_warp;
    if (k0 >= pl.groups) return;
    const uint64_t k1 = min(k0 + pl.per_warp, pl.groups);
    const uint64_t H0 = pl.Hw + k0;  // < 2^(64 - m)
    {  // D(H0): every lane forms it; lane w < W publishes word w
        uint64_t g = ((H0 ^ (H0 >> 1)) << mb) | ((H0 & 1ull) << (mb - 1));
        uint64_t D[W];
#pragma unroll
        for (int w = 0; w < W; ++w) D[w] = 0;
        while (g) {
            xor_row<W>(D, t.B[__ffsll((long long)g) - 1]);
            g &= g - 1;
        }
#pragma unroll
        for (int w = 0; w < W; ++w)
            if (lane == w) s_D[warp * W + w] = D[w];
        __syncwarp();
    }
    // G'(H0): f of consecutive words of G(H0), the last with G(H0 + 1)[0]
    uint64_t G[MW];
    {
        const uint64_t* D = s_D + warp * W;
        const int j = ctz64(H0 + 1);
        const uint64_t next0 = s_S0[0] ^ tile_word<W>(D, n, 0) ^ tile_word<W>(s_C[j], n, 0);
#pragma unroll
        for (int m = 0; m < MW; ++m) {
            const int q = lane + 32 * m;
            uint64_t v = 0;
            if (q < K) {
                v = s_S0[q] ^ tile_word<W>(D, n, (uint32_t)q);
                if (b) v = funnel(v, q + 1 < K ? s_S0[q + 1] ^ tile_word<W>(D, n, (uint32_t)q + 1) : next0, b);
            }
            G[m] = v;
        }
    }
    // blocks whose every word lies inside the stream and before its last
    // word: [ka, kb) (stream word p = k K + q - a of block Hw + k)
    const uint64_t ka = (pl.a + K - 1) / K;
    const uint64_t kb = (pl.words + pl.a - 1) / K;  // k K - a + K <= words - 1
    uint64_t kn = k0 * (uint64_t)K;
    for (uint64_t k = k0;; kn += K) {
        if (k >= ka && k < kb) {
            uint64_t* dst = out + (kn - pl.a);
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int q = lane + 32 * m;
                if (q < K && HLF_IN_BOUNDS(kn - pl.a + q, pl.words, kSiteDenseStore)) st_cs(dst + q, G[m]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int q = lane + 32 * m;
                const uint64_t p = kn + q - pl.a;  // wraps to a huge value when negative
                if (q < K && kn + q >= pl.a && p < pl.words && HLF_IN_BOUNDS(p, pl.words, kSiteDenseStore))
                    st_cs(out + p, p == pl.words - 1 ? (G[m] & pl.last_mask) : G[m]);
            }
        }
        if (++k == k1) break;
        const uint64_t H = pl.Hw + k;  // the block stepped to
        // one of j = ctz(H), j' = ctz(H + 1) is 0: c is the other
        const int c = __ffsll((long long)((H & 1) ? H + 1 : H)) - 1;
        const int row = (H & 1) ? kD3J + c : c;
        if (c < kD3J) {
            const uint64_t* S = s_S + row * K;
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int q = lane + 32 * m;
                if (q < K) G[m] ^= S[q];
            }
        } else {
#pragma unroll
            for (int m = 0; m < MW; ++m) {
                const int q = lane + 32 * m;
                if (q < K) G[m] ^= step_word<W>(s_C[(H & 1) ? 0 : c], s_C[(H & 1) ? c : 0], n, K, (uint32_t)q, b);
            }
        }
    }
}

template <int W, int MW>
hlf_status launch_dense3(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                         cudaStream_t s)
{
    Dense3Plan pl{};
    pl.n = n;
    int sh = 0;  // s: for n < 64 the smallest with n 2^(s+1) > kD3MaxK, so 128 < K <= 256
    if (n < 64)
        while ((n << (sh + 1)) <= kD3MaxK) ++sh;
    else if (2 * n <= MW * 32)  // 64 < n < 128 with 8 words a lane: blocks of two groups
        sh = 1;
    pl.m = 6 + sh;
    pl.K = n << sh;
    pl.Hw = offset >> pl.m;
    pl.groups = ((offset + (count - 1)) >> pl.m) - pl.Hw + 1;  // count >= 1; offset + count - 1 < 2^64
    const uint64_t bits = count * (uint64_t)n;                // <= 2^64 - 64 (checked by the caller)
    pl.words = (bits + 63) / 64;
    pl.last_mask = (bits & 63) ? (1ull << (bits & 63)) - 1 : ~0ull;
    const uint64_t e = (offset & ((1ull << pl.m) - 1)) * (uint64_t)n;
    pl.a = (uint32_t)(e >> 6);
    pl.b = (uint32_t)(e & 63);
    const size_t smem = ((size_t)(2 * kD3J + 1) * pl.K + (size_t)kD3Warps * W) * sizeof(uint64_t);  // <= 34.9 KB
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense3_kernel<W, MW>, kD3Threads, smem) != cudaSuccess)
        return HLF_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    const uint64_t max_warps = (uint64_t)sm_count() * per_sm * kD3Warps;
    const uint64_t warps = pl.groups < max_warps ? pl.groups : max_warps;
    pl.per_warp = (pl.groups + warps - 1) / warps;
    const uint64_t used = (pl.groups + pl.per_warp - 1) / pl.per_warp;
    const unsigned blocks = (unsigned)((used + kD3Warps - 1) / kD3Warps);
    dense3_kernel<W, MW><<<blocks, kD3Threads, smem, s>>>(table, pl, out);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

// n <= 256 takes the group-block walk (dense3_kernel); wider rows place
// their solutions one by one (dense2_kernel).
template <int W>
hlf_status launch_dense2(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                         cudaStream_t s)
{
    if constexpr (W == 2) {
        // n < 128: blocks of two groups (2n words), so a warp's stores leave
        // fewer lanes idle (n = 65: a group is 65 words, three store
        // instructions with one lane in the last; two groups fill 130 of 160
        // lanes): 5.9-6.1 TB/s against 5.5 at n = 65, even elsewhere. n = 128
        // fills every lane with one group and keeps it (6.40 TB/s against 6.33).
        if (n < 128) return launch_dense3<2, 8>(table, n, offset, count, out, s);
        return launch_dense3<2, 4>(table, n, offset, count, out, s);
    } else if constexpr (W <= 4) {
        return launch_dense3<W, 2 * W>(table, n, offset, count, out, s);
    } else {
        if (reinterpret_cast<uintptr_t>(out) % 16 == 0 && n % 2 == 0)
            return launch_dense2_k<W, true, 1>(table, n, offset, count, out, s);
        return launch_dense2_k<W, false, 1>(table, n, offset, count, out, s);
    }
}

}  // namespace

hlf_status launch_store_dense(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                              cudaStream_t s)
{
    if (n == 64) return launch_store(table, 1, offset, count, out, s);  // one whole word per solution
    if (n < 64) {
        const int m = 64 / (n & -n);  // 64 / gcd(n, 64)
        const int M = m < 16 ? 16 : m;
        const bool aligned = (offset & (uint64_t)(M - 1)) == 0;
        // Offsets that are not a multiple of M: the lane runs then need a
        // per-lane step table, and 4 GB windows measured 4.4-5.8 TB/s at
        // n = 33..48 against 6.2 TB/s for the block walk at any offset;
        // from n = 56 the runs stay ahead (6.6 against 6.2 TB/s), as they do
        // at aligned offsets (6.2-6.5 TB/s).
        if (!aligned && n <= 48) return launch_dense3<1, 8>(table, n, offset, count, out, s);
        switch (M) {
        case 16: return aligned ? launch_dense1<16, true>(table, n, offset, count, out, s)
                                : launch_dense1<16, false>(table, n, offset, count, out, s);
        case 32: return aligned ? launch_dense1<32, true>(table, n, offset, count, out, s)
                                : launch_dense1<32, false>(table, n, offset, count, out, s);
        default: return aligned ? launch_dense1<64, true>(table, n, offset, count, out, s)
                                : launch_dense1<64, false>(table, n, offset, count, out, s);
        }
    }
    switch ((n + 63) / 64) {
    case 2: return launch_dense2<2>(table, n, offset, count, out, s);
    case 3: return launch_dense2<3>(table, n, offset, count, out, s);
    case 4: return launch_dense2<4>(table, n, offset, count, out, s);
    case 5: return launch_dense2<5>(table, n, offset, count, out, s);
    case 6: return launch_dense2<6>(table, n, offset, count, out, s);
    case 7: return launch_dense2<7>(table, n, offset, count, out, s);
    case 8: return launch_dense2<8>(table, n, offset, count, out, s);
    case 9: return launch_dense2<9>(table, n, offset, count, out, s);
    case 10: return launch_dense2<10>(table, n, offset, count, out, s);
    case 11: return launch_dense2<11>(table, n, offset, count, out, s);
    case 12: return launch_dense2<12>(table, n, offset, count, out, s);
    case 13: return launch_dense2<13>(table, n, offset, count, out, s);
    case 14: return launch_dense2<14>(table, n, offset, count, out, s);
    case 15: return launch_dense2<15>(table, n, offset, count, out, s);
    case 16: return launch_dense2<16>(table, n, offset, count, out, s);
    default: return HLF_ERR_SIZE;
    }
}

HLF_DEBUG_TAKE(dense)

}  // namespace hlf
