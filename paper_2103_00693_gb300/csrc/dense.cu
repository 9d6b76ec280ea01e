// Stage 2 materialised as one dense bit stream: solution t of a window takes
// bits [t*n, (t+1)*n) of the output (stream bit b = bit b % 64 of word b / 64),
// instead of W whole words. For n = 36 that is 36 bits instead of 64 per
// solution. The solutions are those of hlf_enumerate_store.
//
// A warp produces 64 consecutive solutions per step; 64 solutions of n bits
// are exactly n words, so every group's words start on a word boundary for
// any n. Each lane walks two Gray chains (relative positions 2*lane and
// 2*lane+1 of the group) that advance by 64 in absolute index per step:
// with i = 64 H + l, z(i + 64) = z(i) ^ B_5 ^ B_{6 + ctz(H + 1)} (the
// lane-interleaved identity of enumerate.cu), so a step is one row XOR per
// solution whatever the window's offset. The group's 64 solutions are
// staged in shared memory; output word j of a group holds stream bits
// [64 j, 64 j + 64), which start at bit o of solution s, with (s, o) taken
// from a per-CTA table built once (no division in the loop). Each lane
// assembles whole output words with shifts (at n <= 64: one word of solution
// s, then the next solutions shifted in), and the warp writes the group's n
// words out, coalesced.

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
