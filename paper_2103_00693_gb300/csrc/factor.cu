// Stage 1 for one matrix (the CLA module of Section 2, steps (1)-(4)).
//
// n <= 512 (W <= 8): one CTA runs factor_block (factor_impl.cuh): input
// checks, elimination, kernel vectors, q and z^a in one launch, which is what
// the latency of small and medium instances wants.
//
// n > 512 (W >= 9): the same results from two launches that spread the work
// that does not have to be sequential over many SMs:
//   factor_elim_kernel   CTA 0 runs the Gauss-Jordan elimination (step (1))
//                        with the rows of A in registers, by factor_block's
//                        loop; CTAs 1.. check the input (padding bits,
//                        symmetry by 64 x 64 bit-block transposes) at the
//                        same time, each writing its own status slot.
//   factor_kvec_kernel   one warp per free column f across the GPU: the
//                        kernel vector x_f, q(x_f) mod 4 and the bit z^a_f
//                        (steps (2)-(4)), the paper-order table, and, in
//                        the last CTA to finish, the status and rank.
// At n = 1024 (grid 32 x 32) this takes 355 us against 392 us in one CTA; at
// n = 484 the second launch costs more than it saves (143 us against 124 us),
// hence the threshold.
//
// The elimination itself stays one barrier per pivot column. Measured at
// n = 1024 and dropped:
//   - a split barrier (an mbarrier whose arrive precedes the XOR of the
//     previous pivot row's later words, and whose wait follows it): 607 us;
//   - panels of 8 columns (a Four-Russians scheme: the pivot search on 8-bit
//     slices with a mask of the panel's pivots, then one XOR of a table of
//     pivot-row combinations per row and panel): 367 us with all warps
//     searching, 431 us with one warp searching bit-planes; the barrier and
//     the per-column chain dominate, not the XOR volume.

#include "factor_impl.cuh"

namespace hlf {
namespace {

template <int W>
constexpr int rows_per_thread() { return W <= 8 ? 1 : 2; }

template <int W>
__global__ void __launch_bounds__(512, 1) factor_kernel(const uint64_t* __restrict__ A, int n, FactorOut o)
{
    extern __shared__ __align__(16) unsigned char smem[];
    factor_block<W, rows_per_thread<W>(), HLF_MAX_N>(A, n, o, smem);
}

template <int W>
hlf_status launch_factor_w(const uint64_t* A, int n, const FactorOut& o, cudaStream_t s)
{
    constexpr int R = rows_per_thread<W>();
    const int threads = ((n + R - 1) / R + 31) / 32 * 32;
    const size_t smem = factor_smem_bytes<W, HLF_MAX_N>(n);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(factor_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)factor_smem_bytes<W, HLF_MAX_N>(HLF_MAX_N)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    factor_kernel<W><<<1, threads, smem, s>>>(A, n, o);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

// ------------------------------------------------------------ n > 256

constexpr int kChkCtas = 8;       // CTAs that check the input beside the elimination
constexpr int kWorkR = 16;        // work[16] = r
constexpr int kWorkInternal = 17; // work[17] = HLF_ERR_INTERNAL if some q(x_f) was odd
constexpr int kWorkDone = 18;     // work[18] = CTAs of factor_kvec_kernel done
static_assert(kChkCtas <= kWorkR, "one status slot per checking CTA");

template <int W, int NW>
struct ElimSmem {
    int first[2][NW];         // per warp: its lowest candidate's key, by column parity
    uint64_t crow[2][NW][W];  // and that row's words
    int pivcol[HLF_MAX_N];
};

template <int W, int NW>
constexpr size_t elim_smem_bytes(int n)
{
    return sizeof(ElimSmem<W, NW>) + (size_t)n * basis_stride<W>() * sizeof(uint64_t);
}

// Step (1) for the whole CTA: the reduced row echelon form, pivots and the
// enumeration table, by factor_block's elimination loop; the kernel-vector
// step and the input checks are left to the other CTAs and kernel. Also
// zeroes the z^a rows of both tables (factor_kvec_kernel ORs the bits in) and
// the scratch words the second kernel uses, and publishes r in work[kWorkR].
template <int W, int R, int NW>
__device__ void eliminate_only(const uint64_t* __restrict__ A, int n, const FactorOut& o, unsigned char* smem)
{
    constexpr int kNone = 0x7fffffff;
    using Smem = ElimSmem<W, NW>;
    Smem& sm = *reinterpret_cast<Smem*>(smem);
    constexpr int SW = basis_stride<W>();
    uint64_t* s_rows = reinterpret_cast<uint64_t*>(smem + sizeof(Smem));  // [n][SW]

    const int tid = threadIdx.x;
    const int bs = blockDim.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = bs >> 5;

    uint64_t row[R][W];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = tid + j * bs;
#pragma unroll
        for (int w = 0; w < W; ++w) row[j][w] = i < n ? A[(size_t)i * W + w] : 0ull;
    }
    bool used[R];
    int my_k[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        used[j] = false;
        my_k[j] = -1;
    }
    int rank = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        for (int b = 0; b < 64; ++b) {
            const int c = (w << 6) + b;
            if (c >= n) break;
            const int buf = c & 1;
            int cand = kNone;
#pragma unroll
            for (int j = R - 1; j >= 0; --j)
                if (tid + j * bs < n && !used[j] && ((row[j][w] >> b) & 1ull)) cand = ((tid + j * bs) << 5) | warp;
            const int wmin = __reduce_min_sync(0xffffffffu, cand);
            if (wmin != kNone && cand == wmin) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (tid + j * bs != (wmin >> 5)) continue;
#pragma unroll
                    for (int v = w; v < W; ++v) sm.crow[buf][warp][v] = row[j][v];
                }
            }
            if (lane == 0) sm.first[buf][warp] = wmin;
            __syncthreads();
            int pk = lane < nwarps ? sm.first[buf][lane] : kNone;
            pk = __reduce_min_sync(0xffffffffu, pk);
            if (pk == kNone) continue;  // no pivot in column c (uniform)
            const uint64_t* prow = sm.crow[buf][pk & 31];
            const int p = pk >> 5;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (tid + j * bs == p) {
                    used[j] = true;
                    my_k[j] = rank;
                }
            }
            if (tid == 0) sm.pivcol[rank] = c;
            if constexpr (R == 1) {  // row p; its words below word w are zero
                uint64_t pv[W];
#pragma unroll
                for (int v = w; v < W; ++v) pv[v] = prow[v];
                const uint64_t m = (tid != p && ((row[0][w] >> b) & 1ull)) ? ~0ull : 0ull;
#pragma unroll
                for (int v = w; v < W; ++v) row[0][v] ^= pv[v] & m;
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (tid + j * bs != p && ((row[j][w] >> b) & 1ull)) {
#pragma unroll
                        for (int v = w; v < W; ++v) row[j][v] ^= prow[v];
                    }
                }
            }
            ++rank;
        }
    }
    const int r = rank;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (!used[j]) continue;
#pragma unroll
        for (int v = 0; v < W; ++v) s_rows[my_k[j] * SW + v] = row[j][v];
    }
    __syncthreads();

    // outputs of step (1): B_k in pivot order, pivots, enumeration table rows;
    // both tables' z^a rows and rows past min(r, 64) zero
    const int nb = r < HLF_MAX_VARYING ? r : HLF_MAX_VARYING;
    for (int i = tid; i < r * W; i += bs) {
        const uint64_t v = s_rows[(i / W) * SW + i % W];
        o.basis[i] = v;
        if (i < nb * W) o.table[i] = v;
    }
    for (int i = nb * W + tid; i < kTableTotalRows * W; i += bs) {
        o.table[i] = 0ull;
        if (o.ptable) o.ptable[i] = 0ull;
    }
    for (int k = tid; k < r; k += bs) o.piv[k] = sm.pivcol[k];
    if (tid == 0) {
        o.work[kWorkR] = r;
        o.work[kWorkInternal] = 0;
        o.work[kWorkDone] = 0;
    }
}

// The input checks of factor_block, spread over the checking CTAs: padding
// bits row by row, symmetry by the warp transposes of the 64 x 64 block pairs
// (I, J), I <= J. CTA k writes its verdict (0 or the larger code) to
// work[k]; every slot is written, so nothing needs clearing beforehand.
template <int W>
__device__ void check_input(const uint64_t* __restrict__ A, int n, int cta, int nctas, int32_t* work)
{
    __shared__ int s_bad;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    int bad = 0;
    const int tail = n & 63;
    if (tail)
        for (int i = cta * blockDim.x + threadIdx.x; i < n; i += nctas * blockDim.x)
            if (A[(size_t)i * W + W - 1] >> tail) bad = HLF_ERR_PADDING;
    for (int pr = cta * nwarps + warp; pr < W * (W + 1) / 2; pr += nctas * nwarps) {
        int I = 0, rest = pr;  // pair index -> (I, J), I <= J < W
        while (rest >= W - I) {
            rest -= W - I;
            ++I;
        }
        const int J = I + rest;
        const int ra = 64 * I + lane, rb = 64 * J + lane;
        uint64_t p0 = ra < n ? A[(size_t)ra * W + J] : 0ull;
        uint64_t p1 = ra + 32 < n ? A[(size_t)(ra + 32) * W + J] : 0ull;
        const uint64_t q0 = rb < n ? A[(size_t)rb * W + I] : 0ull;
        const uint64_t q1 = rb + 32 < n ? A[(size_t)(rb + 32) * W + I] : 0ull;
        transpose64_warp(p0, p1, lane);
        const int cols = n - 64 * I;
        const uint64_t cm = cols >= 64 ? ~0ull : ((1ull << cols) - 1ull);
        if ((rb < n && ((p0 ^ q0) & cm)) || (rb + 32 < n && ((p1 ^ q1) & cm))) bad = max(bad, HLF_ERR_NOT_SYMMETRIC);
    }
    if (bad) atomicMax(&s_bad, bad);
    __syncthreads();
    if (threadIdx.x == 0) work[cta] = s_bad;
}

template <int W>
__global__ void __launch_bounds__(512, 1) factor_elim_kernel(const uint64_t* __restrict__ A, int n, FactorOut o)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (blockIdx.x > 0) {
        check_input<W>(A, n, (int)blockIdx.x - 1, (int)gridDim.x - 1, o.work);
        return;
    }
    eliminate_only<W, rows_per_thread<W>(), 16>(A, n, o, smem);
}

// Steps (2)-(4), one warp per free column f: x_f = e_f + sum_k B_k[f] e_{p_k},
// q(x_f) = sum over i in supp(x_f) of popcount(A_i & x_f) mod 4, and
// z^a_f = q(x_f) / 2 (z^a vanishes on the pivots). The paper-order table is
// built by warp 0 of CTA 0, as in factor_block. The last CTA to finish folds
// the checking CTAs' verdicts and the q parity into the status word.
template <int W>
__global__ void __launch_bounds__(256) factor_kvec_kernel(const uint64_t* __restrict__ A, int n, FactorOut o,
                                                          int n_chk)
{
    constexpr int NW = 8;
    __shared__ uint32_t s_pivmask[HLF_MAX_N / 32];
    __shared__ uint64_t s_x[NW][W];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int r = __ldcg(o.work + kWorkR);
    for (int i = threadIdx.x; i < HLF_MAX_N / 32; i += blockDim.x) s_pivmask[i] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        const int c = __ldcg(o.piv + k);
        atomicOr(&s_pivmask[c >> 5], 1u << (c & 31));
    }
    __syncthreads();

    if (blockIdx.x == 0 && warp == 0 && o.ptable && lane < W) {
        // the paper's order: row l = XOR of A's columns (= rows) at p_{r-1}, .., p_{r-1-l}
        const int nb = r < HLF_MAX_VARYING ? r : HLF_MAX_VARYING;
        uint64_t acc = 0;
        for (int l = 0; l < nb; ++l) {
            acc ^= A[(size_t)__ldcg(o.piv + r - 1 - l) * W + lane];
            o.ptable[l * W + lane] = acc;
        }
    }

    int err = 0;
    const int gw = blockIdx.x * NW + warp;
    for (int f = gw; f < n; f += gridDim.x * NW) {
        if ((s_pivmask[f >> 5] >> (f & 31)) & 1u) continue;  // pivot column (uniform per warp)
        const int fw = f >> 6;
        const int fb = f & 63;
        if (lane < W) s_x[warp][lane] = lane == fw ? (1ull << fb) : 0ull;
        __syncwarp();
        // bit p_k of x_f is B_k[f]: each lane sets the bits of its k
        for (int k = lane; k < r; k += 32) {
            if ((__ldcg(o.basis + (size_t)k * W + fw) >> fb) & 1ull) {
                const int pc = __ldcg(o.piv + k);
                atomicOr(reinterpret_cast<unsigned long long*>(&s_x[warp][pc >> 6]), 1ull << (pc & 63));
            }
        }
        __syncwarp();
        unsigned acc = 0;
        for (int i = lane; i < n; i += 32) {
            if ((s_x[warp][i >> 6] >> (i & 63)) & 1ull) {
#pragma unroll
                for (int v = 0; v < W; ++v) acc += __popcll(A[(size_t)i * W + v] & s_x[warp][v]);
            }
        }
        const unsigned q = __reduce_add_sync(0xffffffffu, acc) & 3u;
        if (q & 1u) err = HLF_ERR_INTERNAL;  // q is even on Ker(A) for symmetric A
        if (lane == 0 && (q >> 1)) {
            atomicOr(reinterpret_cast<unsigned long long*>(o.table + kTableZ0Row * W + fw), 1ull << fb);
            if (o.ptable)
                atomicOr(reinterpret_cast<unsigned long long*>(o.ptable + kTableZ0Row * W + fw), 1ull << fb);
        }
        __syncwarp();
    }
    if (err) atomicMax(o.work + kWorkInternal, err);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(o.work + kWorkDone, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        // an input fault first (as factor_block reports it), then an odd q
        int st = 0;
        for (int k = 0; k < n_chk; ++k) st = max(st, __ldcg(o.work + k));
        if (!st) st = __ldcg(o.work + kWorkInternal);
        o.info[0] = st;
        o.info[1] = st ? -1 : r;
    }
}

template <int W>
hlf_status launch_factor_large(const uint64_t* A, int n, const FactorOut& o, cudaStream_t s)
{
    constexpr int R = rows_per_thread<W>();
    if (!o.work) return HLF_ERR_INTERNAL;
    const int threads = ((n + R - 1) / R + 31) / 32 * 32;
    const size_t smem = elim_smem_bytes<W, 16>(n);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(factor_elim_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)elim_smem_bytes<W, 16>(HLF_MAX_N)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    factor_elim_kernel<W><<<1 + kChkCtas, threads, smem, s>>>(A, n, o);
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    // one warp per free column at most: n warps over CTAs of 8
    const int blocks = (n + 7) / 8;
    factor_kvec_kernel<W><<<blocks, 256, 0, s>>>(A, n, o, kChkCtas);
    return cudaGetLastError() == cudaSuccess ? HLF_OK : HLF_ERR_CUDA;
}

}  // namespace

hlf_status launch_factor(const uint64_t* A, int n, int W, const FactorOut& o, cudaStream_t s)
{
    switch (W) {
    case 1: return launch_factor_w<1>(A, n, o, s);
    case 2: return launch_factor_w<2>(A, n, o, s);
    case 3: return launch_factor_w<3>(A, n, o, s);
    case 4: return launch_factor_w<4>(A, n, o, s);
    case 5: return launch_factor_w<5>(A, n, o, s);
    case 6: return launch_factor_w<6>(A, n, o, s);
    case 7: return launch_factor_w<7>(A, n, o, s);
    case 8: return launch_factor_w<8>(A, n, o, s);
    case 9: return launch_factor_large<9>(A, n, o, s);
    case 10: return launch_factor_large<10>(A, n, o, s);
    case 11: return launch_factor_large<11>(A, n, o, s);
    case 12: return launch_factor_large<12>(A, n, o, s);
    case 13: return launch_factor_large<13>(A, n, o, s);
    case 14: return launch_factor_large<14>(A, n, o, s);
    case 15: return launch_factor_large<15>(A, n, o, s);
    case 16: return launch_factor_large<16>(A, n, o, s);
    default: return HLF_ERR_SIZE;
    }
}

}  // namespace hlf
