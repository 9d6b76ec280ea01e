// Stage 1 for one matrix (the CLA module of Section 2, steps (1)-(4)).
//
// n <= 256 (W <= 4): one CTA runs factor_block (factor_impl.cuh): input
// checks, elimination, kernel vectors, q and z^a in one launch, which is what
// the latency of small and medium instances wants.
//
// n > 256 (W >= 5): the same results from two launches that spread the work
// that does not have to be sequential over many SMs:
//   factor_elim_kernel   CTA 0 runs the Gauss-Jordan elimination (step (1))
//                        with the rows of A in registers, in panels of 32
//                        columns (eliminate_only); CTAs 1.. check the input
//                        (padding bits, symmetry by 64 x 64 bit-block
//                        transposes) at the same time, each writing its own
//                        status slot.
//   factor_kvec_kernel   one CTA per free column f across the GPU: the
//                        kernel vector x_f, q(x_f) mod 4 and the bit z^a_f
//                        (steps (2)-(4)), the paper-order table, and, in
//                        the last CTA to finish, the status and rank.
// At n = 1024 this takes 202 us (grid 32 x 32) and 309 us (random
// symmetric); one CTA running factor_block's column loop for everything took
// 392 us. Against the one-CTA path it saves 11-19% on grids from W = 5 on
// (n = 289: 53 us against 60; n = 324: 57 against 70; n = 361: 63 against
// 74), ties on random symmetric matrices there (n = 300: 57.4 against 57.7;
// n = 384: 76.7 against 78.4), ties at n = 256 and loses below (n = 200: 42
// us against 39), hence the threshold.
//
// The elimination's cost is the pivot search: a CTA barrier per column and
// the chain through the exchange (every searching warp's candidate, two warp
// minima, the exchange, the slice and record updates). Per-row records of the
// absorbed pivots replaced a Gauss-Jordan inversion of each panel's pivot
// slices by one warp (91k of 617k cycles at n = 1024). Keeping the pivot rows
// of earlier panels out of the search, and with them every warp that holds no
// live slice, leaves two or three searching warps a panel on grids (grid 32 x
// 32: 269 -> 202 us) at the price of a barrier and the T1 tables a panel on
// dense matrices (random symmetric n = 1024: 301 -> 309 us).
//
// Measured at n = 1024 and
// dropped:
//   - factor_block's loop (every row's full row XORs the pivot row each
//     column, 600 cycles a column): 355 us;
//   - a split barrier (an mbarrier whose arrive precedes the XOR of the
//     previous pivot row's later words, and whose wait follows it): 607 us;
//   - panels of 8 columns searched on 8-bit slices: 367 us;
//   - panels of 64 columns with 64-bit slices and per-row records: 395 us;
//   - the exchange by a shared atomicMin per warp into a per-column slot
//     instead of per-warp slots and a second warp minimum: the search 462k
//     cycles against 394k;
//   - one copy of the panel code for all panels (the word w picked out of
//     the registers by unrolled selects, the updates predicated on v >= w):
//     grid 32 x 32 214 us against 202, random symmetric 327 against 309; with
//     the table build free of divisions and the update dispatched to a copy
//     per w instead of predicated, 211 and 326;
//   - the table builds in one out-of-line function: 218 us against 202 (the
//     call saves and restores the live registers);
//   - two columns per barrier (each warp offering its lowest rows with bit
//     0, with bit 1 and with bit 0 xor bit 1 set, which settles the pivots
//     of both columns): 345 us, the search 405 cycles a column;
//   - the search in one warp with the rows transposed (lane l holding rows
//     32l..32l+31 as column words): no CTA barrier, but 611 cycles a column,
//     the pivot slice's extraction being a chain of dependent ORs (370 us);
//   - a thread-block cluster sharing the rows: its barrier alone takes about
//     400 cycles a round trip on this GPU (any cluster size), and a
//     publish-then-minimum exchange over 8 CTAs about 800, more than the
//     whole column step in one CTA.

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
constexpr int kWorkMask = 32;     // work[32..64) = the pivot columns, one bit each
constexpr int kKvecCtas = 256;    // CTAs of factor_kvec_kernel (one free column at a time each)
static_assert(kWorkMask + HLF_MAX_N / 32 <= kFactorWorkWords, "the pivot mask fits the scratch words");
static_assert(kChkCtas <= kWorkR, "one status slot per checking CTA");

template <int W>
struct ElimSmem {
    int first[2][32];          // per warp: its lowest candidate's key, by column parity
    uint2 cw[2][32];           // and that row's current slice and record, pivot bit added
    int part[32];              // per warp: whether it holds a live slice in the panel
    int npiv;                  // the panel's pivot count, from the searching warps
    int colidx[32];            // pivot index of each column of the panel, -1 if free
    uint32_t H[32];            // reduced pivot row k as a set of the panel's pivot start rows
    uint32_t T1[8 * 16];       // XORs of H over 4 pivot columns, for the earlier pivot rows
    uint32_t pivmask[HLF_MAX_N / 32];  // the pivot columns, for the second kernel
    uint64_t piv[32][W];       // the pivot rows at the panel's start
    uint64_t T2[8 * 16 * (W | 1)];  // their combinations over 4 pivot indices, odd stride
    int pivcol[HLF_MAX_N];
};

template <int W>
constexpr size_t elim_smem_bytes(int n)
{
    return sizeof(ElimSmem<W>) + (size_t)n * basis_stride<W>() * sizeof(uint64_t);
}

// Step (1) for the whole CTA: the reduced row echelon form, pivots and the
// enumeration table, by panels of 32 columns (below); the kernel-vector step
// and the input checks are left to the other CTAs and kernel. Also
// zeroes the z^a rows of both tables (factor_kvec_kernel ORs the bits in) and
// the scratch words the second kernel uses, and publishes r in work[kWorkR].
template <int W, int R>
__device__ void eliminate_only(const uint64_t* __restrict__ A, int n, const FactorOut& o, unsigned char* smem)
{
    constexpr int kNone = 0x7fffffff;
    using Smem = ElimSmem<W>;
    Smem& sm = *reinterpret_cast<Smem*>(smem);
    constexpr int SW = basis_stride<W>();
    uint64_t* s_rows = reinterpret_cast<uint64_t*>(smem + sizeof(Smem));  // [n][SW]

    const int tid = threadIdx.x;
    const int bs = blockDim.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    uint64_t row[R][W];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = tid + j * bs;
#pragma unroll
        for (int w = 0; w < W; ++w) row[j][w] = i < n ? A[(size_t)i * W + w] : 0ull;
    }
    // key = (row << 5) | warp while the row may still become a pivot; kNone
    // for the rows past n and for the pivot rows of earlier panels
    int key[R];
    bool used[R];
    int my_k[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        key[j] = tid + j * bs < n ? (((tid + j * bs) << 5) | warp) : kNone;
        used[j] = false;
        my_k[j] = -1;
    }
    if (tid < 64) (&sm.first[0][0])[tid] = kNone;
    if (tid < 32) sm.part[tid] = 0;  // absent warps never search
    __syncthreads();

    // Panels of 32 columns. (a) Gauss-Jordan on the 32-bit slices of the
    // rows that are not pivots of earlier panels: for each column the lowest
    // such row with the bit that is not yet a pivot becomes the pivot, and
    // every other slice with the bit, the panel's earlier pivots included,
    // absorbs the pivot's; the slices rotate so that bit 0 is the column.
    // Each row also keeps the record cf of what it absorbed, as a set of the
    // panel's pivot rows taken at the panel's start: the pivot of index k
    // publishes its own record with bit k added, and an absorbing row XORs
    // that into its record. Only the warps holding a nonzero slice search,
    // behind a named barrier sized to them (on banded matrices, two or three
    // warps). (b) The reduced pivot row k is the set H_k = its final record
    // plus k. Every row is rebuilt from the panel's start values as itself
    // XOR the start rows of the pivots in its record, read from nibble tables
    // of those start rows (T2); a pivot row of an earlier panel takes, as its
    // record, the XOR of H over the pivot columns its start slice has (nibble
    // tables T1 of H). The result is the Gauss-Jordan elimination of the
    // panel: zeros on its pivot columns outside each pivot's own row, the same
    // span; the pivot rows are zero left of the panel, so only words w..
    // change.
    constexpr int kHalvesUnroll = W > 11 ? 2 : 1;
    int rank = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        // both halves of word w run the same code (the registers it names
        // depend on w only): rolled, W copies in all, save where the rolled
        // loop spills (W > 11, measured slower)
#pragma unroll kHalvesUnroll
        for (int h = 0; h < 2; ++h) {
            const int c0 = (w << 6) + (h << 5);
            if (c0 >= n) break;
            const int ncols = n - c0 < 32 ? n - c0 : 32;
            uint32_t s[R], cf[R];
            int my_kp[R];
            bool live = false;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                s[j] = used[j] ? 0u : (uint32_t)(row[j][w] >> (32 * h));
                cf[j] = 0u;
                my_kp[j] = -1;
                live |= s[j] != 0u;
            }
            live = __any_sync(0xffffffffu, live);
            if (lane == 0) {
                sm.part[warp] = live;
                if (!live) sm.first[0][warp] = sm.first[1][warp] = kNone;  // read by the searching warps
            }
            if (tid < 32) sm.colidx[tid] = -1;
            __syncthreads();  // also: the previous panel's table reads are done
            const unsigned pm = __ballot_sync(0xffffffffu, sm.part[lane] != 0);
            int kp = 0;
            if ((pm >> warp) & 1u) {  // warp-uniform
                const int nthr = __popc(pm) * 32;
                const bool scribe = lane == 0 && warp == __ffs(pm) - 1;  // the lowest searching warp's lane 0
                // unrolled by 4 only: 2W copies of the panel code suit the
                // instruction cache, 64W copies of this body would not (by 4:
                // the search 5% faster than rolled at n = 1024)
#pragma unroll 4
                for (int b = 0; b < ncols; ++b) {
                    const int buf = b & 1;
                    int cand = kNone;
#pragma unroll
                    for (int j = 0; j < R; ++j) cand = min(cand, (s[j] & 1u) ? key[j] : kNone);
                    const int wmin = __reduce_min_sync(0xffffffffu, cand);
                    if (cand == wmin && wmin != kNone) {  // the lane of the warp's candidate
                        uint32_t sv = s[0], cv = cf[0];
#pragma unroll
                        for (int j = 1; j < R; ++j) {
                            sv = cand == key[j] ? s[j] : sv;
                            cv = cand == key[j] ? cf[j] : cv;
                        }
                        sm.cw[buf][warp] = make_uint2(sv, cv ^ (1u << kp));
                    }
                    if (lane == 0) sm.first[buf][warp] = wmin;
                    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
                    const int pk = __reduce_min_sync(0xffffffffu, sm.first[buf][lane]);
                    if (pk != kNone) {  // uniform
                        const uint2 pv = sm.cw[buf][pk & 31];
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            const bool me = key[j] == pk;
                            const bool ab = (s[j] & 1u) && !me;
                            s[j] = ab ? s[j] ^ pv.x : s[j];
                            cf[j] = ab ? cf[j] ^ pv.y : cf[j];
                            my_kp[j] = me ? kp : my_kp[j];
                            key[j] = me ? kNone : key[j];
                        }
                        if (scribe) {
                            sm.colidx[b] = kp;
                            if (HLF_IN_BOUNDS(rank + kp, HLF_MAX_N, kSiteFactorSmem)) sm.pivcol[rank + kp] = c0 + b;
                        }
                        ++kp;
                    }
#pragma unroll
                    for (int j = 0; j < R; ++j) s[j] = __funnelshift_r(s[j], s[j], 1);
                }
                if (scribe) sm.npiv = kp;
            }
            // the pivot rows: start rows (words w..) to T2's source, H_k
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int k = my_kp[j];
                if (k < 0 || !HLF_IN_BOUNDS(k, 32, kSiteFactorSmem)) continue;
                used[j] = true;
                my_k[j] = rank + k;
                sm.H[k] = cf[j] ^ (1u << k);
#pragma unroll
                for (int v = w; v < W; ++v) sm.piv[k][v] = row[j][v];
            }
            __syncthreads();
            kp = pm ? sm.npiv : 0;
            if (kp == 0) continue;  // uniform; nothing absorbs anything
            rank += kp;
            const int V = W - w;
            const int VP = V | 1;  // odd stride: the 16 entries of a table in distinct banks
            // T2[(t, x)][v]: XOR of the start rows' word w + v of the pivots
            // 4t + i, i over the bits of x
            for (int e = tid; e < 128 * V; e += bs) {
                const int v = e % V;
                const int tx = e / V;
                const int k0 = (tx >> 4) << 2;
                uint64_t acc = 0ull;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (((tx >> i) & 1) && k0 + i < kp) acc ^= sm.piv[k0 + i][w + v];
                if (HLF_IN_BOUNDS(tx * VP + v, 128 * (W | 1), kSiteFactorSmem)) sm.T2[tx * VP + v] = acc;
            }
            if (tid < 128) {  // T1[(t, x)]: XOR of H over the pivot columns 4t + i, i over the bits of x
                const int t = tid >> 4;
                uint32_t acc = 0u;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = sm.colidx[4 * t + i];
                    if (((tid >> i) & 1) && k >= 0 && HLF_IN_BOUNDS(k, 32, kSiteFactorSmem)) acc ^= sm.H[k];
                }
                sm.T1[tid] = acc;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < R; ++j) {
                uint32_t coef = cf[j];
                if (used[j] && my_kp[j] < 0) {  // a pivot row of an earlier panel
                    const uint32_t st = (uint32_t)(row[j][w] >> (32 * h));
#pragma unroll
                    for (int t = 0; t < 8; ++t) coef ^= sm.T1[(t << 4) | ((st >> (4 * t)) & 15u)];
                }
                if (!__any_sync(0xffffffffu, coef != 0u)) continue;  // warp-uniform
                const uint64_t* tb[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) tb[t] = sm.T2 + ((t << 4) | (int)((coef >> (4 * t)) & 15u)) * VP;
#pragma unroll
                for (int v = 0; v < V; ++v)
                    row[j][w + v] ^= ((tb[0][v] ^ tb[1][v]) ^ (tb[2][v] ^ tb[3][v])) ^
                                     ((tb[4][v] ^ tb[5][v]) ^ (tb[6][v] ^ tb[7][v]));
            }
            // the next panel's first barrier orders these reads before the
            // tables are written again
        }
    }
    const int r = rank;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (!used[j] || !HLF_IN_BOUNDS(my_k[j], n, kSiteFactorSmem)) continue;
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
    if (tid < HLF_MAX_N / 32) sm.pivmask[tid] = 0u;
    __syncthreads();
    for (int k = tid; k < r; k += bs) atomicOr(&sm.pivmask[sm.pivcol[k] >> 5], 1u << (sm.pivcol[k] & 31));
    __syncthreads();
    if (tid < HLF_MAX_N / 32) o.work[kWorkMask + tid] = (int32_t)sm.pivmask[tid];
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
    eliminate_only<W, rows_per_thread<W>()>(A, n, o, smem);
}

// Steps (2)-(4), one CTA per free column f (the j-th free column, j =
// blockIdx.x, blockIdx.x + gridDim.x, ..., found from the pivot mask the
// elimination left in the scratch words): x_f = e_f + sum_k B_k[f] e_{p_k},
// q(x_f) = sum over i in supp(x_f) of popcount(A_i & x_f) mod 4, and
// z^a_f = q(x_f) / 2 (z^a vanishes on the pivots). Each thread takes every
// 256th k and every 256th row, so a free column costs a few rounds of
// memory latency, not one per row. The paper-order table is built by warp 1
// of CTA 0, as in factor_block. The last CTA to finish folds the checking
// CTAs' verdicts and the q parity into the status word.
template <int W>
__global__ void __launch_bounds__(256) factor_kvec_kernel(const uint64_t* __restrict__ A, int n, FactorOut o,
                                                          int n_chk)
{
    __shared__ uint32_t s_mask[HLF_MAX_N / 32];  // free columns below n, by word
    __shared__ int s_before[HLF_MAX_N / 32];     // free columns in the words before
    __shared__ uint64_t s_x[W];
    __shared__ unsigned s_q;
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int r = __ldcg(o.work + kWorkR);
    if (warp == 0) {
        const int c0 = lane * 32;
        const uint32_t below_n = c0 >= n ? 0u : (n - c0 >= 32 ? ~0u : ((1u << (n - c0)) - 1u));
        const uint32_t fm = ~(uint32_t)__ldcg(o.work + kWorkMask + lane) & below_n;
        const int cnt = __popc(fm);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        s_mask[lane] = fm;
        s_before[lane] = incl - cnt;
    }
    if (blockIdx.x == 0 && warp == 1 && o.ptable && lane < W) {
        // the paper's order: row l = XOR of A's columns (= rows) at p_{r-1}, .., p_{r-1-l}
        const int nb = r < HLF_MAX_VARYING ? r : HLF_MAX_VARYING;
        uint64_t acc = 0;
        for (int l0 = 0; l0 < nb; l0 += 8) {  // eight independent loads in flight
            uint64_t a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                a[u] = l0 + u < nb ? A[(size_t)__ldcg(o.piv + r - 1 - l0 - u) * W + lane] : 0ull;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                acc ^= a[u];
                if (l0 + u < nb) o.ptable[(l0 + u) * W + lane] = acc;
            }
        }
    }
    __syncthreads();

    int err = 0;
    const int nfree = n - r;
    for (int j = blockIdx.x; j < nfree; j += gridDim.x) {
        // the j-th free column: the last mask word with at most j free
        // columns before it holds it
        const int l = 31 - __clz(__ballot_sync(0xffffffffu, s_before[lane] <= j));
        uint32_t m = s_mask[l];
        for (int t = j - s_before[l]; t > 0; --t) m &= m - 1u;
        if (!m) continue;  // not reached: the mask has n - r free columns (uniform)
        const int f = 32 * l + __ffs(m) - 1;
        const int fw = f >> 6;
        const int fb = f & 63;
        if (tid < W) s_x[tid] = tid == fw ? (1ull << fb) : 0ull;
        if (tid == 0) s_q = 0u;
        __syncthreads();
        // bit p_k of x_f is B_k[f]: thread t sets the bits of k = t, t + 256, ...
        for (int k0 = tid; k0 < r; k0 += 1024) {  // four loads in flight
            uint64_t bk[4];
            int pc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + 256 * u;
                bk[u] = k < r ? __ldcg(o.basis + (size_t)k * W + fw) : 0ull;
                pc[u] = k < r ? __ldcg(o.piv + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (((bk[u] >> fb) & 1ull) && HLF_IN_BOUNDS(pc[u] >> 6, W, kSiteFactorKvec))
                    atomicOr(reinterpret_cast<unsigned long long*>(&s_x[pc[u] >> 6]), 1ull << (pc[u] & 63));
        }
        __syncthreads();
        uint64_t xr[W];
#pragma unroll
        for (int v = 0; v < W; ++v) xr[v] = s_x[v];
        unsigned acc = 0;
        for (int i0 = tid; i0 < n; i0 += 512) {  // two rows' loads in flight
            const int i1 = i0 + 256;
            const bool in0 = (s_x[i0 >> 6] >> (i0 & 63)) & 1ull;
            const bool in1 = i1 < n && ((s_x[i1 >> 6] >> (i1 & 63)) & 1ull);
#pragma unroll
            for (int v = 0; v < W; ++v) {
                const uint64_t a0 = in0 ? A[(size_t)i0 * W + v] : 0ull;
                const uint64_t a1 = in1 ? A[(size_t)i1 * W + v] : 0ull;
                acc += __popcll(a0 & xr[v]) + __popcll(a1 & xr[v]);
            }
        }
        acc = __reduce_add_sync(0xffffffffu, acc);
        if (lane == 0) atomicAdd(&s_q, acc);
        __syncthreads();
        if (tid == 0) {
            const unsigned q = s_q & 3u;
            if (q & 1u) err = HLF_ERR_INTERNAL;  // q is even on Ker(A) for symmetric A
            if ((q >> 1) && HLF_IN_BOUNDS(fw, W, kSiteFactorKvec)) {
                atomicOr(reinterpret_cast<unsigned long long*>(o.table + kTableZ0Row * W + fw), 1ull << fb);
                if (o.ptable)
                    atomicOr(reinterpret_cast<unsigned long long*>(o.ptable + kTableZ0Row * W + fw), 1ull << fb);
            }
        }
        __syncthreads();  // s_x and s_q serve the next free column
    }
    if (err) atomicMax(o.work + kWorkInternal, err);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(o.work + kWorkDone, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && tid == 0) {
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
    const size_t smem = elim_smem_bytes<W>(n);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(factor_elim_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)elim_smem_bytes<W>(HLF_MAX_N)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    factor_elim_kernel<W><<<1 + kChkCtas, threads, smem, s>>>(A, n, o);
    if (cudaGetLastError() != cudaSuccess) return HLF_ERR_CUDA;
    factor_kvec_kernel<W><<<kKvecCtas, 256, 0, s>>>(A, n, o, kChkCtas);
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
    case 5: return launch_factor_large<5>(A, n, o, s);
    case 6: return launch_factor_large<6>(A, n, o, s);
    case 7: return launch_factor_large<7>(A, n, o, s);
    case 8: return launch_factor_large<8>(A, n, o, s);
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

HLF_DEBUG_TAKE(factor)

}  // namespace hlf
