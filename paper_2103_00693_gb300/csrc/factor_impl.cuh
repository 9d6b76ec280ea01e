// Stage 1 of the two-stage scheme as a block-level device function: the CLA
// module of Section 2 (Fig. 1(b)), steps (1)-(4), for one matrix per CTA.
//
//   (1) Gauss-Jordan elimination of A over GF(2). Each thread owns R rows of
//       A in registers (W uint64 words each). For each column c, left to
//       right, the candidates are the rows not yet used as a pivot that have
//       bit c set; a min over each warp and then over the warps picks the
//       lowest such row p. The key minimised is (row << 5) | warp, so the
//       minimum also names the warp that holds row p. Each warp stages its
//       lowest candidate's words next to its key, so one barrier per column
//       suffices: after it every thread knows p and reads row p from that
//       warp's slot, and every other row with bit c set XORs it in (rows
//       above and below: Gauss-Jordan, so the result is the unique reduced
//       row echelon form). The slots
//       alternate with the column's parity, so a slot is rewritten only after
//       the next column's barrier, when every read of it is done. A row not
//       yet used as a pivot is zero in every column left of c (each earlier
//       column was cleared by its pivot or had no candidate), so the pivot
//       row's words left of c's word are zero: they are neither staged nor
//       XORed. Rows are never swapped; the pivot row of column c is
//       remembered instead. Unused rows end at zero.
//
//       Measured and rejected: one warp eliminating alone with ballots and
//       shuffles (slower from W = 2 on), and two columns per barrier (three
//       minima per warp; more work per column than the barrier it saves).
//   (2)-(4) Kernel basis, q and z^a. For a free column f the kernel vector is
//       x_f = e_f + sum_k B_k[f] e_{p_k}; q(x_f) = sum over i in supp(x_f) of
//       popcount(A_i & x_f), mod 4, which is x_f^T A x_f mod 4. With z^a
//       chosen to vanish on the pivots, z^a . x_f = z^a_f, so the equation
//       2 z^T x_f = q(x_f) (mod 4) gives z^a_f = q(x_f) / 2 directly.
//
// Also checked here: padding bits (column >= n) are zero and A is symmetric
// (Section 1 defines the problem for symmetric A only), the latter by 64 x 64
// bit-block transposes in registers.
#pragma once

#include "hlf_internal.cuh"

namespace hlf {

// NW: the most warps a CTA running factor_block may have (32 by default).
template <int W, int MAXN, int NW = 32>
struct FactorSmem {
    int first[2][NW];        // per warp: its lowest candidate's key for the column (by column parity)
    uint64_t crow[2][NW][W];  // and that row's words
    int pivcol[MAXN];
    uint32_t pivmask[MAXN / 32];
    uint64_t x[NW][W];
    uint64_t z0[W];
    int err;
};

// Transpose a 64 x 64 bit block held by one warp: lane l has rows l (x0) and
// l + 32 (x1), bit s of a row being column s. Stage j (j = 32, 16, ..., 1)
// swaps the row-index bit of weight j with the column-index bit of weight j:
// it exchanges the bits at column s + j of row t with those at column s of
// row t + j, for s and t with that bit clear. The six stages compose to the
// transpose. Stage 32 pairs the two rows of a lane, the others pair lanes l
// and l ^ j.
__device__ __forceinline__ void transpose64_warp(uint64_t& x0, uint64_t& x1, int lane)
{
    {
        const uint64_t t = ((x0 >> 32) ^ x1) & 0x00000000FFFFFFFFull;
        x1 ^= t;
        x0 ^= t << 32;
    }
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint64_t m = j == 16 ? 0x0000FFFF0000FFFFull
                         : j == 8  ? 0x00FF00FF00FF00FFull
                         : j == 4  ? 0x0F0F0F0F0F0F0F0Full
                         : j == 2  ? 0x3333333333333333ull
                                   : 0x5555555555555555ull;
        const bool upper = (lane & j) != 0;  // this lane's rows are the t + j of their pairs
        const uint64_t o0 = __shfl_xor_sync(0xffffffffu, x0, j);
        const uint64_t o1 = __shfl_xor_sync(0xffffffffu, x1, j);
        const uint64_t t0 = upper ? (((o0 >> j) ^ x0) & m) : (((x0 >> j) ^ o0) & m);
        const uint64_t t1 = upper ? (((o1 >> j) ^ x1) & m) : (((x1 >> j) ^ o1) & m);
        x0 ^= upper ? t0 : t0 << j;
        x1 ^= upper ? t1 : t1 << j;
    }
}

// Row stride of the basis rows in shared memory: odd, so that 32 lanes reading
// one word of 32 consecutive rows hit distinct banks.
template <int W>
constexpr int basis_stride() { return W | 1; }

template <int W, int MAXN, int NW = 32>
constexpr size_t factor_smem_bytes(int n)
{
    return sizeof(FactorSmem<W, MAXN, NW>) + (size_t)n * basis_stride<W>() * sizeof(uint64_t);
}

// Factor the n x n matrix A ([n][W] words, global) with the whole CTA.
// Thread t owns the R rows t, t + blockDim.x, ... in registers. Requires
// R * blockDim.x >= n, blockDim.x a multiple of 32 and at most 32 * NW,
// n <= MAXN. `smem` points to factor_smem_bytes<W, MAXN, NW>(n) bytes of
// shared memory. Writes o.table
// (always), o.basis and o.piv (when non-null) and o.info[0] = status,
// o.info[1] = r (or -1 on a fault). Returns r, or -1.
template <int W, int R, int MAXN, int NW = 32>
__device__ int factor_block(const uint64_t* __restrict__ A, int n, const FactorOut& o, unsigned char* smem)
{
    constexpr int kNone = 0x7fffffff;
    using Smem = FactorSmem<W, MAXN, NW>;
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
    if (tid == 0) sm.err = 0;
    if (tid < W) sm.z0[tid] = 0;
    for (int i = tid; i < MAXN / 32; i += bs) sm.pivmask[i] = 0;
    __syncthreads();

    // ---- input checks: padding bits, then symmetry. A warp takes the 64 x 64
    // blocks (I, J) and (J, I), I <= J, of the W x W block grid, transposes the
    // first in registers and compares it with the second on the rows and
    // columns below n.
    int bad = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int tail = n & 63;
        if (tid + j * bs < n && tail && (row[j][W - 1] >> tail)) bad = HLF_ERR_PADDING;
    }
    for (int pr = warp; pr < W * (W + 1) / 2; pr += nwarps) {
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
    if (bad) atomicMax(&sm.err, bad);
    __syncthreads();
    if (sm.err) {
        const int e = sm.err;
        __syncthreads();
        if (tid == 0) {
            o.info[0] = e;
            o.info[1] = -1;
        }
        return -1;
    }

    // ---- (1) Gauss-Jordan elimination: B_k to s_rows[k][.], its pivot column to sm.pivcol[k]
    int r;
    {
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
#pragma unroll 4  // 9-12% faster than rolled at n = 100..324
            for (int b = 0; b < 64; ++b) {
                const int c = (w << 6) + b;
                if (c >= n) break;
                const int buf = c & 1;
                // this thread's lowest unused row with bit c, keyed (row << 5) | warp
                int cand = kNone;
#pragma unroll
                for (int j = R - 1; j >= 0; --j)
                    if (tid + j * bs < n && !used[j] && ((row[j][w] >> b) & 1ull)) cand = ((tid + j * bs) << 5) | warp;
                const int wmin = __reduce_min_sync(0xffffffffu, cand);
                if (wmin != kNone && cand == wmin) {  // this lane holds the warp's lowest candidate
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
                if (tid == 0 && HLF_IN_BOUNDS(rank, HLF_MAX_N, kSiteFactorSmem)) sm.pivcol[rank] = c;
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
        r = rank;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (!used[j] || !HLF_IN_BOUNDS(my_k[j], n, kSiteFactorSmem)) continue;
#pragma unroll
            for (int v = 0; v < W; ++v) s_rows[my_k[j] * SW + v] = row[j][v];
        }
    }
    const int nb = r < HLF_MAX_VARYING ? r : HLF_MAX_VARYING;
    __syncthreads();

    // ---- outputs of step (1): B_k in pivot order, pivots, enumeration table
    for (int i = tid; i < r * W; i += bs) {
        const uint64_t v = s_rows[(i / W) * SW + i % W];
        if (o.basis) o.basis[i] = v;
        if (i < nb * W) o.table[i] = v;
    }
    for (int i = nb * W + tid; i < kTableRows * W; i += bs) o.table[i] = 0ull;
    for (int k = tid; k < r; k += bs) {
        const int c = sm.pivcol[k];
        if (o.piv) o.piv[k] = c;
        atomicOr(&sm.pivmask[c >> 5], 1u << (c & 31));
    }
    __syncthreads();

    // ---- (2)-(4): one warp per free column f
    int err = 0;
    for (int f = warp; f < n; f += nwarps) {
        if ((sm.pivmask[f >> 5] >> (f & 31)) & 1u) continue;  // pivot column (uniform per warp)
        const int fw = f >> 6;
        const int fb = f & 63;
        if (lane < W) sm.x[warp][lane] = lane == fw ? (1ull << fb) : 0ull;
        __syncwarp();
        // bit p_k of x_f is B_k[f]. pivcol ascends with k, so the lanes of a
        // 32-row chunk that set bits of one word of x_f are contiguous, and
        // an OR over them sets that word.
        for (int k0 = 0; k0 < r; k0 += 32) {
            const int k = k0 + lane;
            const bool has = k < r && ((s_rows[k * SW + fw] >> fb) & 1ull);
            const int pc = has ? sm.pivcol[k] : 0;
            unsigned pending = __ballot_sync(0xffffffffu, has);
            while (pending) {  // one word of x_f per pass (uniform)
                const int wv = __shfl_sync(0xffffffffu, pc >> 6, __ffs(pending) - 1);
                const bool mine = has && (pc >> 6) == wv;
                const uint64_t bit = mine ? 1ull << (pc & 63) : 0ull;
                const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)bit);
                const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(bit >> 32));
                if (lane == 0) sm.x[warp][wv] |= ((uint64_t)hi << 32) | lo;
                pending &= ~__ballot_sync(0xffffffffu, mine);
            }
        }
        __syncwarp();
        unsigned acc = 0;
        for (int i = lane; i < n; i += 32) {
            if ((sm.x[warp][i >> 6] >> (i & 63)) & 1ull) {
#pragma unroll
                for (int v = 0; v < W; ++v) acc += __popcll(A[(size_t)i * W + v] & sm.x[warp][v]);
            }
        }
        const unsigned q = __reduce_add_sync(0xffffffffu, acc) & 3u;
        if (q & 1u) err = HLF_ERR_INTERNAL;  // q is even on Ker(A) for symmetric A
        if (lane == 0 && (q >> 1))
            atomicOr(reinterpret_cast<unsigned long long*>(&sm.z0[fw]), 1ull << fb);
        __syncwarp();
    }
    if (err) atomicMax(&sm.err, err);
    __syncthreads();
    const int e = sm.err;
    if (tid < W) o.table[kTableZ0Row * W + tid] = sm.z0[tid];

    // ---- the paper's own order (Section 2, Eq. 3; the counter of Section 4):
    // counter value t sets R_{p_j} = bit (r - j) of t, y = A R, z = y ^ z^a.
    // Bit l of t selects T_l = column p_{r-1-l} of A (0-based pivots), which is
    // row p_{r-1-l} since A is symmetric. With P_k = T_0 ^ ... ^ T_k, the Gray
    // walk over P visits z(t) in counter order, because bit l of t is the XOR
    // of the Gray code's bits k >= l. One warp builds the prefix XORs.
    if (o.ptable) {
        if (warp == 0 && lane < W) {
            uint64_t acc = 0;
            for (int l = 0; l < nb; ++l) {
                acc ^= A[(size_t)sm.pivcol[r - 1 - l] * W + lane];
                o.ptable[l * W + lane] = acc;
            }
        }
        for (int i = nb * W + tid; i < kTableRows * W; i += bs) o.ptable[i] = 0ull;
        if (tid < W) o.ptable[kTableZ0Row * W + tid] = sm.z0[tid];
    }
    if (tid == 0) {
        o.info[0] = e;
        o.info[1] = e ? -1 : r;
    }
    __syncthreads();  // shared memory may be reused by the caller
    return e ? -1 : r;
}

}  // namespace hlf
