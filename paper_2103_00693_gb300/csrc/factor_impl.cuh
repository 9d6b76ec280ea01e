// Stage 1 of the two-stage scheme as a block-level device function: the CLA
// module of Section 2 (Fig. 1(b)), steps (1)-(4), for one matrix per CTA.
//
//   (1) Gauss-Jordan elimination of A over GF(2). Each thread owns R rows of
//       A in registers (W uint64 words each). For each column c, left to
//       right, the candidates are the rows not yet used as a pivot that have
//       bit c set; a min over each warp and then over the warps picks the
//       lowest such row p. Each warp stages its lowest candidate's words next
//       to its index, so one barrier per column suffices: after it every
//       thread knows p and reads row p from its warp's slot, and every other
//       row with bit c set XORs it in (rows above and below: Gauss-Jordan, so
//       the result is the unique reduced row echelon form). The slots
//       alternate with the column's parity, so a slot is rewritten only after
//       the next column's barrier, when every read of it is done. Rows are
//       never swapped; the pivot row of column c is remembered instead.
//       Unused rows end at zero.
//   (2)-(4) Kernel basis, q and z^a. For a free column f the kernel vector is
//       x_f = e_f + sum_k B_k[f] e_{p_k}; q(x_f) = sum over i in supp(x_f) of
//       popcount(A_i & x_f), mod 4, which is x_f^T A x_f mod 4. With z^a
//       chosen to vanish on the pivots, z^a . x_f = z^a_f, so the equation
//       2 z^T x_f = q(x_f) (mod 4) gives z^a_f = q(x_f) / 2 directly.
//
// Also checked here: padding bits (column >= n) are zero and A is symmetric
// (Section 1 defines the problem for symmetric A only).
#pragma once

#include "hlf_internal.cuh"

namespace hlf {

template <int W, int MAXN>
struct FactorSmem {
    int first[2][32];        // per warp: its lowest candidate row for the column (by column parity)
    uint64_t crow[2][32][W];  // and that row's words
    int pivcol[MAXN];
    uint32_t pivmask[MAXN / 32];
    uint64_t x[32][W];
    uint64_t z0[W];
    int err;
};

template <int W, int MAXN>
constexpr size_t factor_smem_bytes(int n)
{
    return sizeof(FactorSmem<W, MAXN>) + (size_t)n * W * sizeof(uint64_t);
}

// Factor the n x n matrix A ([n][W] words, global) with the whole CTA.
// Thread t owns the R rows t, t + blockDim.x, ... in registers. Requires
// R * blockDim.x >= n, blockDim.x a multiple of 32, n <= MAXN. `smem` points
// to factor_smem_bytes<W, MAXN>(n) bytes of shared memory. Writes o.table
// (always), o.basis and o.piv (when non-null) and o.info[0] = status,
// o.info[1] = r (or -1 on a fault). Returns r, or -1.
template <int W, int R, int MAXN>
__device__ int factor_block(const uint64_t* __restrict__ A, int n, const FactorOut& o, unsigned char* smem)
{
    constexpr int kNone = 0x7fffffff;
    FactorSmem<W, MAXN>& sm = *reinterpret_cast<FactorSmem<W, MAXN>*>(smem);
    uint64_t* s_rows = reinterpret_cast<uint64_t*>(smem + sizeof(FactorSmem<W, MAXN>));  // [n][W]

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
        if (i < n) {
#pragma unroll
            for (int w = 0; w < W; ++w) s_rows[i * W + w] = row[j][w];
        }
    }
    if (tid == 0) sm.err = 0;
    if (tid < W) sm.z0[tid] = 0;
    for (int i = tid; i < MAXN / 32; i += bs) sm.pivmask[i] = 0;
    __syncthreads();

    // ---- input checks: padding, then symmetry (bit j of row i == bit i of row j)
    int bad = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = tid + j * bs;
        if (i >= n) continue;
        const int tail = n & 63;
        if (tail && (row[j][W - 1] >> tail)) bad = HLF_ERR_PADDING;
        const int wi = i >> 6;
        const int bi = i & 63;
        if (bad) continue;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t t = 0;
            for (int b = 0; b < 64; ++b) {
                const int c = (w << 6) + b;
                if (c >= n) break;
                t |= ((s_rows[c * W + wi] >> bi) & 1ull) << b;
            }
            if (t != row[j][w]) bad = HLF_ERR_NOT_SYMMETRIC;
        }
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

    // ---- (1) Gauss-Jordan elimination
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
            int cand = kNone;  // this thread's lowest unused row with bit c
#pragma unroll
            for (int j = R - 1; j >= 0; --j)
                if (tid + j * bs < n && !used[j] && ((row[j][w] >> b) & 1ull)) cand = tid + j * bs;
            const int wmin = __reduce_min_sync(0xffffffffu, cand);
            if (wmin != kNone && cand == wmin) {  // this lane holds the warp's lowest candidate
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (tid + j * bs != wmin) continue;
#pragma unroll
                    for (int v = 0; v < W; ++v) sm.crow[buf][warp][v] = row[j][v];
                }
            }
            if (lane == 0) sm.first[buf][warp] = wmin;
            __syncthreads();
            int p = lane < nwarps ? sm.first[buf][lane] : kNone;
            p = __reduce_min_sync(0xffffffffu, p);
            if (p == kNone) continue;  // no pivot in column c (uniform)
            const uint64_t* prow = sm.crow[buf][(p % bs) >> 5];
            if (tid == p % bs) {
                const int pj = p / bs;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (j != pj) continue;
                    used[j] = true;
                    my_k[j] = rank;
                }
            }
            if (tid == 0) sm.pivcol[rank] = c;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (tid + j * bs != p && ((row[j][w] >> b) & 1ull)) {
#pragma unroll
                    for (int v = 0; v < W; ++v) row[j][v] ^= prow[v];
                }
            }
            ++rank;
        }
    }
    const int r = rank;
    const int nb = r < HLF_MAX_VARYING ? r : HLF_MAX_VARYING;
    __syncthreads();  // all reads of the input rows in s_rows are done

    // ---- outputs of step (1): B_k in pivot order, pivots, enumeration table
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (!used[j]) continue;
        const int k = my_k[j];
#pragma unroll
        for (int v = 0; v < W; ++v) {
            s_rows[k * W + v] = row[j][v];
            if (o.basis) o.basis[(size_t)k * W + v] = row[j][v];
            if (k < HLF_MAX_VARYING) o.table[k * W + v] = row[j][v];
        }
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
        for (int k = lane; k < r; k += 32) {
            if ((s_rows[k * W + fw] >> fb) & 1ull) {
                const int pc = sm.pivcol[k];
                atomicOr(reinterpret_cast<unsigned long long*>(&sm.x[warp][pc >> 6]), 1ull << (pc & 63));
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
