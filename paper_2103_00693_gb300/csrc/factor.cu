// Stage 1 of the two-stage scheme: the CLA module of Section 2 (Fig. 1(b)),
// steps (1)-(4), on one CTA per matrix.
//
//   (1) Gauss-Jordan elimination of A over GF(2). Thread i owns row i of A in
//       registers (W uint64 words). For each column c, left to right, the
//       candidates are the rows not yet used as a pivot that have bit c set;
//       a warp ballot plus a min over warps picks the lowest such row p. Row p
//       is broadcast through shared memory and every other row with bit c set
//       XORs it in (rows above and below: Gauss-Jordan, so the result is the
//       unique reduced row echelon form). Rows are never swapped; the pivot
//       row of column c is remembered instead. Unused rows end at zero.
//   (2)-(4) Kernel basis, q and z^a. For a free column f the kernel vector is
//       x_f = e_f + sum_k B_k[f] e_{p_k}; q(x_f) = sum over i in supp(x_f) of
//       popcount(A_i & x_f), mod 4, which is x_f^T A x_f mod 4. With z^a
//       chosen to vanish on the pivots, z^a . x_f = z^a_f, so the equation
//       2 z^T x_f = q(x_f) (mod 4) gives z^a_f = q(x_f) / 2 directly.
//
// Also checked on the device: padding bits (column >= n) are zero and A is
// symmetric (Section 1 defines the problem for symmetric A only).

#include <cstdio>

#include "hlf_internal.cuh"

namespace hlf {
namespace {

constexpr int kNone = 0x7fffffff;

template <int W>
__global__ void __launch_bounds__(1024) factor_kernel(const uint64_t* __restrict__ A, int n, FactorOut o)
{
    extern __shared__ uint64_t s_rows[];  // [n][W]: input rows, later B_k in pivot order
    __shared__ int s_first[2][32];
    __shared__ uint64_t s_prow[2][W];
    __shared__ int s_pivcol[HLF_MAX_N];
    __shared__ uint32_t s_pivmask[HLF_MAX_N / 32];
    __shared__ uint64_t s_x[32][W];
    __shared__ uint64_t s_z0[W];
    __shared__ int s_err;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;

    uint64_t row[W];
#pragma unroll
    for (int w = 0; w < W; ++w) row[w] = tid < n ? A[(size_t)tid * W + w] : 0ull;
    if (tid < n) {
#pragma unroll
        for (int w = 0; w < W; ++w) s_rows[tid * W + w] = row[w];
    }
    if (tid == 0) s_err = 0;
    if (tid < W) s_z0[tid] = 0;
    for (int i = tid; i < HLF_MAX_N / 32; i += blockDim.x) s_pivmask[i] = 0;
    __syncthreads();

    // ---- input checks: padding, then symmetry (bit j of row i == bit i of row j)
    int bad = 0;
    if (tid < n) {
        const int tail = n & 63;
        if (tail && (row[W - 1] >> tail)) bad = HLF_ERR_PADDING;
        const int wi = tid >> 6;
        const int bi = tid & 63;
        if (!bad) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t t = 0;
                for (int b = 0; b < 64; ++b) {
                    const int j = (w << 6) + b;
                    if (j >= n) break;
                    t |= ((s_rows[j * W + wi] >> bi) & 1ull) << b;
                }
                if (t != row[w]) bad = HLF_ERR_NOT_SYMMETRIC;
            }
        }
    }
    if (bad) atomicMax(&s_err, bad);
    __syncthreads();
    if (s_err) {
        if (tid == 0) {
            o.info[0] = s_err;
            o.info[1] = -1;
        }
        return;
    }

    // ---- (1) Gauss-Jordan elimination
    bool used = false;
    int my_k = -1;
    int rank = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        for (int b = 0; b < 64; ++b) {
            const int c = (w << 6) + b;
            if (c >= n) break;
            const int buf = c & 1;
            const bool cand = tid < n && !used && ((row[w] >> b) & 1ull);
            const unsigned m = __ballot_sync(0xffffffffu, cand);
            if (lane == 0) s_first[buf][warp] = m ? (warp << 5) + __ffs(m) - 1 : kNone;
            __syncthreads();
            int p = lane < nwarps ? s_first[buf][lane] : kNone;
            p = __reduce_min_sync(0xffffffffu, p);
            if (p == kNone) continue;  // no pivot in column c (uniform)
            if (tid == p) {
#pragma unroll
                for (int v = 0; v < W; ++v) s_prow[buf][v] = row[v];
                used = true;
                my_k = rank;
            }
            if (tid == 0) s_pivcol[rank] = c;
            __syncthreads();
            if (tid != p && ((row[w] >> b) & 1ull)) {
#pragma unroll
                for (int v = 0; v < W; ++v) row[v] ^= s_prow[buf][v];
            }
            ++rank;
        }
    }
    const int r = rank;
    const int nb = r < HLF_MAX_VARYING ? r : HLF_MAX_VARYING;
    __syncthreads();  // all reads of the input rows in s_rows are done

    // ---- outputs of step (1): B_k in pivot order, pivots, enumeration table
    if (used) {
#pragma unroll
        for (int v = 0; v < W; ++v) {
            s_rows[my_k * W + v] = row[v];
            o.basis[(size_t)my_k * W + v] = row[v];
            if (my_k < HLF_MAX_VARYING) o.table[my_k * W + v] = row[v];
        }
    }
    for (int i = nb * W + tid; i < kTableRows * W; i += blockDim.x) o.table[i] = 0ull;
    for (int k = tid; k < r; k += blockDim.x) {
        const int c = s_pivcol[k];
        o.piv[k] = c;
        atomicOr(&s_pivmask[c >> 5], 1u << (c & 31));
    }
    __syncthreads();

    // ---- (2)-(4): one warp per free column f
    int err = 0;
    for (int f = warp; f < n; f += nwarps) {
        if ((s_pivmask[f >> 5] >> (f & 31)) & 1u) continue;  // pivot column (uniform per warp)
        const int fw = f >> 6;
        const int fb = f & 63;
        if (lane < W) s_x[warp][lane] = lane == fw ? (1ull << fb) : 0ull;
        __syncwarp();
        for (int k = lane; k < r; k += 32) {
            if ((s_rows[k * W + fw] >> fb) & 1ull) {
                const int pc = s_pivcol[k];
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
        if (lane == 0 && (q >> 1))
            atomicOr(reinterpret_cast<unsigned long long*>(&s_z0[fw]), 1ull << fb);
        __syncwarp();
    }
    if (err) atomicMax(&s_err, err);
    __syncthreads();
    if (tid < W) o.table[kTableZ0Row * W + tid] = s_z0[tid];
    if (tid == 0) {
        o.info[0] = s_err;
        o.info[1] = r;
    }
}

template <int W>
hlf_status launch_factor_w(const uint64_t* A, int n, const FactorOut& o, cudaStream_t s)
{
    const int threads = ((n + 31) / 32) * 32;
    const size_t smem = (size_t)n * W * sizeof(uint64_t);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(factor_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 HLF_MAX_N * HLF_MAX_W * (int)sizeof(uint64_t)) != cudaSuccess)
            return HLF_ERR_CUDA;
        attr_set[dev] = true;
    }
    factor_kernel<W><<<1, threads, smem, s>>>(A, n, o);
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
    case 9: return launch_factor_w<9>(A, n, o, s);
    case 10: return launch_factor_w<10>(A, n, o, s);
    case 11: return launch_factor_w<11>(A, n, o, s);
    case 12: return launch_factor_w<12>(A, n, o, s);
    case 13: return launch_factor_w<13>(A, n, o, s);
    case 14: return launch_factor_w<14>(A, n, o, s);
    case 15: return launch_factor_w<15>(A, n, o, s);
    case 16: return launch_factor_w<16>(A, n, o, s);
    default: return HLF_ERR_SIZE;
    }
}

}  // namespace hlf
