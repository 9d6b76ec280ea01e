// Internal declarations shared by the kernels and the C ABI of libhlf.
//
// Device-side layout of one factorisation (all written by the factor kernel):
//   info  [16] int32   info[0] = status (hlf_status), info[1] = rank r; these
//                      live in pinned, device-mapped host memory, so the host
//                      reads them after an event without a copy
//   piv   [n]  int32   pivot columns p_0 < ... < p_{r-1}
//   basis [n][W]       B_0 .. B_{r-1}: the nonzero RREF rows in pivot order
//   table [66][W]      enumeration table: rows 0..64 hold B_0 .. B_63 with the
//                      rows k >= min(r, 64) zero (row 64 is always zero, it is
//                      the target of ctz = 64 steps), row 65 holds z0.
//   ptable [66][W]     the same layout for the paper's own order: row k is
//                      T_0 ^ ... ^ T_k with T_l = A's column at pivot p_{r-1-l},
//                      so that the Gray walk over ptable visits the paper's
//                      binary counter order (see factor_impl.cuh).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "hlf.h"

namespace hlf {

// NVTX range around a host entry point (stage 1, stage 2, batched and
// served calls), so a profiler's timeline shows which call enqueued which
// kernels. Without a profiler attached a push and pop cost nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kTableRows = 65;      // B_0..B_64 (row 64 always zero)
constexpr int kTableZ0Row = 65;     // z0 follows the basis rows
constexpr int kTableTotalRows = 66;

struct FactorOut {
    uint64_t* basis;   // [n][W]
    int32_t* piv;      // [n]
    uint64_t* table;   // [66][W]
    int32_t* info;     // [16]
    uint64_t* ptable;  // [66][W] or null: the paper-order table (see factor_impl.cuh)
    int32_t* work;     // [kFactorWorkWords] device scratch of the n > 256 path (factor.cu), or null
};

constexpr int kFactorWorkWords = 64;

// ---------------------------------------------------------------- launchers
hlf_status launch_factor(const uint64_t* A, int n, int W, const FactorOut& o, cudaStream_t s);
hlf_status launch_reduce(const uint64_t* table, int W, uint64_t offset, uint64_t count,
                         hlf_reduce* out, cudaStream_t s);
hlf_status launch_reduce_chunks(const uint64_t* table, int W, uint64_t offset, uint64_t chunk,
                                uint64_t n_chunks, hlf_reduce* out, cudaStream_t s);
// out: 8-byte aligned at W = 1, 16-byte aligned at W > 1.
hlf_status launch_store(const uint64_t* table, int W, uint64_t offset, uint64_t count,
                        uint64_t* out, cudaStream_t s);
hlf_status launch_store_dense(const uint64_t* table, int n, uint64_t offset, uint64_t count, uint64_t* out,
                              cudaStream_t s);
hlf_status launch_histogram(const uint64_t* table, int W, uint64_t offset, uint64_t count, int lo, int nbits,
                            uint64_t* out, cudaStream_t s);
hlf_status launch_sample(const uint64_t* table, int W, int nb, const uint64_t* idx, uint64_t m,
                         uint64_t* out, int32_t* info, cudaStream_t s);

// Number of SMs of the current device (cached per device).
int sm_count();

// Lets the current device's default memory pool keep up to 1 GiB of freed
// handle memory (called before the first stream-ordered allocation).
void keep_pool_memory();

// Host-side fault injection (hlf_debug_fail_allocs): true if the calling
// entry point must fail its allocation with HLF_ERR_NOMEM; consumes one
// pending failure.
bool take_injected_alloc_failure();

// ----------------------------------------------------------- device helpers

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): the
// finalizer the reduce applies to every solution word.
__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

// Index of the lowest set bit; 64 for x == 0 (so the zero row 64 is used).
__device__ __forceinline__ int ctz64(uint64_t x) { return __clzll(__brevll(x)); }

// Record the first device-side fault in a status word.
__device__ __forceinline__ void set_status(int32_t* info, int code) { atomicCAS(info, 0, code); }

}  // namespace hlf
