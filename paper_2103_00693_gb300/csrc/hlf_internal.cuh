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

// ---------------------------------------------------------------- debug build
// Bounds checks of the debug build (compiled with -DHLF_DEBUG, the library
// the binding loads when HLF_DEBUG=1): a failed check skips the access it
// guards and records the first failure, 2^63 | (site << 48) | (index mod
// 2^48), in a device word of its translation unit; hlf_debug_violation reads
// and clears the words of all of them. Release builds compile every check to
// `true`. The sites:
enum DebugSite : int {
    kSiteProbe = 1,      // hlf_debug_bounds_probe
    kSiteStore = 2,      // store_kernel, sample_kernel: solution words vs count * W
    kSiteManyStore = 3,  // many_kernel: solution words vs the window's count * W
    kSiteUptoStore = 4,  // store_upto_kernel: solution words vs cap * W
    kSiteBatchStore = 5, // batch_kernel store items: words vs the instance's output
    kSiteDenseStore = 6, // dense kernels: stream words vs the stream's length
    kSiteFactorSmem = 7, // factor: panel tables, pivot lists, basis rows
    kSiteFactorKvec = 8, // factor_kvec_kernel: mask words, x_f words, table words
    kSiteHistBin = 9,    // histogram kernels: bins vs the bin count
};

#ifdef HLF_DEBUG
static __device__ unsigned long long g_hlf_violation;  // one per translation unit

__device__ __forceinline__ bool debug_in_bounds(long long i, long long n, int site)
{
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_hlf_violation, 0ull,
              (1ull << 63) | ((unsigned long long)site << 48) | ((unsigned long long)i & ((1ull << 48) - 1)));
    return false;
}
#define HLF_IN_BOUNDS(i, n, site) ::hlf::debug_in_bounds((long long)(i), (long long)(n), (site))
// [i, i + len) inside [0, n)
#define HLF_RANGE_IN_BOUNDS(i, len, n, site) \
    (HLF_IN_BOUNDS((i), (n), (site)) && HLF_IN_BOUNDS((long long)(i) + (long long)(len) - 1, (n), (site)))
// the host side of a translation unit's word: read it and clear it
#define HLF_DEBUG_TAKE(name)                                                                   \
    uint64_t debug_take_##name()                                                               \
    {                                                                                          \
        unsigned long long v = 0, z = 0;                                                       \
        if (cudaMemcpyFromSymbol(&v, g_hlf_violation, sizeof v) != cudaSuccess) return ~0ull;  \
        cudaMemcpyToSymbol(g_hlf_violation, &z, sizeof z);                                     \
        return v;                                                                              \
    }
constexpr bool kDebugBuild = true;
#else
#define HLF_IN_BOUNDS(i, n, site) true
#define HLF_RANGE_IN_BOUNDS(i, len, n, site) true
#define HLF_DEBUG_TAKE(name) \
    uint64_t debug_take_##name() { return 0; }
constexpr bool kDebugBuild = false;
#endif
// one per translation unit with checks (defined there by HLF_DEBUG_TAKE)
uint64_t debug_take_api();
uint64_t debug_take_enumerate();
uint64_t debug_take_many();
uint64_t debug_take_upto();
uint64_t debug_take_batch();
uint64_t debug_take_dense();
uint64_t debug_take_factor();
uint64_t debug_take_hist();

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
