/*
 * hlf.h -- C ABI of the GB300 (sm_103a) solver for the full-sampling 2D
 * hidden linear function problem (FS2D HLF) of arXiv 2103.00693.
 *
 * Problem (Section 1): for a symmetric binary n x n matrix A, find every
 * z in {0,1}^n with q(x) = 2 z^T x (mod 4) for all x in Ker(A), where
 * q(x) = x^T A x (mod 4). The solutions form the affine space z^a + Col(A)
 * of 2^r elements, r the binary rank (Section 2).
 *
 * The library runs the paper's two stages on one GPU:
 *   stage 1 (the "CLA module" of Section 2, Fig. 1(b)) -- hlf_factor:
 *     GF(2) elimination of A -> rank r, pivot columns P, a basis of Col(A),
 *     q on a basis of Ker(A), and one particular solution z^a;
 *   stage 2 (the "classical parallel circuit" of Section 2, Eqs. 1-3,
 *     Fig. 1(c)) -- hlf_enumerate_*, hlf_sample: the solutions themselves.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Bit layout. A vector of n bits is W = ceil(n / 64) uint64 words; bit j
 *   (0-based; the paper's z_{j+1}) is bit (j % 64) of word j / 64. Padding
 *   bits (j >= n) are 0. A matrix is row-major [n][W]: bit j of row i is
 *   A_{i+1, j+1}.
 * Basis and order (a reading of Section 2, where the paper leaves both
 *   open). B_0 .. B_{r-1} are the nonzero rows of the reduced row echelon
 *   form of A, in increasing order of their pivot columns p_0 < ... < p_{r-1}
 *   (P is the leftmost maximal independent column set L_ind of Section 2).
 *   They span Row(A) = Col(A) = Ker(A)^perp. z^a (here z0) is the unique
 *   solution that is 0 on every pivot column. Solution number i is
 *       z(i) = z0 XOR  XOR_{k : bit k of g(i) is 1} B_k,   g(i) = i ^ (i >> 1),
 *   the reflected Gray code, so z(i+1) = z(i) ^ B_{ctz(i+1)} and z(i)
 *   restricted to P is g(i). Indices run over [0, 2^min(r, 64)): with
 *   r > 64 only B_0 .. B_63 vary (documented limit, not an error).
 * Memory. Every pointer named *_dev is device memory owned by the caller;
 *   every *_host pointer is host memory owned by the caller. The library
 *   owns an hlf_handle and the device buffers behind it until hlf_destroy.
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream). Work is enqueued asynchronously on it; calls that must
 *   read results on the host say so.
 * Errors. Every call returns an hlf_status and never throws or traps.
 *   Arguments are checked on the host before anything is enqueued. Faults
 *   found by a kernel (A not symmetric, padding bits set, an index outside
 *   the space) are written to the handle's device status word and returned
 *   by the next call that synchronises on the handle (hlf_get_rank,
 *   hlf_get_factor, hlf_get_status, and the first enumerate call after
 *   hlf_factor other than hlf_enumerate_store_upto, which does not wait).
 */
#ifndef HLF_H
#define HLF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hlf_status {
    HLF_OK = 0,
    HLF_ERR_ARG = 1,           /* null pointer, bad count, unknown option */
    HLF_ERR_SIZE = 2,          /* n outside [1, HLF_MAX_N] */
    HLF_ERR_NOT_SYMMETRIC = 3, /* A != A^T (the problem needs symmetric A, Section 1) */
    HLF_ERR_PADDING = 4,       /* a padding bit (column >= n) is set */
    HLF_ERR_RANGE = 5,         /* window or index outside [0, 2^min(r,64)) */
    HLF_ERR_NOMEM = 6,         /* device or host allocation failed */
    HLF_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
    HLF_ERR_CUDA = 8,          /* a CUDA runtime call failed */
    HLF_ERR_INTERNAL = 9       /* an invariant of the method failed (e.g. q odd on Ker(A)) */
} hlf_status;

#define HLF_MAX_N 1024      /* largest n (32 x 32 grids) */
#define HLF_MAX_W 16        /* words per row at HLF_MAX_N */
#define HLF_MAX_VARYING 64  /* basis vectors addressable by a 64-bit index */

/* Result of a reduce over a window: the number of solutions, the sum mod 2^64
 * of their hashes, and the XOR of all of them (words >= W are 0). The hash of
 * a solution with words w_0..w_{W-1} is h = mix(w_0), then h = mix(h ^ w_j),
 * with mix the SplitMix64 finalizer (Steele, Lea and Flood, OOPSLA 2014).
 * All three are independent of the order in which solutions are visited. */
typedef struct hlf_reduce {
    uint64_t count;
    uint64_t hsum;
    uint64_t xor_fold[HLF_MAX_W];
} hlf_reduce; /* 144 bytes */

typedef struct hlf_handle hlf_handle;

/* Text for a status code (static storage). */
const char* hlf_status_string(hlf_status s);

/* Number of CUDA devices visible, or -1 if the runtime cannot be reached. */
int32_t hlf_device_count(void);

/* Host-side fault injection for tests of a caller's failure paths (the
 * paper has no counterpart): the next `count` calls that allocate
 * (hlf_factor, hlf_many_create, hlf_batch_create) return HLF_ERR_NOMEM after
 * their argument checks, as if their host or device allocation had failed,
 * without touching the GPU. count = 0 clears it; count < 0 is HLF_ERR_ARG.
 * Process-wide, shared by all threads. */
hlf_status hlf_debug_fail_allocs(int32_t count);

/* The debug build (the paper has no counterpart; it stands in for a race and
 * bounds checker that this GPU pool does not offer). Built with -DHLF_DEBUG
 * (the Python binding loads that library when HLF_DEBUG=1), the kernels test
 * the index of every solution store against its output buffer and of their
 * shared-memory tables against the table; an access that would fall outside
 * is skipped and the first such event recorded on the device.
 * hlf_debug_violation synchronises the current device, writes that record to
 * *first and clears it: 0 if none, else 2^63 | site << 48 | (index mod 2^48),
 * the sites listed in the library's sources (1 = hlf_debug_bounds_probe).
 * *is_debug is 1 in a debug build, 0 in a release build (where *first is
 * always 0). HLF_ERR_ARG if a pointer is null; HLF_ERR_CUDA if the device
 * cannot be read. */
hlf_status hlf_debug_violation(uint64_t* first, int32_t* is_debug);

/* A check of the check: one device thread tests index i against [0, n) at
 * site 1 and touches no memory, so a test can see a failed check recorded
 * (debug build) or not (release build). Asynchronous on stream (a
 * cudaStream_t, 0 for the legacy stream). */
hlf_status hlf_debug_bounds_probe(int64_t i, int64_t n, void* stream);

/*
 * Stage 1, the CLA module (Section 2, steps (1)-(4); Fig. 1(b)).
 * A_dev:  [n][W] uint64, device, caller-owned; read until the factor kernel
 *         ends (i.e. in stream order), not retained.
 * n:      1 .. HLF_MAX_N.
 * stream: cudaStream_t the kernel is launched on.
 * *h:     receives a new handle (library-owned; free with hlf_destroy). Its
 *         few device buffers come from the device's stream-ordered memory
 *         pool (cudaMallocAsync on `stream`), so creating and destroying
 *         handles never synchronises the device.
 * Computes r, P, B_0..B_{r-1} and z0 on the device. Asynchronous: symmetry
 * and padding faults surface on the first synchronising call on *h.
 * Returns HLF_ERR_SIZE for bad n, HLF_ERR_ARG for null pointers,
 * HLF_ERR_NOMEM / HLF_ERR_CUDA when allocation or launch fails (then *h is
 * left NULL).
 */
hlf_status hlf_factor(const uint64_t* A_dev, int32_t n, void* stream, hlf_handle** h);

/* Waits for the factorisation of h and returns its binary rank in *r, or the
 * device-side fault (HLF_ERR_NOT_SYMMETRIC, HLF_ERR_PADDING, ...). */
hlf_status hlf_get_rank(hlf_handle* h, int32_t* r);

/* Waits for the factorisation and copies it to host memory (any pointer may
 * be NULL to skip it): piv_host[r] int32 pivot columns (0-based, ascending),
 * z0_host[W], basis_host[r][W] (B_k, row-major). */
hlf_status hlf_get_factor(hlf_handle* h, int32_t* piv_host, uint64_t* z0_host, uint64_t* basis_host);

/* Enumeration orders. HLF_ORDER_GRAY (the default) is the order of the
 * conventions above. HLF_ORDER_PAPER is the paper's own order (Section 2,
 * Eq. 3, with the binary counter of Section 4): index t sets
 * R_{p_j} = bit (r - j) of t (R^(r) = R_{p_1}..R_{p_r} read as a binary
 * numeral, R_{p_1} most significant; bits of t at or above 64 are 0), every
 * other R_i = 0, and the solution is y ^ z^a with y = A R over GF(2). Both
 * orders enumerate the same set: every index in [0, 2^min(r,64)) names one
 * solution, different indices name different solutions. */
#define HLF_ORDER_GRAY 0
#define HLF_ORDER_PAPER 1

/* Selects the order used by every later hlf_enumerate_*, hlf_sample and
 * hlf_enumerate_store_many call on h. Host-side only; takes effect for work
 * enqueued after it. */
hlf_status hlf_set_order(hlf_handle* h, int32_t order);

/* n and W of the handle's matrix. */
hlf_status hlf_get_shape(hlf_handle* h, int32_t* n, int32_t* W);

/* Waits for all work enqueued so far through h and returns its device status
 * word (HLF_OK if no kernel reported a fault), then clears it. */
hlf_status hlf_get_status(hlf_handle* h);

/*
 * Stage 2, materialised (Section 2, Fig. 1(c): the solutions y ^ z^a one by
 * one). Writes z(offset + t) to out_dev[t][0..W) for t in [0, count).
 * out_dev: device, caller-owned, count * W uint64, 16-byte aligned.
 * Requires offset + count <= 2^min(r, 64) (else HLF_ERR_RANGE, nothing
 * enqueued). count = 0 is a no-op. The first call after hlf_factor waits
 * for the factorisation (it needs r on the host).
 */
hlf_status hlf_enumerate_store(hlf_handle* h, uint64_t offset, uint64_t count, uint64_t* out_dev,
                               void* stream);

/*
 * Stage 2 for small instances, with no host round trip after hlf_factor
 * (Section 2, Eq. 3): out_dev[i][0..W) = z(i) for i < min(2^r, cap), the same
 * solutions in the same order as hlf_enumerate_store over that window. The
 * kernel reads r on the device from the factorisation; nothing is written if
 * the factorisation failed. The number written is min(2^r, cap) with r from
 * hlf_get_rank, which returns at once once `stream` has been synchronised.
 * Work on `stream` first waits for the factor kernel's stream.
 * out_dev: device, caller-owned, cap * W uint64, 8-byte aligned. Requires
 * cap <= HLF_STORE_UPTO_MAX (else HLF_ERR_ARG). Each solution is computed
 * from its index with up to r row XORs, so large windows belong to
 * hlf_enumerate_store.
 */
#define HLF_STORE_UPTO_MAX (1ull << 24)
hlf_status hlf_enumerate_store_upto(hlf_handle* h, uint64_t cap, uint64_t* out_dev, void* stream);

/*
 * Stage 2 reduced for small instances, with no host round trip after
 * hlf_factor: *red_dev (device, one hlf_reduce, overwritten) is the reduce
 * of [0, min(2^min(r,64), cap)), equal to hlf_enumerate_reduce over that
 * window, with r read on the device from the factorisation (all zero if the
 * factorisation failed; the fault is reported by hlf_get_status). Work on
 * `stream` first waits for the factor kernel's stream. The grid is sized for
 * cap, so a cap far above 2^r leaves threads idle.
 */
hlf_status hlf_enumerate_reduce_upto(hlf_handle* h, uint64_t cap, hlf_reduce* red_dev, void* stream);

/*
 * Stage 2, materialised densely: the same solutions as hlf_enumerate_store,
 * n bits each, back to back. Solution z(offset + t) occupies bits
 * [t*n, (t+1)*n) of the stream at out_dev, where stream bit b is bit b % 64
 * of word b / 64 and solution bit j is z_{j+1}. Bits past the last solution
 * in the last word are written as 0.
 * out_dev: device, caller-owned, ceil(count * n / 64) uint64, 8-byte aligned
 * (a 16-byte aligned out_dev is written with bulk TMA stores, which is
 * faster). Same range rule as hlf_enumerate_store. For n = 36 this writes 36
 * bits per solution instead of 64.
 */
hlf_status hlf_enumerate_store_dense(hlf_handle* h, uint64_t offset, uint64_t count, uint64_t* out_dev,
                                     void* stream);

/*
 * Stage 2, reduced on the device: *red_dev (device, caller-owned, one
 * hlf_reduce) is overwritten with (count, hash sum, XOR-fold) of the window
 * [offset, offset + count). Same range rule as hlf_enumerate_store.
 */
hlf_status hlf_enumerate_reduce(hlf_handle* h, uint64_t offset, uint64_t count, hlf_reduce* red_dev,
                                void* stream);

/*
 * Stage 2, counted into a histogram: hist_dev[v] (device, 2^nbits uint64,
 * overwritten) is the number of solutions of the window [offset,
 * offset + count) whose bits bit_lo .. bit_lo + nbits - 1 (bit j is z_{j+1};
 * bit bit_lo is the least significant bit of v) have value v. These are the
 * output distributions of the paper's Figs. 3, 6 and 7, where each square
 * counts one pattern of the first or last bits of z. Requires
 * 1 <= nbits <= HLF_HIST_MAX_BITS and bit_lo + nbits <= n (else HLF_ERR_ARG);
 * same range rule as hlf_enumerate_store. No solution is stored.
 */
#define HLF_HIST_MAX_BITS 20
hlf_status hlf_enumerate_histogram(hlf_handle* h, uint64_t offset, uint64_t count, int32_t bit_lo, int32_t nbits,
                                   uint64_t* hist_dev, void* stream);

/*
 * Stage 2, reduced per chunk: red_dev[c] (device, n_chunks entries) is
 * overwritten with the reduce of [offset + c*chunk, offset + (c+1)*chunk).
 * Requires chunk >= 1 and offset + n_chunks*chunk <= 2^min(r, 64) without
 * overflow. The chunks combine (+, +, XOR) to the reduce of the whole range.
 */
hlf_status hlf_enumerate_reduce_chunks(hlf_handle* h, uint64_t offset, uint64_t chunk,
                                       uint64_t n_chunks, hlf_reduce* red_dev, void* stream);

/*
 * Stage 2 at chosen indices: out_dev[t][0..W) = z(idx_dev[t]) for t < m.
 * idx_dev: device uint64[m]; out_dev: device uint64[m][W]. An index outside
 * the space yields an all-zero row and sets HLF_ERR_RANGE in the handle's
 * status word (reported by hlf_get_status).
 */
hlf_status hlf_sample(hlf_handle* h, const uint64_t* idx_dev, uint64_t m, uint64_t* out_dev,
                      void* stream);

/* Frees the handle. Its device buffers (allocated stream-ordered on the
 * stream given to hlf_factor) are released in stream order after the last
 * work enqueued through the handle; the host does not wait. If every call
 * used one stream, the release is enqueued on that stream (a free, which
 * delays nothing that follows); otherwise on a library stream that waits for
 * each stream's last use. NULL is accepted. */
hlf_status hlf_destroy(hlf_handle* h);

/* ------------------------------------------------------------ many windows
 * Continuous batching for a request loop: windows of several factorisations
 * (any n and W) materialised in ONE launch. Each window is exactly what
 * hlf_enumerate_store writes; only the scheduling is shared.
 */
typedef struct hlf_many hlf_many;

/* Plan for up to max_windows windows per call: two descriptor buffers on the
 * device and two in pinned host memory (about 100 B per window each). */
hlf_status hlf_many_create(int32_t max_windows, hlf_many** m);

/*
 * For j < k: writes z(offsets[j] + t) of handle hs[j] to outs_dev[j][t][0..W_j)
 * for t < counts[j]. hs, offsets, counts and outs_dev are host arrays; each
 * outs_dev[j] is device memory, 16-byte aligned, counts[j] * W_j words.
 * Every window must lie inside its handle's index space (else HLF_ERR_RANGE,
 * nothing enqueued). Waits for the handles' factorisations (their ranks are
 * needed on the host) and for the call before last on this plan (its host
 * staging buffer is reused); otherwise asynchronous on `stream`.
 */
hlf_status hlf_enumerate_store_many(hlf_many* m, hlf_handle* const* hs, const uint64_t* offsets,
                                    const uint64_t* counts, uint64_t* const* outs_dev, int32_t k, void* stream);

/* Frees the plan (waits for its launches). NULL is accepted. */
hlf_status hlf_many_destroy(hlf_many* m);

/* ------------------------------------------------------------------ batched
 * Many independent matrices (the batched workload: thousands of grids of
 * uneven n) factored (stage 1) and enumerated (stage 2) by persistent kernel
 * launches. CTAs pull work items from an on-device queue: one factorisation
 * per matrix, and fixed-size chunks of each matrix's index space; in the
 * fused launch a chunk waits, with a bounded number of polls, for its
 * matrix's factorisation. The paper has no batched mode: this is the same
 * arithmetic as hlf_factor + hlf_enumerate_reduce / hlf_enumerate_store,
 * scheduled across matrices. Each item is worked on by one CTA of 2, 4 or 8
 * warps (hlf_batch_set_tiles).
 *
 * Two forms:
 *   hlf_factor_batched, then hlf_enumerate_batched: the ragged batch is
 *     given as ONE packed buffer and an offsets table of count + 1 entries;
 *     the factorisations stay resident in the plan between the calls, so one
 *     factorisation can be enumerated several times (reduced, then stored);
 *   hlf_batch_factor_reduce: factor and reduce in one launch (word offset
 *     and n per matrix), the shape the batched benchmark times.
 */

#define HLF_BATCH_MAX_N 256 /* largest n in a batch */

typedef struct hlf_batch hlf_batch;

/* Creates a batch plan with device workspace for up to max_instances
 * matrices (per matrix: a 66 x 4-word table, status, rank, n, a ready flag;
 * about 2.1 KiB). The plan is bound to the current device. */
hlf_status hlf_batch_create(int32_t max_instances, hlf_batch** b);

/* Launch shape, chosen by the autotuner: warps per work item (2, 4 or 8: the
 * CTA size; a CTA of 32w threads holds 8/w rows of a matrix per thread),
 * CTAs per SM (0 = as many as fit) and solutions per chunk item (a power of
 * two >= 256). Default: 8 warps, as many CTAs as fit, 2^16. Results do not
 * depend on the shape. */
hlf_status hlf_batch_set_tiles(hlf_batch* b, int32_t warps_per_item, int32_t ctas_per_sm, uint64_t chunk);

/* Bound on the polls a chunk makes while waiting for its matrix (default
 * 2^23 polls of >= 128 ns); past it the chunk is skipped and the batch status
 * becomes HLF_ERR_TIMEOUT. */
hlf_status hlf_batch_set_spin_limit(hlf_batch* b, uint32_t polls);

/* Fault injection for tests of the bounded waits: flags = 1 makes the next
 * launches skip every factorisation item, so no chunk's matrix ever becomes
 * ready and every wait runs out (HLF_ERR_TIMEOUT, results left unwritten).
 * flags = 0 restores normal operation. No GPU fault is involved. */
hlf_status hlf_batch_set_debug(hlf_batch* b, uint32_t flags);

/*
 * Stage 1 of `count` matrices in one launch (Section 2, steps (1)-(4), per
 * matrix), enqueued on `stream` with no host synchronisation.
 *   A_dev        device, all matrices' rows back to back: matrix b is the
 *                words [offsets_dev[b], offsets_dev[b+1]) of A_dev, [n_b][W_b]
 *                with W_b = ceil(n_b / 64). n_b is read from the size
 *                (n * ceil(n/64) words determines n); a size that fits no
 *                n in [1, HLF_BATCH_MAX_N] fails that matrix alone with
 *                HLF_ERR_SIZE.
 *   offsets_dev  device int64[count + 1], nondecreasing, offsets_dev[0] the
 *                first matrix's word offset.
 *   r_dev        device int32[count]: the rank, or -(hlf_status) if that
 *                matrix failed (not symmetric, padding, size).
 * The factorisations stay in the plan until its next factor or fused call.
 * Host-side errors: HLF_ERR_ARG (bad pointers, count > max_instances, plan
 * made on another device).
 */
hlf_status hlf_factor_batched(hlf_batch* b, const uint64_t* A_dev, const int64_t* offsets_dev, int32_t count,
                              int32_t* r_dev, void* stream);

/*
 * Stage 2 of the matrices of the plan's last hlf_factor_batched (or
 * hlf_batch_factor_reduce) call, in one launch: for each matrix b with rank
 * r_b, the solutions z(i), i < total_b = min(2^min(r_b, 64), cap), in the
 * Gray order of the conventions above. Exactly one of:
 *   red_dev  device hlf_reduce[count], overwritten with each matrix's
 *            (count, hash sum, XOR-fold) over [0, total_b);
 *   out_dev + out_offsets_dev  device: matrix b writes z(i) for
 *            i < min(total_b, room_b) to out_dev + out_offsets_dev[b] + i*W_b,
 *            W_b words each, where room_b = (out_offsets_dev[b+1] -
 *            out_offsets_dev[b]) / W_b (an int64[count + 1] offsets table of
 *            the caller's output buffer, 8-byte aligned words).
 * A matrix whose factorisation failed is skipped (its reduce reads 0).
 * Host-side errors: HLF_ERR_ARG (no factorisation in the plan, both or
 * neither output given), HLF_ERR_RANGE (cap needs more than 2^20 chunks).
 */
hlf_status hlf_enumerate_batched(hlf_batch* b, uint64_t cap, hlf_reduce* red_dev, uint64_t* out_dev,
                                 const int64_t* out_offsets_dev, void* stream);

/*
 * Factor and reduce `count` matrices in ONE launch (plus three memsets), all
 * enqueued on `stream` with no host synchronisation (so it can be captured in
 * a CUDA graph). The same results as hlf_factor_batched followed by
 * hlf_enumerate_batched with red_dev; the input is described per matrix
 * instead of by an offsets table:
 *   A_dev        device, the matrices' rows back to back: matrix b is
 *                [n_b][W_b] words starting at word word_off_dev[b].
 *   word_off_dev device int64[count]; n_dev device int32[count], each n_b in
 *                [1, HLF_BATCH_MAX_N] (others fail alone with HLF_ERR_SIZE).
 *   cap          each matrix reduces its solutions [0, min(2^min(r,64), cap)).
 *   r_dev        device int32[count]: the rank, or -(hlf_status) if that
 *                matrix failed (not symmetric, padding, size).
 *   red_dev      device hlf_reduce[count], overwritten.
 * The factorisations stay in the plan, as after hlf_factor_batched.
 * Host-side errors: HLF_ERR_ARG (bad pointers, count > max_instances, plan
 * made on another device), HLF_ERR_RANGE (too many work items).
 */
hlf_status hlf_batch_factor_reduce(hlf_batch* b, const uint64_t* A_dev, const int64_t* word_off_dev,
                                   const int32_t* n_dev, int32_t count, uint64_t cap, int32_t* r_dev,
                                   hlf_reduce* red_dev, void* stream);

/* Waits for the plan's last launch and returns its status word (HLF_OK, or
 * HLF_ERR_TIMEOUT if a bounded wait gave up), then clears it. */
hlf_status hlf_batch_get_status(hlf_batch* b);

/* Frees the plan (waits for its last launch). NULL is accepted. */
hlf_status hlf_batch_destroy(hlf_batch* b);

/*
 * hlf_batch_factor_reduce without allocating anything (the paper has no
 * counterpart; this exists for callers, not for the method).
 *
 * Some callers cannot call cudaMalloc when they need this work done: a host
 * application that owns all device memory and hands a plugin only its input
 * and output pointers; a framework whose memory pool has already reserved the
 * device; a latency-critical loop that must not risk the device-wide
 * synchronisation cudaMalloc and cudaFree can cause. This entry point needs no
 * plan: its workspace is a fixed array in the library's device image, sized
 * for HLF_BATCH_NOALLOC_MAX matrices (about 2.1 MiB), which every GPU that
 * loads the library holds until the process exits. It never calls cudaMalloc,
 * cudaFree or any allocating routine.
 *
 * Arguments, layout and results are those of hlf_batch_factor_reduce with the
 * default launch shape (8 warps per work item; CTAs per SM: as many as fit;
 * 2^16 solutions per work item; 2^23 polls per wait). count > HLF_BATCH_NOALLOC_MAX returns
 * HLF_ERR_SIZE and enqueues nothing. A bounded wait that runs out cannot be
 * reported separately here; it shows as red_dev[b].count below
 * min(2^r_b, cap), which a caller checks to detect it.
 *
 * The first call on each device looks up the workspace's device address
 * (with that device current). CUDA loads a library's device code lazily by
 * default, so that first call may also load the module and reserve the
 * workspace, which can allocate and synchronise: make one call (a warm-up
 * with count = 1 is enough) before the region that must not allocate, and
 * before any stream capture. Later calls allocate nothing. Every call shares the one workspace, and each call clears what must
 * start at zero, so calls whose work overlaps on the GPU (on different streams,
 * or from different host threads) race and give wrong results: issue them in
 * one stream order.
 */
#define HLF_BATCH_NOALLOC_MAX 1024
hlf_status hlf_batch_factor_reduce_noalloc(const uint64_t* A_dev, const int64_t* word_off_dev,
                                           const int32_t* n_dev, int32_t count, uint64_t cap, int32_t* r_dev,
                                           hlf_reduce* red_dev, void* stream);

/* ------------------------------------------------------------ measurement
 * Not part of the method (the paper has no counterpart): a microbenchmark
 * whose rate is the denominator of the histogram's roofline. One wave of CTAs
 * in which every thread performs `iters` 32-bit shared-memory atomic adds,
 * the 32 lanes of a warp on 32 distinct banks (the pattern of
 * hlf_enumerate_histogram's interleaved walk when its lanes land in distinct
 * bins). *sum_dev (device, one uint64, overwritten) receives the total of all
 * counters, which equals *atomics (host), the number of atomics the launch
 * performs. Time the launch with events on `stream`. iters must be a
 * positive multiple of 16 (else HLF_ERR_ARG).
 */
hlf_status hlf_probe_smem_atomics(uint32_t iters, uint64_t* sum_dev, uint64_t* atomics, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HLF_H */
