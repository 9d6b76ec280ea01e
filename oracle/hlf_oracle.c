/*
 * Plain CPU oracle for the two-stage FS2D HLF scheme (arXiv 2103.00693).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only code that loads this library.
 * It shares no code, header, table or helper with the CUDA path: it has its
 * own elimination, its own bit packing and its own hash.
 *
 * Stage 1 -- the CLA module of Section 2 (Fig. 1(b)), one byte per bit:
 *   (1) Gauss-Jordan elimination of A over GF(2): pivot columns
 *       P = {p_1 < ... < p_r} (the leftmost maximal independent column set
 *       L_ind), rank r, and the reduced row echelon rows B_1..B_r;
 *   (2) a basis of Ker(A): one vector x_f per free (non-pivot) column f;
 *   (3) q(x_f) = x_f^T A x_f mod 4, as the integer double sum over i, j;
 *   (4) one solution z^a of 2 z^T x_f = q(x_f) (mod 4) for every f, made
 *       unique by also asking z_p = 0 for every pivot p; solved as a linear
 *       system over GF(2) by the same elimination.
 * Stage 2 -- the classical parallel circuit of Section 2 (Eqs. 1-3,
 * Fig. 1(c)), in uint64 words (bit j of word j/64 is z_{j+1}):
 *   solutions are z^a XOR y for y in Col(A) = Row(A) = span{B_k}; index i
 *   names z(i) = z^a XOR (XOR of B_{k+1} over the set bits k of g(i)), with
 *   g(i) = i ^ (i >> 1) the reflected Gray code. A window is made either index
 *   by index from that formula, or by Gray stepping z(i+1) = z(i) ^ B_{c+1},
 *   c = ctz(i+1). The reduce of a window is (count, XOR of all z, sum of the
 *   chained SplitMix64 finalizer of every z, mod 2^64).
 *   The paper's own order is also provided: a binary counter over
 *   R^(r) = R_{p_1} ... R_{p_r}, y = A R (Eq. 3), z = y XOR z^a.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_NOT_SYMMETRIC -3
#define ORC_ERR_RANGE -5
#define ORC_ERR_NOMEM -6
#define ORC_ERR_INCONSISTENT -9

int orc_version(void) { return 1; }

/* ---------------------------------------------------------------- hashing */

/* SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), the finalizer applied to the
 * state after each increment. */
uint64_t orc_mix64(uint64_t x)
{
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* Hash of one solution of W words: h = mix(w_0), then h = mix(h ^ w_j). */
static uint64_t chain_hash(const uint64_t* z, int W)
{
    uint64_t h = orc_mix64(z[0]);
    for (int j = 1; j < W; ++j) h = orc_mix64(h ^ z[j]);
    return h;
}

/* ------------------------------------------------------ GF(2) elimination */

/* Gauss-Jordan elimination over GF(2) of a rows x cols byte matrix, on its
 * first elim_cols columns: for each column c from left to right, take the
 * first row at or below the current rank with a 1 in column c, swap it up,
 * and clear column c in every other row. Returns the rank; piv[k] is the
 * column of the k-th pivot. */
static int rref_bytes(uint8_t* M, int rows, int cols, int elim_cols, int32_t* piv)
{
    int rank = 0;
    for (int c = 0; c < elim_cols && rank < rows; ++c) {
        int p = -1;
        for (int i = rank; i < rows; ++i)
            if (M[(size_t)i * cols + c]) { p = i; break; }
        if (p < 0) continue;
        if (p != rank) {
            for (int j = 0; j < cols; ++j) {
                uint8_t t = M[(size_t)p * cols + j];
                M[(size_t)p * cols + j] = M[(size_t)rank * cols + j];
                M[(size_t)rank * cols + j] = t;
            }
        }
        for (int i = 0; i < rows; ++i) {
            if (i == rank || !M[(size_t)i * cols + c]) continue;
            for (int j = 0; j < cols; ++j) M[(size_t)i * cols + j] ^= M[(size_t)rank * cols + j];
        }
        piv[rank++] = c;
    }
    return rank;
}

/* ------------------------------------------------------------- stage 1 */

/*
 * A: n*n bytes, each 0 or 1, row-major, A[i*n+j] = A_{i+1,j+1}.
 * Outputs (caller-allocated):
 *   piv[n]        pivot columns, first r valid, ascending
 *   R[n*n]        RREF of A; row k < r is B_{k+1}, rows >= r are zero
 *   X[n*n]        row j < n-r is the kernel vector x_f for f = free_cols[j]
 *   free_cols[n]  free columns, first n-r valid, ascending
 *   q[n]          q[j] = x_f^T A x_f mod 4 for f = free_cols[j]
 *   z0[n]         the particular solution z^a (zero on every pivot)
 * Returns r >= 0, or a negative ORC_ERR_* code.
 */
int orc_factor(const uint8_t* A, int n, int32_t* piv, uint8_t* R, uint8_t* X,
               int32_t* free_cols, int32_t* q, uint8_t* z0)
{
    if (!A || !piv || !R || !X || !free_cols || !q || !z0 || n < 1 || n > 8192) return ORC_ERR_ARG;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            uint8_t a = A[(size_t)i * n + j];
            if (a > 1) return ORC_ERR_ARG;
            if (a != A[(size_t)j * n + i]) return ORC_ERR_NOT_SYMMETRIC;
        }

    /* (1) pivots, rank and the RREF rows */
    memcpy(R, A, (size_t)n * n);
    int r = rref_bytes(R, n, n, n, piv);

    /* (2) kernel basis: x_f has a 1 at f, and at each pivot p_k the entry
     * that makes row k of the RREF vanish on it: B_k[f]. */
    uint8_t* is_piv = (uint8_t*)calloc((size_t)n, 1);
    if (!is_piv) return ORC_ERR_NOMEM;
    for (int k = 0; k < r; ++k) is_piv[piv[k]] = 1;
    memset(X, 0, (size_t)n * n);
    int nf = 0;
    for (int f = 0; f < n; ++f) {
        if (is_piv[f]) continue;
        free_cols[nf] = f;
        uint8_t* x = X + (size_t)nf * n;
        x[f] = 1;
        for (int k = 0; k < r; ++k) x[piv[k]] = R[(size_t)k * n + f];
        ++nf;
    }
    free(is_piv);

    /* (3) q(x) = sum_i sum_j A_ij x_i x_j, reduced mod 4 */
    for (int j = 0; j < nf; ++j) {
        const uint8_t* x = X + (size_t)j * n;
        long long s = 0;
        for (int a = 0; a < n; ++a) {
            if (!x[a]) continue;
            for (int b = 0; b < n; ++b) s += (long long)A[(size_t)a * n + b] * x[b];
        }
        q[j] = (int32_t)(s % 4);
    }

    /* (4) z^a: solve x_f . z = q(x_f)/2 (mod 2) for all f, with z_p = 0 on
     * every pivot, as an n x (n+1) augmented system. */
    uint8_t* M = (uint8_t*)calloc((size_t)n * (n + 1), 1);
    int32_t* piv2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!M || !piv2) { free(M); free(piv2); return ORC_ERR_NOMEM; }
    for (int j = 0; j < nf; ++j) {
        if (q[j] & 1) { free(M); free(piv2); return ORC_ERR_INCONSISTENT; }
        memcpy(M + (size_t)j * (n + 1), X + (size_t)j * n, (size_t)n);
        M[(size_t)j * (n + 1) + n] = (uint8_t)(q[j] / 2);
    }
    for (int k = 0; k < r; ++k) M[(size_t)(nf + k) * (n + 1) + piv[k]] = 1;
    int rk = rref_bytes(M, n, n + 1, n, piv2);
    if (rk != n) { free(M); free(piv2); return ORC_ERR_INCONSISTENT; }
    for (int c = 0; c < n; ++c) z0[c] = M[(size_t)c * (n + 1) + n]; /* identity on the left */
    free(M);
    free(piv2);
    return r;
}

/* ------------------------------------------------------------- stage 2 */

static int words_of(int n) { return (n + 63) / 64; }

static void pack_bits(const uint8_t* bits, int n, uint64_t* w)
{
    memset(w, 0, sizeof(uint64_t) * (size_t)words_of(n));
    for (int j = 0; j < n; ++j)
        if (bits[j]) w[j / 64] |= 1ULL << (j % 64);
}

/* Index space of the enumeration: i in [0, 2^min(r,64)). Checks that the
 * window [offset, offset + count) lies inside it. */
static int window_ok(int r, uint64_t offset, uint64_t count)
{
    if (r < 64) {
        uint64_t space = 1ULL << r;
        return offset <= space && count <= space - offset;
    }
    return count == 0 || count - 1 <= UINT64_MAX - offset;
}

/* The basis vectors that can vary at indices below 2^64, packed: rows
 * B_1..B_nb of the RREF, nb = min(r, 64), plus z^a. */
typedef struct {
    int n, W, nb;
    uint64_t* B;  /* [nb][W] */
    uint64_t* z0; /* [W] */
} packed_t;

static int pack_factor(const uint8_t* R, const uint8_t* z0, int n, int r, packed_t* p)
{
    p->n = n;
    p->W = words_of(n);
    p->nb = r < 64 ? r : 64;
    p->B = (uint64_t*)calloc((size_t)(p->nb ? p->nb : 1) * p->W, sizeof(uint64_t));
    p->z0 = (uint64_t*)calloc((size_t)p->W, sizeof(uint64_t));
    if (!p->B || !p->z0) { free(p->B); free(p->z0); return ORC_ERR_NOMEM; }
    for (int k = 0; k < p->nb; ++k) pack_bits(R + (size_t)k * n, n, p->B + (size_t)k * p->W);
    pack_bits(z0, n, p->z0);
    return ORC_OK;
}

static void unpack_free(packed_t* p) { free(p->B); free(p->z0); }

/* z(i) from its definition: z^a XOR the B_{k+1} selected by the bits of g(i). */
static void z_of_index(const packed_t* p, uint64_t i, uint64_t* out)
{
    uint64_t g = i ^ (i >> 1);
    for (int w = 0; w < p->W; ++w) out[w] = p->z0[w];
    for (int k = 0; k < p->nb; ++k)
        if ((g >> k) & 1)
            for (int w = 0; w < p->W; ++w) out[w] ^= p->B[(size_t)k * p->W + w];
}

static int ctz64(uint64_t x)
{
    int c = 0;
    while (!(x & 1)) { x >>= 1; ++c; }
    return c;
}

/* Window [offset, offset+count) by the direct formula, out[count][W]. */
int orc_window(const uint8_t* R, const uint8_t* z0, int n, int r, uint64_t offset, uint64_t count,
               uint64_t* out)
{
    if (!R || !z0 || (!out && count) || n < 1 || r < 0 || r > n) return ORC_ERR_ARG;
    if (!window_ok(r, offset, count)) return ORC_ERR_RANGE;
    packed_t p;
    if (pack_factor(R, z0, n, r, &p)) return ORC_ERR_NOMEM;
    for (uint64_t c = 0; c < count; ++c) z_of_index(&p, offset + c, out + c * (uint64_t)p.W);
    unpack_free(&p);
    return ORC_OK;
}

/* The same window by Gray stepping from a seed at `offset`. */
int orc_window_gray(const uint8_t* R, const uint8_t* z0, int n, int r, uint64_t offset,
                    uint64_t count, uint64_t* out)
{
    if (!R || !z0 || (!out && count) || n < 1 || r < 0 || r > n) return ORC_ERR_ARG;
    if (!window_ok(r, offset, count)) return ORC_ERR_RANGE;
    if (count == 0) return ORC_OK;
    packed_t p;
    if (pack_factor(R, z0, n, r, &p)) return ORC_ERR_NOMEM;
    uint64_t* z = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)p.W);
    if (!z) { unpack_free(&p); return ORC_ERR_NOMEM; }
    z_of_index(&p, offset, z);
    uint64_t i = offset;
    for (uint64_t c = 0; c < count; ++c) {
        memcpy(out + c * (uint64_t)p.W, z, sizeof(uint64_t) * (size_t)p.W);
        if (c + 1 < count) {
            ++i;
            int k = ctz64(i);
            for (int w = 0; w < p.W; ++w) z[w] ^= p.B[(size_t)k * p.W + w];
        }
    }
    free(z);
    unpack_free(&p);
    return ORC_OK;
}

typedef struct {
    const packed_t* p;
    uint64_t first, len;
    uint64_t count, hsum;
    uint64_t fold[128];
} reduce_part_t;

static void* reduce_part(void* arg)
{
    reduce_part_t* t = (reduce_part_t*)arg;
    const packed_t* p = t->p;
    uint64_t z[128];
    memset(t->fold, 0, sizeof(t->fold));
    t->count = 0;
    t->hsum = 0;
    if (t->len == 0) return NULL;
    z_of_index(p, t->first, z);
    uint64_t i = t->first;
    for (uint64_t c = 0; c < t->len; ++c) {
        t->count += 1;
        for (int w = 0; w < p->W; ++w) t->fold[w] ^= z[w];
        t->hsum += chain_hash(z, p->W);
        if (c + 1 < t->len) {
            ++i;
            int k = ctz64(i);
            for (int w = 0; w < p->W; ++w) z[w] ^= p->B[(size_t)k * p->W + w];
        }
    }
    return NULL;
}

/* Reduce of the window [offset, offset+count): res[0] = count,
 * res[1] = sum of chain_hash(z) mod 2^64, res[2..2+W) = XOR of all z.
 * The window is cut into `nthreads` contiguous parts, one per thread; the
 * three quantities are combined by +, + and XOR, which do not depend on the
 * order of the parts. */
int orc_reduce(const uint8_t* R, const uint8_t* z0, int n, int r, uint64_t offset, uint64_t count,
               int nthreads, uint64_t* res)
{
    if (!R || !z0 || !res || n < 1 || n > 8192 || r < 0 || r > n) return ORC_ERR_ARG;
    if (!window_ok(r, offset, count)) return ORC_ERR_RANGE;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    packed_t p;
    if (pack_factor(R, z0, n, r, &p)) return ORC_ERR_NOMEM;
    if ((uint64_t)nthreads > count) nthreads = count ? (int)count : 1;
    reduce_part_t* parts = (reduce_part_t*)calloc((size_t)nthreads, sizeof(reduce_part_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!parts || !th) { free(parts); free(th); unpack_free(&p); return ORC_ERR_NOMEM; }
    uint64_t base = count / (uint64_t)nthreads, extra = count % (uint64_t)nthreads, at = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t len = base + ((uint64_t)t < extra ? 1 : 0);
        parts[t].p = &p;
        parts[t].first = offset + at;
        parts[t].len = len;
        at += len;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, reduce_part, &parts[t]) != 0) break;
        started = t;
    }
    reduce_part(&parts[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) reduce_part(&parts[t]); /* threads that did not start */
    memset(res, 0, sizeof(uint64_t) * (size_t)(2 + p.W));
    for (int t = 0; t < nthreads; ++t) {
        res[0] += parts[t].count;
        res[1] += parts[t].hsum;
        for (int w = 0; w < p.W; ++w) res[2 + w] ^= parts[t].fold[w];
    }
    free(parts);
    free(th);
    unpack_free(&p);
    return ORC_OK;
}

/* The paper's order (Section 2, Eq. 3; the counter of Section 4): counter
 * value t in [t0, t0+count) sets R_{p_j} to bit (r - j) of t (R^(r) read as
 * a binary numeral, R_{p_1} most significant; a 64-bit counter has no bits at
 * or above 64, so for r > 64 the leading R_{p_j} stay 0), every other R_i to
 * 0; y_i = XOR_j A_ij R_j; z = y XOR z^a. Output out[count][W], packed. */
int orc_paper_order(const uint8_t* A, const int32_t* piv, int r, const uint8_t* z0, int n,
                    uint64_t t0, uint64_t count, uint64_t* out)
{
    if (!A || !piv || !z0 || (!out && count) || n < 1 || r < 0 || r > n) return ORC_ERR_ARG;
    if (!window_ok(r, t0, count)) return ORC_ERR_RANGE;
    int W = words_of(n);
    uint8_t* R = (uint8_t*)malloc((size_t)n);
    uint8_t* z = (uint8_t*)malloc((size_t)n);
    if (!R || !z) { free(R); free(z); return ORC_ERR_NOMEM; }
    for (uint64_t c = 0; c < count; ++c) {
        uint64_t t = t0 + c;
        memset(R, 0, (size_t)n);
        for (int j = 1; j <= r; ++j) R[piv[j - 1]] = r - j < 64 ? (uint8_t)((t >> (r - j)) & 1) : 0;
        for (int i = 0; i < n; ++i) {
            uint8_t y = 0;
            for (int j = 0; j < n; ++j) y ^= (uint8_t)(A[(size_t)i * n + j] & R[j]);
            z[i] = y ^ z0[i];
        }
        pack_bits(z, n, out + c * (uint64_t)W);
    }
    free(R);
    free(z);
    return ORC_OK;
}
