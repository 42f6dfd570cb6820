/*
 * mpgemm.h -- C ABI of the GB300 multiple-precision GEMM / LU library
 * (libmpgemm.so).  Method: arXiv 1410.1599 (Kouya), "Accelerated Multiple
 * Precision Matrix Multiplication using Strassen's Algorithm and Winograd's
 * Variant".
 *
 * Number format (Sec. 1 and Sec. 3: binary floating point with a p-bit
 * mantissa, every operation correctly rounded, as in MPFR):
 *
 *     x = (-1)^sign * f * 2^exp,   f = sum_k limb[k] * 2^(-64(k+1)) in [1/2, 1)
 *
 *   - p (the precision, "prec") is any integer in [MP_PREC_MIN, MP_PREC_MAX];
 *     a number has L = ceil(p/64) 64-bit limbs, limb 0 most significant, and
 *     the 64L - p low bits of the last limb are zero;
 *   - zero is exp == MP_EXP_ZERO with all limbs zero, and keeps its sign;
 *   - every add, subtract, multiply and divide returns the exact result
 *     rounded once to p bits, ties to even; zero signs follow IEEE 754
 *     (x - x = +0, (-0) + (-0) = -0, the sign of a product is the xor);
 *   - nonzero exponents must lie in [-2^62, 2^62]; a result outside that
 *     range is reported as MP_ERR_RANGE by mp_sync_status().
 *
 * Matrix layout (structure of arrays in device memory), element (r, c):
 *     limb k : limb[k * plane + r * ld + c]      (uint64)
 *     exp    : exp[r * ld + c]                   (int64)
 *     sign   : sign[r * ld + c]                  (int8, 0 = +, 1 = -)
 * with ld >= cols and plane >= rows * ld.  All pointers are device
 * pointers owned by the caller; the library never frees them and keeps
 * no reference after a call returns.
 *
 * Calls are ordered on the calling thread's current stream (mp_set_stream;
 * default: the legacy default stream) and return once the work is enqueued.
 * They return MP_OK or a negative MP_ERR_* code for argument and launch
 * errors.  Conditions found on the device (range overflow, a zero pivot)
 * are read back by mp_sync_status(), which synchronises the stream.
 *
 * Library-owned memory: Strassen/Winograd and LU need a workspace.  It is
 * taken from the buffer given to mp_set_workspace() when that is large
 * enough (mpgemm_workspace_size() says how large), else allocated and
 * freed stream-ordered by the library (cudaMallocAsync / cudaFreeAsync).
 */
#ifndef MPGEMM_H
#define MPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MP_EXP_ZERO  INT64_MIN
#define MP_PREC_MIN  2
#define MP_PREC_MAX  8704       /* Sec. 4 runs its ill-conditioned LU at 8192 and 8650 bits */
#define MP_PREC_EXACT_MAX 2048  /* MP_EXACT and MP_SPLIT: MP_ERR_UNSUPPORTED above */

typedef struct mpmat {
    int32_t   prec;      /* p, the mantissa precision in bits */
    int32_t   reserved;  /* must be 0 */
    int64_t   rows, cols;
    int64_t   ld;        /* elements between consecutive rows, >= cols */
    int64_t   plane;     /* elements between limb planes, >= rows * ld */
    uint64_t *limb;      /* device: L planes, limb 0 most significant */
    int64_t  *exp;       /* device: exponents, MP_EXP_ZERO for zero */
    int8_t   *sign;      /* device: 0 = +, 1 = - */
} mpmat_t;

/* GEMM algorithms (Sec. 2) */
enum {
    MP_SIMPLE   = 0,   /* Eq. 1: c_ij = sum_k a_ik b_kj, k ascending */
    MP_BLOCK    = 1,   /* Eq. 2: blocked, same k-ascending sequence per c_ij */
    MP_STRASSEN = 2,   /* Strassen's P1..P7 recursion */
    MP_WINOGRAD = 3,   /* Winograd's variant, S1..S8 / M1..M7 / T1, T2 */
    MP_EXACT    = 4,   /* every c_ij the exact dot product, rounded once (the
                          accuracy reference of Sec. 3's error tables; the
                          result of the split form) */
    MP_SPLIT    = 5    /* the same result as MP_EXACT by the split form: rows of
                          A / columns of B aligned to their largest exponent,
                          cut into signed 8-bit digits, digit products on
                          tensor cores (exact integer fp16 x fp16 -> fp32
                          chunks folded into int64), exact recombination, one
                          rounding; rows/columns whose exponents spread more
                          than 64 bits are computed by the MP_EXACT kernel.
                          By default the lowest weight diagonals of digit
                          products are skipped under a proven bound and the
                          outputs whose rounding the bound leaves open are
                          recomputed by the MP_EXACT kernel (same bits;
                          mp_set_split_truncation) */
};

/* handling of odd dimensions in the recursion (Sec. 2, last paragraph) */
enum {
    MP_PEEL  = 0,      /* peel every odd dimension (default) */
    MP_MIXED = 1       /* pad x = 3 (mod 4) with a zero row/column, peel x = 1 (mod 4) */
};

enum {
    MP_OK              = 0,
    MP_ERR_ARG         = -1,   /* bad dimension, stride, precision, algorithm or aliasing */
    MP_ERR_NOMEM       = -2,   /* workspace allocation failed */
    MP_ERR_SINGULAR    = -3,   /* LU: a pivot column is entirely zero */
    MP_ERR_TIMEOUT     = -4,   /* a device-side wait gave up */
    MP_ERR_CUDA        = -5,   /* a CUDA runtime call failed */
    MP_ERR_RANGE       = -6,   /* an exponent left [-2^62, 2^62] */
    MP_ERR_UNSUPPORTED = -7,
    MP_ERR_SCRATCH     = -8    /* mpgemm_noalloc: needs more than the static scratch */
};

/* ---- per-thread settings ------------------------------------------------ */

/* Stream for the calling thread's subsequent calls (a cudaStream_t; NULL is
 * the legacy default stream).  Always MP_OK. */
int mp_set_stream(void *stream);

/* Caller-owned device buffer used as workspace by later calls of this
 * thread (NULL / 0 to let the library allocate).  Always MP_OK.  It must be
 * device memory of the device the calls run on: MP_SPLIT refuses any other
 * buffer (host, managed or another GPU's memory) with MP_ERR_ARG before it
 * launches anything, because its tensor-core kernel reads the buffer with
 * TMA loads multicast inside a thread-block cluster. */
int mp_set_workspace(void *ptr, size_t bytes);

/* Odd-dimension policy for Strassen / Winograd (MP_PEEL or MP_MIXED). */
int mp_set_odd_policy(int policy);

/* Split form (MP_SPLIT): 1 (default) skips the digit-product diagonals whose
 * sum is provably below the rounding position of typical outputs and
 * recomputes exactly every output the bound leaves undecided; 0 computes
 * all diagonals.  Both give the correctly rounded exact dot product.
 * MP_ERR_ARG for any other value. */
int mp_set_split_truncation(int on);

/* Staging of the Block kernel's operand tiles (MP_BLOCK and the Strassen /
 * Winograd leaves, Sec. 2 Eq. 2; up to 1024 bits): 1 (default) brings each
 * k-slab's A and B limb tiles into shared memory with the GPU's bulk tensor
 * copies (TMA), double-buffered, wherever the operands' layout allows it --
 * a 16-byte aligned limb base and even ld, plane and batch strides, and an
 * even column offset for a leaf read in place from its parent's quadrant;
 * 0, and every other layout, has the CTA's threads load the tiles.  Both
 * give the same bits; launches of the first kind are counted under
 * MP_K_LEAF_TMA by the profiler.  MP_ERR_ARG for any other value. */
int mp_set_leaf_tma(int on);

/* LU settings used by mplu: panel width K (Sec. 4 block size, >= 1), the
 * trailing-update algorithm (MP_SIMPLE .. MP_WINOGRAD) and its cutoff
 * (0: chosen by the library, as for mpgemm). */
int mp_set_lu(int panel, int algo, int cutoff);

/* Row exchanges in mplu: 1 (default) partial pivoting; 0 the paper's LU
 * without pivoting (Sec. 4: no exchange, the pivot of column k is a_kk and
 * piv[k] = k).  MP_ERR_ARG for any other value. */
int mp_set_lu_pivoting(int on);

/* ---- elementwise arithmetic -------------------------------------------- */

/* R = X op Y elementwise on rows x cols views of equal shape and precision,
 * op 0 add, 1 subtract, 2 multiply, 3 divide (Sec. 1: one correct rounding
 * per operation); ops 4..7 are the same four operations formed by one warp
 * per element (the latency-bound form the LU solves use; same bits; up to
 * 1024 bits, MP_ERR_UNSUPPORTED above).  R may alias X or Y exactly (same pointers and strides).
 * A division by zero leaves that entry untouched and makes mp_sync_status()
 * return MP_ERR_ARG. */
int mp_elementwise(int op, const mpmat_t *X, const mpmat_t *Y, mpmat_t *R);

/* R = RN_{R.prec}(X) elementwise (exact when R.prec >= X.prec). */
int mp_convert(const mpmat_t *X, mpmat_t *R);

/* ---- matrix multiplication (Sec. 2) ------------------------------------- */

/* Workspace bytes mpgemm needs for these arguments (0 for Simple/Block). */
size_t mpgemm_workspace_size(int64_t m, int64_t l, int64_t n, int32_t prec,
                             int32_t algo, int32_t cutoff);

/*
 * C := A B with A m x l, B l x n, C m x n, all of precision prec.
 *   algo   : MP_SIMPLE, MP_BLOCK, MP_STRASSEN, MP_WINOGRAD, MP_EXACT or MP_SPLIT;
 *   cutoff : Strassen/Winograd recurse while m, l and n all exceed it
 *            (n_min of Sec. 2, >= 1); below it the leaf product is Block.
 *            0 lets the library choose (the cutoff measured fastest for the
 *            precision class: 64 up to 1024 bits, 32 above); negative is
 *            MP_ERR_ARG.
 * Every c_ij of Simple/Block is (((+0 + a_i1 b_1j) + a_i2 b_2j) + ...) with
 * each product and sum rounded; Strassen/Winograd evaluate the printed
 * formulas left to right with one rounding per matrix add/sub element.
 * MP_EXACT forms each dot product exactly in a fixed-point accumulator and
 * rounds once; an exact zero sum is +0; a row/column pair whose products'
 * exponents spread wider than the accumulator (about 2p bits) is left +0 and
 * mp_sync_status() returns MP_ERR_UNSUPPORTED.  MP_EXACT and MP_SPLIT take
 * prec <= MP_PREC_EXACT_MAX and return MP_ERR_UNSUPPORTED above it.
 * Precisions above 2048 bits run the same algorithms with the numbers in
 * local memory (a slower, wide capacity class).
 * C must not overlap A or B (MP_ERR_ARG).  l = 0 gives C = +0.
 */
int mpgemm(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo, int32_t cutoff,
           const mpmat_t *A, const mpmat_t *B, mpmat_t *C);

/*
 * C_b := A_b B_b for b = 0 .. batch-1, independent equally shaped products
 * (Simple or Block; each C_b exactly as mpgemm would compute it).  The
 * operands are stacked by rows: A is (batch*m) x l with A_b = rows
 * [b*m, (b+1)*m), B is (batch*l) x n, C is (batch*m) x n; one grouped launch
 * covers all of them.  Other algorithms return MP_ERR_UNSUPPORTED.
 */
int mpgemm_batched(int64_t batch, int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo,
                   const mpmat_t *A, const mpmat_t *B, mpmat_t *C);

/*
 * mpgemm_noalloc -- C := A B like mpgemm, for callers that cannot allocate
 * device memory when they multiply: real-time or serving loops that must
 * not touch an allocator (an allocation can synchronise the device and
 * stall the loop), code that runs inside an allocator or memory-pool
 * callback of a host framework (calling back into the allocator there can
 * deadlock), and hosts whose device memory is all handed out in advance by
 * another owner (a new allocation fails).  The paper has no counterpart: it
 * is a deployment variant, not part of the method.
 *
 * It allocates nothing: Strassen/Winograd temporaries live in one
 * file-scope static device array of MP_NOALLOC_SCRATCH_BYTES (64 MiB), which
 * every GPU that loads the library holds until the process exits; Simple
 * and Block need none.  The caller still provides A, B and C.
 *   - algo: MP_SIMPLE, MP_BLOCK, MP_STRASSEN or MP_WINOGRAD, with the
 *     arguments, results, per-thread stream and odd-dimension policy of
 *     mpgemm (the same bits); MP_EXACT and MP_SPLIT return
 *     MP_ERR_UNSUPPORTED; anything else MP_ERR_ARG.
 *   - A product whose recursion needs more than the array holds is rejected
 *     with MP_ERR_SCRATCH before anything is launched (Winograd with cutoff
 *     64 fits n = 200 at 512 bits and n = 256 at 256 bits, not n = 256 at
 *     512 bits).
 *   - The first call on a device looks up the device addresses of the array
 *     and of a static status word (cudaGetSymbolAddress) once; make that
 *     first call before any stream capture.
 *   - Every call uses the same array and leaves its contents behind; the
 *     recursion writes every temporary before reading it.  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on the
 *     array: serialise them.
 *   - Exponent-range overflow is recorded in the static status word and
 *     reported by the next mp_sync_status() on that device (MP_ERR_RANGE).
 */
#define MP_NOALLOC_SCRATCH_BYTES (64u << 20)
int mpgemm_noalloc(int64_t m, int64_t l, int64_t n, int32_t prec, int32_t algo, int32_t cutoff,
                   const mpmat_t *A, const mpmat_t *B, mpmat_t *C);

/* ---- LU decomposition and solve (Sec. 4) -------------------------------- */

/* Workspace bytes mplu needs for an n x n system at prec. */
size_t mplu_workspace_size(int64_t n, int32_t prec);

/*
 * Blocked right-looking LU with partial pivoting (or none, see
 * mp_set_lu_pivoting) of the n x n matrix A
 * (overwritten by L\U, unit lower L), then the solve of A x = b.
 *   piv : device int64[n]; piv[k] is the row exchanged with row k at step k;
 *   b   : n x 1 (read only); x : n x 1 (written), may be NULL to factor only.
 * Each panel of K columns (mp_set_lu) is factored column by column (pivot
 * = first row of largest |a_ik|, l_ik = RN(a_ik / a_kk)), U12 = L11^-1 A12,
 * then A22 = RN(A22 - mpgemm(L21, U12)) with the configured algorithm.
 * A zero pivot makes mp_sync_status() return MP_ERR_SINGULAR.
 */
int mplu(int64_t n, int32_t prec, mpmat_t *A, int64_t *piv, const mpmat_t *b, mpmat_t *x);

/*
 * X := A^-1 B for every column of B (n x nrhs), from the factors L\U and piv
 * that mplu left in A (Sec. 4, the solve Ly = Pb, Ux = y, applied to each
 * column).  Column c of X is bit for bit what mplu returns as x for
 * b = column c of B: forward, y_i = RN(y_i - RN(l_ij y_j)) for j = 0..i-1
 * ascending; backward, x_j = RN(y_j / u_jj) for j = n-1 down to 0, then
 * y_i = RN(y_i - RN(u_ij x_j)) for every i < j.  With B = I, X = A^-1 (the
 * condition number ||A||_1 ||A^-1||_1 of Sec. 4's ill-conditioned matrix).
 * LU n x n, B and X n x nrhs, all of precision prec; piv device int64[n].
 * X must not overlap LU or B (MP_ERR_ARG).  A zero u_jj gives x_j = +0 and
 * mp_sync_status() returns MP_ERR_SINGULAR.  Uses n * nrhs numbers of
 * workspace (mp_set_workspace or stream-ordered allocation).
 */
int mplu_solve(int64_t n, int32_t prec, const mpmat_t *LU, const int64_t *piv, const mpmat_t *B, mpmat_t *X);

/* ---- serving: continuous batching of GEMM and LU-solve requests ---------- */

/*
 * A request loop for mixed MP GEMM and LU-solve requests (sizes and
 * precisions vary per request).  Requests are queued as they arrive and
 * admitted while the device memory they need fits the server's budget and a
 * slot (a CUDA stream) is free; admitted work from different requests runs
 * concurrently.  Small GEMMs of the same precision and size bucket (all of
 * m, l, n <= 512; bucket = next of 64/128/256/512) that ask for Simple or
 * Block are batched into one grouped Block launch, zero-padded to the
 * bucket: the padding only appends exact zero products after each c_ij's
 * k-ascending sequence, so a request's result is the same alone or batched.
 * Other GEMMs of the same precision and size class (largest dimension up to
 * 256, 512, 1024 or 2048) that are queued together form a leaf group (up
 * to 8): each runs its own Strassen/Winograd operand sums and combinations,
 * and the leaf products of all of them (a Simple or Block request, also
 * one that waits beside them in a bucket, is one leaf of its own shape)
 * share grouped Block launches.  Requests whose shape was seen before are
 * left to the graph cache instead.
 * Every request's result depends only on the request (never on the mix).
 *
 * Host buffers use the interchange layout, contiguous: limb[L][rows][cols]
 * (limb 0 most significant), exp[rows][cols], sign[rows][cols]; they must
 * stay valid until the request completes.  Page-locked host memory gives
 * asynchronous copies.
 */
typedef struct mp_server mp_server_t;

enum { MP_REQ_GEMM = 0, MP_REQ_LU_SOLVE = 1 };
enum { MP_REQ_DONE = 0, MP_REQ_PENDING = 1, MP_REQ_RUNNING = 2, MP_REQ_CANCELLED = 3,
       MP_REQ_FAILED = 4 };

typedef struct mp_request {
    int64_t  id;          /* caller's tag, returned by mp_server_poll */
    int32_t  kind;        /* MP_REQ_GEMM: C = A B (A m x l, B l x n);
                             MP_REQ_LU_SOLVE: x = A^-1 b (A m x m, b m x 1; l, n ignored) */
    int32_t  prec;
    int64_t  m, l, n;
    int32_t  algo;        /* GEMM algorithm, or the LU trailing-update algorithm */
    int32_t  cutoff;
    int32_t  lu_panel;    /* LU panel width (0: 128) */
    int32_t  reserved;
    const uint64_t *a_limb; const int64_t *a_exp; const int8_t *a_sign;
    const uint64_t *b_limb; const int64_t *b_exp; const int8_t *b_sign;
    uint64_t *c_limb; int64_t *c_exp; int8_t *c_sign;      /* C, or x for LU */
} mp_request_t;

/* A server on the current device with a device-memory budget (bytes) and a
 * number of slots (concurrent streams, 1..64).  NULL on failure. */
mp_server_t *mp_server_create(size_t budget_bytes, int slots);

/* Queue a request (thread safe).  MP_ERR_ARG for a malformed request,
 * MP_ERR_NOMEM if it could never fit the budget. */
int mp_server_submit(mp_server_t *srv, const mp_request_t *req);

/* Cancel a queued request that has not been admitted yet: MP_OK, or
 * MP_ERR_ARG if it is unknown, running or finished. */
int mp_server_cancel(mp_server_t *srv, int64_t id);

/* Up to max finished requests since the last poll: ids, final status
 * (MP_REQ_DONE / _CANCELLED / _FAILED) and latency in milliseconds from
 * submission to completion.  Returns how many were written. */
int mp_server_poll(mp_server_t *srv, int64_t *ids, int32_t *status, double *latency_ms, int max);

/* Block until every submitted request has finished. */
int mp_server_drain(mp_server_t *srv);

/* Counters: [0] submitted, [1] completed, [2] batches and leaf groups
 * launched, [3] requests that ran inside one of them, [4] peak device bytes in use,
 * [5] budget, [6] currently running, [7] currently queued. */
int mp_server_stats(mp_server_t *srv, int64_t out[8]);

/* Graph cache (no counterpart in the paper; a serving facility).  A single
 * request whose signature (kind, sizes, precision, algorithm, cutoff, LU
 * panel) has been seen before runs from a CUDA graph captured once over
 * buffers the server owns; its operands are copied into those buffers, the
 * graph is launched, the result is copied out.  max_graphs entries at most
 * (default 8; 0 turns the cache off); entries whose footprint exceeds 1/16 of
 * the budget are not cached; cached memory counts against the budget and
 * idle entries are evicted, least recently used first, when a request needs
 * the room.  Results equal those of the uncached path bit for bit.
 * Returns MP_OK or MP_ERR_ARG. */
int mp_server_set_graphs(mp_server_t *srv, int max_graphs);

/* Graph cache counters: [0] graphs captured, [1] requests run from a graph,
 * [2] entries held now, [3] device bytes held by them. */
int mp_server_graph_stats(mp_server_t *srv, int64_t out[4]);

/* Drain, stop the scheduler thread and free the server. */
void mp_server_destroy(mp_server_t *srv);

/* ---- tracing -------------------------------------------------------------- */

/* kernel classes for mp_profile_read */
enum {
    MP_K_LEAF = 0,       /* Block GEMM kernel, tiles loaded by its threads (plain Block,
                            recursion leaves and serving groups the copies do not serve) */
    MP_K_SIMPLE = 1,     /* Simple GEMM kernel */
    MP_K_OPERANDS = 2,   /* Strassen/Winograd operand sums */
    MP_K_COMBINE = 3,    /* Strassen/Winograd C combinations */
    MP_K_FIXUP = 4,      /* peel fix-ups (rank-1 update, last row / column) */
    MP_K_ELEMENTWISE = 5,/* mp_elementwise, mp_convert, fills */
    MP_K_LU = 6,         /* LU panel: pivot searches, column steps, row exchanges */
    MP_K_SPLIT = 7,      /* split form: digit-product (tensor core) kernel */
    MP_K_SPLIT_AUX = 8,  /* split form: alignment, recombination, wide fallback */
    MP_K_EXACT = 9,      /* exact-dot GEMM kernel */
    MP_K_LU_TRSM = 10,   /* LU: U rows by the unit lower triangle (Sec. 4 step 2) */
    MP_K_LU_UPDATE = 11, /* LU: subtractions of the earlier columns' updates (inside
                            a panel by the subtracting Block kernel; A22 - T after a
                            trailing product) */
    MP_K_LU_SOLVE = 12,  /* LU: row permutation of b and the two substitutions */
    MP_K_LEAF_TMA = 13,  /* Block GEMM kernel with TMA-staged tiles (mp_set_leaf_tma) */
    MP_K_COUNT = 14
};

/* While enabled (on != 0), every kernel the library launches from the
 * calling process is bracketed by CUDA events on its stream and counted
 * per class.  Enabling resets the counters.  Always MP_OK. */
int mp_profile_enable(int on);

/* Totals for one class since the last enable: launches, summed device time
 * in milliseconds, and work units (MP multiply-adds for the GEMM classes,
 * numbers read and written for the recursion's operand sums and
 * combinations, elements written or processed for the others).
 * Synchronises the device. */
int mp_profile_read(int cls, int64_t *launches, double *ms, double *units);

/* ---- status ------------------------------------------------------------- */

/* Synchronise the calling thread's stream and return the first error the
 * device recorded since the last call (then clear it), or MP_OK. */
int mp_sync_status(void);

/* Column (0-based) of the zero pivot behind the last MP_ERR_SINGULAR. */
int64_t mp_singular_column(void);

/* Outputs of MP_SPLIT products that the truncated split form left to the
 * exact limb kernel, counted on the device between the last two
 * mp_sync_status calls of this thread (read by the later one). */
int64_t mp_split_fallbacks(void);

/* Failure-detection self-test (no counterpart in the paper).  Every device
 * wait of the library -- the mbarrier waits of the split form's slice kernel
 * and of the TMA-staged Block kernel -- gives up after a bounded number of
 * clock cycles, records MP_ERR_TIMEOUT in the device status word and ends
 * its CTA, so a copy or tensor-core operation that never completes is
 * reported instead of hanging the device.  This call runs one CTA of that
 * wait against an mbarrier that nothing completes, with a limit of about
 * `cycles` SM clock cycles (1 .. 2^32), on the calling thread's stream, and
 * returns what mp_sync_status() then reports: MP_ERR_TIMEOUT when the
 * mechanism works (the status word is cleared again and the device stays
 * usable).  MP_ERR_ARG for a limit outside that range. */
int mp_wait_selftest(int64_t cycles);

const char *mp_strerror(int status);

/* Library version, major * 10000 + minor * 100 + patch. */
int mp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPGEMM_H */
