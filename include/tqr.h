/*
 * tqr.h - C ABI of libtqr, a tiled QR factorization for NVIDIA GB300 (sm_103a).
 *
 * The method is the tiled QR of a p x q tile matrix driven by an elimination list
 * (Bouwmeester, "Tiled Algorithms for Matrix Computations on Multicore Architectures",
 * 2012, Chapter 3): every sub-diagonal tile (i,k) is zeroed by a triangle-on-triangle
 * transformation elim(i, piv(i,k), k) (Section 3.1, Algorithm "Generic QR"), executed as
 * the kernels GEQRT, TTQRT (panel) and UNMQR, TTMQR (update) of Algorithm "elimTR" and
 * Table "Kernels for tiled QR".  The whole task graph runs in one persistent CUDA kernel.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with a leading dimension (LAPACK style).  Device
 *     pointers are CUDA global-memory pointers owned by the caller; the library never
 *     frees them.  "stream" is a cudaStream_t passed as void* (NULL = legacy stream).
 *   - Tiles are nb x nb; p = ceil(m/nb), q = ceil(n/nb).  Matrices that are not a whole
 *     number of tiles are handled as if zero-padded: the results equal the leading part
 *     of the zero-padded problem's results.
 *   - Rows/columns/tiles are 0-based (the thesis counts from 1).
 *   - Every function returns an int status: 0 = TQR_OK; -i = the i-th argument is
 *     invalid (LAPACK style, nothing was done); a positive TQR_E* code otherwise.
 *     No C++ exception crosses this interface.
 *   - Device work is enqueued on "stream".  Unless tqr_set_sync(0) was called, each
 *     call that runs device work synchronizes "stream" before returning so that a
 *     device-side error (TQR_ETIMEOUT) is reported by that call.
 *   - The library keeps per-shape plans (elimination list, task graph, device task
 *     tables) in device memory it allocates itself; tqr_finalize() frees them.  Two
 *     calls that use the same plan must not run concurrently on different streams.
 */
#ifndef TQR_H
#define TQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Elimination trees (Section 3.2): FlatTree (Sameh-Kuck), PlasmaTree(BS), BinaryTree
 * (= PlasmaTree(1)), Fibonacci (Modi-Clarke order 1), Greedy, GrASAP (Definition
 * "grasap": Greedy on the first q-1 columns, ASAP on the last), ASAP on every column. */
typedef enum {
  TQR_FLAT = 0, TQR_PLASMA = 1, TQR_BINARY = 2, TQR_FIBONACCI = 3,
  TQR_GREEDY = 4, TQR_GRASAP = 5, TQR_ASAP = 6
} tqr_tree;

/* Flag OR-ed into any tree argument: the TS form of the tree's list (Section 3.1.1,
 * Algorithm "elimSQ", Table "Kernels for tiled QR").  A TS elimination zeroes a square
 * tile with TSQRT(i,piv,k) (weight 6) and updates its row pair with TSMQR(i,piv,k,j)
 * (weight 12); its row must not have been triangularized, so the TS form zeroes with TS
 * kernels every row that is never a pivot in that column and keeps the TT kernels for
 * the rows that pivot before they are zeroed (those rows get GEQRT/UNMQR as before).
 * TQR_FLAT | TQR_TS is Sameh-Kuck with TS kernels; TQR_PLASMA | TQR_TS is the PLASMA
 * algorithm (TS inside each domain, TT between the domain heads).  A TSQRT stores its
 * reflectors in the whole zeroed tile and its T in the tile's TTQRT slot. */
enum { TQR_TS = 16 };

/* Arithmetic of the factorization.
 *   TQR_FP64   : everything in FP64 (matrix in double).
 *   TQR_FP32   : matrix in float; Householder norms and tau in FP64; updates in FP32.
 *   TQR_BF16X3 : matrix in float; norms/tau in FP64; the UNMQR/TTMQR updates on the
 *                tensor cores as split-bf16 x3 products (x = hi + lo; hi*hi + hi*lo +
 *                lo*hi, ~2^-16 relative) with FP32 accumulation.
 *   TQR_BF16X6 : as TQR_BF16X3 with a three-way split and six products (~2^-24, close
 *                to FP32 updates).
 *   TQR_BF16, TQR_FP16 : as TQR_BF16X3 with one bf16 / fp16 product.
 *   TQR_Z64    : double complex, the thesis's second precision (Section 3.3): matrices,
 *                T and right-hand sides are interleaved (re, im) doubles, leading
 *                dimensions count complex elements; LAPACK's complex reflectors (real
 *                beta, H^H [alpha; x] = [beta; 0]), so R has a real diagonal; tqr_apply_qt
 *                applies Q^H (trans = 0) or Q; nb <= 128; no batched or tensor-core form.
 *                Reported flops are 4 x 2 n^2 (m - n/3) (a complex multiply-add is 8
 *                real flops). */
typedef enum { TQR_FP64 = 0, TQR_BF16 = 1, TQR_FP16 = 2, TQR_BF16X3 = 3, TQR_FP32 = 4,
               TQR_BF16X6 = 5, TQR_Z64 = 6 } tqr_prec;

enum {
  TQR_OK = 0,
  TQR_ECUDA = 1,     /* a CUDA runtime call failed (message: tqr_last_error())   */
  TQR_ENOMEM = 2,    /* the library could not allocate its plan / workspace      */
  TQR_ETIMEOUT = 3,  /* a device-side dependency wait exceeded the wait limit    */
  TQR_ENOCONV = 4,   /* iterative refinement did not reach the tolerance         */
  TQR_EUNSUPPORTED = 5 /* valid arguments this build does not implement          */
};

/* Elimination list of a p x q tile matrix (Section 3.2) and its critical path.
 *   list     : out, 3*E int32 triples (k, i, piv), 0-based, canonical order (by column,
 *              then step, then row); may be NULL to query E only.
 *   len      : in = capacity of list in triples; out = E = number of eliminations.
 *   cp_units : out (may be NULL), the weighted critical path with unbounded
 *              processors in units of nb^3/3 flops, kernel weights GEQRT 4, TTQRT 2,
 *              UNMQR 6, TTMQR 6, TSQRT 6, TSMQR 12 (Table "Kernels for tiled QR",
 *              Section 3.1.3); with TQR_TS in tree, of the TS form.
 *   bs       : PlasmaTree domain size (>= 1), ignored by the other trees.
 * Host only; no device work.  Errors: -1/-2 p or q < 1, -3 unknown tree, -4 bs < 1
 * for PlasmaTree, -6 len NULL or capacity too small while list != NULL. */
int tqr_elimlist(int p, int q, int tree, int bs, int32_t *list, int64_t *len,
                 int64_t *cp_units);

/* Bounded-processor schedule of the factorization task graph (thesis Chapter 5: Sections
 * "ALAP Derived Performance Bound", Eq. (alapbound), and "Critical Path Scheduling";
 * Section 5.5, Table "Schedule lengths for matrix of 5x5 tiles").  The graph is the one
 * of tqr_elimlist (p x q tiles, tree, bs).
 *   nproc      : number of processors, >= 1.
 *   weights    : 4 int64 kernel weights (GEQRT, TTQRT, UNMQR, TTMQR), each >= 1; NULL =
 *                the thesis's 4, 2, 6, 6.  The TS kernels of a TQR_TS tree weigh 3 x TTQRT
 *                (TSQRT) and 2 x TTMQR (TSMQR), the thesis's ratios 6/2 and 12/6.
 *   makespan   : out (may be NULL), the length of the "CP Method" list schedule: every
 *                task gets its Backflow priority (its weight plus the largest priority
 *                of a successor) and at every moment the free processors take the ready
 *                tasks of largest priority, ties to the task earlier in the sequential
 *                program.
 *   alap_bound : out (may be NULL), the ALAP Derived Performance Bound on the makespan,
 *                max(critical path, ceil((T_seq + LA) / nproc)).
 *   lost_area  : out (may be NULL), LA: the idle area of nproc processors at the end of
 *                the as-late-as-possible execution on unbounded processors, walking back
 *                from its end until more than nproc tasks are active.
 * Host only; no device work.  Errors: -1/-2 p or q < 1, -3 unknown tree, -4 bs < 1 for
 * PlasmaTree, -5 nproc < 1, -6 a weight < 1. */
int tqr_schedule(int p, int q, int tree, int bs, int nproc, const int64_t *weights,
                 int64_t *makespan, int64_t *alap_bound, int64_t *lost_area);

/* tqr_schedule with nine weights: the kernels GEQRT, TTQRT, UNMQR, TTMQR, TSQRT, TSMQR
 * (each >= 1; the TS kernels weighed on their own, e.g. by measured task durations); the
 * operand-image preparation tasks of the tensor-core precisions (>= 1: one preparation
 * task after every GEQRT, TTQRT and TSQRT; 0: none); and the 32-column block tasks of a
 * split TTQRT and TSQRT (both >= 1, with preparation tasks: each TT / TS panel as four
 * block tasks, the graph the tensor-core executor runs for ib dividing 32; 0: unsplit).
 * weights must not be NULL (-6); other arguments and errors as tqr_schedule. */
int tqr_schedule_ts(int p, int q, int tree, int bs, int nproc, const int64_t *weights,
                    int64_t *makespan, int64_t *alap_bound, int64_t *lost_area);

/* Claim order of the persistent executor for the factorizations planned after this call
 * (plans are cached per order setting; results never depend on the order).
 *   mode 0: earliest start on unbounded processors with the thesis weights, ties to the
 *           longer remaining path.
 *   mode 1: the start order of tqr_schedule's CP-method list schedule on as many
 *           processors as the executor keeps resident CTAs, with the given per-kind
 *           weights (GEQRT, TTQRT, UNMQR, TTMQR; each >= 1; NULL = 4, 2, 6, 6), e.g.
 *           measured task durations of the chosen precision (TS kernels: 3 x TTQRT and
 *           2 x TTMQR).
 *   mode 2 (default): mode 1 with built-in weights from task durations in
 *           microseconds measured on GB300 - the tensor-core precisions 330, 360, 20, 32,
 *           TSQRT 400, TSMQR 32 (nb 128, panel weights tuned on a 32768 x 4096
 *           factorization), TQR_FP64 5146, 4249, 6394, 6369, TSQRT 6767, TSMQR 9457
 *           (nb 256) - and mode 0 for TQR_FP32.  weights is ignored.
 * Every order is topological, so the executor's dependency waits always end.
 * Host only.  Errors: -1 unknown mode, -2 a weight < 1. */
int tqr_set_claim_order(int mode, const int64_t *weights);
/* tqr_set_claim_order with six weights (GEQRT, TTQRT, UNMQR, TTMQR, TSQRT, TSMQR) for
 * mode 1 (NULL = 4, 2, 6, 6, 6, 12).  Errors as tqr_set_claim_order. */
int tqr_set_claim_order_ts(int mode, const int64_t *weights);
/* tqr_set_claim_order with the nine weights of the tensor-core task graph (GEQRT, TTQRT,
 * UNMQR, TTMQR, TSQRT, TSMQR, operand-image preparation, 32-column TTQRT block, TSQRT
 * block; the weights of tqr_schedule_ts) for mode 1 (NULL = the built-in tensor-core
 * weights).  Errors as tqr_set_claim_order. */
int tqr_set_claim_order_tc(int mode, const int64_t *weights);
/* Column parts of later TQR_FP64 / TQR_FP32 factorization plans.  The critical path of a
 * small task graph (Section 3.2: the lower bound on its execution time however many
 * cores run it) is a chain of panel and update kernels; with column parts each update
 * task UNMQR / TTMQR / TSMQR becomes up to four tasks on 16-column (FP64) or 32-column
 * (FP32) slices of its target tiles, which run on different SMs, while each column's
 * arithmetic stays that of the whole-tile task (the factors are bit for bit the same).
 * mode 0: never; 1 (default): when the split graph's update tasks fit on the GPU's SMs
 * at once (a graph bound by its critical path); 2: always (when the tile holds two
 * slices).  Plans already built keep their form.  Host only.  Errors: -1 unknown mode. */
int tqr_set_column_parts(int mode);

/* Bytes of the caller-owned T workspace of tqr_factor: two ib x nb compact-WY T
 * factors (GEQRT's and TTQRT's, Schreiber-Van Loan form, LAPACK GEQRT layout: block b
 * in columns b*ib..) per tile (i,k), i < p, k < min(p,q), in the precision's element
 * type (double for TQR_FP64, float otherwise), followed for the tensor-core precisions
 * by the split operands of the updates.  Host only. */
int tqr_workspace_size(int64_t m, int64_t n, int nb, int ib, int prec, size_t *T_bytes);

/* Tiled QR factorization A = QR in place (Algorithm "elimTR" over the list of "tree").
 *   A   : device, m x n column-major (double for TQR_FP64, float otherwise), lda >= m.
 *         On exit the upper triangle of A holds R (m >= n: rows 0..n-1), the strictly
 *         lower part of each tile holds its GEQRT reflectors and the upper triangle of
 *         each zeroed tile holds its TTQRT reflectors.
 *   T   : device, tqr_workspace_size() bytes, written.
 *   nb  : tile size, 1..256 for TQR_FP64 and TQR_FP32, exactly 128 for the tensor-core
 *         precisions; ib: inner block, 1 <= ib <= min(nb, 32).
 *   tree: a tqr_tree, optionally | TQR_TS (the TS form: the upper triangle of a tile
 *         zeroed by TSQRT is not R - the whole tile holds its reflectors).
 * Errors: -1..-4 sizes, -5 tree, -6 bs, -7 prec, -8 A NULL, -9 lda < m, -10 T NULL;
 *         TQR_ETIMEOUT, TQR_ECUDA, TQR_ENOMEM, TQR_EUNSUPPORTED. */
int tqr_factor(int64_t m, int64_t n, int nb, int ib, int tree, int bs, int prec,
               void *A, int64_t lda, void *T, void *stream);

/* ---- Batched factorization ------------------------------------------------------
 * Many independent matrices factored by ONE persistent executor launch: the task
 * graphs of all matrices (each the graph of tqr_factor for its own nb, ib and tree)
 * are concatenated into one task table.  The thesis factors one matrix at a time
 * (Chapter 3); batching is this library's own extension of the same task model.
 * Tuning: each matrix takes (nb, ib, tree, bs) from "params" (4 ints per matrix). */

/* Per-matrix tuning from a size-class table.
 *   table : nrows rows of 8 int64 {m_lo, m_hi, n_lo, n_hi, nb, ib, tree, bs}; matrix b
 *           takes the first row with m_lo <= m[b] <= m_hi and n_lo <= n[b] <= n_hi.
 *           Matrices that no row covers (or table NULL) take the library's built-in
 *           size-class rule for "prec".
 *   params: out, 4 * nbatch ints {nb, ib, tree, bs}.
 * Host only.  Errors: -1 nbatch < 1, -2 a size < 1, -3 a table row that
 * tqr_factor would reject, -4 params NULL, -7 prec. */
int tqr_batch_params(int nbatch, const int64_t *m, const int64_t *n, int prec,
                     const int64_t *table, int nrows, int *params);

/* Autotuned size-class table of a batch (device work on "stream", synchronized).  The
 * matrices are grouped into classes: a row bucket (1..1024, 1025..4096, 4097..) times the
 * exact column count.  For each class the library factors a sample of up to 32 of the
 * class's own shapes (seeded pseudo-random entries in scratch device memory it allocates
 * and frees, inputs restored before every timed launch) as one batched launch per
 * candidate and keeps the fastest by device time: the tile size nb in {32, 64, 128, 256}
 * (Greedy, ib = min(nb, 32)), then ib in {8, 16, 32} at that nb, then the tree among
 * Greedy, BinaryTree, Fibonacci, FlatTree, PlasmaTree(4) and the TS forms of FlatTree and
 * PlasmaTree(4).  Tensor-core precisions keep nb = 128 and try ib in {16, 32}.  Results are
 * cached per device, precision and class until tqr_finalize(); a cached class costs
 * nothing.  This tuning is the library's own (the thesis factors one matrix at a time).
 *   table    : out, capacity rows of 8 int64 {m_lo, m_hi, n_lo, n_hi, nb, ib, tree, bs}
 *              (the layout tqr_batch_params reads), or NULL to query the row count.
 *   nrows    : out, the number of classes (rows).
 * Errors: -1 nbatch < 1, -2 NULL or a size < 1, -4 prec, -6 capacity too small, -7 nrows
 * NULL; TQR_ENOMEM, TQR_ECUDA. */
int tqr_batch_autotune(int nbatch, const int64_t *m, const int64_t *n, int prec, int64_t *table,
                       int capacity, int *nrows, void *stream);

/* Offsets of the matrices' T workspaces in one buffer: T of matrix b occupies bytes
 * [offsets[b], offsets[b] + tqr_workspace_size(m[b], n[b], nb_b, ib_b, prec)) and
 * offsets[nbatch] is the total; every offset is a multiple of 256.  Host only. */
int tqr_batch_workspace_size(int nbatch, const int64_t *m, const int64_t *n, int prec,
                             const int *params, size_t *offsets);

/* An uploaded batched task graph bound to fixed device buffers (opaque). */
typedef struct tqr_batch_plan tqr_batch_plan;

/* Builds the concatenated task graph of a batch and uploads it to the current device.
 *   m, n, lda : host arrays of nbatch sizes (lda[b] >= m[b]).
 *   A, T      : host arrays of nbatch DEVICE pointers: matrix b (column-major, double
 *               for TQR_FP64, float otherwise) and its T workspace (tqr_workspace_size
 *               bytes for its nb/ib).  The plan keeps the pointers; the caller keeps the
 *               buffers alive while the plan is used and owns them.
 *   params    : 4 * nbatch ints from tqr_batch_params, or NULL: each matrix takes its
 *               size class's autotuned setting (tqr_batch_autotune, tuned on the legacy
 *               stream on first use, then cached) - size T with tqr_batch_params over the
 *               table tqr_batch_autotune returns.  Tensor-core precisions need nb = 128.
 *   prec      : TQR_FP64, TQR_FP32 or a tensor-core precision.
 * Task order: every matrix's own order (earliest start, then longest remaining path)
 * is kept; matrices are started longest-critical-path first, each offset by the work
 * of the matrices before it divided by the resident CTAs, and the tasks of all
 * matrices are merged by that offset plus their earliest start.  The merged order is
 * topological, so the ticket claim of the executor cannot deadlock.
 * Errors: as tqr_factor, with -1/-2 reporting nbatch and the first bad matrix via
 * tqr_last_error(); TQR_ENOMEM. */
int tqr_batch_plan_create(int nbatch, const int64_t *m, const int64_t *n, void *const *A,
                          const int64_t *lda, const int *params, int prec, void *const *T,
                          tqr_batch_plan **plan);

/* The merged claim order of a batch for "slots" resident CTAs, without building a plan
 * (host only; for inspection and tests).  Position r of the order is task local[r] (an
 * index into matrix mat_of[r]'s own executor order, as tqr_factor would run it).
 *   params : as for tqr_batch_plan_create (NULL: built-in rule).
 *   ntask  : in = capacity of mat_of / local; out = number of tasks.  Pass mat_of or
 *            local NULL to query the count only.
 * Errors: -1 nbatch / sizes, -4 ntask NULL or capacity too small, tqr_factor's status
 * for a bad matrix, TQR_ENOMEM. */
int tqr_batch_order(int nbatch, const int64_t *m, const int64_t *n, int prec, const int *params,
                    int slots, int32_t *mat_of, int32_t *local, int64_t *ntask);

/* Runs a batch plan on "stream": resets the dependency counters, the ticket and the
 * status word (device-to-device copy and memset) and launches the executor once.
 * use_graph != 0 replays a CUDA graph of those three operations, captured on the first
 * such call on a stream owned by the plan.  With synchronization on (tqr_set_sync),
 * waits for the stream and returns TQR_ETIMEOUT if a dependency wait ran out. */
int tqr_batch_plan_run(tqr_batch_plan *plan, int use_graph, void *stream);

/* Waits for "stream" and returns the plan's device status: TQR_OK, or TQR_ETIMEOUT if
 * a dependency wait of its last run ran out (for runs made with synchronization off). */
int tqr_batch_plan_status(tqr_batch_plan *plan, void *stream);

/* out[0] tasks, out[1] dependency edges, out[2] matrices, out[3] resident CTAs the
 * order was planned for, out[4] 1 if a CUDA graph was captured, out[5] nominal flops
 * (sum of 2 n^2 (m - n/3)).  Host only. */
int tqr_batch_plan_info(const tqr_batch_plan *plan, int64_t out[6]);

/* Frees a plan's device buffers and graph (the caller's A and T are untouched). */
void tqr_batch_plan_destroy(tqr_batch_plan *plan);

/* One-shot batched factorization: tqr_batch_plan_create + one tqr_batch_plan_run
 * without a graph + destroy.  The call always synchronizes the stream (the plan's
 * buffers are freed before it returns).  params NULL = the autotuned settings (see
 * tqr_batch_plan_create). */
int tqr_factor_batched(int nbatch, const int64_t *m, const int64_t *n, void *const *A,
                       const int64_t *lda, const int *params, int prec, void *const *T,
                       void *stream);

/* Chapter 3's statement of the problem (its opening, before Section 3.1) motivates the
 * QR factorization A = QR by two uses: solving a linear least-squares problem with m
 * equations and n unknowns, and an orthonormal basis of A's column span (the Q factor).
 * tqr_apply_qt, tqr_trsm and tqr_lstsq are those uses, built on tqr_factor.
 *
 * Apply Q^T (trans = 0) or Q (trans = 1) of a tqr_factor result to B (m x nrhs,
 * column-major, ldb >= m), in place, replaying the UNMQR/TTMQR kernels on B's tile rows
 * (in list order for Q^T, in reverse for Q).  A/T/prec/tree/nb/ib must be those of the
 * factorization.  B is double for every precision; the reflectors are read in the
 * precision A is stored in.
 * With trans = 1 on B = the first n columns of the identity the call forms the explicit
 * thin Q (the orthonormal basis of the column span).
 * Errors: -1..-6 sizes/tree/bs, -7 prec, -8 trans, -9 A, -10 lda, -11 T, -12 B,
 *         -13 ldb, -14 nrhs < 0. */
int tqr_apply_qt(int64_t m, int64_t n, int nb, int ib, int tree, int bs, int prec, int trans,
                 const void *A, int64_t lda, const void *T, double *B, int64_t ldb,
                 int64_t nrhs, void *stream);

/* Solve R X = B (the triangular solve of the least-squares use of A = QR, Chapter 3's
 * statement of the problem) for the n x n upper-triangular R held in the top rows of a factored A
 * (double for TQR_FP64, float otherwise), X overwriting B (n x nrhs double, ldb >= n).
 * Errors: -1 n, -2 prec, -3 A, -4 lda, -5 B, -6 ldb, -7 nrhs. */
int tqr_trsm(int64_t n, int prec, const void *A, int64_t lda, double *B, int64_t ldb,
             int64_t nrhs, void *stream);

/* Same solve as tqr_trsm, for callers that may not allocate device memory: code that
 * runs where cudaMalloc is unavailable or forbidden - under a fixed device-memory budget
 * owned by another allocator, on a path that must never call into the allocator (it can
 * synchronize the device), or between operations that must not change the device's
 * memory map.  This entry point allocates nothing: its scratch (a ticket, one flag per
 * 64-row block and a status word) lives in a fixed array compiled into the library,
 * which every GPU that loads the library keeps until the process exits.
 * (The thesis has no counterpart of this entry point.)
 *   Limit: n <= 262144 (4096 blocks of 64 rows); larger n returns -1 with a message in
 *   tqr_last_error().  Arguments, layout and the other errors are those of tqr_trsm.
 *   The first call on a device looks up the device address of the array (once per
 *   device, with that device current); make that first call before any stream capture.
 *   The address is cached for the life of the device's primary context: after a
 *   cudaDeviceReset, call tqr_finalize() (which forgets it) before the next call.
 *   Every call uses the same array and resets the parts that must start at zero, so
 *   calls that overlap on the GPU (e.g. on two streams at once) race: serialize them. */
int tqr_trsm_static(int64_t n, int prec, const void *A, int64_t lda, double *B, int64_t ldb,
                    int64_t nrhs, void *stream);

/* Least squares min ||A X - B||_2 (m >= n, A of full column rank), all operands double:
 * the linear least-squares problem Chapter 3's statement of the problem names as the
 * first use of the QR factorization (X = R^{-1} (Q^T B)(0:n)).
 *   prec == TQR_FP64 : X = R^{-1} (Q^T B)(0:n) from an FP64 tiled QR.
 *   otherwise        : the tiled QR runs in "prec" on a float copy of A; X is then
 *                      computed by FP64 iterative refinement from X = 0: each step
 *                      forms r = B - A X and A^T r in FP64; a right-hand side is done
 *                      when ||A^T r|| / (||A||_F ||r||) <= tol (least-squares optimal)
 *                      or ||r|| / (||A||_F ||x|| + ||b||) <= tol (backward error of a
 *                      consistent system, e.g. square A); the refinement also stops
 *                      when a step halves neither the worst optimality nor the worst
 *                      backward error (the FP64-attainable level).  Otherwise it solves
 *                      for the correction with LSQR (Paige & Saunders, 1982),
 *                      right-preconditioned with the low-precision R, using LSQR's two
 *                      stopping rules (the normal-equation estimate, and the residual
 *                      estimate against the backward-error threshold); the correction
 *                      solve forms its products with A from an FP32 hi/lo split of A in
 *                      double-float arithmetic (about 2^-47 per product), everything else
 *                      in FP64.
 *   A, B    : device, not modified.  X : device n x nrhs, ldx >= n.
 *   iters   : out (may be NULL), refinement iterations used (max over right-hand sides).
 *   workspace / ws_bytes : device scratch of at least tqr_lstsq_workspace_size() bytes.
 * Errors: -1..-11 sizes/tree/prec/pointers; TQR_ENOCONV when max_iter LSQR iterations
 *         were used while the solution was still improving. */
int tqr_lstsq(int64_t m, int64_t n, int64_t nrhs, int nb, int ib, int tree, int bs, int prec,
              const double *A, int64_t lda, const double *B, int64_t ldb,
              double *X, int64_t ldx, double tol, int max_iter, int *iters,
              void *workspace, size_t ws_bytes, void *stream);
int tqr_lstsq_workspace_size(int64_t m, int64_t n, int64_t nrhs, int nb, int ib, int prec,
                             size_t *bytes);

/* Nominal flop count 2 n^2 (m - n/3) of a QR of an m x n matrix (m >= n) - the count
 * every TFLOP/s figure of this library uses (Theorem "thm.flops"). */
double tqr_nominal_flops(int64_t m, int64_t n);

/* Measured FP64 throughput of the current device (TFLOP/s): the plain FP64 FMA pipe
 * (DFMA: independent FMA chains on every SM) and the FP64 tensor instruction (DMMA:
 * mma.sync m8n8k4 f64, independent accumulators on every warp).  These are the
 * denominators of the FP64 form's fraction of peak; under 0.1 s of device time, on
 * "stream", synchronized.  Errors: -1/-2 NULL output, TQR_ECUDA, TQR_ENOMEM. */
int tqr_fp64_peak(double *dfma_tflops, double *dmma_tflops, void *stream);

/* Maximum time one device-side dependency wait may spin before the kernel gives up
 * with TQR_ETIMEOUT (nanoseconds; default 20 s).  Returns the previous value. */
int64_t tqr_set_wait_limit_ns(int64_t ns);
/* 1 (default): every call synchronizes its stream and reports device errors.
 * 0: calls only enqueue; tqr_sync_status(stream) reports them later.  Returns old. */
int tqr_set_sync(int on);
int tqr_sync_status(void *stream);

/* Device-time accounting of the library's own kernels (for benchmarks).  With timing on,
 * every launch is bracketed by CUDA events on its stream; the elapsed time is added when
 * the call synchronizes (so it needs tqr_set_sync(1)).  kind: 0 = factorization
 * executor, 1 = apply-Q executor, 2 = triangular solve, 3 = refinement kernels.
 * tqr_kernel_time returns the accumulated milliseconds and launch count, then clears
 * them when reset != 0.  Errors: -1 unknown kind. */
int tqr_set_timing(int on);
int tqr_kernel_time(int kind, double *ms_total, int64_t *launches, int reset);
/* Number of CUDA kernels this library has launched in this process (all entry points);
 * reset != 0 clears the count after reading it. */
int64_t tqr_launch_count(int reset);

/* Per-task execution trace (a Gantt chart of the persistent executor).  With tracing on,
 * each executor launch records for every task the globaltimer (ns) when a CTA claimed
 * it, when its dependencies were met, when it finished, the SM it ran on, and the time
 * (ns) spent in up to four phases of the kernel (panels: factorization loops, T build,
 * trailing update, operand images; tensor-core updates: operand conversion, first
 * product, W conversion, second product and epilogue).
 * tqr_trace_fetch copies the last traced launch: 12 int64 per task in executor order =
 * {kind (0 GEQRT, 1 TTQRT, 2 UNMQR, 3 TTMQR, 4/5/8 apply-Q, 6 TSQRT, 7 TSMQR, 9/10 operand
 * images of a GEQRT / of a TTQRT or TSQRT (tensor-core precisions)), i, piv, k | j << 16, claim,
 * start, end, sm, phase0, phase1, phase2, phase3}.  With out == NULL it returns the task count; otherwise the count
 * copied, -1 if cap is too small or nothing was traced, -2 on a CUDA error. */
int tqr_set_trace(int on);
int64_t tqr_trace_fetch(int64_t *out, int64_t cap);

const char *tqr_strerror(int status);
const char *tqr_last_error(void);      /* detail of the last TQR_ECUDA / internal error */
void tqr_finalize(void);               /* free every cached plan and cached scratch address */

/* ---- test hooks (host logic only; no numerics) ----
 * tqr_plan_stats: task and edge counts of the task graph the executor runs for a
 *   factorization of the given shape/tree: out[0..5] = #GEQRT, #TTQRT, #UNMQR, #TTMQR,
 *   #edges, critical path in units (same weights as tqr_elimlist).
 * tqr_debug_drop_edge: when set to e >= 0, the next plan built (a factorization plan or a
 *   batch plan) omits the release of its e-th dependency edge, so that a wait can never
 *   finish; used to check that the kernel returns TQR_ETIMEOUT instead of hanging.  -1
 *   (default) disables it.
 * tqr_debug_claim_order: the executor (claim) order of the factorization task graph of a
 *   p x q tile matrix, built as a plan is: mode 0 = earliest start on unbounded
 *   processors, mode 1 = start order of the CP-method list schedule on nproc processors
 *   with the four kernel weights (NULL = 4, 2, 6, 6; see tqr_set_claim_order).  tasks
 *   receives 5 int32 per task in claim order: kind (0 GEQRT, 1 TTQRT, 2 UNMQR, 3 TTMQR,
 *   6 TSQRT, 7 TSMQR),
 *   i, piv (-1 if none), k, j (-1 if none); NULL to query the count.  ntask: in =
 *   capacity in tasks, out = number of tasks.  Host only.  Errors: -1/-2 p or q < 1,
 *   -3 unknown tree, -4 bs < 1 for PlasmaTree, -5 mode not 0 or 1, -6 nproc < 1, -7 a
 *   weight < 1, -8 ntask NULL or capacity too small while tasks != NULL. */
int tqr_plan_stats(int64_t m, int64_t n, int nb, int tree, int bs, int64_t out[6]);
/* tqr_plan_counts: as tqr_plan_stats with the TS kernels: out[0..7] = #GEQRT, #TTQRT,
 *   #UNMQR, #TTMQR, #TSQRT, #TSMQR, #edges, critical path (tree may carry TQR_TS). */
int tqr_plan_counts(int64_t m, int64_t n, int nb, int tree, int bs, int64_t out[8]);
void tqr_debug_drop_edge(int64_t e);
/* tqr_debug_split_pairs: the FP32 pair split of the least-squares refinement (hi = the
 *   FP32 rounding of x, lo = the FP32 rounding of x - hi; integer instructions on the
 *   device) run on the host for n values: host arrays x (in), hi, lo (out).  Host only.
 *   Errors: -1 n < 0, -2 a NULL array with n > 0. */
int tqr_debug_split_pairs(int64_t n, const double *x, float *hi, float *lo);
int tqr_debug_claim_order(int p, int q, int tree, int bs, int mode, int nproc, const int64_t *weights,
                          int32_t *tasks, int64_t *ntask);

#ifdef __cplusplus
}
#endif
#endif /* TQR_H */
