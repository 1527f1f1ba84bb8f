// Internal declarations of libtqr shared by the host and device translation units.
#pragma once

#include <array>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace tqr {

// One elimination elim(i, piv, k): tile (i,k) is zeroed by row piv in panel k.
struct Elim {
  int k, i, piv;
};

// Kernel weights in units of nb^3/3 flops (Table "Kernels for tiled QR").
constexpr int kWGeqrt = 4, kWTtqrt = 2, kWUnmqr = 6, kWTtmqr = 6;
constexpr int kWTsqrt = 6, kWTsmqr = 12;

// Tree argument flag (TQR_TS in tqr.h): the TS form of the list - every row that is
// never a pivot in a column is zeroed there by TSQRT/TSMQR (Algorithm "elimSQ") while
// still square, the other eliminations keep the TT kernels.
constexpr int kTreeTS = 16;
inline int tree_base(int tree) { return tree & ~kTreeTS; }
inline bool tree_ts(int tree) { return (tree & kTreeTS) != 0; }

// Elimination list of a tree in canonical order (Section 3.2).  Returns false on an
// unknown tree.  The TS flag of "tree" is ignored (the list is the same).  Host only.
bool elimination_list(int p, int q, int tree, int bs, std::vector<Elim> &out);

// Rows of each column zeroed by TS kernels in the TS form of a list: square[k][i] != 0
// when row i is never a pivot of column k's eliminations (and is zeroed in column k).
std::vector<std::vector<char>> ts_square_rows(int p, int q, const std::vector<Elim> &elims);

// Task kinds of the tile task graph.
enum TaskKind : int32_t {
  kGeqrt = 0,   // GEQRT(i,k)
  kTtqrt = 1,   // TTQRT(i,piv,k)
  kUnmqr = 2,   // UNMQR(i,k,j)
  kTtmqr = 3,   // TTMQR(i,piv,k,j)
  kUnmqrB = 4,  // UNMQR(i,k) applied to tile row i of a right-hand-side block
  kTtmqrB = 5,  // TTMQR(i,piv,k) applied to tile rows (piv, i) of a right-hand-side block
  kTsqrt = 6,   // TSQRT(i,piv,k): zeroes the square tile (i,k) under R(piv,k)
  kTsmqr = 7,   // TSMQR(i,piv,k,j)
  kTsmqrB = 8,  // TSMQR(i,piv,k) applied to tile rows (piv, i) of a right-hand-side block
  // tensor-core precisions: the operand images of a factored tile, written by a task of
  // its own so that the next panel task of a chain does not wait for them
  kPrepG = 9,   // images of GEQRT(i,k)'s reflectors (read by UNMQR(i,k,j))
  kPrepT = 10,  // images of the TTQRT / TSQRT that zeroed tile (i,k) (read by TTMQR / TSMQR);
                // its j is 1 after a TSQRT, 0 after a TTQRT
  // tensor-core graphs: a TTQRT / TSQRT split into kPanelSplits tasks of 32 columns each
  // (block j = b), so that the next elimination on the same pivot can start block b as
  // soon as block b of this one has finished with the pivot's row block b
  kTtqrtS = 11,
  kTsqrtS = 12,
};
constexpr int kNumKinds = 13;
constexpr int kPanelSplits = 4;     // 32-column blocks of a 128-column tile
constexpr int kPanelSplitCols = 32;
// Column parts of a small SIMT factorization: each update task (UNMQR, TTMQR, TSMQR)
// becomes kColParts tasks on column slices of its target tile(s), so that the updates on
// the critical path of a graph with fewer tasks than the GPU has SMs run on several SMs.
// The part travels in bits 12.. of Task::j (target column < 4096 then).
constexpr int kColParts = 4;
constexpr int kColShift = 12;
#ifdef __CUDACC__
#define TQR_HOST_DEVICE __host__ __device__
#else
#define TQR_HOST_DEVICE
#endif
// FP32 pair of a double: hi = fl32(v) (round to nearest even), lo = fl32(v - hi) (the
// difference is exact in FP64), formed from the bit pattern with integer instructions -
// GB300 runs FP64 -> FP32 conversions and FP64 arithmetic on its narrow FP64 unit, which
// would bound a pass over a large matrix.  hi's 23 fraction bits are the top of v's 52,
// rounded by the 29 below (a carry moves into the exponent, as rounding does); the
// residual is those 29 bits minus the rounding, an integer of at most 29 bits converted
// with one rounding and scaled by the power of two of its last place.  v with |v| outside
// [2^-74, 2^127) (zero, tiny, huge, inf, NaN) takes the plain conversions.
inline TQR_HOST_DEVICE void split_pair(double v, float &hi, float &lo) {
#ifdef __CUDA_ARCH__
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(v));
#else
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
#endif
  const int e = static_cast<int>((b >> 52) & 0x7ff);
  if (e < 949 || e > 1149) {
    hi = static_cast<float>(v);
    lo = static_cast<float>(v - static_cast<double>(hi));
    return;
  }
  const uint32_t sign = static_cast<uint32_t>(b >> 63) << 31;
  const uint64_t frac = b & ((uint64_t(1) << 52) - 1);
  const uint32_t keep = static_cast<uint32_t>(frac >> 29);
  const uint32_t rem = static_cast<uint32_t>(frac & ((uint64_t(1) << 29) - 1));
  const uint32_t half = uint32_t(1) << 28;
  const uint32_t up = (rem > half || (rem == half && (keep & 1u))) ? 1u : 0u;
  const uint32_t hbits = sign | ((static_cast<uint32_t>(e - 896) << 23) + keep + up);
  const int32_t r = static_cast<int32_t>(rem) - static_cast<int32_t>(up << 29);
  const uint32_t sbits = static_cast<uint32_t>(e - 948) << 23;  // 2^(e - 1075)
#ifdef __CUDA_ARCH__
  hi = __uint_as_float(hbits);
  const float scale = __uint_as_float(sbits);
  const float rf = __int2float_rn(r);
#else
  std::memcpy(&hi, &hbits, sizeof hi);
  float scale;
  std::memcpy(&scale, &sbits, sizeof scale);
  const float rf = static_cast<float>(r);
#endif
  const float mag = rf * scale;
  lo = r == 0 ? 0.f : (sign ? -mag : mag);
}

inline TQR_HOST_DEVICE int task_col(int j, int colparts) { return colparts > 1 ? (j & ((1 << kColShift) - 1)) : j; }
inline TQR_HOST_DEVICE int task_part(int j, int colparts) { return colparts > 1 ? (j >> kColShift) : 0; }

// A task as the device executor reads it (16 bytes).
struct Task {
  int32_t kind;
  int32_t i;    // row of the factored / zeroed tile
  int32_t piv;  // pivot row (TT kernels), else -1
  int16_t k;    // panel column
  int16_t j;    // target column of an update, else -1
};

// The task graph of one factorization or one apply-Q, in executor order.
struct Graph {
  std::vector<Task> tasks;           // executor (priority) order, topological
  std::vector<int32_t> succ_ptr;     // CSR of successors, size tasks+1
  std::vector<int32_t> succ_idx;
  std::vector<int32_t> indeg;        // number of predecessors
  std::vector<int32_t> weight;       // kernel weight per task
  int64_t critical_path = 0;         // longest weighted path (unbounded processors)
  int64_t counts[kNumKinds] = {};    // tasks per kind
  std::vector<int64_t> start;        // earliest start (unbounded processors), executor order
  std::vector<int64_t> bottom;       // longest weighted path to a sink, task included
};

// One matrix of a batched factorization, as the executor reads it.
struct BatchMat {
  void *A;
  int64_t lda, m, n;
  int nb, ib, P, Q;
  void *T;
  void *ops;
  int vec4;
  int pad;
};

// Incremental construction of a task graph in sequential-program order.  Regions are
// integer ids; a task depends on the last writer of every region it reads or writes
// and on every reader (since that write) of a region it writes.  finish[] is the
// earliest finish time with unbounded processors.
struct GraphBuilder {
  explicit GraphBuilder(int nregions);
  int add(const Task &t, int w, const int *reads, int nr, const int *writes, int nw);
  std::vector<Task> tasks;
  std::vector<int32_t> weight;
  std::vector<int64_t> finish;
  std::vector<std::vector<int32_t>> preds;
  std::vector<int32_t> last_writer;
  std::vector<std::vector<int32_t>> readers;
};

// Tile regions of the factorization graph: each tile (i,j) has a strictly-lower part
// (GEQRT reflectors), an upper part (R, then TTQRT reflectors) kept as kPanelSplits row
// blocks (a split panel task writes one row block of its pivot's R), two operand-image
// slots (tensor-core precisions: GEQRT's and the TT/TS elimination's images) and
// kColParts column slices (written by column-part updates; a panel task on the tile
// writes them all).  A task that touches the upper part as a whole touches all of its row
// blocks.
constexpr int kRegionsPerTile = 3 + kPanelSplits + kColParts;
inline int region_L(int q, int i, int j) { return (i * q + j) * kRegionsPerTile; }
inline int region_Ub(int q, int i, int j, int b) { return (i * q + j) * kRegionsPerTile + 1 + b; }
inline int region_ops(int q, int i, int j, int which) {
  return (i * q + j) * kRegionsPerTile + 1 + kPanelSplits + which;
}
inline int region_cp(int q, int i, int j, int c) { return (i * q + j) * kRegionsPerTile + 3 + kPanelSplits + c; }
// Adds GEQRT(i,k) and UNMQR(i,k,j) for every row i >= k of panel k except the rows with
// square[i] != 0 (zeroed by TS kernels); returns the task ids of the GEQRTs (index i - k,
// -1 for a skipped row).  prep: a PREP_G(i,k) task after each GEQRT writes its operand
// images, which the UNMQRs read.
// colparts > 1: each UNMQR as colparts column-part tasks (part in bits kColShift.. of j).
std::vector<int> add_panel_tasks(GraphBuilder &b, int p, int q, int k, const char *square = nullptr,
                                 bool prep = false, int colparts = 1);
// Adds the eliminations of panel k in order: TSQRT / TSMQR(i,piv,k,j) when square[i] != 0,
// TTQRT / TTMQR(i,piv,k,j) otherwise; prep: a PREP_T(i,k) task after each TTQRT / TSQRT;
// split: each TTQRT / TSQRT as kPanelSplits block tasks (kTtqrtS / kTsqrtS, block in j);
// colparts > 1: each TTMQR / TSMQR as colparts column-part tasks.
void add_elim_tasks(GraphBuilder &b, int q, int k, const std::vector<Elim> &col, const char *square = nullptr,
                    bool prep = false, bool split = false, int colparts = 1);
// Orders a built graph for the executor (earliest start, then longest remaining path)
// and fills the successor CSR.
// Executor (claim) order of a factorization graph.  mode 0: earliest start with
// unbounded processors (thesis weights), then the longer remaining path first.  mode 1:
// the bounded-processor list schedule of thesis Chapter 5 ("CP Method") on nproc
// processors with per-kind weights w[kind], tasks ordered by their start in that
// schedule.
struct OrderSpec {
  int mode = 0;
  int nproc = 1;
  // per task kind (TaskKind index; the apply-Q kinds are unused)
  int64_t w[kNumKinds] = {kWGeqrt, kWTtqrt, kWUnmqr, kWTtmqr, kWUnmqr, kWTtmqr, kWTsqrt, kWTsmqr, kWTsmqr, 1, 1, 1, 2};
  int id = 0;  // identity of the weight set in the plan cache (built-in sets < 0)
};
void finalize_graph(GraphBuilder &b, Graph &g, int64_t drop_edge = -1, const OrderSpec *order = nullptr);
// Tasks of the sequential program (all panels, in column order) added to b; ts: the TS
// form of the list.
void add_factor_program(GraphBuilder &b, int p, int q, const std::vector<Elim> &elims, bool ts = false,
                        bool prep = false, bool split = false, int colparts = 1);
// Backflow priorities (a task's weight plus the largest priority of its successors) of
// a graph in program order with successor lists succ and weights w.
std::vector<int64_t> backflow_priorities(const std::vector<std::vector<int32_t>> &succ,
                                         const std::vector<int64_t> &w);
// CP-method list schedule on nproc processors: at every moment free processors take the
// ready tasks of largest priority (ties: earlier in program order).  Returns the
// makespan; start (if not null) receives every task's start time.
int64_t cp_list_schedule(const std::vector<std::vector<int32_t>> &succ, const std::vector<int32_t> &npred,
                         const std::vector<int64_t> &w, const std::vector<int64_t> &prio, int nproc,
                         std::vector<int64_t> *start);
// ALAP Derived Performance Bound of Eq. (alapbound) for nproc processors; *lost (if not
// null) receives the lost area LA_p.
int64_t alap_derived_bound(const std::vector<int64_t> &w, const std::vector<int64_t> &prio, int nproc,
                           int64_t *lost);

// Builds the factorization task graph of a p x q tile matrix with the given list
// (column-by-column program of Algorithm "elimTR"; dependencies from the tile regions
// each kernel reads and writes, Eq. ttdeps / ttdeps2).
// prep: the tensor-core form, with operand-image preparation tasks (PREP_G / PREP_T);
// split: its TTQRT / TSQRT split into 32-column block tasks; colparts > 1: its update
// tasks split into column parts (SIMT executors).
void build_factor_graph(int p, int q, const std::vector<Elim> &elims, Graph &g,
                        int64_t drop_edge = -1, const OrderSpec *order = nullptr, bool ts = false,
                        bool prep = false, bool split = false, int colparts = 1);
// Builds the graph that applies Q^T (or Q when reverse) to a right-hand-side block.
void build_applyq_graph(int p, int q, const std::vector<Elim> &elims, bool reverse, Graph &g, bool ts = false);

void set_error(const std::string &msg);
// The pending tqr_debug_drop_edge value (-1 if none), cleared by the call (batch plans).
int64_t take_debug_drop_edge();
// Number of kernels this library has launched (tqr_launch_count).
void count_launch(int64_t k = 1);
int64_t wait_limit_ns();   // current device-wait limit (tqr_set_wait_limit_ns)
bool sync_enabled();       // tqr_set_sync state

// ---- device side (executor.cuh, solve.cu) -------------------------------------------
// Status word layout written by the device: code in the low 8 bits, task index above.
constexpr int kStatusTimeout = 3;

// Arguments of one persistent executor launch.  Pointers are device pointers.
struct ExecParams {
  void *A;               // factor storage (double or float), column-major
  int64_t lda, m, n;
  int nb, ib, P, Q;      // tile size, inner block, tile grid
  void *T;               // T workspace (same element type as A)
  double *B;             // right-hand-side block for apply-Q tasks (else null)
  int64_t ldb, nrhs;
  int trans;             // apply-Q: 0 = Q^T, 1 = Q
  const Task *tasks;
  const int32_t *succ_ptr, *succ_idx;
  int32_t *counters;     // per-task remaining predecessors (reset before each run)
  int32_t *next;         // task ticket
  int32_t *status;       // 0 or kStatusTimeout | (task << 8)
  int ntask;
  int64_t wait_limit_ns;
  // tensor-core (mixed) mode: split operand images, products per multiply, 16-bit format
  void *ops;             // 2 * P * min(P,Q) slots of 6 operand images (else null)
  int nparts;            // 16-bit parts per operand: 1, 2 (split x3) or 3 (split x6)
  int fmt;               // 1 = bf16, 0 = fp16
  int mixed;             // 1: GEQRT/TTQRT prepare images, UNMQR/TTMQR run on tcgen05
  int vec4;              // A is 16-byte aligned with lda % 4 == 0 (vector loads allowed)
  int cplx;              // 1: double-complex storage (the complex executor runs the graph)
  int64_t *trace;        // optional: per task {claim, start, end, sm} globaltimer stamps
  int colparts;          // > 1: update tasks cover column part task_part(j) of colw columns
  int colw;
  // batched factorization: per-task matrix index and per-matrix geometry (else null)
  const int32_t *mat_of;
  const BatchMat *mats;
};

// Launches the persistent tile-task executor on "stream".  real_is_double selects the
// factor storage type.  Returns a cudaError_t value (0 = success).
int launch_executor(const ExecParams &p, bool real_is_double, void *stream);
// The executor instantiations (exec_*.cu): launch with smem bytes of dynamic shared
// memory; resident CTAs of the whole GPU at that shared-memory size (0 on error).
int exec_launch_f64(const ExecParams &p, void *stream, size_t smem);
int exec_launch_f32(const ExecParams &p, void *stream, size_t smem);
int exec_launch_f32_apply(const ExecParams &p, void *stream, size_t smem);
int exec_launch_mixed(const ExecParams &p, void *stream, size_t smem);
int exec_slots_f64(size_t smem);
int exec_slots_f32(size_t smem);
int exec_slots_mixed(size_t smem);
// The double-complex executor (zexec.cu): shared memory (0 if nb/ib do not fit), launch,
// resident CTAs; and the complex triangular solve R X = B (R upper n x n, lda; B ldb).
size_t zexecutor_smem_bytes(int nb, int ib);
int zexec_launch(const ExecParams &p, void *stream);
int zexec_slots(int nb, int ib);
int launch_ztrsm(int64_t n, const void *R, int64_t lda, void *B, int64_t ldb, int64_t nrhs, void *stream);
// Dynamic shared memory the executor needs (0 if nb/ib do not fit on one SM).
size_t executor_smem_bytes(int nb, int ib, bool real_is_double, bool apply_q);
// Resident factorization CTAs on the current device (SMs x CTAs per SM), 0 on error.
int executor_slots(bool real_is_double, bool mixed, int nb, int ib);

// Argument checks and workspace layout shared by the single and batched entry points.
bool is_tensor_prec(int prec);
int tensor_parts(int prec);  // 16-bit parts per operand of a tensor-core precision
size_t align_up(size_t x, size_t a);
// 0 or the negative status of tqr_factor for bad sizes / tree / prec
int check_tiles(int64_t m, int64_t n, int nb, int ib, int tree, int bs, int prec);
// byte offset of the operand images in T (tensor-core precisions)
size_t ops_offset(int64_t m, int64_t n, int nb, int ib);
size_t factor_workspace_bytes(int64_t m, int64_t n, int nb, int ib, int prec);
// Tile size, bytes per factored tile of operand images, and shared memory of the
// tensor-core (mixed) executor.
constexpr int kMixedNB = 128;
size_t mixed_slot_bytes(int nparts);
size_t mixed_executor_smem_bytes();

// Wavefront triangular solve R X = B (R upper n x n in A, double or float), X over B.
// flags: device int32[ceil(n/TB) + 1] scratch (ticket + per-block flags).
// lower_transposed: solve R^T X = B instead.
int launch_trsm(int64_t n, const void *A, int64_t lda, bool real_is_double, double *B,
                int64_t ldb, int64_t nrhs, int32_t *flags, int32_t *status,
                int64_t wait_limit_ns, void *stream, bool lower_transposed = false);
int trsm_flag_count(int64_t n);
// Forgets the cached device addresses of tqr_trsm_static's fixed scratch (tqr_finalize).
void reset_static_scratch();
// The batched factorization's per-size-class autotuner (autotune.cu): one row {m_lo, m_hi,
// n_lo, n_hi, nb, ib, tree, bs} per class of the batch, tuned on "stream" on first use and
// cached per device, precision and class.  forget_autotune clears the cache.
int autotune_table(int nbatch, const int64_t *m, const int64_t *n, int prec, void *stream,
                   std::vector<std::array<int64_t, 8>> &rows);
void forget_autotune();
// Inverses of the 64 x 64 diagonal blocks of an upper-triangular R (FP64, 64*64 doubles
// per block; identity on the padding of a partial last block).
int launch_diag_inverse(int64_t n, const void *A, int64_t lda, bool real_is_double, double *Dinv, void *stream);

// Preconditioner solves of the refinement (precond.cu): FP64 inverses of R's 512 x 512
// diagonal blocks built once from the 64 x 64 ones (precond_setup), then R X = B or
// R^T X = B by one cooperative launch per four right-hand sides (precond_solve).
// work: precond_work_doubles(n, real_is_double) doubles; bar: one int32 of device scratch.
size_t precond_work_doubles(int64_t n, bool real_is_double);
int precond_setup(int64_t n, const void *R, int64_t ldr, bool real_is_double, const double *Dinv64, double *work,
                  void *stream);
int precond_solve(int64_t n, const void *R, int64_t ldr, bool real_is_double, const double *work, double *B,
                  int64_t ldb, int64_t nrhs, int32_t *bar, int32_t *status, int64_t wait_limit_ns, void *stream,
                  bool lower_transposed);

// LSQR refinement (refine.cu): X (in: x0, out: refined) for min ||A X - B||, operator
// A R^{-1} with the FP32 R of a tensor-core factorization.  work: lsqr_work_doubles()
// doubles (16-byte aligned); flags: trsm_flag_count(n) int32; status: device status word.
// lsqr_prepare runs once per least-squares call, before the factorization: F = fl32(A)
// (ld ldf, the matrix to factor), and A's FP32 pairs and ||A||_F^2 into work.  setup:
// build the preconditioner from R (the first block of right-hand sides; later blocks
// reuse it).  x_zero: X holds zeros on entry (the first residual is B itself).
size_t lsqr_work_doubles(int64_t m, int64_t n, int nrhs);
int lsqr_prepare(int64_t m, int64_t n, const double *A, int64_t lda, float *F, int64_t ldf, double *work,
                 void *stream);
int lsqr_refine(int64_t m, int64_t n, int nrhs, const double *A, int64_t lda, const float *R, int64_t ldr,
                const double *B, int64_t ldb, double *X, int64_t ldx, double tol, int max_iter,
                int *iters_out, bool setup, bool x_zero, double *work, int32_t *flags, int32_t *status,
                int64_t wait_limit_ns, void *stream);

}  // namespace tqr
