/*
 * hm.h -- C ABI of libhm: the product Y = A X of a HODLR or HSS matrix A with
 * a block X of r vectors on one GB300 (sm_103a).
 *
 * Method: the fast products of Sec. 4.1 and Fig. 4.1 of "hm-toolbox: Matlab
 * software for HODLR and HSS matrices" (Massei, Robol, Kressner).  HODLR
 * (Def. 2.2): dense leaf blocks plus, on every level, sibling blocks U V^T.
 * HSS (Def. 2.3, Eq. 2.2): leaf bases, nested translation operators R_U,
 * R_V and core blocks S (B12, B21 in the paper's class).
 *
 * Conventions shared by every call:
 *  - Every function returns an hm_status.  Nothing aborts, nothing prints.
 *    Invalid shapes and pointers are rejected with HM_EINVAL before any work
 *    is queued.  hm_last_error() gives a one-line description of the last
 *    failure on the calling thread.
 *  - Indices are 0-based; blocks passed in are float64, column-major
 *    (Matlab layout), leading dimension = number of rows.
 *  - Node ids are level order: level l (root = 0), position j has id
 *    2^l - 1 + j.  Internal nodes are ids 0..L-2, leaves L-1..2L-2, with
 *    L = 2^p leaves.
 *  - Objects are created by *_create and released by hm_destroy (NULL-safe).
 *    An object may be used from several host threads only if the caller
 *    serialises calls on it, except where a function says otherwise.
 *  - Streams are cudaStream_t values passed as void* (NULL = legacy default
 *    stream).  All GPU work of a call is queued on that stream and is
 *    asynchronous unless stated.
 */
#ifndef HM_H
#define HM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HM_OK = 0,
  HM_EINVAL = 1,        /* bad argument, shape, pointer or handle */
  HM_ENOMEM = 2,        /* device or host allocation failed, or budget exceeded */
  HM_EBUSY = 3,         /* admission refused (no free slot); retry later */
  HM_ETIMEOUT = 4,      /* a bounded wait ran out (host wait or device barrier) */
  HM_ECUDA = 5,         /* a CUDA runtime call failed */
  HM_EUNSUPPORTED = 6   /* valid request outside this library's scope */
} hm_status;

/* Storage / input-output element types.
 * HM_BF16X2 stores every generator entry a as a pair hi = RN_bf16(a),
 * lo = RN_bf16(a - hi); the tensor-core product is hi*xhi + hi*xlo + lo*xhi. */
typedef enum { HM_F64 = 0, HM_F32 = 1, HM_BF16 = 2, HM_BF16X2 = 3 } hm_dtype;

typedef enum { HM_HODLR = 0, HM_HSS = 1 } hm_kind;

typedef struct hm_tree hm_tree;
typedef struct hm_matrix hm_matrix;
typedef struct hm_batch hm_batch;
typedef struct hm_server hm_server;
typedef struct hm_ulv hm_ulv;

/* Static description of a status code; never NULL. */
const char* hm_status_string(hm_status s);
/* Detail of the last failed call on this host thread; never NULL. */
const char* hm_last_error(void);
/* Library version string, e.g. "hm 1.0 sm_103a". */
const char* hm_version(void);

/* ---------------------------------------------------------------------- */
/* Cluster trees (Def. 2.1; vector form of Sec. 3.7; default split Sec. 3.1) */
/* ---------------------------------------------------------------------- */

/* Tree from the leaf-end vector c = [n_1, ..., n_L] (Sec. 3.7): leaf i holds
 * rows c[i-1] .. c[i]-1 (c[-1] = 0).  num_leaves must be a power of two,
 * c non-decreasing, c[L-1] = n.  Empty leaves are allowed (Def. 2.1). */
hm_status hm_tree_create(int64_t n, const int64_t* leaf_ends, int32_t num_leaves, hm_tree** out);

/* Default tree of Sec. 3.1: {1..n} splits into {1..ceil(n/2)} and the rest;
 * every node of a level splits while some node of the level exceeds n_min. */
hm_status hm_tree_default(int64_t n, int64_t n_min, hm_tree** out);

/* n, depth p and number of leaves 2^p of a tree (any pointer may be NULL). */
hm_status hm_tree_shape(const hm_tree* t, int64_t* n, int32_t* depth, int32_t* num_leaves);

/* Copies the leaf-end vector (num_leaves entries) into leaf_ends. */
hm_status hm_tree_leaf_ends(const hm_tree* t, int64_t* leaf_ends);

/* ---------------------------------------------------------------------- */
/* Generators                                                              */
/* ---------------------------------------------------------------------- */

/* HODLR generators, the hodlr class of Sec. 2.1 flattened in node order.
 * For internal node q with children a (left) and b (right):
 *   A(I_a, I_b) = U12[q] * V12[q]^T,  U12[q]: |I_a| x k12[q], V12[q]: |I_b| x k12[q]
 *   A(I_b, I_a) = U21[q] * V21[q]^T,  U21[q]: |I_b| x k21[q], V21[q]: |I_a| x k21[q]
 * D[i] is the m_i x m_i diagonal block of leaf i.  Pointers may be host or
 * device memory (unified addressing); a pointer to an empty block may be NULL.
 * Arrays D has L entries; U12, V12, U21, V21, k12, k21 have L-1 entries. */
typedef struct {
  const double* const* D;
  const double* const* U12;
  const double* const* V12;
  const double* const* U21;
  const double* const* V21;
  const int32_t* k12;
  const int32_t* k21;
} hm_hodlr_gens;

/* HSS generators, the hss class of Sec. 2.2 flattened in node order.
 * ku[q], kv[q]: ranks of the row basis U_q and the column basis V_q of node q
 * (2L-1 entries; the root's are ignored).  Leaf i (node L-1+i):
 *   D[i]: m_i x m_i, U[i]: m_i x ku, V[i]: m_i x kv.
 * Internal non-root node q with children a, b (Eq. 2.2):
 *   RU[q] = [Rl; Rr]: (ku[a] + ku[b]) x ku[q],  RV[q] = [Wl; Wr]: (kv[a] + kv[b]) x kv[q]
 *   (arrays of 2L-1 entries indexed by node id; other entries ignored).
 * Internal node q (root included), core blocks of its children:
 *   B12[q]: ku[a] x kv[b] so that A(I_a, I_b) = U_a B12[q] V_b^T,
 *   B21[q]: ku[b] x kv[a] so that A(I_b, I_a) = U_b B21[q] V_a^T  (L-1 entries). */
typedef struct {
  const double* const* D;
  const double* const* U;
  const double* const* V;
  const double* const* RU;
  const double* const* RV;
  const double* const* B12;
  const double* const* B21;
  const int32_t* ku;
  const int32_t* kv;
} hm_hss_gens;

/* ---------------------------------------------------------------------- */
/* Matrices                                                                */
/* ---------------------------------------------------------------------- */

/* Creates a HODLR matrix (Def. 2.2) on the current CUDA device.  The
 * generators are copied, converted to `storage` (round to nearest even) and
 * packed into library-owned device memory; the caller may free its buffers
 * when the call returns.  Ranks are padded with zero columns to the largest
 * rank of each level; the padded product is exact.  Synchronous. */
hm_status hm_hodlr_create(const hm_tree* t, const hm_hodlr_gens* g, hm_dtype storage, hm_matrix** out);

/* Creates an HSS matrix (Def. 2.3 with Eq. 2.2) on the current device; same
 * ownership and padding rules as hm_hodlr_create.  Translation and coupling
 * operators are held in float64 for HM_F64 storage and in float32 otherwise. */
hm_status hm_hss_create(const hm_tree* t, const hm_hss_gens* g, hm_dtype storage, hm_matrix** out);

typedef struct {
  int32_t kind;          /* hm_kind */
  int32_t storage;       /* hm_dtype */
  int64_t n;
  int32_t depth;         /* p */
  int32_t num_leaves;    /* 2^p */
  int32_t leaf_pad;      /* padded leaf width used by the kernels */
  int32_t rank_total;    /* HODLR: sum over levels of the padded ranks; HSS: padded row-basis (U) rank */
  int64_t generator_elements;  /* unpadded count: HODLR n m + 2 n k p; HSS as Sec. 2.2 */
  size_t  generator_bytes;     /* algorithmic bytes of the generators in `storage` */
  size_t  device_bytes;        /* bytes the library holds on the device for A */
  int32_t tree_cluster;        /* tree phases of the last product: CTAs per cluster of the
                                  one-launch tree kernel, 0 = per-level kernels (or none yet) */
  int32_t tree_columns;        /* right-hand-side columns per cluster (0 likewise) */
  int32_t tree_ring;           /* operator ring slots per CTA (HSS; 0 likewise or HODLR) */
  int32_t rank_col;            /* HSS: padded column-basis (V) rank; HODLR: rank_total */
} hm_matrix_info_t;

hm_status hm_matrix_info(const hm_matrix* A, hm_matrix_info_t* out);

/* Algorithmic generator bytes (the figure a roofline divides by time). */
hm_status hm_matrix_bytes(const hm_matrix* A, size_t* bytes);

/* A^T as a new matrix of the same kind, tree and storage type, built on the
 * current device from A's device storage (products with A^* next to products
 * with A: the constructors of Sec. 3.2-3.3, Table 3.1; real data, so A^T).
 * The generators are relabelled block by block, (A^T)(I, J) = A(J, I)^T:
 * D_i -> D_i^T; HODLR (Def. 2.2) U12' = V21, V12' = U21, U21' = V12,
 * V21' = U12; HSS (Def. 2.3, Eq. 2.2) U' = V, V' = U, R_U' = R_V,
 * R_V' = R_U, B12' = B21^T, B21' = B12^T.  Every stored value is copied, not
 * recomputed, so A^T holds A's values exactly in every storage type and the
 * transpose of the result is A bit for bit.  Products with the result go
 * through hm_hodlr_matmat / hm_hss_matmat like any other matrix.
 * Ownership: *out is a new handle owned by the caller (hm_destroy); A is not
 * modified and may be destroyed first.  Memory: as much device memory as A.
 * Synchronous (runs on the legacy default stream and waits for it).
 * Errors: HM_EINVAL for a NULL out, a handle that is not a matrix, or a
 * current device other than A's; HM_ENOMEM when device memory runs out;
 * HM_ECUDA for another CUDA error.  *out is NULL on any error. */
hm_status hm_matrix_transpose(const hm_matrix* A, hm_matrix** out);

/* The HODLR form of an HSS matrix (hss2hodlr, Sec. 3.5) as a new HODLR matrix
 * on the current device, built from S's device storage.  With the nested
 * bases of Eq. 2.2 written out for every node, the sibling blocks of
 * Def. 2.3 give the HODLR factors of Def. 2.2: U12 = U_a B12, V12 = V_b,
 * U21 = U_b B21, V21 = V_a; the diagonal blocks are copied.  Arithmetic is in
 * the type of S's translation operators (float64 for HM_F64 storage, float32
 * otherwise); every factor is rounded once to S's storage type (HM_BF16X2:
 * hi and lo of the float32 value), so for reduced storage the result differs
 * from S by that rounding.  Every level of the result has S's padded column
 * rank, so its rank_total is p times that rank and it holds about
 * (m + 2 p k) n elements against S's (m + 2 k) n.
 * Ownership: *out is a new handle owned by the caller (hm_destroy); S is not
 * modified.  Synchronous (legacy default stream).
 * Errors: HM_EINVAL for a NULL out, a handle that is not an HSS matrix, or a
 * current device other than S's; HM_EUNSUPPORTED when the ranks need more
 * than 200 KB of shared memory per block (16 (Ke + Kp) elements);
 * HM_ENOMEM / HM_ECUDA for allocation and other CUDA failures.  *out is NULL
 * on any error. */
hm_status hm_hss_to_hodlr(const hm_matrix* S, hm_matrix** out);

/* The Hadamard (entrywise) product C = A o B of two HODLR or two HSS
 * matrices on the same cluster tree, as a new matrix on the current device
 * (Sec. 4.4, Eq. 4.1, Fig. 4.3): D_C = D_A o D_B; every factor of C is the
 * transpose Khatri-Rao product of A's and B's (row i = kron(row i of A's
 * factor, row i of B's), column a1 * k_B + a2); HSS couplings
 * B12_C = B12_A (x) B12_B, B21_C likewise, and each child's block of the
 * stacked translation operators R_U = [R_l; R_r], R_V = [W_l; W_r] is the
 * Kronecker product of A's and B's blocks for that child.  Ranks multiply
 * (HODLR: per level; the padded ranks as stored); no recompression.
 * Products are formed in the translation operators' type (float64 for HM_F64
 * storage, float32 otherwise) and each stored entry of D and of the factors
 * is rounded once to the storage type.
 * Ownership: *out is a new handle owned by the caller (hm_destroy); A and B
 * are not modified (they may be the same matrix).  Synchronous (legacy
 * default stream).
 * Errors: HM_EINVAL for a NULL out, handles that are not matrices, different
 * kinds, storage types or cluster trees, or a current device other than
 * theirs; HM_EUNSUPPORTED when a rank of C exceeds 4096; HM_ENOMEM /
 * HM_ECUDA for allocation and other CUDA failures.  *out is NULL on any
 * error. */
hm_status hm_hadamard(const hm_matrix* A, const hm_matrix* B, hm_matrix** out);

/* Reserves device scratch for products with up to r_max right-hand sides so
 * that later calls allocate nothing (needed before CUDA-graph capture).
 * Synchronous. */
hm_status hm_matrix_reserve(hm_matrix* A, int64_t r_max);

/* ---------------------------------------------------------------------- */
/* Products                                                                */
/* ---------------------------------------------------------------------- */

/* Y = A X (overwrite) for a HODLR matrix: dense leaf blocks times X plus, on
 * every level, each sibling block's U (V^T X) (Sec. 4.1; Fig. 4.1, left).
 *   X: n x r, column-major, leading dimension ldx >= max(n, 1), type xt
 *      (HM_F64, HM_F32 or HM_BF16); Y: n x r, ldy >= max(n, 1), type yt
 *      (HM_F64 or HM_F32).  HM_F64 storage requires xt = yt = HM_F64.
 *   X and Y may be device pointers (used asynchronously on `stream`) or host
 *   pointers (then the call stages them through device scratch and returns
 *   after Y has been written back).  X and Y must not overlap.
 *   r = 0 or n = 0 is a no-op.  Calls on the same matrix must not run
 *   concurrently on different streams: they share the matrix's scratch.
 * Results are deterministic: the reduction order does not depend on timing
 * or on other work on the device. */
hm_status hm_hodlr_matmat(const hm_matrix* A, int64_t r, const void* X, int64_t ldx, hm_dtype xt,
                          void* Y, int64_t ldy, hm_dtype yt, void* stream);

/* Y = A X for an HSS matrix (Sec. 4.1; Fig. 4.1, right): leaf V^T X, upsweep
 * through R_V, couplings S on levels 1..p, downsweep through R_U, leaf U plus
 * D X.  Arguments and rules as hm_hodlr_matmat. */
hm_status hm_hss_matmat(const hm_matrix* A, int64_t r, const void* X, int64_t ldx, hm_dtype xt,
                        void* Y, int64_t ldy, hm_dtype yt, void* stream);

/* Y = A X like hm_hodlr_matmat / hm_hss_matmat (chosen by the matrix's
 * kind), but allocating nothing.  This entry point has no counterpart in the
 * paper; it exists for callers that cannot allocate device memory where they
 * need a product: latency-bound serving loops that must not stall on
 * cudaMalloc's implicit device synchronisation, and applications whose own
 * allocator (a caching allocator or a pool sized at start-up) owns all device
 * memory, so that a library-side allocation could fail or fragment it.
 *   - The per-call scratch lives in one fixed 8 MiB device array compiled into
 *     the library (every GPU that loads the library holds it until the process
 *     exits).  A product whose scratch would exceed 8 MiB -- about
 *     (2L-1) * r * (rank terms) * 4 bytes, see hm_matrix_info -- is rejected
 *     with HM_EINVAL and a message naming the limit; split the columns of X.
 *   - X and Y must be device memory (host buffers would need staging memory)
 *     and must not overlap (HM_EINVAL).
 *   - The first call on a device looks up the array's device address (a
 *     runtime query, no allocation).
 *   - Every call shares the array and it keeps the previous call's contents;
 *     the call clears what must start at zero on `stream`.  Calls whose
 *     kernels overlap on the GPU (concurrent streams or host threads) race on
 *     it and must be serialised by the caller.
 *   - No cudaMalloc, cudaFree or allocating library routine is called. */
hm_status hm_matmat_noalloc(const hm_matrix* A, int64_t r, const void* X, int64_t ldx, hm_dtype xt,
                            void* Y, int64_t ldy, hm_dtype yt, void* stream);

/* Waits for `stream` and reports whether a device-side bounded wait of this
 * library timed out since the last call (HM_ETIMEOUT), then clears the flag. */
hm_status hm_device_status(void* stream);

/* ---------------------------------------------------------------------- */
/* Failure detection and fault injection (not in the paper).  None of these */
/* faults, traps or hangs the GPU: device waits give up after a time limit  */
/* and report through hm_device_status; host failures are simulated.        */
/* ---------------------------------------------------------------------- */

/* Every bounded wait in this library's kernels (mbarrier phases of the TMA
 * and tensor-core pipelines, the tree kernel's operator-ring slots) gives up
 * after `ns` nanoseconds of %globaltimer, records an error code in the
 * device status block, skips its stores and lets the kernel exit.  Default
 * 2e9 (2 s); process-wide; applies to kernels launched after the call.
 * 1e3 <= ns <= 6e10, else HM_EINVAL.  Short limits are for tests of the
 * timeout path: a legitimate wait that outlasts the limit fails the product.
 * Synchronous. */
hm_status hm_set_device_wait_limit(uint64_t ns);
hm_status hm_get_device_wait_limit(uint64_t* ns);

/* Queues on `stream` one small self-test kernel whose two waits can never be
 * satisfied: an mbarrier transaction that is never issued and a flag word
 * that nothing sets.  Each gives up after the device wait limit and records
 * its code (31, 32); the kernel then exits normally, so the context stays
 * usable and the next hm_device_status on the stream returns HM_ETIMEOUT.
 * It touches only its own shared memory and the library's status block. */
hm_status hm_selftest_device_timeout(void* stream);

/* Host-side fault injection: the next `count` device allocations made by the
 * library (generators at create time, product scratch, host staging, batch
 * and server buffers) fail as if the device were out of memory, so the call
 * that needed them returns HM_ENOMEM and leaves no partial object behind.
 * count = 0 disarms.  Process-wide. */
hm_status hm_inject_alloc_failures(int32_t count);

/* Selects the kernel family for later products on this matrix:
 * 0 = automatic (tensor cores when r is wide enough and storage is BF16 or
 * BF16X2), 1 = SIMT only, 2 = tensor cores whenever supported. */
hm_status hm_matrix_set_path(hm_matrix* A, int32_t path);

/* Kernels for the tree phases of later products on this matrix (Sec. 4.1:
 * the HSS upsweep, couplings and downsweep, or the HODLR per-level sums):
 * 0 = automatic, 1 = one launch per phase with per-level handoffs through
 * global memory, 2 = one launch of thread-block clusters that keeps the
 * levels in shared memory, when the shape fits (else as 1).  Both sum in the
 * same order, so the results are identical; 0 picks 2 when it fits. */
hm_status hm_matrix_set_tree(hm_matrix* A, int32_t mode);

/* Chooses the launch shape of the one-launch tree kernel (levels shared by a
 * thread-block cluster, right-hand-side columns per cluster, operator-ring
 * slots) for products with r columns of types xt, yt by timing the whole
 * product (three each, on zero inputs) with every shape that fits on this
 * device, instead of the built-in cost estimate; later products with r
 * columns use the fastest.  The product is timed, not the tree alone,
 * because the expansion starts while the tree drains and competes with it
 * for SMs.  No result changes: every shape sums in the same order.
 * Allocates the scratch for r columns if needed and temporary X, Y buffers;
 * synchronous.  *best_ms (may be NULL) receives the chosen shape's time per
 * product.  HM_EUNSUPPORTED when the tree runs as per-level kernels for this
 * matrix (or F64 storage with other X, Y types). */
hm_status hm_matrix_tune_tree(hm_matrix* A, int64_t r, hm_dtype xt, hm_dtype yt, double* best_ms);

/* Pins the launch shape of the one-launch tree kernel for products of r
 * columns (not in the paper): clusters of cluster_ctas CTAs (2, 4, 8 or 16,
 * at most 2^depth), each cluster taking `columns` (1, 2, 4 or 8) of the
 * right-hand-side columns, with ring_slots (2..12; 0 for HODLR) operator
 * slots per CTA.  Every shape sums in the same order, so results do not
 * depend on it; only the time does.  HM_EINVAL for values outside those
 * sets; HM_EUNSUPPORTED when the shape does not fit this matrix in shared
 * memory or no cluster of it can be resident, or when the tree runs as
 * per-level kernels.  A later hm_matrix_tune_tree replaces it. */
hm_status hm_matrix_set_tree_shape(hm_matrix* A, int64_t r, int32_t cluster_ctas, int32_t columns,
                                   int32_t ring_slots);

/* Per-kernel timing of later products on this matrix: with enable = 1 every
 * kernel launch of a product is bracketed by CUDA events recorded on the
 * product's stream; enable = 0 stops recording.  Not for use under CUDA-graph
 * capture. */
hm_status hm_matrix_profile(hm_matrix* A, int32_t enable);

/* Device time accumulated per phase since the last read, in milliseconds,
 * and the number of launches: phase 0 = leaf projection (V^T X), 1 = tree
 * upsweep (HSS: translations R_V and couplings; HODLR: per-level sums),
 * 2 = HSS downsweep, 3 = leaf expansion, 4 = the diagonal-block product D X
 * when it runs as a launch of its own (FP64 storage with wide X; the
 * expansion then adds E Z to it).  Waits for the recorded events, then
 * resets the accumulators. */
hm_status hm_matrix_phase_times(hm_matrix* A, double ms[5], int64_t launches[5]);

/* ---------------------------------------------------------------------- */
/* Solves with an HSS matrix (Sec. 4.3)                                     */
/* ---------------------------------------------------------------------- */

/* Factors an HSS matrix A (F64 storage) for solves by the implicit ULV
 * scheme of Sec. 4.3, on A's device.  Level by level from the leaves: a QL
 * factorization of each node's row basis (Q^T U = [0; Ut], Step 1), an LQ of
 * the top rows of Q^T D that triangularizes them (Z, Step 1), the split of
 * the product into a block-triangular factor and a reduced system on the
 * trailing ku x ku blocks (Step 2), and the merge of sibling nodes into the
 * next level's blocks (Step 3); the root's block gets a full LQ.  Kept per
 * node on the device: Q^T and Z (n x n), the inverse of the triangular block,
 * the blocks that carry solved parts across levels.  Memory: about three
 * times the dense leaf blocks (leaves padded with identity rows to at least
 * ku + 1).  The reflectors are chosen without pivoting, as in the paper; a
 * singular A (or one whose eliminated blocks are singular) gives infinities.
 * Requires equal padded row and column ranks and depth >= 1 (HM_EUNSUPPORTED
 * otherwise).  A must outlive the factorization (its translation operators
 * are read by hm_ulv_solve).  Synchronous.
 * Errors: HM_EINVAL (NULL out, not an HSS matrix, wrong device),
 * HM_EUNSUPPORTED, HM_ENOMEM, HM_ECUDA.  *out is NULL on any error. */
hm_status hm_ulv_factor(const hm_matrix* A, hm_ulv** out);

/* X = A^{-1} B with the factorization F: B and X are n x r float64 device
 * buffers, column-major with leading dimensions ldb, ldx >= n; they may be
 * the same buffer only if ldb = ldx.  Applies Q^T, the triangular solves and
 * the merges upward, the root's solve, then Z downward (Step 4): a sequence
 * of batched FP64 products queued on `stream`.  The first call with a given
 * r allocates the work space (and synchronises); calls on one factorization
 * must not run concurrently. */
hm_status hm_ulv_solve(const hm_ulv* F, int64_t r, const void* B, int64_t ldb, void* X, int64_t ldx, void* stream);

/* ---------------------------------------------------------------------- */
/* Batched products (the paper runs one product at a time; batching many   */
/* matrices is this library's addition)                                    */
/* ---------------------------------------------------------------------- */

typedef struct {
  int32_t count;             /* products in the batch */
  int32_t launches_per_run;  /* persistent kernel launches per run (at most 6) */
  int64_t items[6];          /* work items per phase: SIMT projection, tensor-core
                                projection, upsweep, downsweep, SIMT expansion,
                                tensor-core expansion */
  int32_t grid[6];           /* persistent blocks per phase */
  int32_t graph;             /* 1 if runs replay a captured CUDA graph */
  int32_t tuned;             /* 0 defaults, 1 tuned by timing, 2 read from the cache file */
  int32_t grid_mult;         /* tuned launch shapes: persistent blocks per SM, */
  int32_t rc_cap;            /*   widest SIMT column chunk, */
  int32_t rct_cap;           /*   widest tree column chunk, */
  int32_t tile_rows;         /*   rows per SIMT expansion tile */
  int32_t capture_error;     /* CUDA error that prevented graph capture (runs then launch directly), 0 if none */
} hm_batch_info_t;

/* Groups `count` products Y_j = A_j X_j (r[j] right-hand sides each) into one
 * batch.  Matrices may differ in kind (HODLR/HSS), size, tree, rank, storage
 * (HM_F32, HM_BF16, HM_BF16X2; HM_F64 returns HM_EUNSUPPORTED) and r, but
 * must live on one device and outlive the batch.  Scratch for every product is
 * reserved and the work lists of the six phases are built (each product keeps
 * exactly the blocking it has alone, so its result is bit-identical in the
 * batch and alone).  Synchronous. */
hm_status hm_batch_create(hm_matrix* const* A, const int64_t* r, int32_t count, hm_batch** out);

/* Chooses the launch shapes (persistent blocks per SM, SIMT and tree column
 * chunk widths, SIMT tile height) by timing candidates on the device with
 * temporary zero inputs (coordinate descent).  With cache_path != NULL a stored
 * choice for the same batch signature (kinds, storages, sizes, ranks, r) is
 * reused, and a new choice is appended to the file.  None of the shapes
 * changes any result.  Synchronous; allocates temporary buffers. */
hm_status hm_batch_tune(hm_batch* b, const char* cache_path);

/* Runs every product of the batch: X[j] (n_j x r_j, column-major, ld = n_j,
 * type xt: HM_F32, HM_BF16 or HM_F64) and Y[j] (ld = n_j, type yt: HM_F32 or
 * HM_F64) are device pointers.  The work is one persistent launch per
 * non-empty phase (SIMT and tensor-core projection, tree upsweep, HSS
 * downsweep, SIMT and tensor-core expansion), recorded into a CUDA graph at
 * the first run and replayed after.
 * Asynchronous on `stream`; runs of one batch must not overlap. */
hm_status hm_batch_run(hm_batch* b, const void* const* X, void* const* Y, hm_dtype xt, hm_dtype yt, void* stream);

hm_status hm_batch_info(const hm_batch* b, hm_batch_info_t* out);

/* ---------------------------------------------------------------------- */
/* Serving (continuous batching of product requests; not in the paper)    */
/* ---------------------------------------------------------------------- */

typedef struct {
  int64_t submitted;        /* requests offered to hm_serve_submit */
  int64_t admitted;         /* accepted */
  int64_t rejected;         /* refused with HM_EBUSY */
  int64_t completed;        /* finished */
  int64_t launches;         /* merged products launched */
  int32_t pending;          /* admitted and not yet completed */
  int32_t max_merged;       /* most requests merged into one product */
  size_t resident_bytes;    /* device bytes of registered matrices and their buffers */
  double p50_us;            /* submit-to-completion latency percentiles and mean, */
  double p99_us;            /*   over completed requests since creation or reset */
  double mean_us;
  double throughput_rps;    /* completed requests per second (first submit to last completion) */
  double gbs;               /* algorithmic bytes of the launched products per second */
} hm_serve_stats_t;

/* Creates a server on the current device: at most max_slots requests may be
 * admitted and unfinished at once, and registered matrices plus admitted
 * requests' buffers may use at most mem_budget device bytes.  A worker thread
 * takes the queued requests continuously, merges requests for the same matrix
 * into one product with up to 64 columns, and runs products of different
 * matrices on separate streams so they overlap. */
hm_status hm_serve_create(size_t mem_budget, int32_t max_slots, hm_server** out);

/* Makes a matrix resident for serving (F32, BF16 or BF16X2 storage).  Its
 * scratch and merge buffers are reserved now and counted, with the matrix
 * itself, against the budget (HM_ENOMEM if they do not fit).  The matrix's
 * kernel family is fixed (tensor cores for BF16/BF16X2, SIMT otherwise) so
 * that a request's result does not depend on the requests it is merged with.
 * The matrix must outlive the server.  *id receives the matrix's id. */
hm_status hm_serve_register(hm_server* s, hm_matrix* A, int32_t* id);

/* Queues Y = A_id X for X, Y device buffers of n x r float32 values,
 * column-major with leading dimension n (1 <= r <= 64).  Non-blocking:
 * returns HM_EBUSY, without queuing, when no slot or budget is free.  *ticket
 * identifies the request for hm_serve_wait / hm_serve_poll. */
hm_status hm_serve_submit(hm_server* s, int32_t id, int64_t r, const void* X, void* Y, uint64_t* ticket);

/* Waits up to timeout_ms for a request: HM_OK (Y is written), HM_ETIMEOUT
 * (still pending; the ticket stays valid) or the error of its product.  Never
 * waits longer than the timeout. */
hm_status hm_serve_wait(hm_server* s, uint64_t ticket, int32_t timeout_ms);

/* Non-blocking: HM_OK when the request has finished, HM_EBUSY while pending. */
hm_status hm_serve_poll(hm_server* s, uint64_t ticket);

/* Withdraws a request that is still queued: HM_OK (it will never run, Y is
 * not written, its slot and budget are released and the ticket becomes
 * unknown); HM_EBUSY when it is already running or finished (wait for it
 * instead); HM_EINVAL for an unknown ticket. */
hm_status hm_serve_cancel(hm_server* s, uint64_t ticket);

/* pause = 1: the worker stops taking queued requests (products already
 * launched finish); requests are still admitted and wait in the queue, as
 * when a worker stalls.  pause = 0 resumes.  For tests of hm_serve_wait's
 * timeout and of cancellation. */
hm_status hm_serve_pause(hm_server* s, int32_t pause);

hm_status hm_serve_stats(hm_server* s, hm_serve_stats_t* out);
hm_status hm_serve_reset_stats(hm_server* s);

/* Releases any object created by this library (tree, matrix, batch, server,
 * ULV factorization).
 * NULL-safe.  A matrix registered with a server must be released after the
 * server. */
void hm_destroy(void* any);

#ifdef __cplusplus
}
#endif

#endif /* HM_H */
