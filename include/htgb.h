/*
 * htgb.h -- C-ABI of the GB300 (sm_103a) library for the HSVD truncation of
 * tensors in the Hierarchical Tucker (HT) format after HT addition.
 *
 * Method: Grasedyck & Loebbert, "Distributed Hierarchical SVD in the
 * Hierarchical Tucker Format".  Each call below names the section / equation
 * that defines what it computes.  Every floating-point step runs in this
 * library's CUDA kernels on the tensor's stream; there is no CPU fallback.
 *
 * Conventions
 *  - Modes and tree nodes are 0-based.  The dimension tree is the balanced
 *    tree of Sec. 2.1 (eq. "balanced"): node {mu..nu} has the sons
 *    {mu..floor((mu+nu-1)/2)} and the rest (1-based), numbered in pre-order,
 *    root = 0.  ht_tree_node gives the structure.
 *  - Ranks are given per node in pre-order; the root's entry is 1 (k_D = 1).
 *  - Leaf {mu}: frame U (n_mu x k_t), column-major, ld = n_mu.
 *  - Inner node t with sons s1, s2: transfer tensor B_t (k_t x k_s1 x k_s2),
 *    element (i,j,l) at (i*k_s1 + j)*k_s2 + l, so M_{2,3}(B_t) is the
 *    column-major (k_s1 k_s2) x k_t matrix.  The root holds B_D (k_t1 x k_t2)
 *    as [j][l].
 *  - "Packed blob": the node arrays above concatenated in pre-order, in the
 *    tensor's dtype.  ht_tensor_upload / ht_tensor_download use it.
 *  - Ownership: handles are owned by the library (free them with the
 *    matching *_free).  Pointers passed in are borrowed for the duration of
 *    the call; device pointers returned by *_ptr calls stay valid until the
 *    tensor is freed or changed by an in-place call.
 *  - Errors: every call returns an ht_status; nothing is thrown across the
 *    ABI.  ht_last_error() gives a thread-local message for the last failure.
 *  - Streams: each tensor carries a cudaStream_t (passed as void*; NULL is
 *    the legacy default stream).  Calls enqueue work on it and return without
 *    waiting, except where a call is marked "synchronises".
 */
#ifndef HTGB_H
#define HTGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ht_tree ht_tree;
typedef struct ht_tensor ht_tensor;

typedef enum {
  HT_OK = 0,
  HT_EINVAL = 1,       /* bad argument (sizes, ranks, null pointer, mismatched trees) */
  HT_ENOMEM = 2,       /* device or host allocation failed */
  HT_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  HT_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  HT_ENUMERIC = 5,     /* non-finite values met where finite ones are required */
  HT_EUNSUPPORTED = 6  /* valid request this build does not handle (e.g. dtype/precision mix) */
} ht_status;

typedef enum { HT_F64 = 0, HT_F32 = 1 } ht_dtype;

/* Arithmetic of the truncation.  HT_PREC_FP64: every step in FP64 (F64
 * tensors).  HT_PREC_FP32: storage and dense contractions in FP32, the small
 * k x k Gramian eigendecompositions solved in FP32 and refined to FP64-level
 * accuracy (one Ogita-Aishima step with double-float products, about 48
 * bits) (F32 tensors).
 * HT_PREC_FP32_SQRT: as HT_PREC_FP32, but the reduced Gramians of Sec. 3.3
 * are carried as square-root factors Ghat_t = S_t S_t^T (top-down: the sons'
 * Gramians are Gram products of B_t contracted with S_t, accumulated exactly
 * in double-float with FP64 results; S_s is their semidefinite Cholesky
 * factor), so FP32 rounding perturbs the singular values by O(u_32 sigma_max)
 * instead of O(sqrt(u_32) sigma_max); the eps rule's noise floor becomes
 * (4 sqrt(2d-1) u_32)^2 sigma_{t,1}^2.  F32 tensors.  This is the direction
 * the paper's conclusion names for avoiding B^T B products.
 * HT_PREC_MIXED: F64 tensors; the R-factor QRs (Sec. 3.4) and the Gramian
 * eigendecompositions stay in FP64, and every dense contraction (mode products
 * of Lemma "transfer tensor transformation", Gramian contractions of eqs.
 * "acctransferSon1/2", leaf products, TSQR recombination) runs on the tcgen05
 * tensor cores: each FP64 operand row is put on a common fixed-point grid and
 * cut into 5 BF16 slices of 8 bits, the slice products with index sum <= 4 are
 * accumulated in FP32 (exactly for the leading ones, over chunks of at most
 * 256 products) and the chunks are summed in FP64.  Per product about 2^-40
 * of |a| |b| (normwise), against 2^-53 for FP64 and 2^-24 for FP32; the eps
 * rule is the FP64 one (nu_t = 0). */
typedef enum { HT_PREC_FP64 = 0, HT_PREC_FP32 = 1, HT_PREC_FP32_SQRT = 2, HT_PREC_MIXED = 3 } ht_prec;

typedef enum { HT_TRUNC_RANK = 0, HT_TRUNC_EPS = 1 } ht_trunc_mode;

/* Launch schedule: all nodes of one tree level in one batched launch per
 * step (default), or one launch per tree node (the plain reference schedule). */
typedef enum { HT_SCHED_LEVEL = 0, HT_SCHED_NODE = 1 } ht_schedule;

/* Options of the truncation T(X) (Sec. 3.3; Sec. 3.5 "to prescribed ranks or
 * to prescribed accuracy"; Sec. 5: absolute eps with a rank cap).
 *  mode = HT_TRUNC_RANK: r_t = min(ranks[t] (or rank_cap if ranks == NULL),
 *         rank_cap if > 0, rank available after orthogonalization).
 *  mode = HT_TRUNC_EPS:  r_t = smallest r >= 1 with sum_{i>r} (sigma_{t,i}^2 + nu_t)
 *         <= eps_abs^2 / (2d-3), eps_abs = eps * ||X|| if eps_relative, then
 *         capped as above.  On F64 tensors nu_t = 0: the computed tail alone
 *         decides.  On F32 tensors nu_t = 4 sqrt(2d-1) u_32 sigma_{t,1}^2 (its
 *         square for HT_PREC_FP32_SQRT) is the noise floor of an eigenvalue of
 *         an FP32-computed Gramian: an eps below what that arithmetic resolves
 *         keeps rank.  The two sons of the root have the same singular values
 *         and share one rank (decided on the first son).
 *  prec: HT_PREC_FP64 and HT_PREC_MIXED need an F64 tensor, HT_PREC_FP32 and
 *         HT_PREC_FP32_SQRT an F32 tensor.
 *  tensor_caps: NULL, or (batch calls) one rank cap per tensor, host array of
 *         count entries, used instead of rank_cap for that tensor. */
typedef struct {
  int mode;
  double eps;
  int eps_relative;
  int rank_cap;
  const int *ranks; /* host, one per node in pre-order, or NULL */
  int prec;
  int schedule;
  const int *tensor_caps; /* host, one per tensor of a batch call, or NULL */
  int qr_kernel;          /* TSQR row-block kernel: 0 by shape and launch size (default;
                             HT_PREC_MIXED: double-float blocks, about 2^-47 relative,
                             on the FP32 pipe), 1 the one-column kernel, 2 the
                             two-column kernel (F32 blocks of 64 columns; smaller
                             blocks keep their kernel), 3 HT_PREC_MIXED with FP64
                             Householder blocks */
} ht_trunc_opts;

/* Optional report (pass NULL to skip; synchronises when given).  With a
 * report the truncation returns HT_ENUMERIC (after filling the report) when a
 * tensor's ||X|| or one of its Gramian eigenvalues is not finite, e.g. NaN or
 * Inf in the input; without one, ht_device_status reports it.
 *  norm         ||X|| = ||B_D||_F after orthogonalization (Sec. 3.4)
 *  discarded_sq sum over non-root nodes of the discarded sigma^2 (root pair once)
 *  bound        sqrt(discarded_sq): the a-priori error bound of [Gr10]
 *  ranks_out    caller array of 2d-1 ints, or NULL: the truncated ranks
 *  korth_out    caller array of 2d-1 ints, or NULL: ranks after orthogonalization
 *  sigma_out    caller array, or NULL: for every non-root node in pre-order,
 *               korth_out[t] singular values (descending), concatenated */
typedef struct {
  double norm;
  double discarded_sq;
  double bound;
  int *ranks_out;
  int *korth_out;
  double *sigma_out;
} ht_trunc_report;

/* ---- dimension tree (Sec. 2.1) ---------------------------------------- */

/* Balanced dimension tree for d >= 2 modes (eq. "balanced"). */
ht_status ht_tree_balanced(int d, ht_tree **out);
void ht_tree_free(ht_tree *tree);
/* Number of nodes (2d-1), or -1 for NULL. */
int ht_tree_num_nodes(const ht_tree *tree);
/* Structure of node t: mode range [lo, hi], parent (-1 at the root), sons
 * (-1 at leaves), depth (root 0) and height (leaves 0).  Any output may be NULL. */
ht_status ht_tree_node(const ht_tree *tree, int t, int *lo, int *hi, int *parent, int *son1, int *son2,
                       int *depth, int *height);

/* ---- HT container (Sec. 2.2) ------------------------------------------ */

/* Allocate an HT tensor on the current device: n[d] mode sizes, ranks[2d-1]
 * (root entry ignored, taken as 1), dtype, stream.  Contents are zero. */
ht_status ht_tensor_create(const ht_tree *tree, const int64_t *n, const int *ranks, ht_dtype dtype, void *stream,
                           ht_tensor **out);
ht_status ht_tensor_free(ht_tensor *x);
/* Current ranks (2d-1 ints); synchronises if ranks were decided on the device. */
ht_status ht_tensor_ranks(ht_tensor *x, int *ranks);
/* Number of elements of the packed blob at the current ranks (synchronises like ht_tensor_ranks). */
ht_status ht_tensor_blob_size(ht_tensor *x, int64_t *count);
/* Copy a packed blob (current ranks, tensor dtype) from host memory into the
 * tensor: asynchronous on the tensor's stream; pinned host memory overlaps. */
ht_status ht_tensor_upload(ht_tensor *x, const void *host_blob);
/* Copy the tensor out as a packed blob into host memory (synchronises). */
ht_status ht_tensor_download(ht_tensor *x, void *host_blob);
/* Device pointer of node t's array (leaf frame / transfer tensor / root),
 * and its element count at the current ranks. */
ht_status ht_tensor_node_ptr(ht_tensor *x, int t, void **dev, int64_t *count);
/* Multiply the tensor by alpha (scales the root transfer matrix). */
ht_status ht_scale(ht_tensor *x, double alpha);

/* ---- arithmetic --------------------------------------------------------- */

/* HT addition, Lemma "sum of two H-tensors" (Sec. 3.5, eq. "sumleafframes"):
 * W = [U, V] at the leaves, H_t = blockdiag(B_t, F_t) inside, H_D =
 * blockdiag(B_D, F_D) at the root.  Allocates *out (ranks k + kbar) on a's
 * stream.  a and c must share d, n and dtype. */
ht_status ht_add(const ht_tensor *a, const ht_tensor *c, ht_tensor **out);
/* Same, into an existing tensor whose ranks already equal k + kbar (no allocation). */
ht_status ht_add_into(const ht_tensor *a, const ht_tensor *c, ht_tensor *out);

/* Application of an H-operator to an H-tensor, Lemma "operator" (Sec. 3.6):
 * out = L X.  The operator L is an HT tensor over the index pairs
 * (j_mu, i_mu) (eq. "operatorastensor"), i.e. an ht_tensor with mode sizes
 * m_mu n_mu whose leaf columns are column-major m_mu x n_mu matrices W_r
 * (pair (j, i) at j + i m_mu); X has mode sizes n_mu; out must be created with
 * mode sizes m_mu and capacities kbar_t k_t (kbar: ranks of L, k: of X).
 * Leaves: V[:, r k + l] = W_r U[:, l] (eq. "operatorleafframes", batched
 * products); inner nodes: F_t = H_t (x) B_t, the pair (p, i) of (operator
 * rank, tensor rank) at p k_t + i.  The ranks of out become kbar_t k_t;
 * truncate it with ht_truncate.  Same tree and dtype for all three.  Errors:
 * HT_EINVAL (shapes, capacities), HT_ENOMEM, HT_ECUDA. */
ht_status ht_apply(const ht_tensor *op, const ht_tensor *x, ht_tensor *out);

/* Orthogonalization, Sec. 3.4 (leaves -> root): QR of every leaf frame and of
 * M_{2,3}(B_t) of every inner node after B_t <- (I, R_s1, R_s2) o B_t; the root
 * becomes R_t1 B_D R_t2^T.  In place; ranks become min(n, k) at leaves and
 * min(k_t, k_s1 k_s2) inside (eq. "qrtransfer").  prec as in ht_trunc_opts. */
ht_status ht_orthogonalize(ht_tensor *x, int prec);

/* Reduced Gramians Bhat_t = V_t^T V_t of an ORTHOGONAL tensor, Sec. 3.3: eq.
 * "acctransferroot" for the sons of the root, eqs. "acctransferSon1/2"
 * top-down.  dev_out: device FP64 buffer, for every node in pre-order a
 * k_t x k_t block (column-major; the root's block is the 1x1 matrix 1). */
ht_status ht_gramians(ht_tensor *x_orth, double *dev_out, int prec);

/* Same result as ht_gramians, but the call allocates no device memory.
 * (Not a step of the paper: it serves callers that cannot let a library
 * allocate, e.g. a program that reserves all device memory up front under a
 * fixed budget or hands every buffer out from its own allocator, so that a
 * hidden cudaMalloc/cudaMallocAsync would break its accounting or fail.)
 * The workspace is one fixed device array of HT_NOALLOC_SCRATCH_BYTES that
 * every GPU loading this library keeps until the process exits; the caller
 * still provides the tensor and dev_out.  The first call on a device looks up
 * the array's device address (with that device current).  A tensor whose
 * workspace needs more than the array holds is rejected with HT_ENOMEM and a
 * message giving both sizes.
 * All calls share the one array and its contents persist between calls:
 * calls that can run at the same time on the GPU (different streams, or
 * several host threads) race on it and must be serialised by the caller. */
#define HT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
ht_status ht_gramians_noalloc(ht_tensor *x_orth, double *dev_out, int prec);
/* (The fixed array used is the current device's: the tensor's stream must run
 * on the current device, else HT_EINVAL.) */

/* HSVD truncation T(X), Sec. 3.3 after Sec. 3.4, in place: orthogonalize,
 * Gramians of all non-root nodes, their eigendecompositions (singular values
 * of every matricization), ranks, then the projection U <- U Q|_r,
 * B_t <- (Q_t|_r^T, Q_s1|_r^T, Q_s2|_r^T) o B_t (eq. "transfertransformationtrunc"),
 * B_D <- Q_t1^T B_D Q_t2. */
ht_status ht_truncate(ht_tensor *x, const ht_trunc_opts *opts, ht_trunc_report *report);
/* Truncate count tensors (any d, n, ranks; one dtype) with the same options,
 * each tree level of all tensors in one batched launch.  report: NULL or an
 * array of count reports. */
ht_status ht_truncate_batch(ht_tensor *const *xs, int count, const ht_trunc_opts *opts, ht_trunc_report *reports);

/* CUDA graph of the hot path: out[i] = T(a[i] + c[i]) for i < count, i.e.
 * the addition of Sec. 3.5 (Lemma "sum of two H-tensors": leaf frames side by
 * side, transfer tensors block-diagonal) followed by the truncation of
 * ht_truncate_batch with options opts, recorded once and replayed by
 * ht_graph_launch without host work.
 * a, c: count summand pairs (same d, n, dtype per pair).  out: count tensors
 * created with capacities a[i] ranks + c[i] ranks (as ht_add_into requires);
 * each replay overwrites them (their ranks become the truncated ranks).
 * All tensors must use one stream, on which every replay is enqueued.  The
 * graph borrows the tensors: they must outlive it and keep their ranks
 * (a[i], c[i] unchanged between replays).  Its device workspace (the
 * truncation workspace plus descriptors) is allocated here, once, and freed
 * by ht_graph_free.  Errors: HT_EINVAL (shapes, streams, options),
 * HT_ENOMEM, HT_ECUDA (capture or instantiation refused by the driver). */
typedef struct ht_graph ht_graph;
ht_status ht_graph_add_truncate(const ht_tensor *const *a, const ht_tensor *const *c, ht_tensor *const *out, int count,
                                const ht_trunc_opts *opts, ht_graph **graph);
/* Enqueue one replay on the tensors' stream (asynchronous). */
ht_status ht_graph_launch(ht_graph *graph);
/* Number of kernel nodes one replay launches. */
ht_status ht_graph_kernels(const ht_graph *graph, int *kernels);
/* Wait for the graph's stream, then release the graph and its workspace. */
ht_status ht_graph_free(ht_graph *graph);

/* ||X||: orthogonalizes a copy, returns ||B_D||_F (Sec. 3.4).  Synchronises. */
ht_status ht_norm(const ht_tensor *x, double *out);
/* Inner product <X, Y> (Sec. 3.2, Lemma "phi"): Phi_t = U_t^T V_t computed
 * bottom-up from the leaves (Phi = U^T V) through the transfer tensors,
 * Phi_t = M_1(B_t) (Phi_s1 (x) Phi_s2) M_1(B'_t)^T, one batched launch per
 * contraction and tree level; the root's 1 x 1 Phi is <X, Y>.  X and Y: same
 * d, mode sizes and dtype, any ranks; neither needs to be orthogonal.  The
 * sum runs in the tensors' dtype (F32: FP32 contractions, long reductions
 * split with FP64 partial sums).  Synchronises.  Errors: HT_EINVAL. */
ht_status ht_inner(const ht_tensor *x, const ht_tensor *y, double *out);

/* Entries X[idx[e*d + 0], ..., idx[e*d + d-1]] for e < m (Sec. 3.1, eq.
 * "transfermult").  idx and out are host arrays.  Synchronises. */
ht_status ht_eval_entries(const ht_tensor *x, const int64_t *idx, int64_t m, double *out);

/* ---- tracing ------------------------------------------------------------- */

/* Kernel families of this library, for launch accounting and timing. */
typedef enum {
  HT_K_GEMM = 0,    /* strided batched contractions (mode products, Gramians, leaf products, TSQR recombination) */
  HT_K_QR = 1,      /* Householder QR of shared-memory row blocks (TSQR) */
  HT_K_EIG = 2,     /* symmetric eigensolver (FP64, or FP32 + refinement) */
  HT_K_COPY = 3,    /* copies, casts, identity fills */
  HT_K_COMPACT = 4, /* packing of projected transfer tensors */
  HT_K_RANKS = 5,   /* rank selection and ||X|| */
  HT_K_ADD = 6,     /* HT addition packing */
  HT_K_EVAL = 7,    /* entry evaluation */
  HT_K_MISC = 8,    /* norms, scaling */
  HT_K_SPLIT = 9,   /* BF16 slicing of the tensor-core contractions' operands (mixed path);
                       its "flops" in ht_profile_read are algorithmic bytes */
  HT_K_COUNT = 10
} ht_kernel_kind;

/* Record CUDA events around every launch of the kinds set in mask (bit
 * 1 << kind) on the launching stream; 0 switches recording off.  Not thread-safe. */
ht_status ht_profile_set(unsigned mask);
/* Launches, summed device time (ms) and summed algorithmic flops (counted at
 * the launches' maximal dimensions: 2 m n k for contractions (on the mixed
 * path the BF16 work of the tensor cores, S (S + 1) / 2 slice products of
 * 2 m n k each),
 * 4 m n^2 - 4 n^3 / 3 per QR block, 9 k^3 per eigendecomposition) of one kind
 * recorded since the last reset; synchronises on the recorded events.
 * reset != 0 clears the record.  Any output may be NULL. */
ht_status ht_profile_read(int kind, int64_t *launches, double *total_ms, double *flops, int reset);
/* Number of kernels this library has launched since it was loaded (all kinds). */
ht_status ht_launch_count(int64_t *total);

/* Synchronises the device, then reads and clears the library's device
 * status words:
 *  - bounded waits: every wait of a library kernel (the tcgen05 contractions'
 *    mbarrier waits, the self-test below) is limited in time; one that gave
 *    up marks its results invalid, sets a word and returns -> HT_ETIMEOUT;
 *  - an eigensolver sweep that reached its iteration limit -> HT_ENUMERIC;
 *  - a non-finite ||X|| or Gramian eigenvalue met by a truncation (NaN or Inf
 *    in the input) -> HT_ENUMERIC.
 * HT_ECUDA if the device reports an error, else HT_OK. */
ht_status ht_device_status(void);

/* Self-test of the bounded-wait machinery (no counterpart in the paper):
 * enqueues on `stream` one kernel whose single thread waits for a device flag
 * that no code ever sets, with the library's time bound set to limit_ms
 * (0 <= limit_ms <= 1000); the wait runs out, marks the wait status word and
 * the kernel returns.  The next ht_device_status returns HT_ETIMEOUT and the
 * context stays usable.  Errors: HT_EINVAL (limit), HT_ECUDA (launch). */
ht_status ht_selftest_wait(double limit_ms, void *stream);

/* Tile-shape rule of the SIMT contraction kernel: launches whose flops lie
 * mostly (share >= tall_share) in items with M >= tall_m use 128-row tiles,
 * those with square_share in items with M, N >= tall_m 128 x 128 tiles.  The
 * defaults are the committed autotuner table; tall_m < 0 restores them.  Used
 * by the autotuner to time candidates without rebuilding; not thread-safe. */
ht_status ht_set_gemm_tuning(int tall_m, double tall_share, double square_share);

/* Message of the last failing call on this thread ("" if none). */
const char *ht_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HTGB_H */
