// internal.h -- work items and kernel launchers shared by the library's
// translation units.  Every kernel walks a device array of work items, so
// one launch covers all nodes of one tree level (or of many tensors).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace htgb {

constexpr int kSmCount = 152;  // GB300: two dies x 76 SMs

// ---------------------------------------------------------------------------
// Strided batched contraction ("GEMM" item):
//   C[m,n] (b) = alpha * sum_{ko<Ko} sum_{k<K} A[m,k,ko](b) * B[k,ko,n](b) + beta * C[m,n](b)
// element addresses:  A + b*sab + m*sam + k*sak + ko*sako
//                     B + b*sbb + k*sbk + ko*sbko + n*sbn
//                     C + b*scb + m*scm + n*scn
// Dimensions marked by a rank reference (>= 0) are read on the device:
//   dim = min(dim_literal, ranks[ref] * mult)
// which lets the projection run on ranks decided on the device (eps mode).
// Split-K: the Ko range is cut into `ksplit` chunks whose partial sums go to
// `part` (dense M x N per chunk and batch, column-major); a second kernel sums
// them in a fixed order.
// ---------------------------------------------------------------------------
struct GemmItem {
  const void *A, *B;
  void *C;
  void *part;  // split-K partial buffer (ksplit * batch * M * N elements) or null
  int64_t sam, sak, sako, sab;
  int64_t sbk, sbko, sbn, sbb;
  int64_t scm, scn, scb;
  int M, N, K, Ko, batch;
  int m_ref, n_ref, b_ref;  // rank refs (-1: none)
  int n_mult, b_mult;
  int ksplit;
  double alpha, beta;
  int tiles_m, tiles_n;  // tile grid at the literal (maximal) dims
  int tile0;             // first global tile index of this item
  int tc_tiles_m, tc_tiles_n, tc_tile0;  // same for the tensor-core kernel's 128 x 128 tiles (k_oz.cu)
  int64_t k_total;  // >= 0: only flat reduction indices ko * K + k < k_total take part (ragged last chunk)
  // tensor-core path (k_oz.cu): BF16 slices of A and B in 8 KB stage blocks,
  // per-(row, chunk) exponents, stages per chunk, first CTA of the split launch
  void *oza, *ozb;
  int *oea, *oeb;
  int oz_stages;
  int oz_split0;
  int oz_share;  // bit 0: A, bit 1: B is the same for every batch entry (sliced once)
  // bit 0: A's slices and exponents are given in oza / oea (made by an earlier
  // launch), not by this launch's split; bit 1: a slicing-only item (operand A
  // only, no B, no tiles, no output)
  int oz_pre;
  int oz_row0;  // slicing-only items: first row of A's slices within its 128-row block
};

// Householder QR of one row block (m >= n) held in shared memory.
//   in  A (m x n, column-major, lda)
//   out Q (m x n, column-major, ldq), R (n x n upper triangular, column-major,
//   ldr; rows below the diagonal written as zero).  Q may alias A.
struct QrItem {
  const void *A;
  void *Q, *R;
  int64_t lda, ldq, ldr;
  int m, n;
};

// Symmetric eigendecomposition (FP64) of one k x k matrix.
struct EigItem {
  const double *G;  // k x k column-major (symmetrised on load)
  double *V;        // k x k column-major eigenvectors (descending eigenvalues)
  double *lam;      // k eigenvalues, descending
  int k;
};

// Semidefinite Cholesky factor of one k x k FP64 Gramian: G = S S^T, S lower
// triangular (FP32 output, zeros above the diagonal); W is a k x k FP64
// working array.  Pivots at or below tau = 4 k u_64 max_i G_ii give a zero
// column (the Gramian is singular there to working accuracy).
struct CholItem {
  const double *G;
  double *W;
  float *S;
  int k;
};

// 2-D strided copy with optional cast, identity or zero fill, scaling.
//   dst[r*dr + c*dc] = (src ? alpha*src[r*sr + c*sc] : (zero ? 0 : (r == c ? 1 : 0))) + beta*dst[...]
// rows/cols may be rank references like GemmItem dims (-1: literal).
struct CopyItem {
  const void *src;
  void *dst;
  int64_t sr, sc, dr, dc;
  int rows, cols;
  int rows_ref, cols_ref;
  int src_f64, dst_f64;
  double alpha, beta;
  int zero;
};

// Packed copy of an inner node into its truncated, compact layout:
//   dst[(a*r1 + b)*r2 + c] = src[(a*ld1 + b)*ld2 + c], a<r0, b<r1, c<r2
// with r0, r1, r2 read from the device rank array.
struct CompactItem {
  const void *src;
  void *dst;
  int ref0, ref1, ref2;  // rank refs (ref0 < 0: r0 = 1)
  int ld1, ld2;
  int max0, max1, max2;
};

// Rank selection for one tensor.  Nodes are listed in pre-order from node0.
struct RankItem {
  const double *lam;      // eigenvalues of all nodes (offset table lam_off)
  const int64_t *lam_off; // per node (device)
  const int *korth;       // ranks after orthogonalization (device)
  const int *target;      // per node target (rank mode) or null
  int *r_out;             // truncated ranks (device)
  double *stats;          // [norm, discarded_sq, tail2] out
  const double *root;     // orthogonalized root matrix (for ||X||)
  int root_f64;
  int64_t root_count;
  int nn, t1, t2, d;
  int mode, eps_rel, cap;
  double eps;
  double noise;  // per-eigenvalue noise floor, relative to the node's largest eigenvalue
};
// RankItem.stats: [0] ||X||, [1] discarded sigma^2 (root pair once), [2] per-node
// squared threshold, [3] 1 if ||X|| or an eigenvalue was not finite, else 0.

// ---------------------------------------------------------------------------
// launchers (stream-ordered; return cudaGetLastError())
// ---------------------------------------------------------------------------
// variant: SIMT tile shape (0: 64 x 64, 1: 128 x 64, 2: 128 x 128, the last
// without compensation only); items' tiles_m / tiles_n / tile0 must be laid
// out for that shape (gemm_tile_shape).  comp: Kahan-compensated FP32
// accumulation across the BK-wide tiles of a CTA.  df (FP32 only): double-float
// accumulation of exact products, FP64 output and split-K partials.
// uniform > 0: every item has that many tiles (tile -> item by division).
template <typename T>
cudaError_t launch_gemm(const GemmItem *d_items, int n_items, int total_tiles, const int *d_ranks,
                        bool any_split, int tc_tiles, cudaStream_t s, int variant, bool comp, bool df,
                        int uniform = 0);
void gemm_tile_shape(int variant, int *bm, int *bn);
// Split-K partial sums of FP64 items added in chunk order (k_gemm.cu).
cudaError_t launch_gemm_reduce_f64(const GemmItem *d_items, int n_items, const int *d_ranks, cudaStream_t s);
// FP64 contractions on the tensor cores by exact BF16 slicing (k_oz.cu), in
// two launches: the split of every item's operands into BF16 slices
// (split_blocks CTAs), then the persistent GEMM over `tiles` tiles of
// oz_tile_m() x oz_gemm_tile_n() (followed by the split-K reduction if
// any_split).  Every item needs K * ceil(Ko / ksplit) <= 256 (products per
// exactness chunk); slices in [2, 6].
cudaError_t launch_oz_split(const GemmItem *d_items, int n_items, int split_blocks, const int *d_ranks, int slices,
                            cudaStream_t s);
// tile_item: the item of every tile (device array of `tiles` ints).
cudaError_t launch_oz_gemm(const GemmItem *d_items, const int *tile_item, int n_items, int tiles, const int *d_ranks,
                           bool any_split, int slices, cudaStream_t s);
int oz_tile_m();       // rows of a GEMM tile and of a split block
int oz_tile_n();       // rows of a split block of B (output columns)
int oz_gemm_tile_n();  // output columns of a GEMM tile
int oz_stage_k();
int oz_block_bytes();
unsigned oz_take_status();  // bit 0: a bounded wait of the tensor-core kernel gave up (read and clear)
// qr_kernel: 0 picks the block kernel by shape and launch size; 1 forces the
// one-column kernel, 2 the two-column kernel (FP32, 64-column blocks).
template <typename T>
cudaError_t launch_qr(const QrItem *d_items, int n_items, int max_m, int max_n, cudaStream_t s, int qr_kernel = 0);
// The same row blocks (FP64 in and out) factored in double-float arithmetic
// on the FP32 pipe, about 2^-47 relative (k_qr_df.cu); max_n <= 32, max_m <= 256.
cudaError_t launch_qr_df(const QrItem *d_items, int n_items, int max_m, int max_n, cudaStream_t s);
// mode 0: FP64 QL; mode 1: FP32 QL followed by one double-float refinement step;
// mode 2: FP64 QL recurrence (the eigenvalues) with the eigenvector rotations
// applied in double-float on the FP32 pipe (about 2^-47 per rotation).
// scratch: 4 * max_k^2 doubles per item when max_k exceeds the shared-memory sizes (eig_scratch_needed).
cudaError_t launch_eig(const EigItem *d_items, int n_items, int max_k, double *scratch, cudaStream_t s, int mode);
cudaError_t launch_copy(const CopyItem *d_items, int n_items, const int *d_ranks, int f64_any, cudaStream_t s);
cudaError_t launch_chol(const CholItem *d_items, int n_items, cudaStream_t s);
template <typename T>
cudaError_t launch_compact(const CompactItem *d_items, int n_items, const int *d_ranks, cudaStream_t s);
cudaError_t launch_ranks(const RankItem *d_items, int n_items, cudaStream_t s);
template <typename T>
cudaError_t launch_pack_add(const void *a, const void *c, void *out, const int64_t *d_desc, int n_nodes,
                            int64_t max_elems, cudaStream_t s);
// Kronecker transfer tensors of an operator application (6 int64 per node descriptor)
template <typename T>
cudaError_t launch_kron(const void *h, const void *b, void *f, const int64_t *d_desc, int n_nodes, int64_t max_elems,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_eval_level(const void *x, const int64_t *node_off, const int *ranks, const int *tree,
                              const int64_t *n, const int64_t *idx, const int64_t *row_off, int64_t rows_per,
                              const int *level_nodes, int n_level, int64_t m, int d, double *rows, double *out,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_sumsq(const void *x, int64_t count, double *out, cudaStream_t s);
template <typename T>
cudaError_t launch_scale(void *x, int64_t count, double alpha, cudaStream_t s);

// Status words of the eigensolvers (bit 0: a QL sweep hit its iteration
// limit) and of the rank selection (bit 0: a non-finite norm or eigenvalue):
// read and clear; ~0u if the read failed.  Synchronise the device.
unsigned eig_take_status();
unsigned misc_take_status();
// Bounded-wait self-test (k_misc.cu): one kernel waits limit_ns on a flag that
// nothing sets, then marks the wait status word (read and cleared by
// wait_take_status) and returns.
cudaError_t launch_selftest_wait(int64_t limit_ns, cudaStream_t s);
unsigned wait_take_status();

// launch accounting / tracing (api.cu)
void count_launch(int n = 1);
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s, double flops);

// maximum rows of one QR block that fit in shared memory for n columns
int qr_max_rows(int n, int elem_bytes);
// largest k whose eigenproblem is solved in shared memory (larger k use a global scratch slab)
int eig_smem_k();
// FP64 eigensolves of more matrices than SMs keep their eigenvectors in the
// scratch slab instead of shared memory, so that several CTAs share an SM
inline bool eig_z_global(int max_k, int n_items) { return max_k <= 128 && n_items > kSmCount; }
inline bool eig_scratch_needed(int max_k, int mode, int n_items) {
  return mode == 0 ? (max_k > 128 || eig_z_global(max_k, n_items)) : max_k > 64;
}

}  // namespace htgb
