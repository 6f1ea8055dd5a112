/*
 * ht_oracle.c -- plain, slow, CPU FP64 oracle of the HSVD truncation of a
 * Hierarchical Tucker (HT) tensor after HT addition.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline and reference legs of the benchmark may load this file.  The
 * product (the CUDA library) shares no code with it.
 *
 * Every routine follows the paper (Grasedyck & Loebbert, "Distributed
 * Hierarchical SVD in the Hierarchical Tucker Format"), cited by section and
 * equation name; the order of the steps is the paper's order.  There is no
 * blocking and no fusion; loops are written so that each formula can be read
 * off directly.  Own Householder QR and own cyclic Jacobi eigensolver.
 *
 * Data conventions (shared interface with the library's upload format):
 *   - tree: balanced dimension tree (Sec. 2.1, eq. "balanced"), nodes numbered
 *     in pre-order, root = 0.  Modes are 0-based.
 *   - leaf {mu}: frame U (n_mu x k_t), column-major (ld = n_mu).
 *   - inner node t with sons s1, s2: transfer tensor B_t (k_t x k_s1 x k_s2),
 *     element (i,j,l) at (i*k_s1 + j)*k_s2 + l  (l fastest).  The root has
 *     k_root = 1, so B_root is the k_t1 x k_t2 matrix [j][l].
 *   - a tensor is one "packed blob": the nodes in pre-order, each node's
 *     array as above, concatenated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Dimension tree (Sec. 2.1)                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d, nn;
  int *lo, *hi, *par, *s1, *s2, *depth, *height;
} otree;

/* Node {mu..nu} (1-based) splits into {mu..floor((mu+nu-1)/2)} and the rest
 * (eq. "balanced").  With 0-based lo = mu-1, hi = nu-1 the last mode of the
 * first son is floor((lo+hi+1)/2) - 1. */
static int tree_build_rec(otree *T, int lo, int hi, int parent, int depth) {
  int id = T->nn++;
  T->lo[id] = lo;
  T->hi[id] = hi;
  T->par[id] = parent;
  T->depth[id] = depth;
  if (lo == hi) {
    T->s1[id] = T->s2[id] = -1;
    T->height[id] = 0;
    return id;
  }
  int last1 = (lo + hi + 1) / 2 - 1;
  int a = tree_build_rec(T, lo, last1, id, depth + 1);
  int b = tree_build_rec(T, last1 + 1, hi, id, depth + 1);
  T->s1[id] = a;
  T->s2[id] = b;
  T->height[id] = 1 + (T->height[a] > T->height[b] ? T->height[a] : T->height[b]);
  return id;
}

static int tree_init(otree *T, int d) {
  int nn = 2 * d - 1;
  T->d = d;
  T->nn = 0;
  int *buf = (int *)malloc(sizeof(int) * 7 * (size_t)nn);
  if (!buf) return -1;
  T->lo = buf;
  T->hi = buf + nn;
  T->par = buf + 2 * nn;
  T->s1 = buf + 3 * nn;
  T->s2 = buf + 4 * nn;
  T->depth = buf + 5 * nn;
  T->height = buf + 6 * nn;
  tree_build_rec(T, 0, d - 1, -1, 0);
  return 0;
}

static void tree_free(otree *T) { free(T->lo); }

static int is_leaf(const otree *T, int t) { return T->s1[t] < 0; }

static int tree_max_height(const otree *T) { return T->height[0]; }

static int tree_max_depth(const otree *T) {
  int m = 0;
  for (int t = 0; t < T->nn; ++t)
    if (T->depth[t] > m) m = T->depth[t];
  return m;
}

/* number of doubles of node t for ranks k */
static int64_t node_size(const otree *T, const int64_t *n, const int *k, int t) {
  if (is_leaf(T, t)) return n[T->lo[t]] * (int64_t)k[t];
  int kt = (t == 0) ? 1 : k[t];
  return (int64_t)kt * k[T->s1[t]] * k[T->s2[t]];
}

static void node_offsets(const otree *T, const int64_t *n, const int *k, int64_t *off) {
  int64_t o = 0;
  for (int t = 0; t < T->nn; ++t) {
    off[t] = o;
    o += node_size(T, n, k, t);
  }
  off[T->nn] = o;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (plain loops)                                               */
/* ------------------------------------------------------------------------ */

/* Householder QR: A (m x n, column-major, lda) = Q R with p = min(m,n),
 * Q (m x p, column-major, ld m) with orthonormal columns, R (p x n, row-major)
 * upper trapezoidal.  Reflector j maps W[j:m, j] to beta e_1; H_j = I - tau v v^T
 * with v_0 = 1.  Q is formed explicitly by applying H_{p-1} ... H_0 to [I_p; 0]. */
static void hh_qr(int64_t m, int n, const double *A, int64_t lda, double *Q, double *R) {
  int p = (int)(m < n ? m : n);
  double *W = (double *)malloc(sizeof(double) * (size_t)m * n);
  double *tau = (double *)malloc(sizeof(double) * (size_t)(p > 0 ? p : 1));
  for (int c = 0; c < n; ++c) memcpy(W + (int64_t)c * m, A + (int64_t)c * lda, sizeof(double) * (size_t)m);
  for (int j = 0; j < p; ++j) {
    double *x = W + (int64_t)j * m;
    double alpha = x[j], s2 = 0.0;
    for (int64_t i = j + 1; i < m; ++i) s2 += x[i] * x[i];
    if (s2 == 0.0) {
      tau[j] = 0.0; /* already of the form beta e_1: no reflection */
      continue;
    }
    double nrm = sqrt(alpha * alpha + s2);
    double beta = (alpha <= 0.0) ? nrm : -nrm;
    double v0 = alpha - beta;
    tau[j] = (beta - alpha) / beta;
    for (int64_t i = j + 1; i < m; ++i) x[i] /= v0; /* v = [1; x[j+1:]/v0] */
    x[j] = beta;
    for (int c = j + 1; c < n; ++c) { /* apply H_j to the trailing columns */
      double *y = W + (int64_t)c * m;
      double s = y[j];
      for (int64_t i = j + 1; i < m; ++i) s += x[i] * y[i];
      s *= tau[j];
      y[j] -= s;
      for (int64_t i = j + 1; i < m; ++i) y[i] -= s * x[i];
    }
  }
  for (int r = 0; r < p; ++r)
    for (int c = 0; c < n; ++c) R[(int64_t)r * n + c] = (c >= r) ? W[(int64_t)c * m + r] : 0.0;
  for (int c = 0; c < p; ++c) {
    double *q = Q + (int64_t)c * m;
    for (int64_t i = 0; i < m; ++i) q[i] = (i == c) ? 1.0 : 0.0;
  }
  for (int j = p - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
    const double *x = W + (int64_t)j * m;
    for (int c = 0; c < p; ++c) {
      double *q = Q + (int64_t)c * m;
      double s = q[j];
      for (int64_t i = j + 1; i < m; ++i) s += x[i] * q[i];
      s *= tau[j];
      q[j] -= s;
      for (int64_t i = j + 1; i < m; ++i) q[i] -= s * x[i];
    }
  }
  free(W);
  free(tau);
}

/* Cyclic Jacobi eigensolver for a symmetric n x n matrix A (row-major, read
 * only).  Rotations in the (p,q) planes, row-by-row cyclic order, until the
 * off-diagonal mass is below rounding level.  Output: w (descending) and V
 * (n x n, column-major: column c is the eigenvector of w[c]). */
static void jacobi_eig(int n, const double *A, double *w, double *V) {
  double *a = (double *)malloc(sizeof(double) * (size_t)n * n);
  double *v = (double *)malloc(sizeof(double) * (size_t)n * n);
  memcpy(a, A, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i * n + j] = (i == j) ? 1.0 : 0.0; /* v row-major: v[r*n+c] */
  double fro2 = 0.0;
  for (int i = 0; i < n * n; ++i) fro2 += a[i] * a[i];
  const double tol2 = fro2 * 1e-36; /* (1e-18 ||A||_F)^2 */
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off2 = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off2 += 2.0 * a[p * n + q] * a[p * n + q];
    if (off2 <= tol2 || off2 == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (apq == 0.0) continue;
        double app = a[p * n + p], aqq = a[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* A <- J^T A J with J_pp = J_qq = c, J_pq = s, J_qp = -s */
        for (int r = 0; r < n; ++r) { /* columns p, q */
          double arp = a[r * n + p], arq = a[r * n + q];
          a[r * n + p] = c * arp - s * arq;
          a[r * n + q] = s * arp + c * arq;
        }
        for (int r = 0; r < n; ++r) { /* rows p, q */
          double apr = a[p * n + r], aqr = a[q * n + r];
          a[p * n + r] = c * apr - s * aqr;
          a[q * n + r] = s * apr + c * aqr;
        }
        a[p * n + q] = a[q * n + p] = 0.0;
        for (int r = 0; r < n; ++r) { /* V <- V J */
          double vrp = v[r * n + p], vrq = v[r * n + q];
          v[r * n + p] = c * vrp - s * vrq;
          v[r * n + q] = s * vrp + c * vrq;
        }
      }
    }
  }
  /* sort descending (selection sort; n is small) */
  int *idx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i) {
    int best = i;
    for (int j = i + 1; j < n; ++j)
      if (a[idx[j] * n + idx[j]] > a[idx[best] * n + idx[best]]) best = j;
    int tmp = idx[i];
    idx[i] = idx[best];
    idx[best] = tmp;
  }
  for (int c = 0; c < n; ++c) {
    w[c] = a[idx[c] * n + idx[c]];
    for (int r = 0; r < n; ++r) V[(int64_t)c * n + r] = v[r * n + idx[c]];
  }
  free(idx);
  free(a);
  free(v);
}

/* (M1, M2, M3) o B, the mode products of Lemma "transfer tensor
 * transformation":  out[a,b,c] = sum_{i,j,l} M1[a,i] M2[b,j] M3[c,l] B[i,j,l].
 * B is kt x k1 x k2 ([i][j][l]); M1 is r0 x kt, M2 r1 x k1, M3 r2 x k2, all
 * row-major.  Evaluated mode 1, then mode 2, then mode 3. */
static void mode_products(int kt, int k1, int k2, const double *B, int r0, const double *M1, int r1,
                          const double *M2, int r2, const double *M3, double *out) {
  double *T1 = (double *)calloc((size_t)r0 * k1 * k2, sizeof(double));
  double *T2 = (double *)calloc((size_t)r0 * r1 * k2, sizeof(double));
  for (int a = 0; a < r0; ++a)
    for (int i = 0; i < kt; ++i) {
      double m = M1[(int64_t)a * kt + i];
      if (m == 0.0) continue;
      const double *src = B + (int64_t)i * k1 * k2;
      double *dst = T1 + (int64_t)a * k1 * k2;
      for (int64_t e = 0; e < (int64_t)k1 * k2; ++e) dst[e] += m * src[e];
    }
  for (int a = 0; a < r0; ++a)
    for (int b = 0; b < r1; ++b)
      for (int j = 0; j < k1; ++j) {
        double m = M2[(int64_t)b * k1 + j];
        if (m == 0.0) continue;
        const double *src = T1 + ((int64_t)a * k1 + j) * k2;
        double *dst = T2 + ((int64_t)a * r1 + b) * k2;
        for (int l = 0; l < k2; ++l) dst[l] += m * src[l];
      }
  for (int a = 0; a < r0; ++a)
    for (int b = 0; b < r1; ++b) {
      const double *src = T2 + ((int64_t)a * r1 + b) * k2;
      double *dst = out + ((int64_t)a * r1 + b) * r2;
      for (int c = 0; c < r2; ++c) {
        double s = 0.0;
        for (int l = 0; l < k2; ++l) s += M3[(int64_t)c * k2 + l] * src[l];
        dst[c] = s;
      }
    }
  free(T1);
  free(T2);
}

/* ------------------------------------------------------------------------ */
/* Public oracle API                                                         */
/* ------------------------------------------------------------------------ */

static int g_threads = 0;

int ho_set_threads(int nthreads) {
  g_threads = nthreads;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int ho_num_nodes(int d) { return 2 * d - 1; }

/* Tree description in pre-order.  Arrays of length 2d-1. */
int ho_tree_info(int d, int *lo, int *hi, int *parent, int *son1, int *son2, int *depth, int *height) {
  if (d < 2) return -1;
  otree T;
  if (tree_init(&T, d)) return -2;
  for (int t = 0; t < T.nn; ++t) {
    lo[t] = T.lo[t];
    hi[t] = T.hi[t];
    parent[t] = T.par[t];
    son1[t] = T.s1[t];
    son2[t] = T.s2[t];
    depth[t] = T.depth[t];
    height[t] = T.height[t];
  }
  tree_free(&T);
  return 2 * d - 1;
}

int64_t ho_size(int d, const int64_t *n, const int *k) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T.nn + 1));
  node_offsets(&T, n, k, off);
  int64_t s = off[T.nn];
  free(off);
  tree_free(&T);
  return s;
}

/* HT addition, Lemma "The sum of two H-tensors" (Sec. 3.5, eq.
 * "sumleafframes"): leaf frames are concatenated, W = [U, V]; transfer
 * tensors are stacked block-diagonally, H_t = diag(B_t, F_t); the root
 * becomes the 2x2 block-diagonal matrix diag(B_D, F_D).  No arithmetic. */
int ho_add(int d, const int64_t *n, const int *ka, const double *xa, const int *kc, const double *xc, int *kout,
           double *xout) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  for (int t = 0; t < T.nn; ++t) kout[t] = (t == 0) ? 1 : ka[t] + kc[t];
  int64_t *oa = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(T.nn + 1));
  int64_t *oc = oa + T.nn + 1, *oo = oc + T.nn + 1;
  node_offsets(&T, n, ka, oa);
  node_offsets(&T, n, kc, oc);
  node_offsets(&T, n, kout, oo);
  memset(xout, 0, sizeof(double) * (size_t)oo[T.nn]);
  for (int t = 0; t < T.nn; ++t) {
    const double *A = xa + oa[t], *C = xc + oc[t];
    double *O = xout + oo[t];
    if (is_leaf(&T, t)) {
      int64_t nm = n[T.lo[t]];
      for (int c = 0; c < ka[t]; ++c)
        for (int64_t i = 0; i < nm; ++i) O[(int64_t)c * nm + i] = A[(int64_t)c * nm + i];
      for (int c = 0; c < kc[t]; ++c)
        for (int64_t i = 0; i < nm; ++i) O[(int64_t)(ka[t] + c) * nm + i] = C[(int64_t)c * nm + i];
    } else {
      int s1 = T.s1[t], s2 = T.s2[t];
      int at = (t == 0) ? 1 : ka[t], a1 = ka[s1], a2 = ka[s2];
      int ct = (t == 0) ? 1 : kc[t], c1 = kc[s1], c2 = kc[s2];
      int ot = (t == 0) ? 1 : kout[t], o1 = kout[s1], o2 = kout[s2];
      (void)ot;
      for (int i = 0; i < at; ++i)
        for (int j = 0; j < a1; ++j)
          for (int l = 0; l < a2; ++l) O[((int64_t)i * o1 + j) * o2 + l] = A[((int64_t)i * a1 + j) * a2 + l];
      int ioff = (t == 0) ? 0 : at; /* the root's single index is shared (k_D = 1) */
      for (int i = 0; i < ct; ++i)
        for (int j = 0; j < c1; ++j)
          for (int l = 0; l < c2; ++l)
            O[((int64_t)(ioff + i) * o1 + a1 + j) * o2 + a2 + l] = C[((int64_t)i * c1 + j) * c2 + l];
    }
  }
  free(oa);
  tree_free(&T);
  return 0;
}

/* Orthogonalization, Sec. 3.4, steps 1-3 (leaves -> root).
 *   1. leaves: reduced QR U = Q R, U <- Q, R goes to the father;
 *   2. inner nodes (by height): B <- (I, R_s1, R_s2) o B, then reduced QR of
 *      M_{2,3}(B) as in eq. "qrtransfer", B[q,j,l] <- Q[(j,l),q], R_t to the
 *      father.  The new rank is min(k_t, k_s1 k_s2);
 *   3. root: B_D <- R_t1 B_D R_t2^T.
 * k is updated in place (ranks after orthogonalization); x is read with the
 * input ranks and xout written with the new ranks (xout may not alias x). */
int ho_orthogonalize(int d, const int64_t *n, int *k, const double *x, double *xout) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  int nn = T.nn;
  int *kin = (int *)malloc(sizeof(int) * (size_t)nn);
  memcpy(kin, k, sizeof(int) * (size_t)nn);
  int64_t *oin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  node_offsets(&T, n, kin, oin);
  double **R = (double **)calloc((size_t)nn, sizeof(double *)); /* R_t: knew[t] x kin[t], row-major */
  double **node = (double **)calloc((size_t)nn, sizeof(double *));
  int H = tree_max_height(&T);
  for (int h = 0; h <= H; ++h) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nn; ++t) {
      if (T.height[t] != h) continue;
      if (is_leaf(&T, t)) {
        int64_t m = n[T.lo[t]];
        int kt = kin[t];
        int p = (int)(m < kt ? m : kt);
        node[t] = (double *)malloc(sizeof(double) * (size_t)(m * p));
        R[t] = (double *)malloc(sizeof(double) * (size_t)p * kt);
        hh_qr(m, kt, x + oin[t], m, node[t], R[t]);
        k[t] = p;
      } else {
        int s1 = T.s1[t], s2 = T.s2[t];
        int kt = (t == 0) ? 1 : kin[t];
        int k1 = kin[s1], k2 = kin[s2], p1 = k[s1], p2 = k[s2];
        /* B <- (I, R_s1, R_s2) o B   (I of size kt) */
        double *I = (double *)calloc((size_t)kt * kt, sizeof(double));
        for (int i = 0; i < kt; ++i) I[i * kt + i] = 1.0;
        double *Bp = (double *)malloc(sizeof(double) * (size_t)kt * p1 * p2);
        mode_products(kt, k1, k2, x + oin[t], kt, I, p1, R[s1], p2, R[s2], Bp);
        free(I);
        if (t == 0) {
          node[t] = Bp;
        } else {
          /* M_{2,3}(B) is (p1 p2) x kt, column i = slab B[i,:,:] */
          int64_t m = (int64_t)p1 * p2;
          int p = (int)(m < kt ? m : kt);
          double *Q = (double *)malloc(sizeof(double) * (size_t)(m * p));
          R[t] = (double *)malloc(sizeof(double) * (size_t)p * kt);
          hh_qr(m, kt, Bp, m, Q, R[t]);
          free(Bp);
          node[t] = Q; /* B[q,j,l] = Q[(j,l), q]: column-major Q is exactly [q][j][l] */
          k[t] = p;
        }
      }
    }
  }
  int64_t *oout = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  k[0] = 1;
  node_offsets(&T, n, k, oout);
  for (int t = 0; t < nn; ++t) {
    memcpy(xout + oout[t], node[t], sizeof(double) * (size_t)(oout[t + 1] - oout[t]));
    free(node[t]);
    free(R[t]);
  }
  free(R);
  free(node);
  free(oin);
  free(oout);
  free(kin);
  tree_free(&T);
  return 0;
}

/* Reduced Gramians Bhat_t = V_t^T V_t of an orthogonal tensor, Sec. 3.3:
 * root sons by eq. "acctransferroot" (Bhat_t1 = B_D B_D^T, Bhat_t2 =
 * B_D^T B_D), then top-down by eqs. "acctransferSon1" / "acctransferSon2":
 *   Bhat_s1[p,q] = sum_{i1,i2,l} B[i1,p,l] Bhat_t[i1,i2] B[i2,q,l]
 *   Bhat_s2[p,q] = sum_{i1,i2,j} B[i1,j,p] Bhat_t[i1,i2] B[i2,j,q]
 * With Bhat_D = 1 the root case is the same formula.  The sum over i1 is
 * taken first: C[i2,p,l] = sum_{i1} Bhat_t[i1,i2] B[i1,p,l].
 * Output g: for each node t in pre-order a k_t x k_t row-major block (root 1x1). */
int ho_gramians(int d, const int64_t *n, const int *k, const double *x, double *g) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  int nn = T.nn;
  int64_t *ox = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  int64_t *og = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  node_offsets(&T, n, k, ox);
  int64_t o = 0;
  for (int t = 0; t < nn; ++t) {
    og[t] = o;
    int kt = (t == 0) ? 1 : k[t];
    o += (int64_t)kt * kt;
  }
  g[0] = 1.0;
  int D = tree_max_depth(&T);
  for (int lev = 0; lev <= D; ++lev) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nn; ++t) {
      if (T.depth[t] != lev || is_leaf(&T, t)) continue;
      int s1 = T.s1[t], s2 = T.s2[t];
      int kt = (t == 0) ? 1 : k[t], k1 = k[s1], k2 = k[s2];
      const double *B = x + ox[t], *G = g + og[t];
      double *C = (double *)calloc((size_t)kt * k1 * k2, sizeof(double));
      for (int i2 = 0; i2 < kt; ++i2)
        for (int i1 = 0; i1 < kt; ++i1) {
          double gv = G[(int64_t)i1 * kt + i2];
          const double *src = B + (int64_t)i1 * k1 * k2;
          double *dst = C + (int64_t)i2 * k1 * k2;
          for (int64_t e = 0; e < (int64_t)k1 * k2; ++e) dst[e] += gv * src[e];
        }
      double *G1 = g + og[s1], *G2 = g + og[s2];
      for (int p = 0; p < k1; ++p)
        for (int q = 0; q < k1; ++q) {
          double s = 0.0;
          for (int i = 0; i < kt; ++i)
            for (int l = 0; l < k2; ++l)
              s += C[((int64_t)i * k1 + p) * k2 + l] * B[((int64_t)i * k1 + q) * k2 + l];
          G1[(int64_t)p * k1 + q] = s;
        }
      for (int p = 0; p < k2; ++p)
        for (int q = 0; q < k2; ++q) {
          double s = 0.0;
          for (int i = 0; i < kt; ++i)
            for (int j = 0; j < k1; ++j)
              s += C[((int64_t)i * k1 + j) * k2 + p] * B[((int64_t)i * k1 + j) * k2 + q];
          G2[(int64_t)p * k2 + q] = s;
        }
      free(C);
    }
  }
  free(ox);
  free(og);
  tree_free(&T);
  return 0;
}

/* Options of the truncation T(X) (Sec. 3.3 and 3.5): to prescribed ranks, or
 * to accuracy eps (absolute, or relative to ||X||), with a rank cap. */
typedef struct {
  int mode;          /* 0: ranks, 1: eps */
  double eps;        /* accuracy for mode 1 */
  int eps_relative;  /* 1: eps_abs = eps * ||X|| */
  int rank_cap;      /* <= 0: none */
  const int *ranks;  /* mode 0: target rank per node (pre-order), or NULL = rank_cap */
  double noise;      /* mode 1: charge per dropped eigenvalue, relative to the node's largest (0: none) */
} ho_opts;

/* Rank rule for one node (reading of the eps truncation of [Gr10]): the
 * smallest r >= 1 whose discarded tail sum_{i>r} (max(lambda_i,0) + nu) is
 * <= tail2, then capped.  nu = noise * max(lambda_1, 0) is an optional charge
 * per dropped eigenvalue (0 gives the plain rule: the computed tail alone). */
static int eps_rank(const double *lam, int k, double tail2, double noise) {
  const double nu = noise * (lam[0] > 0.0 ? lam[0] : 0.0);
  double tail = 0.0;
  int r = k;
  for (int i = k - 1; i >= 1; --i) { /* can we drop lambda_i (0-based)? */
    double l = (lam[i] > 0.0 ? lam[i] : 0.0) + nu;
    if (tail + l <= tail2) {
      tail += l;
      r = i;
    } else {
      break;
    }
  }
  return r;
}

/* HSVD truncation T(X), Sec. 3.3 (with Sec. 3.4 first, since the frames
 * must be orthonormal):
 *   a. orthogonalize;
 *   b. reduced Gramians Bhat_t for all non-root nodes (top-down);
 *   c. eigendecomposition Bhat_t = Q_t Lambda_t Q_t^T (descending); the
 *      singular values of M_t(X) are sqrt(max(lambda,0));
 *   c'. ranks r_t;
 *   d. leaves U <- U Q|_r; inner nodes B <- (Q_t|_r^T, Q_s1|_r^T, Q_s2|_r^T) o B
 *      (eq. "transfertransformationtrunc"); root B_D <- Q_t1^T B_D Q_t2.
 *      All Gramians and eigenvectors are computed before any node is changed.
 * In:  k (input ranks), x.  Out: k (truncated ranks), korth (ranks after
 * orthogonalization), xout (truncated tensor, capacity = size of x),
 * sigma (for every non-root node, korth[t] singular values, pre-order,
 * concatenated), info[0] = ||X||, info[1] = sum of discarded sigma^2
 * (root pair counted once), info[2] = eps threshold per node (squared), info[3] = number of counted nodes. */
int ho_truncate(int d, const int64_t *n, int *k, const double *x, const ho_opts *opts, int *korth, double *xout,
                double *sigma, double *info) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  int nn = T.nn;
  int64_t sz = ho_size(d, n, k);
  double *xo = (double *)malloc(sizeof(double) * (size_t)sz);
  memcpy(korth, k, sizeof(int) * (size_t)nn);
  ho_orthogonalize(d, n, korth, x, xo);
  int64_t *ox = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  node_offsets(&T, n, korth, ox);
  /* b. Gramians */
  int64_t gsz = 0;
  int64_t *og = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  for (int t = 0; t < nn; ++t) {
    og[t] = gsz;
    int kt = (t == 0) ? 1 : korth[t];
    gsz += (int64_t)kt * kt;
  }
  og[nn] = gsz;
  double *g = (double *)malloc(sizeof(double) * (size_t)gsz);
  ho_gramians(d, n, korth, xo, g);
  /* c. eigen */
  double *Q = (double *)malloc(sizeof(double) * (size_t)gsz); /* column-major k_t x k_t per node */
  double *lam = (double *)malloc(sizeof(double) * (size_t)gsz);
  int64_t *ol = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  {
    int64_t o = 0;
    for (int t = 0; t < nn; ++t) {
      ol[t] = o;
      o += (t == 0) ? 1 : korth[t];
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 1; t < nn; ++t) jacobi_eig(korth[t], g + og[t], lam + ol[t], Q + og[t]);
  Q[og[0]] = 1.0;
  lam[ol[0]] = 1.0;
  /* ||X|| = ||B_D||_F of the orthogonal representation (Sec. 3.4) */
  double nrm2 = 0.0;
  for (int64_t e = ox[0]; e < ox[1]; ++e) nrm2 += xo[e] * xo[e];
  double nrm = sqrt(nrm2);
  /* c'. ranks */
  int t1 = T.s1[0], t2 = T.s2[0];
  int counted = 2 * d - 3;
  double tail2 = 0.0;
  if (opts->mode == 1) {
    double e = opts->eps_relative ? opts->eps * nrm : opts->eps;
    tail2 = e * e / (double)counted;
  }
  int *r = (int *)malloc(sizeof(int) * (size_t)nn);
  r[0] = 1;
  for (int t = 1; t < nn; ++t) {
    int avail = korth[t];
    int rt;
    if (opts->mode == 1) {
      rt = eps_rank(lam + ol[t], avail, tail2, opts->noise);
    } else {
      rt = (opts->ranks) ? opts->ranks[t] : opts->rank_cap;
      if (rt <= 0) rt = avail;
    }
    if (opts->rank_cap > 0 && rt > opts->rank_cap) rt = opts->rank_cap;
    if (rt > avail) rt = avail;
    if (rt < 1) rt = 1;
    r[t] = rt;
  }
  {
    /* the two sons of the root have the same nonzero singular values
     * (M_t2 = M_t1^T): one shared rank, decided on t1 */
    int rr = r[t1];
    if (opts->mode == 0 && r[t2] < rr) rr = r[t2];
    if (rr > korth[t2]) rr = korth[t2];
    r[t1] = r[t2] = rr;
  }
  double disc = 0.0;
  for (int t = 1; t < nn; ++t) {
    if (t == t2) continue;
    for (int i = r[t]; i < korth[t]; ++i) disc += (lam[ol[t] + i] > 0.0 ? lam[ol[t] + i] : 0.0);
  }
  for (int t = 1; t < nn; ++t)
    for (int i = 0; i < korth[t]; ++i) {
      double l = lam[ol[t] + i];
      sigma[ol[t] - 1 + i] = sqrt(l > 0.0 ? l : 0.0);
    }
  /* d. projection */
  int64_t *oo = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  node_offsets(&T, n, r, oo);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < nn; ++t) {
    const double *src = xo + ox[t];
    double *dst = xout + oo[t];
    if (is_leaf(&T, t)) {
      int64_t m = n[T.lo[t]];
      int kt = korth[t];
      const double *Qt = Q + og[t];
      for (int c = 0; c < r[t]; ++c)
        for (int64_t i = 0; i < m; ++i) {
          double s = 0.0;
          for (int j = 0; j < kt; ++j) s += src[(int64_t)j * m + i] * Qt[(int64_t)c * kt + j];
          dst[(int64_t)c * m + i] = s;
        }
    } else {
      int s1 = T.s1[t], s2 = T.s2[t];
      int kt = (t == 0) ? 1 : korth[t], k1 = korth[s1], k2 = korth[s2];
      int r0 = r[t], r1 = r[s1], r2 = r[s2];
      /* M1 = Q_t|_r^T (r0 x kt), M2 = Q_s1|_r^T, M3 = Q_s2|_r^T, row-major */
      double *M1 = (double *)malloc(sizeof(double) * (size_t)r0 * kt);
      double *M2 = (double *)malloc(sizeof(double) * (size_t)r1 * k1);
      double *M3 = (double *)malloc(sizeof(double) * (size_t)r2 * k2);
      for (int a = 0; a < r0; ++a)
        for (int i = 0; i < kt; ++i) M1[(int64_t)a * kt + i] = Q[og[t] + (int64_t)a * kt + i];
      for (int b = 0; b < r1; ++b)
        for (int j = 0; j < k1; ++j) M2[(int64_t)b * k1 + j] = Q[og[s1] + (int64_t)b * k1 + j];
      for (int c = 0; c < r2; ++c)
        for (int l = 0; l < k2; ++l) M3[(int64_t)c * k2 + l] = Q[og[s2] + (int64_t)c * k2 + l];
      mode_products(kt, k1, k2, src, r0, M1, r1, M2, r2, M3, dst);
      free(M1);
      free(M2);
      free(M3);
    }
  }
  memcpy(k, r, sizeof(int) * (size_t)nn);
  info[0] = nrm;
  info[1] = disc;
  info[2] = tail2;
  info[3] = (double)counted;
  free(r);
  free(oo);
  free(ol);
  free(lam);
  free(Q);
  free(g);
  free(og);
  free(ox);
  free(xo);
  tree_free(&T);
  return 0;
}

/* Entry evaluation, Sec. 3.1: leaves select row i_mu of U; each inner node
 * forms its row by eq. "transfermult",
 *   u_t[q] = sum_{j,l} B_t[q,j,l] u_s1[j] u_s2[l],
 * and the root gives the scalar sum_{j,l} B_D[j,l] u_t1[j] u_t2[l].
 * idx: m x d (row-major), out: m. */
int ho_eval(int d, const int64_t *n, const int *k, const double *x, int64_t m, const int64_t *idx, double *out) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  int nn = T.nn;
  int64_t *ox = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  node_offsets(&T, n, k, ox);
  int64_t rows = 0;
  int64_t *orow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
  for (int t = 0; t < nn; ++t) {
    orow[t] = rows;
    rows += (t == 0) ? 1 : k[t];
  }
  int H = tree_max_height(&T);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    double *u = (double *)malloc(sizeof(double) * (size_t)rows);
    for (int h = 0; h <= H; ++h)
      for (int t = 0; t < nn; ++t) {
        if (T.height[t] != h) continue;
        const double *X = x + ox[t];
        if (is_leaf(&T, t)) {
          int mu = T.lo[t];
          int64_t nm = n[mu], i = idx[e * d + mu];
          for (int c = 0; c < k[t]; ++c) u[orow[t] + c] = X[(int64_t)c * nm + i];
        } else {
          int s1 = T.s1[t], s2 = T.s2[t];
          int kt = (t == 0) ? 1 : k[t], k1 = k[s1], k2 = k[s2];
          const double *u1 = u + orow[s1], *u2 = u + orow[s2];
          for (int q = 0; q < kt; ++q) {
            double s = 0.0;
            for (int j = 0; j < k1; ++j) {
              double sj = 0.0;
              for (int l = 0; l < k2; ++l) sj += X[((int64_t)q * k1 + j) * k2 + l] * u2[l];
              s += sj * u1[j];
            }
            u[orow[t] + q] = s;
          }
        }
      }
    out[e] = u[orow[0]];
    free(u);
  }
  free(orow);
  free(ox);
  tree_free(&T);
  return 0;
}

/* Inner product <A,C> by the recursion of Definition "phi" / Lemma "phi"
 * (Sec. 3.2): Phi_leaf = U^T V; Phi_t[jt,jbt] = sum B[jt,j1,j2] Phi_s1[j1,jb1]
 * Phi_s2[j2,jb2] F[jbt,jb1,jb2]; <A,C> = Phi_root.  Used as a cross-check. */
double ho_inner(int d, const int64_t *n, const int *ka, const double *xa, const int *kc, const double *xc) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return NAN;
  int nn = T.nn;
  int64_t *oa = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(nn + 1));
  int64_t *oc = oa + nn + 1;
  node_offsets(&T, n, ka, oa);
  node_offsets(&T, n, kc, oc);
  double **phi = (double **)calloc((size_t)nn, sizeof(double *));
  int H = tree_max_height(&T);
  for (int h = 0; h <= H; ++h)
    for (int t = 0; t < nn; ++t) {
      if (T.height[t] != h) continue;
      if (is_leaf(&T, t)) {
        int64_t nm = n[T.lo[t]];
        int a = ka[t], c = kc[t];
        phi[t] = (double *)malloc(sizeof(double) * (size_t)a * c);
        for (int p = 0; p < a; ++p)
          for (int q = 0; q < c; ++q) {
            double s = 0.0;
            for (int64_t i = 0; i < nm; ++i) s += xa[oa[t] + (int64_t)p * nm + i] * xc[oc[t] + (int64_t)q * nm + i];
            phi[t][p * c + q] = s;
          }
      } else {
        int s1 = T.s1[t], s2 = T.s2[t];
        int at = (t == 0) ? 1 : ka[t], a1 = ka[s1], a2 = ka[s2];
        int ct = (t == 0) ? 1 : kc[t], c1 = kc[s1], c2 = kc[s2];
        const double *B = xa + oa[t], *F = xc + oc[t];
        const double *P1 = phi[s1], *P2 = phi[s2];
        phi[t] = (double *)malloc(sizeof(double) * (size_t)at * ct);
        /* W[jt, jb1, j2] = sum_{j1} B[jt,j1,j2] Phi_s1[j1,jb1] */
        double *W = (double *)calloc((size_t)at * c1 * a2, sizeof(double));
        for (int i = 0; i < at; ++i)
          for (int j1 = 0; j1 < a1; ++j1)
            for (int b1 = 0; b1 < c1; ++b1) {
              double pv = P1[j1 * c1 + b1];
              for (int j2 = 0; j2 < a2; ++j2) W[((int64_t)i * c1 + b1) * a2 + j2] += B[((int64_t)i * a1 + j1) * a2 + j2] * pv;
            }
        /* Y[jt, jb1, jb2] = sum_{j2} W[jt,jb1,j2] Phi_s2[j2,jb2] */
        double *Y = (double *)calloc((size_t)at * c1 * c2, sizeof(double));
        for (int i = 0; i < at; ++i)
          for (int b1 = 0; b1 < c1; ++b1)
            for (int j2 = 0; j2 < a2; ++j2) {
              double wv = W[((int64_t)i * c1 + b1) * a2 + j2];
              for (int b2 = 0; b2 < c2; ++b2) Y[((int64_t)i * c1 + b1) * c2 + b2] += wv * P2[j2 * c2 + b2];
            }
        for (int i = 0; i < at; ++i)
          for (int ib = 0; ib < ct; ++ib) {
            double s = 0.0;
            for (int64_t e = 0; e < (int64_t)c1 * c2; ++e) s += Y[(int64_t)i * c1 * c2 + e] * F[(int64_t)ib * c1 * c2 + e];
            phi[t][i * ct + ib] = s;
          }
        free(W);
        free(Y);
      }
    }
  double res = phi[0][0];
  for (int t = 0; t < nn; ++t) free(phi[t]);
  free(phi);
  free(oa);
  tree_free(&T);
  return res;
}

/* Direct access to the dense building blocks, for their own pins. */
/* Application of an H-operator to an H-tensor, Lemma "operator" (Sec. 3.6):
 * C = L A with L stored as an HT tensor over the index pairs (j_mu, i_mu)
 * (eq. "operatorastensor"), pair (j, i) flattened as j + i m_mu, i.e. the
 * leaf columns of L are column-major m_mu x n_mu matrices W_r.  Ranks of C
 * are kbar_t k_t, the pair index (p, i) of (operator rank, tensor rank)
 * flattened as p k_t + i.  Leaves: V[:, r k + l] = W_r U[:, l]
 * (eq. "operatorleafframes"); inner nodes: F_t = H_t (x) B_t,
 * F[(p,i),(q,j),(r,l)] = H[p,q,r] B[i,j,l].
 *   d, n (tensor mode sizes), m (output mode sizes), kop/xop (operator, mode
 *   sizes m n), kx/xx (tensor), kout/xout (result). */
int ho_apply(int d, const int64_t *n, const int64_t *m, const int *kop, const double *xop, const int *kx,
             const double *xx, int *kout, double *xout) {
  otree T;
  if (d < 2 || tree_init(&T, d)) return -1;
  int64_t *mn = (int64_t *)malloc(sizeof(int64_t) * (size_t)d);
  for (int mu = 0; mu < d; ++mu) mn[mu] = m[mu] * n[mu];
  for (int t = 0; t < T.nn; ++t) kout[t] = (t == 0) ? 1 : kop[t] * kx[t];
  int64_t *oo = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(T.nn + 1));
  int64_t *ox = oo + T.nn + 1, *oc = ox + T.nn + 1;
  node_offsets(&T, mn, kop, oo);
  node_offsets(&T, n, kx, ox);
  node_offsets(&T, m, kout, oc);
  for (int t = 0; t < T.nn; ++t) {
    const double *H = xop + oo[t], *B = xx + ox[t];
    double *F = xout + oc[t];
    if (is_leaf(&T, t)) {
      const int mu = T.lo[t];
      const int64_t mm = m[mu], nm = n[mu];
      const int kb = kop[t], k = kx[t];
      for (int r = 0; r < kb; ++r)
        for (int l = 0; l < k; ++l)
          for (int64_t j = 0; j < mm; ++j) {
            double acc = 0.0;
            for (int64_t i = 0; i < nm; ++i) acc += H[(int64_t)r * mm * nm + j + i * mm] * B[(int64_t)l * nm + i];
            F[((int64_t)r * k + l) * mm + j] = acc;
          }
    } else {
      const int s1 = T.s1[t], s2 = T.s2[t];
      const int pt = (t == 0) ? 1 : kop[t], p1 = kop[s1], p2 = kop[s2];
      const int it = (t == 0) ? 1 : kx[t], i1 = kx[s1], i2 = kx[s2];
      const int o1 = p1 * i1, o2 = p2 * i2;
      for (int p = 0; p < pt; ++p)
        for (int i = 0; i < it; ++i)
          for (int q = 0; q < p1; ++q)
            for (int j = 0; j < i1; ++j)
              for (int r = 0; r < p2; ++r)
                for (int l = 0; l < i2; ++l) {
                  const int64_t I = (int64_t)p * it + i, J = (int64_t)q * i1 + j, L = (int64_t)r * i2 + l;
                  F[(I * o1 + J) * o2 + L] =
                      H[((int64_t)p * p1 + q) * p2 + r] * B[((int64_t)i * i1 + j) * i2 + l];
                }
    }
  }
  free(oo);
  free(mn);
  tree_free(&T);
  return 0;
}

void ho_qr(int64_t m, int n, const double *A, double *Q, double *R) { hh_qr(m, n, A, m, Q, R); }
void ho_eig_sym(int n, const double *A, double *w, double *V) { jacobi_eig(n, A, w, V); }
