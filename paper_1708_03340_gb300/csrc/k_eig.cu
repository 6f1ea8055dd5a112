// k_eig.cu -- batched symmetric eigendecompositions of the reduced Gramians
// (Sec. 3.3: Bhat_t Q_t = Q_t Sigma_t^2 gives the singular values and left
// singular vectors of every matricization).  One CTA per matrix.
//
// eig_ql_kernel<T>: Householder reduction to tridiagonal form, explicit H
// from the reflectors, implicit QL with Wilkinson shifts, sort.  The matrix is
// scaled by 1/max|G| first.  One thread runs the scalar QL recurrence of a
// sweep and logs its Givens rotations; every thread then applies the logged
// rotations to its own rows of H.  On GB300 a dependent FP64 operation costs
// ~64 cycles and an FP64 divide or square root ~430-670 cycles, so the
// recurrence uses one reciprocal square root per rotation and no divides.
//
// refine_kernel: one step of the Ogita-Aishima iterative refinement
// (Ogita & Aishima, "Iterative refinement for symmetric eigenvalue
// decomposition", Japan J. Indust. Appl. Math. 35, 2018), written from its
// first-order conditions: with X the current eigenvectors, R = I - X^T X,
// S = X^T G X, lambda_i = S_ii / (1 - R_ii) and E solving
// E + E^T = R, (S + E^T S + S E) diagonal to first order:
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   if |lambda_i - lambda_j| > delta
//   E_ij = R_ij / 2                                           otherwise (cluster)
// X <- X (I + E).  Used in FP64 after an FP32 QL solve: the dense products
// keep every warp's FP64 pipe busy instead of a one-lane scalar chain.
#include "internal.h"

namespace htgb {

namespace {

constexpr int EIG_THREADS = 256;
constexpr int kEigSmemK = 128;

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ T block_sum_t(T v, T *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_t(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = (lane < nw) ? red[lane] : T(0);
  return warp_sum_t(s);
}

__device__ double block_max_d(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  return s;
}

// Position of eigenvalue i in descending order (ties by index; NaN last):
// every thread ranks its own values, so the order costs O(k) per thread.
template <typename T>
__device__ __forceinline__ int desc_rank(const T *lam, int k, int i) {
  const double li = isnan((double)lam[i]) ? -INFINITY : (double)lam[i];
  int r = 0;
  for (int j = 0; j < k; ++j) {
    const double lj = isnan((double)lam[j]) ? -INFINITY : (double)lam[j];
    r += (lj > li || (lj == li && j < i)) ? 1 : 0;
  }
  return r;
}

struct EigShared {
  int count;
  int lo;
  int done;
  int status;
};

// Givens rotation with r = sqrt(f^2 + g^2), s = f / r, c = g / r.
__device__ __forceinline__ void givens(double f, double g, double &r, double &s, double &c) {
  const double q = f * f + g * g;  // the matrix is scaled to O(1): no overflow, underflow only at 1e-154
  if (q == 0.0) {
    r = 0.0;
    s = 0.0;
    c = 1.0;
    return;
  }
  const double ri = rsqrt(q);
  r = q * ri;
  s = f * ri;
  c = g * ri;
}
__device__ __forceinline__ void givens(float f, float g, float &r, float &s, float &c) {
  const float m = fmaxf(fabsf(f), fabsf(g));
  if (m == 0.0f) {
    r = 0.0f;
    s = 0.0f;
    c = 1.0f;
    return;
  }
  // scale by 1/max(m, 1e-30) to keep f^2 + g^2 away from FP32 underflow; the
  // floor keeps the scale finite when m is subnormal (1/m would overflow to
  // inf and turn the rotation into NaN), and q stays a normal number then
  const float sc = fmaxf(m, 1e-30f);
  const float im = 1.0f / sc;
  const float fs = f * im, gs = g * im;
  const float q = fs * fs + gs * gs;
  const float ri = rsqrtf(q);
  r = sc * q * ri;
  s = fs * ri;
  c = gs * ri;
}

template <typename T>
__global__ void __launch_bounds__(EIG_THREADS) eig_ql_kernel(const EigItem *__restrict__ items, void *scratch,
                                                             int64_t scratch_stride, int z_in_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x;
  // layout: [32 doubles][Z: k*k T, when the launch's largest k fits][6k + 32 T][k ints];
  // the FP64 scratch comes first so that it stays 8-byte aligned for any k.
  // z_in_smem is decided per launch (from its largest k), since the dynamic
  // shared memory is sized for the launch, not for the item.
  double *redd = reinterpret_cast<double *>(smem_raw);
  T *Z;
  T *tail;
  if (z_in_smem) {
    Z = reinterpret_cast<T *>(redd + 32);
    tail = Z + (int64_t)k * k;
  } else {
    Z = static_cast<T *>(scratch) + (int64_t)blockIdx.x * scratch_stride;
    tail = reinterpret_cast<T *>(redd + 32);
  }
  T *dg = tail;
  T *eo = dg + k;
  T *tau = eo + k;
  T *pv = tau + k;
  T *rc = pv + k;
  T *rs = rc + k;
  T *red = rs + k;
  int *perm = reinterpret_cast<int *>(red + 32);
  __shared__ EigShared sh;
  const int ld = k;
  // scale to max |G| = 1 (symmetrised)
  double mx = 0.0;
  for (int e = tid; e < k * k; e += nt) mx = fmax(mx, fabs(it.G[e]));
  mx = block_max_d(mx, redd);
  const double scale = (mx > 0.0) ? mx : 1.0;
  const double inv_scale = 1.0 / scale;
  for (int e = tid; e < k * k; e += nt) {
    int c = e / k, r = e - c * k;
    Z[e] = T(0.5 * (it.G[(int64_t)c * k + r] + it.G[(int64_t)r * k + c]) * inv_scale);
  }
  __syncthreads();
  // 1. tridiagonalisation: step j annihilates Z[j+2:k, j]
  for (int j = 0; j + 2 < k; ++j) {
    T *x = Z + (int64_t)j * ld;
    T part = T(0);
    for (int r = j + 2 + tid; r < k; r += nt) part += x[r] * x[r];
    const T s2 = block_sum_t(part, red);
    const T alpha = x[j + 1];
    T tj = T(0), beta = alpha;
    if (s2 != T(0)) {
      const T nrm = sqrt(alpha * alpha + s2);
      beta = (alpha <= T(0)) ? nrm : -nrm;
      const T inv_v0 = T(1) / (alpha - beta);
      tj = (beta - alpha) / beta;
      for (int r = j + 2 + tid; r < k; r += nt) x[r] *= inv_v0;
    }
    __syncthreads();
    if (tid == 0) {
      tau[j] = tj;
      dg[j] = x[j];
      eo[j] = beta;
    }
    if (tj != T(0)) {
      const int L = k - j - 1;
      for (int rr = tid; rr < L; rr += nt) {
        const int r = j + 1 + rr;
        T s = Z[(int64_t)(j + 1) * ld + r];
        for (int cc = 1; cc < L; ++cc) s += Z[(int64_t)(j + 1 + cc) * ld + r] * x[j + 1 + cc];
        pv[rr] = tj * s;
      }
      __syncthreads();
      T pp = T(0);
      for (int rr = tid; rr < L; rr += nt) pp += pv[rr] * (rr == 0 ? T(1) : x[j + 1 + rr]);
      const T kk = T(0.5) * tj * block_sum_t(pp, red);
      for (int rr = tid; rr < L; rr += nt) pv[rr] -= kk * (rr == 0 ? T(1) : x[j + 1 + rr]);
      __syncthreads();
      for (int e = tid; e < L * L; e += nt) {
        const int cc = e / L, rr = e - cc * L;
        const T vr = (rr == 0) ? T(1) : x[j + 1 + rr];
        const T vc = (cc == 0) ? T(1) : x[j + 1 + cc];
        Z[(int64_t)(j + 1 + cc) * ld + (j + 1 + rr)] -= vr * pv[cc] + pv[rr] * vc;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (k >= 2) {
      dg[k - 2] = Z[(int64_t)(k - 2) * ld + (k - 2)];
      eo[k - 2] = Z[(int64_t)(k - 2) * ld + (k - 1)];
    }
    dg[k - 1] = Z[(int64_t)(k - 1) * ld + (k - 1)];
    eo[k - 1] = T(0);
  }
  __syncthreads();
  // 2. explicit H = H_0 ... H_{k-3}; column j+1 carries reflector j
  for (int j = k - 3; j >= 0; --j) {
    for (int r = j + 2 + tid; r < k; r += nt) Z[(int64_t)(j + 1) * ld + r] = Z[(int64_t)j * ld + r];
    __syncthreads();
  }
  for (int e = tid; e < k; e += nt) {
    Z[e] = (e == 0) ? T(1) : T(0);
    if (e > 0) Z[(int64_t)e * ld] = T(0);
  }
  __syncthreads();
  for (int c = k - 1; c >= 1; --c) {
    const int j = c - 1;
    const T tj = (j <= k - 3) ? tau[j] : T(0);
    const T *v = Z + (int64_t)c * ld;
    if (tj != T(0)) {
      const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
      for (int cc = c + 1 + warp; cc < k; cc += nw) {
        T *y = Z + (int64_t)cc * ld;
        T s = T(0);
        for (int r = c + 1 + lane; r < k; r += 32) s += v[r] * y[r];
        s = warp_sum_t(s) + y[c];
        s *= tj;
        if (lane == 0) y[c] -= s;
        for (int r = c + 1 + lane; r < k; r += 32) y[r] -= s * v[r];
      }
    }
    __syncthreads();
    T *x = Z + (int64_t)c * ld;
    for (int r = 1 + tid; r < k; r += nt) {
      if (r < c) x[r] = T(0);
      else if (r == c) x[r] = T(1) - tj;
      else x[r] = -tj * x[r];
    }
    __syncthreads();
  }
  // 3. implicit QL; deflation when |e_m| <= eps ||T|| (normwise: the Gramians
  //    need eigenvalues to within eps * lambda_max only)
  if (tid == 0) {
    sh.done = 0;
    sh.status = 0;
  }
  int l = 0, iter = 0;
  T tol = T(0);
  if (tid == 0) {
    T tn = T(0);
    for (int i = 0; i < k; ++i) {
      T v = fabs(dg[i]) + fabs(eo[i]) + (i > 0 ? fabs(eo[i - 1]) : T(0));
      tn = tn > v ? tn : v;
    }
    const T eps = (sizeof(T) == 8) ? T(2.220446049250313e-16) : T(1.1920929e-7);
    tol = eps * tn;
  }
  for (;;) {
    if (tid == 0) {
      sh.count = 0;
      while (l < k && sh.count == 0) {
        int mm;
        for (mm = l; mm < k - 1; ++mm)
          if (fabs(eo[mm]) <= tol) break;
        if (mm == l) {
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > 64) {
          sh.status = 1;
          ++l;
          iter = 0;
          continue;
        }
        // Wilkinson-type shift from the leading 2x2 block
        T g = (dg[l + 1] - dg[l]) / (T(2) * eo[l]);
        T r = sqrt(g * g + T(1));
        g = dg[mm] - dg[l] + eo[l] / (g + copysign(r, g));
        T s = T(1), c = T(1), p = T(0);
        bool deflated = false;
        for (int i = mm - 1; i >= l; --i) {
          const T f = s * eo[i], b = c * eo[i];
          givens(f, g, r, s, c);
          eo[i + 1] = r;
          if (r == T(0)) {
            dg[i + 1] -= p;
            eo[mm] = T(0);
            deflated = true;
            break;
          }
          g = dg[i + 1] - p;
          r = (dg[i] - g) * s + T(2) * c * b;
          p = s * r;
          dg[i + 1] = g + p;
          g = c * r - b;
          rc[sh.count] = c;
          rs[sh.count] = s;
          sh.count++;
        }
        sh.lo = mm - 1;
        if (!deflated) {
          dg[l] -= p;
          eo[l] = g;
          eo[mm] = T(0);
        }
      }
      if (l >= k && sh.count == 0) sh.done = 1;
    }
    __syncthreads();
    if (sh.done) break;
    const int cnt = sh.count, i0 = sh.lo;
    for (int row = tid; row < k; row += nt) {
      for (int q = 0; q < cnt; ++q) {
        const int i = i0 - q;
        T *zi = Z + (int64_t)i * ld + row;
        T *zi1 = Z + (int64_t)(i + 1) * ld + row;
        const T f = *zi1;
        *zi1 = rs[q] * (*zi) + rc[q] * f;
        *zi = rc[q] * (*zi) - rs[q] * f;
      }
    }
    __syncthreads();
  }
  // 4. sort descending, unscale
  for (int i = tid; i < k; i += nt) perm[desc_rank(dg, k, i)] = i;
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {
    int c = e / k, r = e - c * k;
    it.V[e] = (double)Z[(int64_t)perm[c] * ld + r];
  }
  for (int c = tid; c < k; c += nt) it.lam[c] = (double)dg[perm[c]] * scale;
}

// ---- FP64 refinement ---------------------------------------------------------
// C = op(A) * B for k x k column-major matrices in shared or global memory;
// transA: C[i][j] = sum_l A[l][i] B[l][j].  Each thread computes 4x4 outputs.
__device__ void small_gemm(const double *A, const double *B, double *C, int k, bool transA) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tiles = (k + 3) / 4;
  for (int t = tid; t < tiles * tiles; t += nt) {
    const int ti = (t % tiles) * 4, tj = (t / tiles) * 4;
    double acc[4][4] = {};
    for (int l = 0; l < k; ++l) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = ti + u, j = tj + u;
        a[u] = (i < k) ? (transA ? A[(int64_t)i * k + l] : A[(int64_t)l * k + i]) : 0.0;
        b[u] = (j < k) ? B[(int64_t)j * k + l] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (ti + u < k && tj + v < k) C[(int64_t)(tj + v) * k + ti + u] = acc[u][v];
  }
}

__global__ void __launch_bounds__(EIG_THREADS) refine_kernel(const EigItem *__restrict__ items, double *scratch,
                                                             int64_t scratch_stride, int buf_in_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x;
  const int64_t kk = (int64_t)k * k;
  // buf_in_smem: decided per launch from its largest k (the shared memory is sized for the launch)
  double *buf = buf_in_smem ? reinterpret_cast<double *>(smem_raw) : scratch + (int64_t)blockIdx.x * scratch_stride;
  double *A = buf, *X = buf + kk, *W1 = buf + 2 * kk, *W2 = buf + 3 * kk;
  double *small = buf_in_smem ? buf + 4 * kk : reinterpret_cast<double *>(smem_raw);
  double *lam = small;          // k
  double *red = small + k;      // 32
  int *perm = reinterpret_cast<int *>(red + 32);
  double mx = 0.0;
  for (int e = tid; e < kk; e += nt) mx = fmax(mx, fabs(it.G[e]));
  mx = block_max_d(mx, red);
  const double scale = (mx > 0.0) ? mx : 1.0, inv_scale = 1.0 / scale;
  for (int e = tid; e < kk; e += nt) {
    const int c = (int)(e / k), r = (int)(e - (int64_t)c * k);
    A[e] = 0.5 * (it.G[(int64_t)c * k + r] + it.G[(int64_t)r * k + c]) * inv_scale;
    X[e] = it.V[e];
  }
  __syncthreads();
  small_gemm(A, X, W1, k, false);  // W1 = A X
  __syncthreads();
  small_gemm(X, W1, W2, k, true);  // W2 = S = X^T A X
  __syncthreads();
  small_gemm(X, X, W1, k, true);   // W1 = X^T X
  __syncthreads();
  for (int e = tid; e < kk; e += nt) {
    const int c = (int)(e / k), r = (int)(e - (int64_t)c * k);
    W1[e] = ((r == c) ? 1.0 : 0.0) - W1[e];  // R = I - X^T X
  }
  __syncthreads();
  for (int i = tid; i < k; i += nt) lam[i] = W2[(int64_t)i * k + i] / (1.0 - W1[(int64_t)i * k + i]);
  // cluster threshold from the sizes of the first-order residuals
  double so = 0.0, ro = 0.0, lm = 0.0;
  for (int e = tid; e < kk; e += nt) {
    const int c = (int)(e / k), r = (int)(e - (int64_t)c * k);
    if (r != c) so = fmax(so, fabs(W2[e]));
    ro = fmax(ro, fabs(W1[e]));
  }
  __syncthreads();
  for (int i = tid; i < k; i += nt) lm = fmax(lm, fabs(lam[i]));
  so = block_max_d(so, red);
  ro = block_max_d(ro, red);
  lm = block_max_d(lm, red);
  const double delta = 2.0 * (so + lm * ro) * (double)k;
  for (int e = tid; e < kk; e += nt) {
    const int c = (int)(e / k), r = (int)(e - (int64_t)c * k);
    const double Rv = W1[e];
    double Ev;
    if (r == c) {
      Ev = 0.5 * Rv;
    } else {
      const double gap = lam[c] - lam[r];
      Ev = (fabs(gap) > delta) ? (W2[e] + lam[c] * Rv) / gap : 0.5 * Rv;
    }
    W2[e] = Ev;
  }
  __syncthreads();
  small_gemm(X, W2, W1, k, false);  // W1 = X E
  __syncthreads();
  for (int e = tid; e < kk; e += nt) W1[e] += X[e];
  for (int i = tid; i < k; i += nt) perm[desc_rank(lam, k, i)] = i;
  __syncthreads();
  for (int e = tid; e < kk; e += nt) {
    const int c = (int)(e / k), r = (int)(e - (int64_t)c * k);
    it.V[e] = W1[(int64_t)perm[c] * k + r];
  }
  for (int c = tid; c < k; c += nt) it.lam[c] = lam[perm[c]] * scale;
}

// ---- double-float refinement (k <= kDfMaxK) ---------------------------------
// The same Ogita-Aishima step with its four k x k products on the FP32 pipes:
// every product of FP32 operands is carried exactly as a pair (p, e) with p =
// a b rounded and e = fma(a, b, -p), and summed into a double-float (hi, lo)
// with a two-sum (Dekker / Knuth error-free transformations); the symmetrised
// scaled Gramian A is split into A_hi + A_lo (48 bits), the FP32 solve's
// eigenvectors X are FP32 numbers.  The sums are accurate to about 2^-48
// relative, far below the FP32 Gramian's own error; lambda, R, S and E are
// formed in FP64 from the double-float results.  GB300 runs FP32 at 64 times
// its FP64 rate, so this is several times faster than FP64 products.
constexpr int kDfMaxK = 64;

__device__ __forceinline__ void df_mac(float &hi, float &lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);  // a b = p + e exactly
  const float t = __fadd_rn(hi, p);
  const float bp = __fsub_rn(t, hi);
  const float e2 = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));  // hi + p = t + e2 exactly
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(e2, e));
}

// C = op(A) B for k x k column-major matrices in shared memory (leading
// dimension ld), A = Ah (+ Al), B = Bh (+ Bl): high parts multiplied exactly,
// the cross terms rounded into the low word.  op(A)_il = A[i ld + l] when
// kTransA, else A[l ld + i].  Each thread accumulates a 4 x 4 block; the
// threads of a warp share their rows (broadcast reads of A).
template <bool kTransA, bool kALo, bool kBLo>
__device__ void df_gemm(const float *Ah, const float *Al, const float *Bh, const float *Bl, float *Ch, float *Cl,
                        int k, int ld) {
  const int tiles = (k + 3) / 4;
  for (int t = threadIdx.x; t < tiles * tiles; t += blockDim.x) {
    const int ti = (t / tiles) * 4, tj = (t % tiles) * 4;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) hi[u][v] = lo[u][v] = 0.0f;
    for (int l = 0; l < k; ++l) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = ti + u, j = tj + u;
        const int ia = kTransA ? i * ld + l : l * ld + i;
        ah[u] = (i < k) ? Ah[ia] : 0.0f;
        al[u] = (kALo && i < k) ? Al[ia] : 0.0f;
        bh[u] = (j < k) ? Bh[j * ld + l] : 0.0f;
        bl[u] = (kBLo && j < k) ? Bl[j * ld + l] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          df_mac(hi[u][v], lo[u][v], ah[u], bh[v]);
          if (kALo) lo[u][v] = __fmaf_rn(al[u], bh[v], lo[u][v]);
          if (kBLo) lo[u][v] = __fmaf_rn(ah[u], bl[v], lo[u][v]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (ti + u < k && tj + v < k) {
          const float s = __fadd_rn(hi[u][v], lo[u][v]);  // renormalise: |lo| <= ulp(hi) / 2
          Ch[(tj + v) * ld + ti + u] = s;
          Cl[(tj + v) * ld + ti + u] = __fsub_rn(lo[u][v], __fsub_rn(s, hi[u][v]));
        }
  }
}

size_t refine_df_smem(int max_k) {
  return (size_t)(kDfMaxK + 32) * sizeof(double) + (size_t)kDfMaxK * sizeof(int) +
         7 * (size_t)max_k * (max_k + 1) * sizeof(float);
}

__global__ void __launch_bounds__(EIG_THREADS) refine_df_kernel(const EigItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x, ld = k + 1;  // odd ld: 2-way bank conflicts at most
  const int sz = k * ld;
  double *lam = reinterpret_cast<double *>(smem_raw);  // k
  double *red = lam + kDfMaxK;                          // 32
  int *rank = reinterpret_cast<int *>(red + 32);        // k
  float *Ah = reinterpret_cast<float *>(rank + kDfMaxK);
  float *Al = Ah + sz, *X = Al + sz, *Th = X + sz, *Tl = Th + sz, *Sh = Tl + sz, *Sl = Sh + sz;
  double mx = 0.0;
  for (int e = tid; e < k * k; e += nt) mx = fmax(mx, fabs(it.G[e]));
  mx = block_max_d(mx, red);
  const double scale = (mx > 0.0) ? mx : 1.0, inv_scale = 1.0 / scale;
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, r = e - c * k;
    const double a = 0.5 * (it.G[(int64_t)c * k + r] + it.G[(int64_t)r * k + c]) * inv_scale;
    const float ah = (float)a;
    Ah[c * ld + r] = ah;
    Al[c * ld + r] = (float)(a - (double)ah);
    X[c * ld + r] = (float)it.V[e];  // the FP32 solve's eigenvectors: exact
  }
  __syncthreads();
  df_gemm<false, true, false>(Ah, Al, X, nullptr, Th, Tl, k, ld);  // T = A X
  __syncthreads();
  df_gemm<true, false, true>(X, nullptr, Th, Tl, Sh, Sl, k, ld);   // S = X^T T
  __syncthreads();
  df_gemm<true, false, false>(X, nullptr, X, nullptr, Ah, Al, k, ld);  // P = X^T X = I - R
  __syncthreads();
  // lambda_i = S_ii / (1 - R_ii) = S_ii / P_ii
  for (int i = tid; i < k; i += nt)
    lam[i] = ((double)Sh[i * ld + i] + (double)Sl[i * ld + i]) / ((double)Ah[i * ld + i] + (double)Al[i * ld + i]);
  double so = 0.0, ro = 0.0;
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, r = e - c * k;
    const double P = (double)Ah[c * ld + r] + (double)Al[c * ld + r];
    if (r != c) so = fmax(so, fabs((double)Sh[c * ld + r] + (double)Sl[c * ld + r]));
    ro = fmax(ro, fabs((r == c ? 1.0 : 0.0) - P));
  }
  __syncthreads();
  double lm = 0.0;
  for (int i = tid; i < k; i += nt) lm = fmax(lm, fabs(lam[i]));
  so = block_max_d(so, red);
  ro = block_max_d(ro, red);
  lm = block_max_d(lm, red);
  const double delta = 2.0 * (so + lm * ro) * (double)k;
  // E (FP64, stored as a float pair in T's place)
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, r = e - c * k;
    const double Rv = (r == c ? 1.0 : 0.0) - ((double)Ah[c * ld + r] + (double)Al[c * ld + r]);
    double Ev;
    if (r == c) {
      Ev = 0.5 * Rv;
    } else {
      const double gap = lam[c] - lam[r];
      const double Sv = (double)Sh[c * ld + r] + (double)Sl[c * ld + r];
      Ev = (fabs(gap) > delta) ? (Sv + lam[c] * Rv) / gap : 0.5 * Rv;
    }
    const float eh = (float)Ev;
    Th[c * ld + r] = eh;
    Tl[c * ld + r] = (float)(Ev - (double)eh);
  }
  for (int i = tid; i < k; i += nt) rank[i] = desc_rank(lam, k, i);
  __syncthreads();
  df_gemm<false, false, true>(X, nullptr, Th, Tl, Sh, Sl, k, ld);  // X E
  __syncthreads();
  // X <- X (I + E), columns in descending eigenvalue order
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, r = e - c * k;
    it.V[(int64_t)rank[c] * k + r] = (double)X[c * ld + r] + ((double)Sh[c * ld + r] + (double)Sl[c * ld + r]);
  }
  for (int c = tid; c < k; c += nt) it.lam[rank[c]] = lam[c] * scale;
}

template <typename T>
size_t ql_smem(int max_k) {
  size_t tail = 32 * sizeof(double) + (size_t)(6 * max_k + 32) * sizeof(T) + (size_t)max_k * sizeof(int);
  return (max_k <= kEigSmemK) ? (size_t)max_k * max_k * sizeof(T) + tail : tail;
}

// ---- semidefinite Cholesky (square-root Gramian factors) --------------------
// Right-looking, one column per step: pivot d = A_jj; d <= tau gives a zero
// column, otherwise L_jj = sqrt(d), L_ij = A_ij / L_jj and the trailing lower
// triangle takes A_ip -= L_ij L_pj.  tau = 4 k u_64 max_i G_ii.
__global__ void __launch_bounds__(EIG_THREADS) chol_kernel(const CholItem *__restrict__ items) {
  const CholItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x;
  double *A = it.W;
  __shared__ double red[32];
  __shared__ double piv, pinv;
  double mx = 0.0;
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, r = e - c * k;
    const double v = 0.5 * (it.G[(int64_t)c * k + r] + it.G[(int64_t)r * k + c]);
    A[e] = v;
    if (r == c) mx = fmax(mx, v);
  }
  mx = block_max_d(mx, red);
  const double tau = 4.0 * k * 1.1102230246251565e-16 * mx;
  for (int j = 0; j < k; ++j) {
    __syncthreads();  // the previous update is complete
    if (tid == 0) {
      const double d = A[(int64_t)j * k + j];
      piv = (d > tau) ? sqrt(d) : 0.0;
      pinv = (d > tau) ? 1.0 / piv : 0.0;
      A[(int64_t)j * k + j] = piv;
    }
    __syncthreads();
    const double pi = pinv;
    for (int i = j + 1 + tid; i < k; i += nt) A[(int64_t)j * k + i] *= pi;
    __syncthreads();
    if (pi == 0.0) continue;
    const int m = k - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int p = j + 1 + e / m, i = j + 1 + e % m;
      if (i >= p) A[(int64_t)p * k + i] -= A[(int64_t)j * k + i] * A[(int64_t)j * k + p];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, r = e - c * k;
    it.S[e] = (r >= c) ? (float)A[e] : 0.0f;
  }
}

}  // namespace

cudaError_t launch_chol(const CholItem *d_items, int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  chol_kernel<<<n_items, EIG_THREADS, 0, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_eig(const EigItem *d_items, int n_items, int max_k, double *scratch, cudaStream_t s, int mode) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e;
  if (mode == 0) {  // FP64 QL
    const size_t smem = ql_smem<double>(max_k);
    e = cudaFuncSetAttribute(eig_ql_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    eig_ql_kernel<double><<<n_items, EIG_THREADS, smem, s>>>(d_items, scratch, (int64_t)max_k * max_k,
                                                             max_k <= kEigSmemK ? 1 : 0);
    count_launch();
    return cudaGetLastError();
  }
  // FP32 QL, then one refinement step (double-float for k <= kDfMaxK, else FP64)
  const size_t smem = ql_smem<float>(max_k);
  e = cudaFuncSetAttribute(eig_ql_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eig_ql_kernel<float><<<n_items, EIG_THREADS, smem, s>>>(d_items, scratch, (int64_t)max_k * max_k,
                                                            max_k <= kEigSmemK ? 1 : 0);
  count_launch();
  if (max_k <= kDfMaxK) {  // double-float refinement in shared memory
    const size_t dsm = refine_df_smem(max_k);
    e = cudaFuncSetAttribute(refine_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (e != cudaSuccess) return e;
    refine_df_kernel<<<n_items, EIG_THREADS, dsm, s>>>(d_items);
    count_launch();
    return cudaGetLastError();
  }
  const size_t rsm = (max_k <= 64) ? (size_t)(4 * max_k * max_k + max_k + 32) * sizeof(double) + max_k * sizeof(int)
                                   : (size_t)(max_k + 32) * sizeof(double) + max_k * sizeof(int);
  e = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
  if (e != cudaSuccess) return e;
  refine_kernel<<<n_items, EIG_THREADS, rsm, s>>>(d_items, scratch, 4 * (int64_t)max_k * max_k, max_k <= 64 ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

int eig_smem_k() { return kEigSmemK; }

}  // namespace htgb
