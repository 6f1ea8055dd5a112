// k_qr.cu -- Householder QR of row blocks held in registers (the leaf level
// of a TSQR).  Used for the reduced QR decompositions of Sec. 3.4:
// leaf frames U = Q R and M_{2,3}(B_t) = Q R_t (eq. "qrtransfer").  A tall
// matrix is cut into row blocks that fit one CTA; the stacked R factors are
// factorised again by the same kernel and Q is recombined by a batched
// product (see the TSQR driver in api.cu).
#include "internal.h"

namespace htgb {

namespace {

constexpr int kRegRows = 256;  // rows of a register-resident block (32 x NI)

// ---------------------------------------------------------------------------
// Register-resident variant for n <= 4*NW columns and m <= 32*NI rows.
//
// Warp w owns columns 4w..4w+3, one per group of 8 lanes; lane s of a group
// holds rows 32i + 4s + e (i < NI, e < 4) of its column, so a column's dot
// products reduce over the 8 lanes of its group (3 shuffles) and shared
// vectors are read four rows at a time.
//
// Column j's reflector is kept as H_j = I - kappa_j y_j y_j^T, y_j zero above
// row j, y_j(j) = alpha_j - beta_j and the column itself below j (stored
// before the scalars are known; kappa_j from one division).  The warp owning
// column j forms ||.||^2 below the diagonal, beta_j = R(j, j) and kappa_j
// from its registers and stores y_j and kappa_j in shared memory; after one
// barrier every warp holding a column right of j applies H_j with one dot
// product (one 8-lane sum) and one axpy: a -= kappa_j (y_j^T a) y_j.  Row j
// needs no special case.  The owner of column j+1 forms the next reflector
// right after its own update.  One barrier per column.
//
// The y_j stay in shared memory, so Q = H_0 ... H_{n-1} [I; 0] is then
// accumulated backwards on the columns in registers without barriers.
// ---------------------------------------------------------------------------
constexpr int REG_MR = kRegRows;  // leading dimension of the reflector array (rows)

__device__ __forceinline__ void ld4(const float *p, float (&x)[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&x)[4]) {
  const double2 t0 = reinterpret_cast<const double2 *>(p)[0], t1 = reinterpret_cast<const double2 *>(p)[1];
  x[0] = t0.x; x[1] = t0.y; x[2] = t1.x; x[3] = t1.y;
}
__device__ __forceinline__ void st4(float *p, const float (&x)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&x)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(x[0], x[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(x[2], x[3]);
}

// Sum over the 8 lanes of a group (lanes 8g .. 8g+7).
template <typename T>
__device__ __forceinline__ T group_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// Row j (< 64) of column c of the lane's warp, broadcast to the group that
// holds column c (one select tree and one shuffle).
template <typename T, int NI>
__device__ __forceinline__ T row_value(const T (&a)[NI][4], int j, int lane) {
  const int e = j & 3;
  const T y0 = (e & 1) ? a[0][1] : a[0][0], y1 = (e & 1) ? a[0][3] : a[0][2];
  const T z0 = (e & 1) ? a[1][1] : a[1][0], z1 = (e & 1) ? a[1][3] : a[1][2];
  const T y = (e & 2) ? y1 : y0, z = (e & 2) ? z1 : z0;
  return __shfl_sync(0xffffffffu, (j >> 5) ? z : y, (lane & ~7) | ((j >> 2) & 7));
}

// Smallest alpha^2 + ||w||^2 for which the reflector is formed (4 x the
// smallest normal number): below it the column is treated as zero (identity
// reflector), which also keeps kappa below 1 / (4 x the smallest normal).
__device__ __forceinline__ float min_norm2(float) { return 4.0f * 1.17549435e-38f; }
__device__ __forceinline__ double min_norm2(double) { return 4.0 * 2.2250738585072014e-308; }

// Form column j's reflector from the lane's registers (called by the whole
// warp that owns column j, after H_0..H_{j-1} reached it).  With alpha the
// diagonal entry and w the part below it, beta = R(j, j) = -sign(alpha)
// sqrt(alpha^2 + ||w||^2) and u = alpha - beta, the reflector is
// H_j = I - kappa y y^T with y = [0; u; w] and kappa = -1 / (beta u)
// (kappa ||y||^2 = 2).  The owner group stores w before the scalars are known
// (one division, sqrt and IEEE division), then u and kappa; its lanes set
// R(j, j) = beta in their registers (rows below j are held in y).
template <typename T, int NI>
__device__ __forceinline__ void form_reflector(T (&a)[NI][4], T *yj, T *kappa_j, int j, int lane, bool me) {
  const int s = lane & 7;
  T q0 = T(0), q1 = T(0), q2 = T(0), q3 = T(0);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    T x[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 32 * i + 4 * s + e;
      x[e] = (i >= 2 || r > j) ? a[i][e] : T(0);  // j < 64: rows of chunks i >= 2 lie below j
    }
    q0 += x[0] * x[0];
    q1 += x[1] * x[1];
    q2 += x[2] * x[2];
    q3 += x[3] * x[3];
    if (me) st4(yj + 32 * i + 4 * s, x);
  }
  const T s2 = group_sum((q0 + q1) + (q2 + q3));
  const T alpha = row_value<T, NI>(a, j, lane);
  T kappa = T(0), beta = alpha, u = T(0);
  const T x2 = alpha * alpha + s2;
  if (s2 != T(0) && x2 >= min_norm2(T(0))) {
    const T nrm = sqrt(x2);
    beta = (alpha <= T(0)) ? nrm : -nrm;
    u = alpha - beta;
    kappa = T(-1) / (beta * u);
  }
  if (!me) return;
#pragma unroll
  for (int i = 0; i < 2 && i < NI; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (32 * i + 4 * s + e == j) {
        yj[j] = u;
        a[i][e] = beta;
      }
  if (s == 0) *kappa_j = kappa;
}

// a <- a - kappa (y^T a) y for the lane's column (y in shared memory).
// upd = false leaves a unchanged (the reduction spans the warp, so every
// lane takes part).  kKeep keeps y in registers between the two passes.
template <typename T, int NI, bool kKeep>
__device__ __forceinline__ void apply_reflector(T (&a)[NI][4], const T *vj, T tj, bool upd, int s) {
  T v[kKeep ? NI : 1][4];
  T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    T x[4];
    ld4(vj + 32 * i + 4 * s, x);
    d0 += x[0] * a[i][0];
    d1 += x[1] * a[i][1];
    d2 += x[2] * a[i][2];
    d3 += x[3] * a[i][3];
    if (kKeep) {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[kKeep ? i : 0][e] = x[e];
    }
  }
  const T sum = group_sum((d0 + d1) + (d2 + d3));
  const T d = upd ? tj * sum : T(0);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    T x[4];
    if (kKeep) {
#pragma unroll
      for (int e = 0; e < 4; ++e) x[e] = v[kKeep ? i : 0][e];
    } else {
      ld4(vj + 32 * i + 4 * s, x);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) a[i][e] -= d * x[e];
  }
}

template <typename T, int NW, int NI, bool KEEP>
__global__ void __launch_bounds__(NW * 32, (sizeof(T) == 8 && NW == 8) ? 2 : 1) qr_reg_kernel(const QrItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QrItem it = items[blockIdx.x];
  const int m = it.m, n = it.n;
  T *V = reinterpret_cast<T *>(smem_raw);  // REG_MR x n: y_j in column j
  T *tau = V + (int64_t)REG_MR * n;        // n: kappa_j
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 3, s = lane & 7;
  const int c = 4 * warp + g;  // this lane's column
  T a[NI][4];
  const T *A = static_cast<const T *>(it.A) + (int64_t)c * it.lda;
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 32 * i + 4 * s + e;
      a[i][e] = (c < n && r < m) ? A[r] : T(0);
    }
  if (warp == 0) form_reflector<T, NI>(a, V, tau, 0, lane, g == 0);
  for (int j = 0; j + 1 < n; ++j) {
    __syncthreads();                  // y_j and kappa_j are in shared memory
    if (4 * warp + 3 <= j) continue;  // no column of this warp lies right of j
    const T *vj = V + (int64_t)j * REG_MR;
    apply_reflector<T, NI, KEEP>(a, vj, tau[j], c > j, s);
    if (warp == ((j + 1) >> 2))       // the owner of column j+1 forms its reflector
      form_reflector<T, NI>(a, V + (int64_t)(j + 1) * REG_MR, tau + j + 1, j + 1, lane, g == ((j + 1) & 3));
  }
  __syncthreads();
  // R (n x n upper triangular) from the registers
  T *R = static_cast<T *>(it.R) + (int64_t)c * it.ldr;
  if (c < n) {
#pragma unroll
    for (int i = 0; i < 2 && i < NI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        if (r < n) R[r] = (r <= c) ? a[i][e] : T(0);
      }
  }
  // Explicit Q = H_0 H_1 ... H_{n-1} [I; 0], accumulated backwards on the
  // columns of [I; 0].  Column c is untouched by H_j for j > c (v_j is zero
  // above row j, column c is e_c there), so warp w starts at j = 4w + 3.
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) a[i][e] = (32 * i + 4 * s + e == c) ? T(1) : T(0);
  for (int j = min(n - 1, 4 * warp + 3); j >= 0; --j)
    apply_reflector<T, NI, KEEP>(a, V + (int64_t)j * REG_MR, tau[j], true, s);
  T *Q = static_cast<T *>(it.Q) + (int64_t)c * it.ldq;
  if (c < n) {
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        if (r < m) Q[r] = a[i][e];
      }
  }
}

// ---------------------------------------------------------------------------
// Two-column variant for launches with more blocks than SMs (FP32, n <= 64):
// 8 warps, and group g of warp w holds columns c0 = 8w + g and c1 = 8w + 4 + g
// (64 data registers a thread), so that two blocks share an SM and fill each
// other's barrier and shared-memory waits.  Every column goes through the
// same reflector, dot-product and axpy steps as in qr_reg_kernel; R comes out
// bit-identical on random blocks, Q within a few units in the last place (the
// compiled backward accumulation rounds differently).  The warp that owns the
// next reflector's column updates that column's set first, forms the
// reflector, then updates its other set; the other warps update both of their
// columns with one pass over y_j.
// ---------------------------------------------------------------------------

// Both of a lane's columns: a <- a - kappa (y^T a) y and b likewise, y read
// once per pass (the dot products and axpys are those of apply_reflector).
template <typename T, int NI>
__device__ __forceinline__ void apply_reflector2(T (&a)[NI][4], T (&b)[NI][4], const T *vj, T tj, bool upda,
                                                 bool updb, int s) {
  T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
  T f0 = T(0), f1 = T(0), f2 = T(0), f3 = T(0);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    T x[4];
    ld4(vj + 32 * i + 4 * s, x);
    d0 += x[0] * a[i][0];
    d1 += x[1] * a[i][1];
    d2 += x[2] * a[i][2];
    d3 += x[3] * a[i][3];
    f0 += x[0] * b[i][0];
    f1 += x[1] * b[i][1];
    f2 += x[2] * b[i][2];
    f3 += x[3] * b[i][3];
  }
  const T suma = group_sum((d0 + d1) + (d2 + d3));
  const T sumb = group_sum((f0 + f1) + (f2 + f3));
  const T da = upda ? tj * suma : T(0);
  const T db = updb ? tj * sumb : T(0);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    T x[4];
    ld4(vj + 32 * i + 4 * s, x);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      a[i][e] -= da * x[e];
      b[i][e] -= db * x[e];
    }
  }
}

template <typename T, int NI>
__global__ void __launch_bounds__(256, 2) qr_reg2_kernel(const QrItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QrItem it = items[blockIdx.x];
  const int m = it.m, n = it.n;
  T *V = reinterpret_cast<T *>(smem_raw);  // REG_MR x n: y_j in column j
  T *tau = V + (int64_t)REG_MR * n;        // n: kappa_j
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 3, s = lane & 7;
  const int c0 = 8 * warp + g, c1 = c0 + 4;  // this lane's columns
  T a0[NI][4], a1[NI][4];
  {
    const T *A0 = static_cast<const T *>(it.A) + (int64_t)c0 * it.lda;
    const T *A1 = static_cast<const T *>(it.A) + (int64_t)c1 * it.lda;
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        a0[i][e] = (c0 < n && r < m) ? A0[r] : T(0);
        a1[i][e] = (c1 < n && r < m) ? A1[r] : T(0);
      }
  }
  if (warp == 0) form_reflector<T, NI>(a0, V, tau, 0, lane, g == 0);
  for (int j = 0; j + 1 < n; ++j) {
    __syncthreads();                  // y_j and kappa_j are in shared memory
    if (8 * warp + 7 <= j) continue;  // no column of this warp lies right of j
    const T *vj = V + (int64_t)j * REG_MR;
    const T tj = tau[j];
    const int o = j + 1;  // column of the next reflector
    if ((o >> 3) == warp) {
      T *vo = V + (int64_t)o * REG_MR;
      if ((o & 4) == 0) {  // o is in the c0 set; every c1 column lies right of j
        apply_reflector<T, NI, false>(a0, vj, tj, c0 > j, s);
        form_reflector<T, NI>(a0, vo, tau + o, o, lane, g == (o & 3));
        apply_reflector<T, NI, false>(a1, vj, tj, true, s);
      } else {  // o is in the c1 set; no c0 column lies right of j
        apply_reflector<T, NI, false>(a1, vj, tj, c1 > j, s);
        form_reflector<T, NI>(a1, vo, tau + o, o, lane, g == (o & 3));
      }
    } else if (8 * warp + 3 > j) {
      apply_reflector2<T, NI>(a0, a1, vj, tj, c0 > j, c1 > j, s);
    } else {
      apply_reflector<T, NI, false>(a1, vj, tj, c1 > j, s);
    }
  }
  __syncthreads();
  // R (n x n upper triangular) from the registers
  {
    T *R0 = static_cast<T *>(it.R) + (int64_t)c0 * it.ldr;
    T *R1 = static_cast<T *>(it.R) + (int64_t)c1 * it.ldr;
#pragma unroll
    for (int i = 0; i < 2 && i < NI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        if (c0 < n && r < n) R0[r] = (r <= c0) ? a0[i][e] : T(0);
        if (c1 < n && r < n) R1[r] = (r <= c1) ? a1[i][e] : T(0);
      }
  }
  // Explicit Q, accumulated backwards as in qr_reg_kernel: column c is
  // untouched by H_j for j > c, so the c1 set starts at j = 8w + 7 and the
  // c0 set joins at j = 8w + 3.
#pragma unroll
  for (int i = 0; i < NI; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 32 * i + 4 * s + e;
      a0[i][e] = (r == c0) ? T(1) : T(0);
      a1[i][e] = (r == c1) ? T(1) : T(0);
    }
  for (int j = min(n - 1, 8 * warp + 7); j >= 0; --j) {
    const T *vj = V + (int64_t)j * REG_MR;
    if (j > 8 * warp + 3)
      apply_reflector<T, NI, false>(a1, vj, tau[j], true, s);
    else
      apply_reflector2<T, NI>(a0, a1, vj, tau[j], true, true, s);
  }
  {
    T *Q0 = static_cast<T *>(it.Q) + (int64_t)c0 * it.ldq;
    T *Q1 = static_cast<T *>(it.Q) + (int64_t)c1 * it.ldq;
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        if (c0 < n && r < m) Q0[r] = a0[i][e];
        if (c1 < n && r < m) Q1[r] = a1[i][e];
      }
  }
}

template <typename T, int NW, int NI>
cudaError_t launch_qr_reg(const QrItem *d_items, int n_items, int max_n, cudaStream_t s) {
  constexpr bool kKeep = sizeof(T) * NI <= 32;  // FP32 keeps w in registers, FP64 reads it twice
  const size_t smem = ((size_t)REG_MR * max_n + max_n) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(qr_reg_kernel<T, NW, NI, kKeep>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_reg_kernel<T, NW, NI, kKeep><<<n_items, NW * 32, smem, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int qr_max_rows(int n, int elem_bytes) {
  (void)elem_bytes;
  return (n <= 64) ? kRegRows : 0;  // wider matrices are factored in 64-column panels
}

static cudaError_t launch_qr_reg2(const QrItem *d_items, int n_items, int max_n, cudaStream_t s) {
  const size_t smem = ((size_t)REG_MR * max_n + max_n) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(qr_reg2_kernel<float, kRegRows / 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // two blocks of up to 65 KB each: ask for the largest shared-memory carveout
  e = cudaFuncSetAttribute(qr_reg2_kernel<float, kRegRows / 32>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  qr_reg2_kernel<float, kRegRows / 32><<<n_items, 256, smem, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

// Two-column kernel for FP32 launches with more blocks than SMs (two blocks
// per SM instead of one); qr_kernel 1 or 2 forces the choice either way.
static bool use_qr_reg2(int n_items, int qr_kernel) {
  if (qr_kernel == 1) return false;
  if (qr_kernel == 2) return true;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  return n_items > sms;
}

template <typename T>
cudaError_t launch_qr(const QrItem *d_items, int n_items, int max_m, int max_n, cudaStream_t s, int qr_kernel) {
  if (n_items <= 0) return cudaSuccess;
  if (max_n > 64 || max_m > kRegRows) return cudaErrorInvalidValue;  // the TSQR driver never asks for more
  if (max_n <= 16) return launch_qr_reg<T, 4, kRegRows / 32>(d_items, n_items, max_n, s);
  if (max_n <= 32) return launch_qr_reg<T, 8, kRegRows / 32>(d_items, n_items, max_n, s);
  if (sizeof(T) == 4 && use_qr_reg2(n_items, qr_kernel)) return launch_qr_reg2(d_items, n_items, max_n, s);
  return launch_qr_reg<T, 16, kRegRows / 32>(d_items, n_items, max_n, s);
}

template cudaError_t launch_qr<double>(const QrItem *, int, int, int, cudaStream_t, int);
template cudaError_t launch_qr<float>(const QrItem *, int, int, int, cudaStream_t, int);

}  // namespace htgb
