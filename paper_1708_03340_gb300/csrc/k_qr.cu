// k_qr.cu -- Householder QR of row blocks held in shared memory (the leaf
// level of a TSQR).  Used for the reduced QR decompositions of Sec. 3.4:
// leaf frames U = Q R and M_{2,3}(B_t) = Q R_t (eq. "qrtransfer").  A tall
// matrix is cut into row blocks that fit one CTA; the stacked R factors are
// factorised again by the same kernel and Q is recombined by a batched
// product (see the TSQR driver in api.cu).
#include "internal.h"

namespace htgb {

namespace {

constexpr int QR_THREADS = 512;
constexpr int kSmemLimit = 232448;  // opt-in shared memory per CTA on sm_103
constexpr int kSmemReserve = 2048;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduction over the block; every thread gets the sum.  red has >= 32 slots.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = (lane < nw) ? red[lane] : T(0);
  return warp_sum(s);
}

// Apply H = I - tau v v^T (v = [1; W[j+1:m, j]]) to columns c0..n-1 of W,
// rows j..m-1.  One warp per column.
template <typename T>
__device__ __forceinline__ void apply_reflector(T *W, int ld, int m, int n, int j, int c0, T tau) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T *v = W + (int64_t)j * ld;
  for (int c = c0 + warp; c < n; c += nw) {
    T *y = W + (int64_t)c * ld;
    T s = T(0);
    for (int r = j + 1 + lane; r < m; r += 32) s += v[r] * y[r];
    s = warp_sum(s) + y[j];
    s *= tau;
    if (lane == 0) y[j] -= s;
    for (int r = j + 1 + lane; r < m; r += 32) y[r] -= s * v[r];
  }
}

template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qr_block_kernel(const QrItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QrItem it = items[blockIdx.x];
  const int m = it.m, n = it.n, ld = it.m;
  T *W = reinterpret_cast<T *>(smem_raw);
  T *tau = W + (int64_t)m * n;
  T *red = tau + n;
  const int tid = threadIdx.x;
  const T *A = static_cast<const T *>(it.A);
  for (int c = 0; c < n; ++c)
    for (int r = tid; r < m; r += blockDim.x) W[(int64_t)c * ld + r] = A[(int64_t)c * it.lda + r];
  __syncthreads();
  // factorisation: column j of W becomes [R(0:j, j); beta; v tail]
  for (int j = 0; j < n; ++j) {
    T *x = W + (int64_t)j * ld;
    T part = T(0);
    for (int r = j + 1 + tid; r < m; r += blockDim.x) part += x[r] * x[r];
    const T s2 = block_sum(part, red);
    const T alpha = x[j];
    T tj = T(0);
    if (s2 != T(0)) {
      const T nrm = sqrt(alpha * alpha + s2);
      const T beta = (alpha <= T(0)) ? nrm : -nrm;
      const T inv_v0 = T(1) / (alpha - beta);
      tj = (beta - alpha) / beta;
      for (int r = j + 1 + tid; r < m; r += blockDim.x) x[r] *= inv_v0;
      __syncthreads();
      if (tid == 0) x[j] = beta;
    }
    if (tid == 0) tau[j] = tj;
    __syncthreads();
    if (tj != T(0)) apply_reflector(W, ld, m, n, j, j + 1, tj);
    __syncthreads();
  }
  // R: upper triangle, zeros below
  T *R = static_cast<T *>(it.R);
  for (int e = tid; e < n * n; e += blockDim.x) {
    int c = e / n, r = e - c * n;
    R[(int64_t)c * it.ldr + r] = (r <= c) ? W[(int64_t)c * ld + r] : T(0);
  }
  __syncthreads();
  // explicit Q = H_0 ... H_{n-1} [I; 0], formed in place from the last reflector back
  for (int j = n - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (j < n - 1 && tj != T(0)) apply_reflector(W, ld, m, n, j, j + 1, tj);
    __syncthreads();
    T *x = W + (int64_t)j * ld;
    for (int r = tid; r < m; r += blockDim.x) {
      if (r < j) x[r] = T(0);
      else if (r == j) x[r] = T(1) - tj;
      else x[r] = -tj * x[r];
    }
    __syncthreads();
  }
  T *Q = static_cast<T *>(it.Q);
  for (int c = 0; c < n; ++c)
    for (int r = tid; r < m; r += blockDim.x) Q[(int64_t)c * it.ldq + r] = W[(int64_t)c * ld + r];
}

// ---------------------------------------------------------------------------
// Register-resident variant for n <= 16*CPW columns and m <= 32*ROWS rows.
// Warp w owns columns w, w+16, ...; lane l owns rows l, l+32, ....  The
// factorisation needs one barrier per column: the owner warp of column j
// builds the reflector from its registers and publishes v_j in shared
// memory, then every warp applies H_j to its own columns (the dot products of
// its active columns reduced together).  Q = H_0 ... H_{n-1} [I; 0] is then
// accumulated backwards by every warp on its own columns, from the stored
// reflectors, without further barriers.
// ---------------------------------------------------------------------------
constexpr int REG_ROWS = 8;   // rows per lane -> m <= 256
constexpr int REG_WARPS = 16;

// a[q] <- (I - tau v v^T) a[q] for the owned columns q >= q0 (warp-uniform),
// v read from shared memory (one column of V, rows lane + 32 i); the dot
// products of the active columns are reduced together.
template <typename T, int CPW>
__device__ __forceinline__ void qr_apply_reflector(T (&a)[CPW][REG_ROWS], const T *vcol, T tj, int q0, int lane) {
  T v[REG_ROWS];
#pragma unroll
  for (int i = 0; i < REG_ROWS; ++i) v[i] = vcol[lane + 32 * i];
  T sd[CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    sd[q] = T(0);
    if (q >= q0) {
#pragma unroll
      for (int i = 0; i < REG_ROWS; ++i) sd[q] += v[i] * a[q][i];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < CPW; ++q)
      if (q >= q0) sd[q] += __shfl_xor_sync(0xffffffffu, sd[q], o);
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    if (q < q0) continue;
    const T sq = sd[q] * tj;
#pragma unroll
    for (int i = 0; i < REG_ROWS; ++i) a[q][i] -= sq * v[i];
  }
}

template <typename T, int CPW>
__global__ void __launch_bounds__(REG_WARPS * 32) qr_reg_kernel(const QrItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QrItem it = items[blockIdx.x];
  const int m = it.m, n = it.n;
  constexpr int MR = 32 * REG_ROWS + 1;  // leading dimension of V (odd: no bank conflicts across columns)
  T *V = reinterpret_cast<T *>(smem_raw);  // MR x n, column-major
  T *tau = V + (int64_t)MR * n;            // n
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T a[CPW][REG_ROWS];
  const T *A = static_cast<const T *>(it.A);
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + REG_WARPS * q;
#pragma unroll
    for (int i = 0; i < REG_ROWS; ++i) {
      const int r = lane + 32 * i;
      a[q][i] = (c < n && r < m) ? A[(int64_t)c * it.lda + r] : T(0);
    }
  }
  for (int j = 0; j < n; ++j) {
    const int ow = j % REG_WARPS, qj = j / REG_WARPS;
    if (warp == ow) {
      T alpha = T(0), s2 = T(0);
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        if (q != qj) continue;
#pragma unroll
        for (int i = 0; i < REG_ROWS; ++i) {
          const int r = lane + 32 * i;
          if (r == j) alpha = a[q][i];
          if (r > j) s2 += a[q][i] * a[q][i];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {  // both sums in one butterfly; one lane holds alpha, the others 0
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
      }
      T tj = T(0), beta = alpha, scale = T(0);
      if (s2 != T(0)) {
        const T nrm = sqrt(alpha * alpha + s2);
        beta = (alpha <= T(0)) ? nrm : -nrm;
        tj = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
      }
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        if (q != qj) continue;
#pragma unroll
        for (int i = 0; i < REG_ROWS; ++i) {
          const int r = lane + 32 * i;
          const T v = (r < j) ? T(0) : (r == j ? T(1) : a[q][i] * scale);
          V[(int64_t)j * MR + r] = v;
          if (r == j) a[q][i] = beta;
          else if (r > j) a[q][i] = T(0);
        }
      }
      if (lane == 0) tau[j] = tj;
    }
    __syncthreads();
    const T tj = tau[j];
    const int q0 = (j - warp + REG_WARPS) / REG_WARPS;  // first owned column right of j (j - warp + 16 >= 1)
    if (tj != T(0) && q0 < CPW) qr_apply_reflector<T, CPW>(a, V + (int64_t)j * MR, tj, q0, lane);
  }
  // R (n x n upper triangular) from the registers
  T *R = static_cast<T *>(it.R);
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + REG_WARPS * q;
    if (c >= n) continue;
#pragma unroll
    for (int i = 0; i < REG_ROWS; ++i) {
      const int r = lane + 32 * i;
      if (r < n) R[(int64_t)c * it.ldr + r] = (r <= c) ? a[q][i] : T(0);
    }
  }
  // Explicit Q = H_0 H_1 ... H_{n-1} [I; 0], accumulated backwards: every
  // warp applies H_{n-1}, ..., H_0 to its own columns of [I; 0] in registers.
  // Column c is untouched by H_j for j > c (rows above j are zero in v_j, and
  // column c of the partial product is e_c there), so H_j acts on c >= j only.
#pragma unroll
  for (int q = 0; q < CPW; ++q)
#pragma unroll
    for (int i = 0; i < REG_ROWS; ++i) a[q][i] = (lane + 32 * i == warp + REG_WARPS * q) ? T(1) : T(0);
  for (int j = n - 1; j >= 0; --j) {
    const T tj = tau[j];
    const int q0 = (j - warp + REG_WARPS - 1) / REG_WARPS;  // first owned column >= j (j - warp + 15 >= 0)
    if (tj != T(0) && q0 < CPW) qr_apply_reflector<T, CPW>(a, V + (int64_t)j * MR, tj, q0, lane);
  }
  T *Q = static_cast<T *>(it.Q);
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + REG_WARPS * q;
    if (c >= n) continue;
#pragma unroll
    for (int i = 0; i < REG_ROWS; ++i) {
      const int r = lane + 32 * i;
      if (r < m) Q[(int64_t)c * it.ldq + r] = a[q][i];
    }
  }
}

template <typename T, int CPW>
cudaError_t launch_qr_reg(const QrItem *d_items, int n_items, int max_n, cudaStream_t s) {
  const size_t smem = ((size_t)(32 * REG_ROWS + 1) * max_n + max_n) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(qr_reg_kernel<T, CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_reg_kernel<T, CPW><<<n_items, REG_WARPS * 32, smem, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int qr_max_rows(int n, int elem_bytes) {
  if (n <= 16 * 4) return 32 * REG_ROWS;  // register-resident kernel
  int64_t avail = kSmemLimit - kSmemReserve - (int64_t)(n + 32) * elem_bytes;
  return (int)(avail / ((int64_t)n * elem_bytes));
}

template <typename T>
cudaError_t launch_qr(const QrItem *d_items, int n_items, int max_m, int max_n, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (max_n <= 64 && max_m <= 32 * REG_ROWS) {
    if (max_n <= 16) return launch_qr_reg<T, 1>(d_items, n_items, max_n, s);
    if (max_n <= 32) return launch_qr_reg<T, 2>(d_items, n_items, max_n, s);
    return launch_qr_reg<T, 4>(d_items, n_items, max_n, s);
  }
  size_t smem = ((size_t)max_m * max_n + max_n + 32) * sizeof(T);
  if (smem > (size_t)kSmemLimit) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(qr_block_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_block_kernel<T><<<n_items, QR_THREADS, smem, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_qr<double>(const QrItem *, int, int, int, cudaStream_t);
template cudaError_t launch_qr<float>(const QrItem *, int, int, int, cudaStream_t);

}  // namespace htgb
