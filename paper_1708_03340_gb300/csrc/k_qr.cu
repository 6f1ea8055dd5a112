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

}  // namespace

int qr_max_rows(int n, int elem_bytes) {
  int64_t avail = kSmemLimit - kSmemReserve - (int64_t)(n + 32) * elem_bytes;
  return (int)(avail / ((int64_t)n * elem_bytes));
}

template <typename T>
cudaError_t launch_qr(const QrItem *d_items, int n_items, int max_m, int max_n, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  size_t smem = ((size_t)max_m * max_n + max_n + 32) * sizeof(T);
  if (smem > (size_t)kSmemLimit) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(qr_block_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_block_kernel<T><<<n_items, QR_THREADS, smem, s>>>(d_items);
  return cudaGetLastError();
}

template cudaError_t launch_qr<double>(const QrItem *, int, int, int, cudaStream_t);
template cudaError_t launch_qr<float>(const QrItem *, int, int, int, cudaStream_t);

}  // namespace htgb
