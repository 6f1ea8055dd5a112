// k_gemm.cu -- strided batched contraction on the SIMT pipes (FP64 / FP32).
//
// All dense contractions of the truncation are expressed as GemmItem work
// items (see internal.h): the transfer-tensor mode products of Lemma
// "transfer tensor transformation" (R-apply and projection), the reduced
// Gramian contractions of eqs. "acctransferSon1/2", the leaf products U Q|_r
// and the TSQR recombination.  One launch walks all items of a tree level.
#include "internal.h"

namespace htgb {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, THREADS = 256;

__device__ __forceinline__ int eff_dim(int lit, int ref, int mult, const int *ranks) {
  if (ref < 0) return lit;
  int v = ranks[ref] * mult;
  return v < lit ? v : lit;
}

__device__ __forceinline__ int find_item(const GemmItem *items, int n, int tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(THREADS) gemm_kernel(const GemmItem *__restrict__ items, int n_items,
                                                        const int *__restrict__ ranks) {
  __shared__ __align__(16) T As[BK][BM];
  __shared__ __align__(16) T Bs[BK][BN];
  const int tile = blockIdx.x;
  const GemmItem &it = items[find_item(items, n_items, tile)];
  int local = tile - it.tile0;
  const int tm = local % it.tiles_m;
  local /= it.tiles_m;
  const int tn = local % it.tiles_n;
  local /= it.tiles_n;
  const int b = local % it.batch;
  const int chunk = local / it.batch;
  const int M = eff_dim(it.M, it.m_ref, 1, ranks);
  const int N = eff_dim(it.N, it.n_ref, it.n_mult, ranks);
  const int batch = eff_dim(it.batch, it.b_ref, it.b_mult, ranks);
  const int m0 = tm * BM, n0 = tn * BN;
  if (m0 >= M || n0 >= N || b >= batch) return;
  const int K = it.K;
  const int ko_begin = (int)((int64_t)chunk * it.Ko / it.ksplit);
  const int ko_end = (int)((int64_t)(chunk + 1) * it.Ko / it.ksplit);
  const T *A = static_cast<const T *>(it.A) + (int64_t)b * it.sab;
  const T *B = static_cast<const T *>(it.B) + (int64_t)b * it.sbb;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // thread owns rows 4tx..4tx+3, cols 4ty..4ty+3
  const bool a_mfast = (it.sam == 1);
  const bool b_nfast = (it.sbn == 1) && (it.sbk != 1);
  // FP32: each 16-wide k-tile is summed in registers, then added to the
  // running sum with Kahan compensation (compensated summation of the long
  // Gramian reductions); FP64 sums directly.
  constexpr bool kComp = sizeof(T) == 4;
  T acc[4][4], sum[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = sum[i][j] = cmp[i][j] = T(0);

  for (int ko = ko_begin; ko < ko_end; ++ko) {
    const T *Ak = A + (int64_t)ko * it.sako;
    const T *Bk = B + (int64_t)ko * it.sbko;
    for (int k0 = 0; k0 < K; k0 += BK) {
      // A tile: BM x BK elements, 4 per thread
#pragma unroll
      for (int r = 0; r < (BM * BK) / THREADS; ++r) {
        int e = tid + r * THREADS;
        int mm, kk;
        if (a_mfast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
        int gm = m0 + mm, gk = k0 + kk;
        T v = T(0);
        if (gm < M && gk < K && (it.k_total < 0 || (int64_t)ko * K + gk < it.k_total))
          v = Ak[(int64_t)gm * it.sam + (int64_t)gk * it.sak];
        As[kk][mm] = v;
      }
#pragma unroll
      for (int r = 0; r < (BN * BK) / THREADS; ++r) {
        int e = tid + r * THREADS;
        int nn, kk;
        if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
        int gn = n0 + nn, gk = k0 + kk;
        T v = T(0);
        if (gn < N && gk < K && (it.k_total < 0 || (int64_t)ko * K + gk < it.k_total))
          v = Bk[(int64_t)gk * it.sbk + (int64_t)gn * it.sbn];
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][4 * tx + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][4 * ty + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
      if (kComp) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const T y = acc[i][j] - cmp[i][j];
            const T t = sum[i][j] + y;
            cmp[i][j] = (t - sum[i][j]) - y;
            sum[i][j] = t;
            acc[i][j] = T(0);
          }
      }
      __syncthreads();
    }
  }
  if (kComp) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = sum[i][j];
  }
  if (it.ksplit > 1) {
    T *P = static_cast<T *>(it.part) + ((int64_t)chunk * it.batch + b) * (int64_t)it.M * it.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gm = m0 + 4 * tx + i, gn = n0 + 4 * ty + j;
        if (gm < M && gn < N) P[(int64_t)gn * it.M + gm] = acc[i][j];
      }
    return;
  }
  T *C = static_cast<T *>(it.C) + (int64_t)b * it.scb;
  const T alpha = T(it.alpha), beta = T(it.beta);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gm = m0 + 4 * tx + i, gn = n0 + 4 * ty + j;
      if (gm < M && gn < N) {
        T *c = C + (int64_t)gm * it.scm + (int64_t)gn * it.scn;
        T v = alpha * acc[i][j];
        if (beta != T(0)) v += beta * *c;
        *c = v;
      }
    }
}

// Sum the split-K partials of every split item in chunk order.
template <typename T>
__global__ void gemm_reduce_kernel(const GemmItem *__restrict__ items, const int *__restrict__ ranks) {
  const GemmItem &it = items[blockIdx.y];
  if (it.ksplit <= 1) return;
  const int M = eff_dim(it.M, it.m_ref, 1, ranks);
  const int N = eff_dim(it.N, it.n_ref, it.n_mult, ranks);
  const int batch = eff_dim(it.batch, it.b_ref, it.b_mult, ranks);
  const int64_t per = (int64_t)M * N;
  const int64_t total = per * batch;
  const T *P = static_cast<const T *>(it.part);
  const int64_t stride_chunk = (int64_t)it.batch * it.M * it.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int b = (int)(e / per);
    int64_t r = e - (int64_t)b * per;
    int gn = (int)(r / M), gm = (int)(r - (int64_t)gn * M);
    const T *p = P + (int64_t)b * it.M * it.N + (int64_t)gn * it.M + gm;
    double s = 0.0;  // partial sums are added in FP64
    for (int c = 0; c < it.ksplit; ++c) s += (double)p[c * stride_chunk];
    T *cp = static_cast<T *>(it.C) + (int64_t)b * it.scb + (int64_t)gm * it.scm + (int64_t)gn * it.scn;
    double v = it.alpha * s;
    if (it.beta != 0.0) v += it.beta * (double)*cp;
    *cp = T(v);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_gemm(const GemmItem *d_items, int n_items, int total_tiles, const int *d_ranks, bool any_split,
                        int tc_tiles, cudaStream_t s) {
  if (n_items <= 0 || total_tiles <= 0) return cudaSuccess;
  if (sizeof(T) == 4 && tc_tiles > 0) {
    cudaError_t e = launch_gemm_tc(d_items, n_items, tc_tiles, d_ranks, s);
    if (e != cudaSuccess) return e;
  } else {
    gemm_kernel<T><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, d_ranks);
    count_launch();
  }
  if (any_split) {
    for (int base = 0; base < n_items; base += 65535) {
      const int cnt = n_items - base < 65535 ? n_items - base : 65535;
      gemm_reduce_kernel<T><<<dim3(64, cnt), 256, 0, s>>>(d_items + base, d_ranks);
      count_launch();
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmItem *, int, int, const int *, bool, int, cudaStream_t);
template cudaError_t launch_gemm<float>(const GemmItem *, int, int, const int *, bool, int, cudaStream_t);

}  // namespace htgb
