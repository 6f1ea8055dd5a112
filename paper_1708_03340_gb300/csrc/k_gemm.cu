// k_gemm.cu -- strided batched contraction on the SIMT pipes (FP64 / FP32).
//
// All dense contractions of the truncation are expressed as GemmItem work
// items (see internal.h): the transfer-tensor mode products of Lemma
// "transfer tensor transformation" (R-apply and projection), the reduced
// Gramian contractions of eqs. "acctransferSon1/2", the leaf products U Q|_r
// and the TSQR recombination.  One launch walks all items of a tree level.
#include <type_traits>

#include "internal.h"

namespace htgb {

namespace {

constexpr int THREADS = 256;

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

template <typename T, int TM>
__device__ __forceinline__ void lds_vec(const T *p, T (&x)[TM]) {
  if (sizeof(T) == 4 && TM % 4 == 0) {
#pragma unroll
    for (int i = 0; i < TM; i += 4) {
      const float4 v = *reinterpret_cast<const float4 *>(p + i);
      x[i] = (T)v.x; x[i + 1] = (T)v.y; x[i + 2] = (T)v.z; x[i + 3] = (T)v.w;
    }
  } else if (sizeof(T) == 8 && TM % 2 == 0) {
#pragma unroll
    for (int i = 0; i < TM; i += 2) {
      const double2 v = *reinterpret_cast<const double2 *>(p + i);
      x[i] = (T)v.x; x[i + 1] = (T)v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < TM; ++i) x[i] = p[i];
  }
}

// Asynchronous element copy global -> shared (cp.async, 4 or 8 bytes); with
// valid == false nothing is read (src-size 0) and the destination is
// zero-filled.  src is always an aligned address inside the operand.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst_smem, const T *src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
  const int n = valid ? (int)sizeof(T) : 0;
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
// 16-byte asynchronous copy with zero-fill beyond `bytes` (0..16); src is a
// 16-byte aligned address inside the operand even when bytes == 0.
__device__ __forceinline__ void cp_async_16(void *dst_smem, const void *src, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One BM x BN tile of C per CTA, TM x TN outputs per thread, K walked in
// BK-wide tiles through NS shared-memory stages filled by cp.async: the
// copies of tile q + NS - 1 are in flight while tile q is multiplied, and
// every element lands directly at its (possibly transposed) place, zero
// outside the matrix.  A thread's TM rows are groups of 4 consecutive rows,
// 4 (BM / TM) apart, so that a warp's 16-byte shared-memory reads are
// contiguous; rows of the shared tiles are padded by 4 elements, which keeps
// those reads aligned and spreads the transposing writes of k-fast operands
// over the banks.  kComp (FP32 only): every BK-wide tile is summed in
// registers and added to the running sum with Kahan compensation
// (compensated summation of the long Gramian reductions); chosen per launch
// from the longest per-CTA reduction.  kAcc = 2 (FP32 inputs only): every
// product is carried exactly as a pair (p, e) with p = a b rounded and
// e = fma(a, b, -p), and summed into a double-float (hi, lo) with a two-sum
// (Dekker / Knuth error-free transformations), so the sum is FP64-accurate;
// the output (and any split-K partials) are FP64.
template <typename T, int BM, int BN, int TM, int TN, int BK, int kAcc>
__global__ void __launch_bounds__(THREADS, sizeof(T) != 4 ? 1
                                           : (BM * BN <= 64 * 64 ? (kAcc == 0 ? 3 : 2) : (BM * BN <= 128 * 64 && kAcc == 0 ? 2 : 1)))
    gemm_kernel(const GemmItem *__restrict__ items, int n_items, int uniform,
                                                        const int *__restrict__ ranks) {
  constexpr bool kComp = (kAcc == 1);
  constexpr bool kDF = (kAcc == 2) && sizeof(T) == 4;  // double-float accumulation, FP64 output
  using OutT = typename std::conditional<kDF, double, T>::type;
  static_assert((BM / TM) * (BN / TN) == THREADS, "one output block per thread");
  static_assert(TM % 4 == 0 && TN % 4 == 0, "rows and columns in groups of 4");
  constexpr int LA = (BM * BK) / THREADS, LB = (BN * BK) / THREADS;
  constexpr int PAD = 4, NS = 3;
  __shared__ __align__(16) T As[NS][BK][BM + PAD];
  __shared__ __align__(16) T Bs[NS][BK][BN + PAD];
  const int tile = blockIdx.x;
  // all items of most launches have the same tile count: no search then
  const GemmItem &it = items[uniform > 0 ? tile / uniform : find_item(items, n_items, tile)];
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
  const int kt = (K + BK - 1) / BK;                 // BK-tiles per outer chunk
  const int nq = (ko_end - ko_begin) * kt;          // BK-tiles of this CTA
  const T *A = static_cast<const T *>(it.A) + (int64_t)b * it.sab;
  const T *B = static_cast<const T *>(it.B) + (int64_t)b * it.sbb;
  const int tid = threadIdx.x;
  const int tx = tid % (BM / TM), ty = tid / (BM / TM);
  // row of output i: group i/4 of 4 rows, groups 4 (BM / TM) apart; columns likewise
  auto row_of = [&](int i) { return (i >> 2) * (4 * (BM / TM)) + 4 * tx + (i & 3); };
  auto col_of = [&](int j) { return (j >> 2) * (4 * (BN / TN)) + 4 * ty + (j & 3); };
  const bool a_mfast = (it.sam == 1);
  const bool b_nfast = (it.sbn == 1) && (it.sbk != 1);
  // FP32 operands whose fast dimension is the tile's (A along m, B along n)
  // and whose every 4-element chunk starts 16-byte aligned are copied 16 bytes
  // at a time (chunks cut by M or N are zero-filled past the edge)
  constexpr int LAV = (BM * BK) / (4 * THREADS), LBV = (BN * BK) / (4 * THREADS);
  const bool vecA = sizeof(T) == 4 && LAV >= 1 && a_mfast && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
                    (it.sak & 3) == 0 && (it.sako & 3) == 0;
  const bool vecB = sizeof(T) == 4 && LBV >= 1 && b_nfast && (reinterpret_cast<uintptr_t>(B) & 15) == 0 &&
                    (it.sbk & 3) == 0 && (it.sbko & 3) == 0;

  // Per copied element of this thread: its place in the tile and its global
  // offset without the k tile (fixed for the CTA); a tile adds k0 and ko.
  int offa[LA], offb[LB];  // 32-bit: the plan keeps every tile offset below 2^31 elements
  unsigned vmask = 0;  // bit r: row of A element r inside M; bit LA + r: column of B element r inside N
  if (vecA) {  // chunk r: rows m0 + 4 (e % (BM/4)) .. +3 of tile row e / (BM/4)
#pragma unroll
    for (int r = 0; r < LAV; ++r) {
      const int e = tid + r * THREADS;
      const int gm = m0 + 4 * (e % (BM / 4)), kk = e / (BM / 4);
      offa[r] = (gm < M) ? (int)(gm + (int64_t)kk * it.sak) : 0;
    }
  } else {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      const int e = tid + r * THREADS;
      int mm, kk;
      if (a_mfast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int gm = m0 + mm;
      offa[r] = (gm < M) ? (int)((int64_t)gm * it.sam + (int64_t)kk * it.sak) : 0;
      if (gm < M) vmask |= 1u << r;
    }
  }
  if (vecB) {  // chunk r: columns n0 + 4 (e % (BN/4)) .. +3 of tile row e / (BN/4)
#pragma unroll
    for (int r = 0; r < LBV; ++r) {
      const int e = tid + r * THREADS;
      const int gn = n0 + 4 * (e % (BN / 4)), kk = e / (BN / 4);
      offb[r] = (gn < N) ? (int)((int64_t)kk * it.sbk + gn) : 0;
    }
  } else {
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      const int e = tid + r * THREADS;
      int nn, kk;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int gn = n0 + nn;
      offb[r] = (gn < N) ? (int)((int64_t)kk * it.sbk + (int64_t)gn * it.sbn) : 0;
      if (gn < N) vmask |= 1u << (LA + r);
    }
  }
  // issue the copies of BK-tile q into stage st (one commit group per call)
  auto issue = [&](int q, int st) {
    if (q < nq) {
      const int ko = ko_begin + q / kt, k0 = (q % kt) * BK;
      const T *Ak = A + (int64_t)ko * it.sako + (int64_t)k0 * it.sak;
      const T *Bk = B + (int64_t)ko * it.sbko + (int64_t)k0 * it.sbk;
      // k limit of this tile: K, or the flat cut of a ragged last chunk
      int klim = K - k0;
      if (it.k_total >= 0) {
        const int64_t rest = it.k_total - ((int64_t)ko * K + k0);
        if (rest < klim) klim = (int)(rest > 0 ? rest : 0);
      }
      if (vecA) {
#pragma unroll
        for (int r = 0; r < LAV; ++r) {
          const int e = tid + r * THREADS;
          const int mm = 4 * (e % (BM / 4)), kk = e / (BM / 4);
          const int rows = M - (m0 + mm);
          const int bytes = (kk < klim) ? 4 * (rows < 0 ? 0 : (rows > 4 ? 4 : rows)) : 0;
          cp_async_16(&As[st][kk][mm], Ak + (bytes ? offa[r] : 0), bytes);
        }
      } else {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
          const int e = tid + r * THREADS;
          int mm, kk;
          if (a_mfast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
          const bool v = ((vmask >> r) & 1u) && kk < klim;
          cp_async_elem<T>(&As[st][kk][mm], Ak + (v ? offa[r] : 0), v);
        }
      }
      if (vecB) {
#pragma unroll
        for (int r = 0; r < LBV; ++r) {
          const int e = tid + r * THREADS;
          const int nn = 4 * (e % (BN / 4)), kk = e / (BN / 4);
          const int cols = N - (n0 + nn);
          const int bytes = (kk < klim) ? 4 * (cols < 0 ? 0 : (cols > 4 ? 4 : cols)) : 0;
          cp_async_16(&Bs[st][kk][nn], Bk + (bytes ? offb[r] : 0), bytes);
        }
      } else {
#pragma unroll
        for (int r = 0; r < LB; ++r) {
          const int e = tid + r * THREADS;
          int nn, kk;
          if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
          const bool v = ((vmask >> (LA + r)) & 1u) && kk < klim;
          cp_async_elem<T>(&Bs[st][kk][nn], Bk + (v ? offb[r] : 0), v);
        }
      }
    }
    cp_async_commit();
  };

  T acc[TM][TN], sum[(kComp || kDF) ? TM : 1][(kComp || kDF) ? TN : 1], cmp[(kComp || kDF) ? TM : 1][(kComp || kDF) ? TN : 1];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  if (kComp || kDF) {
#pragma unroll
    for (int i = 0; i < ((kComp || kDF) ? TM : 1); ++i)
#pragma unroll
      for (int j = 0; j < ((kComp || kDF) ? TN : 1); ++j) sum[i][j] = cmp[i][j] = T(0);
  }
#pragma unroll
  for (int st = 0; st < NS - 1; ++st) issue(st, st);
  for (int q = 0; q < nq; ++q) {
    const int buf = q % NS;
    cp_async_wait<NS - 2>();  // this thread's copies of tile q have landed
    __syncthreads();          // everybody's have; and stage (q - 1) % NS is no longer read
    issue(q + NS - 1, (q + NS - 1) % NS);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int g = 0; g < TM / 4; ++g) {
        T x[4];
        lds_vec<T, 4>(&As[buf][kk][g * 4 * (BM / TM) + 4 * tx], x);
#pragma unroll
        for (int u = 0; u < 4; ++u) a[4 * g + u] = x[u];
      }
#pragma unroll
      for (int g = 0; g < TN / 4; ++g) {
        T x[4];
        lds_vec<T, 4>(&Bs[buf][kk][g * 4 * (BN / TN) + 4 * ty], x);
#pragma unroll
        for (int u = 0; u < 4; ++u) bb[4 * g + u] = x[u];
      }
      if (kDF) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const int ii = kDF ? i : 0, jj = kDF ? j : 0;
            // the _rn intrinsics keep every rounding in place (no contraction into FMAs)
            const float pr = __fmul_rn((float)a[i], (float)bb[j]);
            const float er = __fmaf_rn((float)a[i], (float)bb[j], -pr);  // a b = pr + er exactly
            const float hi = (float)sum[ii][jj];
            const float t = __fadd_rn(hi, pr);
            const float bp = __fsub_rn(t, hi);
            const float e2 = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(pr, bp));  // hi + pr = t + e2
            sum[ii][jj] = (T)t;
            cmp[ii][jj] = (T)__fadd_rn((float)cmp[ii][jj], __fadd_rn(e2, er));
          }
      } else {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
    }
    if (kComp) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const T y = acc[i][j] - cmp[kComp ? i : 0][kComp ? j : 0];
          const T t = sum[kComp ? i : 0][kComp ? j : 0] + y;
          cmp[kComp ? i : 0][kComp ? j : 0] = (t - sum[kComp ? i : 0][kComp ? j : 0]) - y;
          sum[kComp ? i : 0][kComp ? j : 0] = t;
          acc[i][j] = T(0);
        }
    }
  }
  cp_async_wait<0>();  // no copy may be left in flight when the CTA exits
  if (kComp) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = sum[kComp ? i : 0][kComp ? j : 0];
  }
  auto result = [&](int i, int j) -> OutT {
    if (kDF) {
      const int ii = kDF ? i : 0, jj = kDF ? j : 0;
      return (OutT)((double)sum[ii][jj] + (double)cmp[ii][jj]);
    }
    return (OutT)acc[i][j];
  };
  // A thread's rows come in groups of 4 consecutive rows: where the output is
  // FP32 with unit row stride, a group is one 16-byte store if aligned and
  // inside M.
  if (it.ksplit > 1) {
    OutT *P = static_cast<OutT *>(it.part) + ((int64_t)chunk * it.batch + b) * (int64_t)it.M * it.N;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + col_of(j);
      if (gn >= N) continue;
#pragma unroll
      for (int gi = 0; gi < TM / 4; ++gi) {
        const int gm0 = m0 + row_of(4 * gi);
        OutT *pp = P + (int64_t)gn * it.M + gm0;
        if (sizeof(OutT) == 4 && gm0 + 3 < M && (reinterpret_cast<uintptr_t>(pp) & 15) == 0) {
          *reinterpret_cast<float4 *>(pp) = make_float4((float)result(4 * gi, j), (float)result(4 * gi + 1, j),
                                                        (float)result(4 * gi + 2, j), (float)result(4 * gi + 3, j));
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (gm0 + u < M) pp[u] = result(4 * gi + u, j);
        }
      }
    }
    return;
  }
  OutT *C = static_cast<OutT *>(it.C) + (int64_t)b * it.scb;
  const OutT alpha = OutT(it.alpha), beta = OutT(it.beta);
  const bool vec = sizeof(OutT) == 4 && it.scm == 1 && beta == OutT(0);
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int gn = n0 + col_of(j);
    if (gn >= N) continue;
#pragma unroll
    for (int gi = 0; gi < TM / 4; ++gi) {
      const int gm0 = m0 + row_of(4 * gi);
      OutT *cp = C + (int64_t)gm0 * it.scm + (int64_t)gn * it.scn;
      if (vec && gm0 + 3 < M && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
        *reinterpret_cast<float4 *>(cp) =
            make_float4((float)(alpha * result(4 * gi, j)), (float)(alpha * result(4 * gi + 1, j)),
                        (float)(alpha * result(4 * gi + 2, j)), (float)(alpha * result(4 * gi + 3, j)));
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (gm0 + u < M) {
            OutT *c = cp + (int64_t)u * it.scm;
            OutT v = alpha * result(4 * gi + u, j);
            if (beta != OutT(0)) v += beta * *c;
            *c = v;
          }
        }
      }
    }
  }
}

// Sum the split-K partials of every split item in chunk order.
template <typename T>
__global__ void gemm_reduce_kernel(const GemmItem *__restrict__ items, const int *__restrict__ ranks) {
  const GemmItem &it = items[blockIdx.y];
  if (it.ksplit <= 1 || (it.oz_pre & 2)) return;  // slicing-only items have no partial sums
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
                        int tc_tiles, cudaStream_t s, int variant, bool comp, bool df, int uniform) {
  if (n_items <= 0 || total_tiles <= 0) return cudaSuccess;
  (void)tc_tiles;
  {
    // Kahan compensation only for FP32 launches with long per-CTA reductions;
    // double-float accumulation (FP64 output) when asked for
    const bool c = (sizeof(T) == 4) && comp;
    if (sizeof(T) == 4 && df) {
      gemm_kernel<T, 64, 64, 4, 4, 16, 2><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, uniform, d_ranks);
    } else if (variant == 2 && !c) {
      gemm_kernel<T, 128, 128, 8, 8, 16, 0><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, uniform, d_ranks);
    } else if (variant >= 1) {
      if (c) gemm_kernel<T, 128, 64, 8, 4, 16, 1><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, uniform, d_ranks);
      else gemm_kernel<T, 128, 64, 8, 4, 16, 0><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, uniform, d_ranks);
    } else {
      if (c) gemm_kernel<T, 64, 64, 4, 4, 16, 1><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, uniform, d_ranks);
      else gemm_kernel<T, 64, 64, 4, 4, 16, 0><<<total_tiles, THREADS, 0, s>>>(d_items, n_items, uniform, d_ranks);
    }
    count_launch();
  }
  if (any_split) {
    for (int base = 0; base < n_items; base += 65535) {
      const int cnt = n_items - base < 65535 ? n_items - base : 65535;
      if (sizeof(T) == 4 && df)
        gemm_reduce_kernel<double><<<dim3(64, cnt), 256, 0, s>>>(d_items + base, d_ranks);
      else
        gemm_reduce_kernel<T><<<dim3(64, cnt), 256, 0, s>>>(d_items + base, d_ranks);
      count_launch();
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmItem *, int, int, const int *, bool, int, cudaStream_t, int, bool,
                                         bool, int);
template cudaError_t launch_gemm<float>(const GemmItem *, int, int, const int *, bool, int, cudaStream_t, int, bool,
                                       bool, int);

cudaError_t launch_gemm_reduce_f64(const GemmItem *d_items, int n_items, const int *d_ranks, cudaStream_t s) {
  for (int base = 0; base < n_items; base += 65535) {
    const int cnt = n_items - base < 65535 ? n_items - base : 65535;
    gemm_reduce_kernel<double><<<dim3(64, cnt), 256, 0, s>>>(d_items + base, d_ranks);
    count_launch();
  }
  return cudaGetLastError();
}

void gemm_tile_shape(int variant, int *bm, int *bn) {
  *bm = (variant >= 1) ? 128 : 64;
  *bn = (variant == 2) ? 128 : 64;
}

}  // namespace htgb
