// k_qr_df.cu -- Householder QR of FP64 row blocks in double-float arithmetic
// (every value an unevaluated sum h + l of two FP32 numbers, about 2^-47
// relative), for the mixed-precision path.  The same factorisation as the
// FP64 register-resident kernel of k_qr.cu (the leaf level of the TSQR behind
// the reduced QR decompositions of Sec. 3.4: leaf frames U = Q R and
// M_{2,3}(B_t) = Q R_t, eq. "qrtransfer"), with the arithmetic moved from the
// FP64 pipe (about 1/62 of the FP32 rate on this GPU) to the FP32 pipe: one
// FP64 multiply-add becomes about 13 FP32 instructions.
//
// Layout: as in k_qr.cu, warp w owns columns 4w..4w+3, one per group of 8
// lanes; lane s of a group holds rows 32i + 4s + e (i < 8, e < 4) of its
// column as (h, l) pairs, the reflectors y_j live in shared memory as (h, l)
// pairs and kappa_j beside them.  One barrier per column; Q = H_0 ... H_{n-1}
// [I; 0] is accumulated backwards on the columns in registers at the end.
//
// Range: FP32 has an 8-bit exponent, so every column of the block is scaled
// by 2^-E_c, E_c its largest exponent in the block (|a| < 2^E_c), when it is
// converted to double-float.  Householder QR commutes with positive column
// scaling: Q is unchanged and column c of R is scaled back by 2^E_c when it is
// written.  Entries below 2^-126 of their column's largest are dropped, far
// below the 2^-47 resolution of the arithmetic.  Conversions in both
// directions are integer operations (no FP64 instruction per element).
//
// Arithmetic: products are exact in two FP32 terms (FMA), sums use Knuth's
// two-sum; dot products accumulate lazily (the high parts by two-sum, all
// low-order terms in one FP32 word) and are renormalised once; every updated
// entry is renormalised (Dekker's fast two-sum), so the pairs stay canonical
// through the cancellation that the reflectors cause.
#include "internal.h"
#include "dfloat.cuh"

namespace htgb {

namespace {

constexpr int kDfRows = 256;  // rows of a block (32 x 8)
constexpr int kDfNI = kDfRows / 32;

// Lazy accumulation: (sh, sl) += a b, sh by two-sum, every low-order term in sl.
__device__ __forceinline__ void df_dot_acc(float &sh, float &sl, float ah, float al, float bh, float bl) {
  float p, e, s, t;
  df_prod(ah, al, bh, bl, p, e);
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// Canonical pair of a lazy accumulator (any relative size of its parts).
__device__ __forceinline__ void df_norm(float &h, float &l) {
  float s, t;
  two_sum(h, l, s, t);
  h = s;
  l = t;
}

// a <- a - d y (one entry), renormalised.
__device__ __forceinline__ void df_axpy_neg(float &ah, float &al, float dh, float dl, float yh, float yl) {
  float p, e, s, t;
  df_prod(dh, dl, yh, yl, p, e);
  two_sum(ah, -p, s, t);
  t = __fadd_rn(t, __fsub_rn(al, e));
  fast_two_sum(s, t, ah, al);
}

// sqrt(x) for x > 0: the FP32 root and one correction term.
__device__ __forceinline__ void df_sqrt(float xh, float xl, float &h, float &l) {
  const float r = __fsqrt_rn(xh);
  const float d = __fadd_rn(__fmaf_rn(-r, r, xh), xl);  // x - r^2
  fast_two_sum(r, __fmul_rn(d, __frcp_rn(__fmul_rn(2.0f, r))), h, l);
}

// 1 / b: the FP32 reciprocal and one Newton correction.
__device__ __forceinline__ void df_rcp(float bh, float bl, float &h, float &l) {
  const float r = __frcp_rn(bh);
  const float e = __fmaf_rn(-bl, r, __fmaf_rn(-bh, r, 1.0f));  // 1 - b r
  fast_two_sum(r, __fmul_rn(r, e), h, l);
}

__device__ __forceinline__ uint32_t abs_hi32(double x) {
  return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
}

// Sum of a pair over the 8 lanes of a group (lanes 8g .. 8g+7).
__device__ __forceinline__ void df_group_sum(float &h, float &l) {
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol, h, l);
  }
}

// Four lazy accumulators of a lane to one canonical pair.
__device__ __forceinline__ void df_sum4(float (&sh)[4], float (&sl)[4], float &h, float &l) {
#pragma unroll
  for (int e = 0; e < 4; ++e) df_norm(sh[e], sl[e]);
  float ah, al, bh, bl;
  df_add(sh[0], sl[0], sh[1], sl[1], ah, al);
  df_add(sh[2], sl[2], sh[3], sl[3], bh, bl);
  df_add(ah, al, bh, bl, h, l);
}

__device__ __forceinline__ void ld4(const float2 *p, float (&xh)[4], float (&xl)[4]) {
  const float4 t0 = reinterpret_cast<const float4 *>(p)[0], t1 = reinterpret_cast<const float4 *>(p)[1];
  xh[0] = t0.x; xl[0] = t0.y; xh[1] = t0.z; xl[1] = t0.w;
  xh[2] = t1.x; xl[2] = t1.y; xh[3] = t1.z; xl[3] = t1.w;
}
__device__ __forceinline__ void st4(float2 *p, const float (&xh)[4], const float (&xl)[4]) {
  reinterpret_cast<float4 *>(p)[0] = make_float4(xh[0], xl[0], xh[1], xl[1]);
  reinterpret_cast<float4 *>(p)[1] = make_float4(xh[2], xl[2], xh[3], xl[3]);
}

// The scalars of a column's reflector from alpha (its diagonal entry) and s2
// (the squared norm below it): beta = R(j, j) = -sign(alpha) sqrt(alpha^2 + s2),
// u = alpha - beta (the reflector's entry at the diagonal; the part below is
// the column itself) and kappa = -1 / (beta u), so that H = I - kappa y y^T
// with kappa ||y||^2 = 2.  A column below 4 x the smallest normal FP32 number
// in alpha^2 + s2 (after its column scaling) keeps the identity reflector.
__device__ __forceinline__ void df_reflector_scalars(float alh, float all, float s2h, float s2l, float &kh, float &kl,
                                                     float &bh, float &bl, float &uh, float &ul) {
  float x2h, x2l, t0h, t0l;
  df_mul(alh, all, alh, all, t0h, t0l);
  df_add(t0h, t0l, s2h, s2l, x2h, x2l);
  kh = 0.0f;
  kl = 0.0f;
  bh = alh;
  bl = all;
  uh = 0.0f;
  ul = 0.0f;
  if (s2h != 0.0f && x2h >= 4.0f * 1.17549435e-38f) {
    float nh, nl;
    df_sqrt(x2h, x2l, nh, nl);
    if (alh <= 0.0f) {
      bh = nh;
      bl = nl;
    } else {
      bh = -nh;
      bl = -nl;
    }
    df_add(alh, all, -bh, -bl, uh, ul);
    float ph, pl, rh, rl;
    df_mul(bh, bl, uh, ul, ph, pl);
    df_rcp(ph, pl, rh, rl);
    kh = -rh;
    kl = -rl;
  }
}

// Sum of a pair over the whole warp.
__device__ __forceinline__ void df_warp_sum(float &h, float &l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol, h, l);
  }
}

// One step of the look-ahead warp (lane l holds rows 32 i + l of one column):
// the column c (j + 1) as its owner left it in `stage` (H_0 .. H_{j-1} applied)
// takes H_j (y_j, kappa_j) unless `apply` is false (c = 0), and its reflector
// y_c, kappa_c and R(c, c) = beta_c are written (c < 32).
__device__ __forceinline__ void df_lookahead_step(const float2 *stage, const float2 *yj, float2 tj, bool apply,
                                                  float2 *yc, float2 *kappa_c, float2 *rdiag_c, int c, int lane) {
  float xh[kDfNI], xl[kDfNI];
#pragma unroll
  for (int i = 0; i < kDfNI; ++i) {
    const float2 v = stage[32 * i + lane];
    xh[i] = v.x;
    xl[i] = v.y;
  }
  if (apply) {
    float d0h = 0.f, d0l = 0.f, d1h = 0.f, d1l = 0.f;
#pragma unroll
    for (int i = 0; i < kDfNI; i += 2) {
      const float2 y0 = yj[32 * i + lane], y1 = yj[32 * (i + 1) + lane];
      df_dot_acc(d0h, d0l, y0.x, y0.y, xh[i], xl[i]);
      df_dot_acc(d1h, d1l, y1.x, y1.y, xh[i + 1], xl[i + 1]);
    }
    df_norm(d0h, d0l);
    df_norm(d1h, d1l);
    float dh, dl;
    df_add(d0h, d0l, d1h, d1l, dh, dl);
    df_warp_sum(dh, dl);
    float ch, cl;
    df_mul(tj.x, tj.y, dh, dl, ch, cl);
#pragma unroll
    for (int i = 0; i < kDfNI; ++i) {
      const float2 y = yj[32 * i + lane];
      df_axpy_neg(xh[i], xl[i], ch, cl, y.x, y.y);
    }
  }
  float q0h = 0.f, q0l = 0.f, q1h = 0.f, q1l = 0.f;
#pragma unroll
  for (int i = 0; i < kDfNI; i += 2) {
    const bool b0 = 32 * i + lane > c, b1 = 32 * (i + 1) + lane > c;
    const float h0 = b0 ? xh[i] : 0.f, l0 = b0 ? xl[i] : 0.f;
    const float h1 = b1 ? xh[i + 1] : 0.f, l1 = b1 ? xl[i + 1] : 0.f;
    df_dot_acc(q0h, q0l, h0, l0, h0, l0);
    df_dot_acc(q1h, q1l, h1, l1, h1, l1);
  }
  df_norm(q0h, q0l);
  df_norm(q1h, q1l);
  float s2h, s2l;
  df_add(q0h, q0l, q1h, q1l, s2h, s2l);
  df_warp_sum(s2h, s2l);
  const float alh = __shfl_sync(0xffffffffu, xh[0], c), all = __shfl_sync(0xffffffffu, xl[0], c);
  float kh, kl, bh, bl, uh, ul;
  df_reflector_scalars(alh, all, s2h, s2l, kh, kl, bh, bl, uh, ul);
#pragma unroll
  for (int i = 0; i < kDfNI; ++i) {
    const int r = 32 * i + lane;
    yc[r] = r > c ? make_float2(xh[i], xl[i]) : (r == c ? make_float2(uh, ul) : make_float2(0.f, 0.f));
  }
  if (lane == 0) {
    *kappa_c = make_float2(kh, kl);
    *rdiag_c = make_float2(bh, bl);
  }
}

// a <- a - kappa (y^T a) y for the lane's column; upd = false leaves a
// unchanged (the group reduction needs every lane).
__device__ __forceinline__ void df_apply_reflector(float (&ah)[kDfNI][4], float (&al)[kDfNI][4], const float2 *vj,
                                                   float2 tj, bool upd, int s) {
  float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kDfNI; ++i) {
    float yh[4], yl[4];
    ld4(vj + 32 * i + 4 * s, yh, yl);
#pragma unroll
    for (int e = 0; e < 4; ++e) df_dot_acc(dh[e], dl[e], yh[e], yl[e], ah[i][e], al[i][e]);
    asm volatile("" ::: "memory");  // one chunk of y in registers at a time
  }
  float sh, sl;
  df_sum4(dh, dl, sh, sl);
  df_group_sum(sh, sl);
  float ch = 0.0f, cl = 0.0f;
  if (upd) df_mul(tj.x, tj.y, sh, sl, ch, cl);
  // read y again rather than keep 64 registers of it live across the passes
  asm volatile("" ::: "memory");
#pragma unroll
  for (int i = 0; i < kDfNI; ++i) {
    float yh[4], yl[4];
    ld4(vj + 32 * i + 4 * s, yh, yl);
#pragma unroll
    for (int e = 0; e < 4; ++e) df_axpy_neg(ah[i][e], al[i][e], ch, cl, yh[e], yl[e]);
    asm volatile("" ::: "memory");
  }
}

// NW warps hold the block's columns (four each); warp NW is the look-ahead
// warp: while the others apply H_j to their columns it brings column j + 1 up
// to date and forms its reflector, so that the barrier of step j + 1 waits
// for the longest update rather than for an update followed by a reflector.
// The owner of column j + 2 leaves it in a staging buffer (two, alternating)
// after applying H_j.  R's diagonal comes from the look-ahead warp.
template <int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) qr_df_kernel(const QrItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QrItem it = items[blockIdx.x];
  const int m = it.m, n = it.n;
  // 16-byte vector accesses go to V and stage only; both start at multiples of
  // 2 KB (kDfRows pairs), tau and rdiag (8-byte accesses) come after them
  float2 *V = reinterpret_cast<float2 *>(smem_raw);  // kDfRows x n: y_j in column j
  float2 *stage = V + (int64_t)kDfRows * n;          // 2 x kDfRows: the next column, alternating
  float2 *tau = stage + 2 * kDfRows;                 // n: kappa_j
  float2 *rdiag = tau + n;                           // n: R(j, j)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool look = warp == NW;
  const int g = lane >> 3, s = lane & 7;
  const int c = 4 * warp + g;  // this lane's column (regular warps)
  float ah[kDfNI][4], al[kDfNI][4];
  int Ec = 0;
  if (!look) {
    const double *A = static_cast<const double *>(it.A) + (int64_t)c * it.lda;
    // the column's largest exponent in the block (integer compares of the high words)
    uint32_t mh = 0u;
#pragma unroll
    for (int i = 0; i < kDfNI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        if (c < n && r < m) mh = max(mh, abs_hi32(A[r]));
      }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) mh = max(mh, __shfl_xor_sync(0xffffffffu, mh, o));
    const bool bad = mh >= 0x7FF00000u;  // Inf or NaN in the column: NaN throughout
    Ec = (mh >> 20) ? (int)(mh >> 20) - 1022 : 0;
#pragma unroll
    for (int i = 0; i < kDfNI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        df_from_f64((c < n && r < m) ? A[r] : 0.0, Ec, ah[i][e], al[i][e]);
        if (bad) ah[i][e] = __uint_as_float(0x7FC00000u);
      }
    if (c < 2 && c < n)  // columns 0 and 1 for the look-ahead warp
#pragma unroll
      for (int i = 0; i < kDfNI; ++i) st4(stage + c * kDfRows + 32 * i + 4 * s, ah[i], al[i]);
  }
  __syncthreads();
  if (look) df_lookahead_step(stage, V, make_float2(0.f, 0.f), false, V, tau, rdiag, 0, lane);
  for (int j = 0; j + 1 < n; ++j) {
    __syncthreads();  // y_j and kappa_j are in shared memory, column j + 1 is staged
    if (look) {
      df_lookahead_step(stage + ((j + 1) & 1) * kDfRows, V + (int64_t)j * kDfRows, tau[j], true,
                        V + (int64_t)(j + 1) * kDfRows, tau + j + 1, rdiag + j + 1, j + 1, lane);
    } else if (4 * warp + 3 > j) {  // some column of this warp lies right of j
      df_apply_reflector(ah, al, V + (int64_t)j * kDfRows, tau[j], c > j, s);
      if (j + 2 < n && c == j + 2)  // the owner of column j + 2 stages it
#pragma unroll
        for (int i = 0; i < kDfNI; ++i) st4(stage + ((j + 2) & 1) * kDfRows + 32 * i + 4 * s, ah[i], al[i]);
    }
  }
  __syncthreads();
  if (look) return;  // no barrier follows
  // R (n x n upper triangular), column c scaled back by 2^Ec; n <= 32 rows: chunk 0
  double *R = static_cast<double *>(it.R) + (int64_t)c * it.ldr;
  if (c < n) {
    const float2 dgc = rdiag[c];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 4 * s + e;
      if (r < n) R[r] = (r < c) ? df_to_f64(ah[0][e], al[0][e], Ec) : (r == c ? df_to_f64(dgc.x, dgc.y, Ec) : 0.0);
    }
  }
  // Q = H_0 H_1 ... H_{n-1} [I; 0], accumulated backwards on the columns of
  // [I; 0]; column c is untouched by H_j for j > c, so warp w starts at j = 4w + 3
#pragma unroll
  for (int i = 0; i < kDfNI; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ah[i][e] = (32 * i + 4 * s + e == c) ? 1.0f : 0.0f;
      al[i][e] = 0.0f;
    }
  for (int j = min(n - 1, 4 * warp + 3); j >= 0; --j)
    df_apply_reflector(ah, al, V + (int64_t)j * kDfRows, tau[j], true, s);
  double *Q = static_cast<double *>(it.Q) + (int64_t)c * it.ldq;
  if (c < n) {
#pragma unroll
    for (int i = 0; i < kDfNI; ++i)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 32 * i + 4 * s + e;
        if (r < m) Q[r] = df_to_f64(ah[i][e], al[i][e], 0);
      }
  }
}

template <int NW>
cudaError_t launch_qr_df_nw(const QrItem *d_items, int n_items, int max_n, cudaStream_t s) {
  const size_t smem = ((size_t)kDfRows * max_n + max_n + 2 * kDfRows + max_n) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(qr_df_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_df_kernel<NW><<<n_items, (NW + 1) * 32, smem, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_qr_df(const QrItem *d_items, int n_items, int max_m, int max_n, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (max_n > 32 || max_m > kDfRows) return cudaErrorInvalidValue;  // mixed-path panels are 32 columns wide
  if (max_n <= 16) return launch_qr_df_nw<4>(d_items, n_items, max_n, s);
  return launch_qr_df_nw<8>(d_items, n_items, max_n, s);
}

}  // namespace htgb
