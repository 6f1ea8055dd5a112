// k_qr_df.cu -- Householder QR of FP64 row blocks in double-float arithmetic
// (every value an unevaluated sum h + l of two FP32 numbers, about 2^-47
// relative), for the mixed-precision path.  The same factorisation as the
// FP64 register-resident kernel of k_qr.cu (the leaf level of the TSQR behind
// the reduced QR decompositions of Sec. 3.4: leaf frames U = Q R and
// M_{2,3}(B_t) = Q R_t, eq. "qrtransfer"), with the arithmetic moved from the
// FP64 pipe (about 1/64 of the FP32 rate on this GPU) to the FP32 pipe: one
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

// (p, e) with p + e = (ah + al)(bh + bl) up to the al bl term and the
// rounding of e (both below 2^-48 of the product).
__device__ __forceinline__ void df_prod(float ah, float al, float bh, float bl, float &p, float &e) {
  p = __fmul_rn(ah, bh);
  e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
}

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

// (h, l) = a + b for canonical pairs.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &h, float &l) {
  float s, t;
  two_sum(ah, bh, s, t);
  t = __fadd_rn(t, __fadd_rn(al, bl));
  fast_two_sum(s, t, h, l);
}

// (h, l) = a b.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &h, float &l) {
  float p, e;
  df_prod(ah, al, bh, bl, p, e);
  fast_two_sum(p, e, h, l);
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

// x 2^-E as a pair (|x| < 2^E): h = x's sign, scaled exponent and top 23
// fraction bits; l = the next 23 fraction bits at their place.  Zero, FP64
// subnormals and results below 2^-126 give zero (l alone below 2^-126 is
// dropped).
__device__ __forceinline__ void df_from_f64(double x, int E, float &h, float &l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int fe = ex - 1023 - E + 127;  // biased FP32 exponent of x 2^-E
  h = 0.0f;
  l = 0.0f;
  if (ex == 0 || fe < 1) return;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  h = __uint_as_float(sign | ((uint32_t)fe << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
  const uint32_t k = (uint32_t)(b >> 6) & 0x7FFFFFu;  // fraction bits 28 .. 6
  if (k != 0u && fe > 46) {
    // k exactly as a float (1.5 2^23 trick without the half), times 2^(fe - 127 - 46)
    const float kf = __fsub_rn(__uint_as_float(0x4B000000u | k), 8388608.0f);
    l = __uint_as_float(__float_as_uint(__fmul_rn(kf, __uint_as_float((uint32_t)(fe - 46) << 23))) | sign);
  }
}

__device__ __forceinline__ double df_to_f64(float h, float l, int E) {
  return __longlong_as_double((long long)df_to_f64_bits(h, l, E));
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

// Row j (< 32) of the lane's column, broadcast to its group.
__device__ __forceinline__ void df_row_value(const float (&ah)[kDfNI][4], const float (&al)[kDfNI][4], int j, int lane,
                                             float &h, float &l) {
  const int e = j & 3;
  const float yh0 = (e & 1) ? ah[0][1] : ah[0][0], yh1 = (e & 1) ? ah[0][3] : ah[0][2];
  const float yl0 = (e & 1) ? al[0][1] : al[0][0], yl1 = (e & 1) ? al[0][3] : al[0][2];
  const int src = (lane & ~7) | (j >> 2);
  h = __shfl_sync(0xffffffffu, (e & 2) ? yh1 : yh0, src);
  l = __shfl_sync(0xffffffffu, (e & 2) ? yl1 : yl0, src);
}

// Column j's reflector (j < 32), formed by the warp that owns column j (each
// group for its own column; group `me` holds column j and stores):
// alpha the diagonal entry, w the part below it, beta = R(j, j) = -sign(alpha)
// sqrt(alpha^2 + ||w||^2), u = alpha - beta, y = [0; u; w], kappa = -1 / (beta u).
// A column below 4 x the smallest normal FP32 number in alpha^2 + ||w||^2 (after
// its column scaling) keeps the identity reflector.
__device__ __forceinline__ void df_form_reflector(float (&ah)[kDfNI][4], float (&al)[kDfNI][4], float2 *yj,
                                                  float2 *kappa_j, int j, int lane, bool me) {
  const int s = lane & 7;
  float qh[4] = {0.f, 0.f, 0.f, 0.f}, ql[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kDfNI; ++i) {
    float xh[4], xl[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool below = 32 * i + 4 * s + e > j;
      xh[e] = below ? ah[i][e] : 0.0f;
      xl[e] = below ? al[i][e] : 0.0f;
      df_dot_acc(qh[e], ql[e], xh[e], xl[e], xh[e], xl[e]);
    }
    if (me) st4(yj + 32 * i + 4 * s, xh, xl);
  }
  float s2h, s2l;
  df_sum4(qh, ql, s2h, s2l);
  df_group_sum(s2h, s2l);
  float alh, all;
  df_row_value(ah, al, j, lane, alh, all);
  float x2h, x2l, t0h, t0l;
  df_mul(alh, all, alh, all, t0h, t0l);
  df_add(t0h, t0l, s2h, s2l, x2h, x2l);
  float kh = 0.0f, kl = 0.0f, bh = alh, bl = all, uh = 0.0f, ul = 0.0f;
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
  if (!me) return;
  if ((j >> 2) == s) {  // row j of chunk 0 lies in this lane
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e == (j & 3)) {
        yj[j] = make_float2(uh, ul);
        ah[0][e] = bh;
        al[0][e] = bl;
      }
  }
  if (s == 0) *kappa_j = make_float2(kh, kl);
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

template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 2 : 4) qr_df_kernel(const QrItem *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QrItem it = items[blockIdx.x];
  const int m = it.m, n = it.n;
  float2 *V = reinterpret_cast<float2 *>(smem_raw);  // kDfRows x n: y_j in column j
  float2 *tau = V + (int64_t)kDfRows * n;            // n: kappa_j
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 3, s = lane & 7;
  const int c = 4 * warp + g;  // this lane's column
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
  const int Ec = (mh >> 20) ? (int)(mh >> 20) - 1022 : 0;
  float ah[kDfNI][4], al[kDfNI][4];
#pragma unroll
  for (int i = 0; i < kDfNI; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 32 * i + 4 * s + e;
      df_from_f64((c < n && r < m) ? A[r] : 0.0, Ec, ah[i][e], al[i][e]);
      if (bad) ah[i][e] = __uint_as_float(0x7FC00000u);
    }
  if (warp == 0) df_form_reflector(ah, al, V, tau, 0, lane, g == 0);
  for (int j = 0; j + 1 < n; ++j) {
    __syncthreads();                  // y_j and kappa_j are in shared memory
    if (4 * warp + 3 <= j) continue;  // no column of this warp lies right of j
    df_apply_reflector(ah, al, V + (int64_t)j * kDfRows, tau[j], c > j, s);
    if (warp == ((j + 1) >> 2))       // the owner of column j+1 forms its reflector
      df_form_reflector(ah, al, V + (int64_t)(j + 1) * kDfRows, tau + j + 1, j + 1, lane, g == ((j + 1) & 3));
  }
  __syncthreads();
  // R (n x n upper triangular), column c scaled back by 2^Ec; n <= 32 rows: chunk 0
  double *R = static_cast<double *>(it.R) + (int64_t)c * it.ldr;
  if (c < n) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 4 * s + e;
      if (r < n) R[r] = (r <= c) ? df_to_f64(ah[0][e], al[0][e], Ec) : 0.0;
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
  const size_t smem = ((size_t)kDfRows * max_n + max_n) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(qr_df_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  qr_df_kernel<NW><<<n_items, NW * 32, smem, s>>>(d_items);
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
