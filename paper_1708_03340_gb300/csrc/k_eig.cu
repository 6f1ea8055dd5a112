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
// The eigenvector matrix lives in shared memory, or, for launches with more
// matrices than SMs, in the L2-resident scratch so that four CTAs share an SM
// and overlap their recurrences.  On the mixed path (df_rot) the rotations are
// applied to the eigenvectors in double-float on the FP32 pipe; the recurrence
// itself, which decides the eigenvalues, stays in FP64.
//
// refine_df_kernel: one step of the Ogita-Aishima iterative refinement
// (Ogita & Aishima, "Iterative refinement for symmetric eigenvalue
// decomposition", Japan J. Indust. Appl. Math. 35, 2018), written from its
// first-order conditions: with X the current eigenvectors, R = I - X^T X,
// S = X^T G X, lambda_i = S_ii / (1 - R_ii) and E solving
// E + E^T = R, (S + E^T S + S E) diagonal to first order:
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   if |lambda_i - lambda_j| > delta
//   E_ij = R_ij / 2                                           otherwise (cluster)
// X <- X (I + E).  Used after an FP32 QL solve, with its dense products in
// double-float on the FP32 pipes (see the kernel).
#include "internal.h"
#include "dfloat.cuh"

namespace htgb {

// Device status word of the eigensolvers: bit 0 is set when a QL sweep gave
// up on an eigenvalue after its iteration limit (the result is then not an
// eigendecomposition to working accuracy).  Read and cleared by eig_take_status.
__device__ unsigned g_eig_status = 0;


namespace {

constexpr int EIG_THREADS = 256;
constexpr int REFINE_THREADS = 512;  // one thread per 4 x 2 outputs of a 64 x 64 product
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

// Leading dimension of a k x k eigenvector array in shared memory: k rounded
// up to 32, plus 4, so that the 4 lanes of a quad reading consecutive rows of
// 8 different columns hit 32 different banks.
__host__ __device__ __forceinline__ int ql_ld(int k) { return ((k + 31) / 32) * 32 + 4; }

// y[i] = alpha * sum_{l < L} Z[(o + i) ld + o + l] x[l] for i < L: column i of
// the trailing block at (o, o) read down its rows, 4 lanes per output (lane
// q takes l = q, q + 4, ...) and a 2-shuffle quad sum.  All threads call it.
template <typename T>
__device__ __forceinline__ void quad_colvec(const T *Z, int ld, int o, int L, const T *x, T *y, T alpha) {
  const int q = threadIdx.x & 3;
  for (int i0 = 0; i0 < L; i0 += (int)(blockDim.x >> 2)) {
    const int i = i0 + (int)(threadIdx.x >> 2);
    T acc = T(0);
    if (i < L) {
      const T *col = Z + (int64_t)(o + i) * ld + o;
      for (int l = q; l < L; l += 4) acc += col[l] * x[l];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (q == 0 && i < L) y[i] = alpha * acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(EIG_THREADS, 4) eig_ql_kernel(const EigItem *__restrict__ items, void *scratch,
                                                             int64_t scratch_stride, int z_in_smem, int df_rot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int ld = ql_ld(k);
  // layout: [32 doubles][Z: k x ld T, when the launch's largest k fits][8k + 32 T][k ints];
  // the FP64 scratch comes first so that it stays 8-byte aligned for any k.
  // z_in_smem is decided per launch (from its largest k), since the dynamic
  // shared memory is sized for the launch, not for the item.
  double *redd = reinterpret_cast<double *>(smem_raw);
  T *Z;
  T *tail;
  if (z_in_smem) {
    Z = reinterpret_cast<T *>(redd + 32);
    tail = Z + (int64_t)k * ld;
  } else {
    Z = static_cast<T *>(scratch) + (int64_t)blockIdx.x * scratch_stride;
    tail = reinterpret_cast<T *>(redd + 32);
  }
  T *dg = tail;    // diagonal of the tridiagonal matrix, then eigenvalues
  T *eo = dg + k;  // off-diagonal
  T *tau = eo + k;
  T *vv = tau + k;   // Householder vectors (vv[0] = 1) of the even steps
  T *vv2 = vv + k;   // and of the odd steps
  T *pv = vv2 + k;   // p of the current step
  T *rc = pv + k;
  T *rs = rc + k;
  // df_rot: the sweep's rotations as double-float pairs (8-byte aligned: the
  // tail starts after 32 doubles and holds only 8-byte elements for T = double)
  float2 *rcf = reinterpret_cast<float2 *>(rs + k);
  float2 *rsf = rcf + k;
  T *red = reinterpret_cast<T *>(rsf + k);
  int *perm = reinterpret_cast<int *>(red + 32);
  __shared__ EigShared sh;
  // scale to max |G| = 1 and symmetrise: coalesced copy, then the
  // symmetrisation inside shared memory
  double mx = 0.0;
  for (int e = tid; e < k * k; e += nt) mx = fmax(mx, fabs(it.G[e]));
  mx = block_max_d(mx, redd);
  const double scale = (mx > 0.0) ? mx : 1.0;
  const double inv_scale = 1.0 / scale;
  for (int c = warp; c < k; c += nw)
    for (int r = lane; r < k; r += 32) Z[(int64_t)c * ld + r] = T(it.G[(int64_t)c * k + r] * inv_scale);
  __syncthreads();
  for (int c = warp; c < k; c += nw)
    for (int r = c + 1 + lane; r < k; r += 32) {
      const T v = T(0.5) * (Z[(int64_t)c * ld + r] + Z[(int64_t)r * ld + c]);
      Z[(int64_t)c * ld + r] = v;
      Z[(int64_t)r * ld + c] = v;
    }
  __syncthreads();
  // 1. tridiagonalisation: step j annihilates Z[j+2:k, j] with the reflector
  //    I - tau v v^T (v(j+1) = 1, tail kept in Z[j+2:k, j]); the trailing
  //    block A = Z[j+1:, j+1:] takes A - v w^T - w v^T, w = p - (tau/2)(p^T v) v, p = tau A v.
  //    Two barriers per step: every warp forms (p^T v) itself, and warp 0,
  //    which updates column j+1 first, forms reflector j+1 (into the other
  //    vector buffer) while the other warps finish the update.
  auto form = [&](int j, T *vb) {  // warp 0
    const int o = j + 1;
    T *x = Z + (int64_t)j * ld;
    T part = T(0);
    for (int r = o + 1 + lane; r < k; r += 32) part += x[r] * x[r];
    const T s2 = warp_sum_t(part);
    const T alpha = x[o];
    T tj = T(0), beta = alpha, inv_v0 = T(0);
    if (s2 != T(0)) {
      const T nrm = sqrt(alpha * alpha + s2);
      beta = (alpha <= T(0)) ? nrm : -nrm;
      inv_v0 = T(1) / (alpha - beta);
      tj = (beta - alpha) / beta;
    }
    for (int r = o + 1 + lane; r < k; r += 32) {
      const T v = x[r] * inv_v0;
      x[r] = v;
      vb[r - o] = v;
    }
    if (lane == 0) {
      vb[0] = T(1);
      tau[j] = tj;
      dg[j] = x[j];
      eo[j] = beta;
    }
  };
  if (warp == 0 && k >= 3) form(0, vv);
  __syncthreads();
  for (int j = 0; j + 2 < k; ++j) {
    const int o = j + 1, L = k - o;
    const T *vc = (j & 1) ? vv2 : vv;
    T *vn = (j & 1) ? vv : vv2;
    const bool next = (j + 3 < k);
    const T tj = tau[j];
    if (tj != T(0)) {  // uniform: every thread read the same tau
      quad_colvec(Z, ld, o, L, vc, pv, tj);  // p = tau A v (A symmetric)
      __syncthreads();
      T part = T(0);
      for (int r = lane; r < L; r += 32) part += pv[r] * vc[r];
      const T kk = T(0.5) * tj * warp_sum_t(part);  // the same value in every warp
      for (int c = warp; c < L; c += nw) {
        T *col = Z + (int64_t)(o + c) * ld + o;
        const T vcc = vc[c], wc = pv[c] - kk * vcc;
        for (int r = lane; r < L; r += 32) col[r] -= vc[r] * wc + (pv[r] - kk * vc[r]) * vcc;
        if (c == 0 && next) {  // warp 0: column j+1 is final, form reflector j+1
          __syncwarp();
          form(j + 1, vn);
        }
      }
    } else if (warp == 0 && next) {
      form(j + 1, vn);  // column j+1 is unchanged
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
  // 2. explicit H = H_0 ... H_{k-3} in place, backwards: after step j the
  //    columns >= j+1 hold H_j ... H_{k-3} (restricted to rows/columns >= 1);
  //    v_j is read from column j (consumed before column j is rewritten)
  for (int r = tid; r < k; r += nt) Z[(int64_t)(k - 1) * ld + r] = (r == k - 1) ? T(1) : T(0);
  __syncthreads();
  for (int j = k - 3; j >= 0; --j) {
    const int o = j + 1, L = k - o;
    const T tj = tau[j];
    const T *v = Z + (int64_t)j * ld;  // v(o) = 1, v(o+1..) = column j below o
    if (tj != T(0)) {
      // w_c = v^T Z[o:, c] for the columns c > o; Z[o:, c] -= tau v w_c
      const int q = tid & 3;
      for (int i0 = 0; i0 < L - 1; i0 += nt >> 2) {
        const int i = i0 + (tid >> 2);
        T acc = T(0);
        const T *col = Z + (int64_t)(o + 1 + i) * ld + o;
        if (i < L - 1)
          for (int l = q; l < L; l += 4) acc += col[l] * (l == 0 ? T(1) : v[o + l]);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (q == 0 && i < L - 1) pv[i] = tj * acc;
      }
      __syncthreads();
      for (int c = warp; c < L - 1; c += nw) {
        T *col = Z + (int64_t)(o + 1 + c) * ld + o;
        const T wc = pv[c];
        for (int r = lane; r < L; r += 32) col[r] -= (r == 0 ? T(1) : v[o + r]) * wc;
      }
    }
    __syncthreads();
    // column o = H_j e_o: 1 - tau at row o, -tau v below, zero above
    T *co = Z + (int64_t)o * ld;
    for (int r = tid; r < k; r += nt) {
      T val;
      if (r < o) val = T(0);
      else if (r == o) val = T(1) - tj;
      else val = -tj * v[r];
      co[r] = val;
    }
    __syncthreads();
  }
  for (int r = tid; r < k; r += nt) {
    Z[r] = (r == 0) ? T(1) : T(0);                  // column 0 = e_0
    if (r > 0) Z[(int64_t)r * ld] = T(0);           // row 0 of the other columns
  }
  __syncthreads();
  // 3. implicit QL; deflation when |e_m| <= eps ||T|| (normwise: the Gramians
  //    need eigenvalues to within eps * lambda_max only)
  if (tid == 0) {
    sh.done = 0;
    sh.status = 0;
  }
  int l = 0, iter = 0;
  T tol = T(0);
  if (warp == 0) {
    T tn = T(0);
    for (int i = lane; i < k; i += 32) {
      T v = fabs(dg[i]) + fabs(eo[i]) + (i > 0 ? fabs(eo[i - 1]) : T(0));
      tn = tn > v ? tn : v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T o2 = __shfl_xor_sync(0xffffffffu, tn, off);
      tn = tn > o2 ? tn : o2;
    }
    const T eps = (sizeof(T) == 8) ? T(2.220446049250313e-16) : T(1.1920929e-7);
    tol = eps * tn;
  }
  // df_rot (mixed path): the eigenvectors are accumulated in double-float on
  // the FP32 pipe (about 2^-47 per rotation); the QL recurrence, which alone
  // decides the eigenvalues, stays in FP64.  Entries are at most 1 in
  // magnitude, so no scaling is needed; each is converted in place.
  if (df_rot) {
    float2 *Zf = reinterpret_cast<float2 *>(Z);
    for (int e = tid; e < k * k; e += nt) {
      const int c = e / k, r = e - c * k;
      float h, l;
      df_from_f64((double)Z[(int64_t)c * ld + r], 0, h, l);
      Zf[(int64_t)c * ld + r] = make_float2(h, l);
    }
  }
  for (;;) {
    // warp 0 finds the next unreduced block (a ballot over 32 off-diagonals
    // at a time); lane 0 runs the sweep's rotation recurrence
    if (warp == 0) {
      int cnt = 0;
      while (l < k && cnt == 0) {
        int mm = k - 1;
        for (int base = l; base < k - 1; base += 32) {
          const int m = base + lane;
          const unsigned hit = __ballot_sync(0xffffffffu, m < k - 1 && fabs(eo[m]) <= tol);
          if (hit) {
            mm = base + __ffs(hit) - 1;
            break;
          }
        }
        if (mm == l) {
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > 64) {
          if (lane == 0) {
            sh.status = 1;
            atomicOr(&g_eig_status, 1u);  // reported by ht_device_status / truncation reports
          }
          ++l;
          iter = 0;
          continue;
        }
        if (lane == 0) {
          // Wilkinson-type shift from the leading 2x2 block
          T g = (dg[l + 1] - dg[l]) / (T(2) * eo[l]);
          T r = sqrt(g * g + T(1));
          g = dg[mm] - dg[l] + eo[l] / (g + copysign(r, g));
          T s = T(1), c = T(1), p = T(0);
          bool deflated = false;
          T e_i = eo[mm - 1], d_i = dg[mm - 1], d_i1 = dg[mm];  // operands of step i, loaded one step ahead
          for (int i = mm - 1; i >= l; --i) {
            const T e_n = (i > l) ? eo[i - 1] : T(0), d_n = (i > l) ? dg[i - 1] : T(0);
            const T f = s * e_i, b = c * e_i;
            givens(f, g, r, s, c);
            eo[i + 1] = r;
            if (r == T(0)) {
              dg[i + 1] = d_i1 - p;
              eo[mm] = T(0);
              deflated = true;
              break;
            }
            g = d_i1 - p;
            r = (d_i - g) * s + T(2) * c * b;
            p = s * r;
            dg[i + 1] = g + p;
            g = c * r - b;
            rc[cnt] = c;
            rs[cnt] = s;
            ++cnt;
            e_i = e_n;
            d_i1 = d_i;
            d_i = d_n;
          }
          sh.lo = mm - 1;
          if (!deflated) {
            dg[l] = d_i1 - p;
            eo[l] = g;
            eo[mm] = T(0);
          }
        }
        cnt = __shfl_sync(0xffffffffu, cnt, 0);
        __syncwarp();  // lane 0's updates of eo / dg before the next scan
      }
      if (lane == 0) {
        sh.count = cnt;
        sh.done = (l >= k && cnt == 0) ? 1 : 0;
      }
    }
    __syncthreads();
    if (sh.done) break;
    const int cnt = sh.count, i0 = sh.lo;
    if (df_rot) {
      for (int q = tid; q < cnt; q += nt) {
        float h, l;
        df_from_f64((double)rc[q], 0, h, l);
        rcf[q] = make_float2(h, l);
        df_from_f64((double)rs[q], 0, h, l);
        rsf[q] = make_float2(h, l);
      }
      __syncthreads();
      float2 *Zf = reinterpret_cast<float2 *>(Z);
      for (int row = tid; row < k; row += nt) {
        float2 z1 = Zf[(int64_t)(i0 + 1) * ld + row];
        for (int q0 = 0; q0 < cnt; q0 += 8) {
          float2 zb[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            zb[u] = (q0 + u < cnt) ? Zf[(int64_t)(i0 - q0 - u) * ld + row] : make_float2(0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int q = q0 + u;
            if (q < cnt) {
              const float2 c = rcf[q], sn = rsf[q];
              float p1, e1, p2, e2, t, ah, al, bh, bl;
              // a = s zb + c z1, b = c zb - s z1, each renormalised
              df_prod(sn.x, sn.y, zb[u].x, zb[u].y, p1, e1);
              df_prod(c.x, c.y, z1.x, z1.y, p2, e2);
              two_sum(p1, p2, ah, t);
              fast_two_sum(ah, __fadd_rn(t, __fadd_rn(e1, e2)), ah, al);
              df_prod(c.x, c.y, zb[u].x, zb[u].y, p1, e1);
              df_prod(sn.x, sn.y, z1.x, z1.y, p2, e2);
              two_sum(p1, -p2, bh, t);
              fast_two_sum(bh, __fadd_rn(t, __fsub_rn(e1, e2)), bh, bl);
              Zf[(int64_t)(i0 - q + 1) * ld + row] = make_float2(ah, al);
              z1 = make_float2(bh, bl);
            }
          }
        }
        Zf[(int64_t)(i0 + 1 - cnt) * ld + row] = z1;
      }
      __syncthreads();
      continue;
    }
    for (int row = tid; row < k; row += nt) {
      T zi1 = Z[(int64_t)(i0 + 1) * ld + row];
      // the sweep's columns in groups of 8: the loads of a group are issued
      // together (Z may live in global memory), then its 8 rotations
      for (int q0 = 0; q0 < cnt; q0 += 8) {
        T zb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) zb[u] = (q0 + u < cnt) ? Z[(int64_t)(i0 - q0 - u) * ld + row] : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u;
          if (q < cnt) {
            Z[(int64_t)(i0 - q + 1) * ld + row] = rs[q] * zb[u] + rc[q] * zi1;
            zi1 = rc[q] * zb[u] - rs[q] * zi1;
          }
        }
      }
      Z[(int64_t)(i0 + 1 - cnt) * ld + row] = zi1;
    }
    __syncthreads();
  }
  if (df_rot) {  // eigenvectors back to FP64, in place
    const float2 *Zf = reinterpret_cast<const float2 *>(Z);
    for (int e = tid; e < k * k; e += nt) {
      const int c = e / k, r = e - c * k;
      const float2 v = Zf[(int64_t)c * ld + r];
      Z[(int64_t)c * ld + r] = T(df_to_f64(v.x, v.y, 0));
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

// ---- double-float refinement --------------------------------------------------
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
  constexpr int BI = 4, BJ = 2;  // outputs per thread: 4 rows x 2 columns
  const int ti_n = (k + BI - 1) / BI, tj_n = (k + BJ - 1) / BJ;
  for (int t = threadIdx.x; t < ti_n * tj_n; t += blockDim.x) {
    const int ti = (t / tj_n) * BI, tj = (t % tj_n) * BJ;
    float hi[BI][BJ], lo[BI][BJ];
#pragma unroll
    for (int u = 0; u < BI; ++u)
#pragma unroll
      for (int v = 0; v < BJ; ++v) hi[u][v] = lo[u][v] = 0.0f;
    for (int l = 0; l < k; ++l) {
      float ah[BI], al[BI], bh[BJ], bl[BJ];
#pragma unroll
      for (int u = 0; u < BI; ++u) {
        const int i = ti + u;
        const int ia = kTransA ? i * ld + l : l * ld + i;
        ah[u] = (i < k) ? Ah[ia] : 0.0f;
        al[u] = (kALo && i < k) ? Al[ia] : 0.0f;
      }
#pragma unroll
      for (int v = 0; v < BJ; ++v) {
        const int j = tj + v;
        bh[v] = (j < k) ? Bh[j * ld + l] : 0.0f;
        bl[v] = (kBLo && j < k) ? Bl[j * ld + l] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < BI; ++u)
#pragma unroll
        for (int v = 0; v < BJ; ++v) {
          df_mac(hi[u][v], lo[u][v], ah[u], bh[v]);
          if (kALo) lo[u][v] = __fmaf_rn(al[u], bh[v], lo[u][v]);
          if (kBLo) lo[u][v] = __fmaf_rn(ah[u], bl[v], lo[u][v]);
        }
    }
#pragma unroll
    for (int u = 0; u < BI; ++u)
#pragma unroll
      for (int v = 0; v < BJ; ++v)
        if (ti + u < k && tj + v < k) {
          const float s = __fadd_rn(hi[u][v], lo[u][v]);  // renormalise: |lo| <= ulp(hi) / 2
          Ch[(tj + v) * ld + ti + u] = s;
          Cl[(tj + v) * ld + ti + u] = __fsub_rn(lo[u][v], __fsub_rn(s, hi[u][v]));
        }
  }
}

// Shared memory of the refinement: lambda (max_k doubles), 32 doubles, the
// ranks (max_k ints), and the seven k x (k+1) float arrays when they fit
// (max_k <= kDfMaxK); larger Gramians keep the arrays in a global scratch
// slab per item (L2-resident).
__host__ __device__ size_t refine_df_smem(int max_k, bool arrays) {
  const size_t base = (size_t)(max_k + 32) * sizeof(double) + (((size_t)max_k * sizeof(int) + 15) & ~size_t(15));
  return base + (arrays ? 7 * (size_t)max_k * (max_k + 1) * sizeof(float) : 0);
}

__global__ void __launch_bounds__(REFINE_THREADS) refine_df_kernel(const EigItem *__restrict__ items, double *scratch,
                                                                int64_t scratch_stride, int max_k, int in_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x, ld = k + 1;  // odd ld: 2-way bank conflicts at most
  const int sz = k * ld;
  double *lam = reinterpret_cast<double *>(smem_raw);  // k
  double *red = lam + max_k;                            // 32
  int *rank = reinterpret_cast<int *>(red + 32);        // k
  float *Ah = in_smem ? reinterpret_cast<float *>(smem_raw + refine_df_smem(max_k, false))
                      : reinterpret_cast<float *>(scratch + (int64_t)blockIdx.x * scratch_stride);
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
size_t ql_tail_smem(int max_k) {  // everything but the eigenvector array
  return 32 * sizeof(double) + (size_t)(8 * max_k + 32) * sizeof(T) + 2 * (size_t)max_k * sizeof(float2) +
         (size_t)max_k * sizeof(int);
}
template <typename T>
size_t ql_smem(int max_k) {
  const size_t tail = ql_tail_smem<T>(max_k);
  return (max_k <= kEigSmemK) ? (size_t)max_k * ql_ld(max_k) * sizeof(T) + tail : tail;
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
  if (mode == 0 || mode == 2) {  // FP64 QL (mode 2: eigenvector rotations in double-float)
    // eigenvectors in shared memory allow one CTA per SM at k = 128; with more
    // matrices than SMs they go to the scratch slab (L2-resident) instead, so
    // that four CTAs share an SM and overlap their one-thread QL recurrences
    const bool z_smem = max_k <= kEigSmemK && !(scratch && eig_z_global(max_k, n_items));
    const size_t smem = z_smem ? ql_smem<double>(max_k) : ql_tail_smem<double>(max_k);
    e = cudaFuncSetAttribute(eig_ql_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    eig_ql_kernel<double><<<n_items, EIG_THREADS, smem, s>>>(d_items, scratch, (int64_t)max_k * ql_ld(max_k),
                                                             z_smem ? 1 : 0, mode == 2 ? 1 : 0);
    count_launch();
    return cudaGetLastError();
  }
  // FP32 QL, then one double-float refinement step
  const size_t smem = ql_smem<float>(max_k);
  e = cudaFuncSetAttribute(eig_ql_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eig_ql_kernel<float><<<n_items, EIG_THREADS, smem, s>>>(d_items, scratch, (int64_t)max_k * ql_ld(max_k),
                                                            max_k <= kEigSmemK ? 1 : 0, 0);
  count_launch();
  const bool in_smem = max_k <= kDfMaxK;  // else the arrays use the scratch slab (4 max_k^2 doubles per item)
  if (!in_smem && !scratch) return cudaErrorInvalidValue;
  const size_t dsm = refine_df_smem(max_k, in_smem);
  e = cudaFuncSetAttribute(refine_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
  if (e != cudaSuccess) return e;
  refine_df_kernel<<<n_items, REFINE_THREADS, dsm, s>>>(d_items, scratch, 4 * (int64_t)max_k * max_k, max_k,
                                                     in_smem ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

int eig_smem_k() { return kEigSmemK; }

unsigned eig_take_status() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_eig_status, sizeof(v)) != cudaSuccess) return ~0u;
  if (v) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_eig_status, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return v;
}

}  // namespace htgb
