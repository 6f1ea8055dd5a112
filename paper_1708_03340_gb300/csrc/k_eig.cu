// k_eig.cu -- batched symmetric eigendecomposition in FP64 (Sec. 3.3:
// Bhat_t Q_t = Q_t Sigma_t^2 gives the singular values and left singular
// vectors of every matricization).  One CTA per matrix:
//   1. Householder reduction to tridiagonal form, T = H^T G H;
//   2. explicit H from the stored reflectors;
//   3. implicit QL iteration with Wilkinson shifts on (d, e).  One thread
//      runs the scalar recurrence of a sweep and logs its Givens rotations;
//      then every thread applies the logged rotations to its own rows of H;
//   4. eigenvalues sorted descending, eigenvectors permuted alike.
// Matrices with k <= kEigSmemK live in shared memory, larger ones in a
// global scratch slab of the item.
#include "internal.h"

namespace htgb {

namespace {

constexpr int EIG_THREADS = 256;
constexpr int kEigSmemK = 128;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = (lane < nw) ? red[lane] : 0.0;
  return warp_sum_d(s);
}

struct EigShared {
  int count;  // rotations logged in this sweep
  int lo;     // first index of the rotation chain (rotations act on (i, i+1), i from hi-1 down to lo)
  int done;
  int status;
};

__global__ void __launch_bounds__(EIG_THREADS) eig_kernel(const EigItem *__restrict__ items, double *scratch,
                                                          int64_t scratch_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigItem it = items[blockIdx.x];
  const int k = it.k, tid = threadIdx.x, nt = blockDim.x;
  double *Z;
  double *tail;
  if (k <= kEigSmemK) {
    Z = reinterpret_cast<double *>(smem_raw);
    tail = Z + (int64_t)k * k;
  } else {
    Z = scratch + (int64_t)blockIdx.x * scratch_stride;
    tail = reinterpret_cast<double *>(smem_raw);
  }
  double *dg = tail;        // diagonal, k
  double *eo = dg + k;      // off-diagonal, k
  double *tau = eo + k;     // reflector factors, k
  double *pv = tau + k;     // work vector p / w, k
  double *rc = pv + k;      // rotation cosines, k
  double *rs = rc + k;      // rotation sines, k
  double *red = rs + k;     // 32
  int *perm = reinterpret_cast<int *>(red + 32);
  __shared__ EigShared sh;
  const int ld = k;
  // load, symmetrised
  for (int e = tid; e < k * k; e += nt) {
    int c = e / k, r = e - c * k;
    Z[e] = 0.5 * (it.G[(int64_t)c * k + r] + it.G[(int64_t)r * k + c]);
  }
  __syncthreads();
  // 1. tridiagonalisation: step j annihilates Z[j+2:k, j]
  for (int j = 0; j + 2 < k; ++j) {
    double *x = Z + (int64_t)j * ld;  // column j; reflector acts on rows j+1..k-1
    double part = 0.0;
    for (int r = j + 2 + tid; r < k; r += nt) part += x[r] * x[r];
    const double s2 = block_sum_d(part, red);
    const double alpha = x[j + 1];
    double tj = 0.0, beta = alpha;
    if (s2 != 0.0) {
      const double nrm = sqrt(alpha * alpha + s2);
      beta = (alpha <= 0.0) ? nrm : -nrm;
      const double inv_v0 = 1.0 / (alpha - beta);
      tj = (beta - alpha) / beta;
      for (int r = j + 2 + tid; r < k; r += nt) x[r] *= inv_v0;
    }
    __syncthreads();
    if (tid == 0) {
      tau[j] = tj;
      dg[j] = x[j];
      eo[j] = beta;
    }
    if (tj != 0.0) {
      // v = [1; x[j+2:k]] on rows j+1..k-1; trailing block A' = Z[j+1:, j+1:]
      const int L = k - j - 1;
      // p = tau A' v
      for (int rr = tid; rr < L; rr += nt) {
        const int r = j + 1 + rr;
        double s = Z[(int64_t)(j + 1) * ld + r];  // v[0] = 1
        for (int cc = 1; cc < L; ++cc) s += Z[(int64_t)(j + 1 + cc) * ld + r] * x[j + 1 + cc];
        pv[rr] = tj * s;
      }
      __syncthreads();
      double pp = 0.0;
      for (int rr = tid; rr < L; rr += nt) pp += pv[rr] * (rr == 0 ? 1.0 : x[j + 1 + rr]);
      const double kk = 0.5 * tj * block_sum_d(pp, red);
      // w = p - kk v
      for (int rr = tid; rr < L; rr += nt) pv[rr] -= kk * (rr == 0 ? 1.0 : x[j + 1 + rr]);
      __syncthreads();
      // A' -= v w^T + w v^T
      for (int e = tid; e < L * L; e += nt) {
        const int cc = e / L, rr = e - cc * L;
        const double vr = (rr == 0) ? 1.0 : x[j + 1 + rr];
        const double vc = (cc == 0) ? 1.0 : x[j + 1 + cc];
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
    eo[k - 1] = 0.0;
  }
  __syncthreads();
  // 2. explicit H = H_0 ... H_{k-3} (each H_j acts on indices j+1..k-1).
  //    Shift reflector tails one column right so that column j+1 holds v_j
  //    below row j+1, then accumulate backwards on the trailing block.
  for (int j = k - 3; j >= 0; --j) {
    for (int r = j + 2 + tid; r < k; r += nt) Z[(int64_t)(j + 1) * ld + r] = Z[(int64_t)j * ld + r];
    __syncthreads();
  }
  for (int e = tid; e < k; e += nt) {
    Z[e] = (e == 0) ? 1.0 : 0.0;             // column 0
    if (e > 0) Z[(int64_t)e * ld] = 0.0;     // row 0
  }
  __syncthreads();
  // column c = j+1 of H carries reflector j; rows/cols 1..k-1 form the block
  for (int c = k - 1; c >= 1; --c) {
    const int j = c - 1;  // reflector index, exists for j <= k-3
    const double tj = (j <= k - 3) ? tau[j] : 0.0;
    const double *v = Z + (int64_t)c * ld;  // tail v[c+1..k-1], v[c] = 1 implicit
    if (tj != 0.0) {
      const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
      for (int cc = c + 1 + warp; cc < k; cc += nw) {
        double *y = Z + (int64_t)cc * ld;
        double s = 0.0;
        for (int r = c + 1 + lane; r < k; r += 32) s += v[r] * y[r];
        s = warp_sum_d(s) + y[c];
        s *= tj;
        if (lane == 0) y[c] -= s;
        for (int r = c + 1 + lane; r < k; r += 32) y[r] -= s * v[r];
      }
    }
    __syncthreads();
    double *x = Z + (int64_t)c * ld;
    for (int r = 1 + tid; r < k; r += nt) {
      if (r < c) x[r] = 0.0;
      else if (r == c) x[r] = 1.0 - tj;
      else x[r] = -tj * x[r];
    }
    __syncthreads();
  }
  // 3. implicit QL on (dg, eo); eigenvectors = columns of Z
  if (tid == 0) {
    sh.done = 0;
    sh.status = 0;
  }
  int l = 0, iter = 0;  // thread 0's state
  const double eps = 2.220446049250313e-16;
  for (;;) {
    if (tid == 0) {
      sh.count = 0;
      while (l < k && sh.count == 0) {
        int mm;
        for (mm = l; mm < k - 1; ++mm) {
          const double dd = fabs(dg[mm]) + fabs(dg[mm + 1]);
          if (fabs(eo[mm]) <= eps * dd) break;
        }
        if (mm == l) {
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > 64) {  // no convergence: keep what we have
          sh.status = 1;
          ++l;
          iter = 0;
          continue;
        }
        double g = (dg[l + 1] - dg[l]) / (2.0 * eo[l]);
        double r = hypot(g, 1.0);
        g = dg[mm] - dg[l] + eo[l] / (g + copysign(r, g));
        double s = 1.0, c = 1.0, p = 0.0;
        int i;
        bool deflated = false;
        for (i = mm - 1; i >= l; --i) {
          double f = s * eo[i], b = c * eo[i];
          r = hypot(f, g);
          eo[i + 1] = r;
          if (r == 0.0) {
            dg[i + 1] -= p;
            eo[mm] = 0.0;
            deflated = true;
            break;
          }
          s = f / r;
          c = g / r;
          g = dg[i + 1] - p;
          r = (dg[i] - g) * s + 2.0 * c * b;
          p = s * r;
          dg[i + 1] = g + p;
          g = c * r - b;
          // rotation on columns (i, i+1), logged in chain order
          rc[sh.count] = c;
          rs[sh.count] = s;
          sh.count++;
        }
        sh.lo = mm - 1;  // first logged rotation acts on (mm-1, mm)
        if (!deflated) {
          dg[l] -= p;
          eo[l] = g;
          eo[mm] = 0.0;
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
        double *zi = Z + (int64_t)i * ld + row;
        double *zi1 = Z + (int64_t)(i + 1) * ld + row;
        const double f = *zi1;
        *zi1 = rs[q] * (*zi) + rc[q] * f;
        *zi = rc[q] * (*zi) - rs[q] * f;
      }
    }
    __syncthreads();
  }
  // 4. sort descending
  if (tid == 0) {
    for (int i = 0; i < k; ++i) perm[i] = i;
    for (int i = 0; i < k; ++i) {
      int best = i;
      for (int j = i + 1; j < k; ++j)
        if (dg[perm[j]] > dg[perm[best]]) best = j;
      int t = perm[i];
      perm[i] = perm[best];
      perm[best] = t;
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {
    int c = e / k, r = e - c * k;
    it.V[e] = Z[(int64_t)perm[c] * ld + r];
  }
  for (int c = tid; c < k; c += nt) it.lam[c] = dg[perm[c]];
}

}  // namespace

cudaError_t launch_eig(const EigItem *d_items, int n_items, int max_k, double *scratch, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  size_t tail = (size_t)(6 * max_k + 32) * sizeof(double) + (size_t)max_k * sizeof(int);
  size_t smem = (max_k <= kEigSmemK) ? (size_t)max_k * max_k * sizeof(double) + tail : tail;
  cudaError_t e = cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eig_kernel<<<n_items, EIG_THREADS, smem, s>>>(d_items, scratch, (int64_t)max_k * max_k);
  return cudaGetLastError();
}

int eig_smem_k() { return kEigSmemK; }

}  // namespace htgb
