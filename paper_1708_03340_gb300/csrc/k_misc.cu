// k_misc.cu -- memory-bound helper kernels of the truncation path:
//   * HT addition packing (Lemma "sum of two H-tensors"),
//   * strided copies / casts / identity fills (trivial QR cases, casts of the
//     small k x k factors between FP64 and FP32),
//   * compaction of projected transfer tensors into their truncated layout,
//   * rank selection (rank or eps rule) and ||X|| = ||B_D||_F,
//   * entry evaluation (Sec. 3.1, eq. "transfermult"),
//   * sum of squares and scaling.
#include "internal.h"
#include "wait.cuh"

namespace htgb {

namespace {

__device__ __forceinline__ int ref_dim(int lit, int ref, const int *ranks) {
  if (ref < 0) return lit;
  int v = ranks[ref];
  return v < lit ? v : lit;
}

// ---- copy -----------------------------------------------------------------
__global__ void copy_kernel(const CopyItem *__restrict__ items, const int *__restrict__ ranks) {
  const CopyItem it = items[blockIdx.y];
  const int rows = ref_dim(it.rows, it.rows_ref, ranks);
  const int cols = ref_dim(it.cols, it.cols_ref, ranks);
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / rows), r = (int)(e - (int64_t)c * rows);
    double v;
    if (it.src) {
      v = it.src_f64 ? static_cast<const double *>(it.src)[r * it.sr + c * it.sc]
                     : (double)static_cast<const float *>(it.src)[r * it.sr + c * it.sc];
      v *= it.alpha;
    } else {
      v = (!it.zero && r == c) ? 1.0 : 0.0;
    }
    const int64_t o = r * it.dr + c * it.dc;
    if (it.dst_f64) {
      double *d = static_cast<double *>(it.dst) + o;
      *d = (it.beta != 0.0) ? v + it.beta * *d : v;
    } else {
      float *d = static_cast<float *>(it.dst) + o;
      *d = (it.beta != 0.0) ? (float)(v + it.beta * (double)*d) : (float)v;
    }
  }
}

// ---- compaction -------------------------------------------------------------
template <typename T>
__global__ void compact_kernel(const CompactItem *__restrict__ items, const int *__restrict__ ranks) {
  const CompactItem it = items[blockIdx.y];
  const int r0 = it.ref0 < 0 ? 1 : ranks[it.ref0];
  const int r1 = ranks[it.ref1], r2 = ranks[it.ref2];
  const int64_t total = (int64_t)r0 * r1 * r2;
  const T *src = static_cast<const T *>(it.src);
  T *dst = static_cast<T *>(it.dst);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % r2);
    const int64_t ab = e / r2;
    const int b = (int)(ab % r1), a = (int)(ab / r1);
    dst[e] = src[((int64_t)a * it.ld1 + b) * it.ld2 + c];
  }
}

// Device status word of the rank selection: bit 0 is set when ||X|| or a
// Gramian eigenvalue is not finite (NaN or Inf in the input, or produced on
// the way).  Read and cleared by misc_take_status.
__device__ unsigned g_numeric_status = 0;


// ---- bounded-wait self-test -------------------------------------------------
// Status word of the bounded waits outside the tensor-core kernels: bit 0 is
// set when a wait gave up.  The self-test kernel waits on a flag that no code
// sets, so its wait always runs out after limit_ns and the kernel returns:
// it exercises the time bound, the status word and the host's report without
// any fault or hang.
__device__ unsigned g_wait_status = 0;
__device__ int g_selftest_flag = 0;  // never written

__global__ void selftest_wait_kernel(int64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (*(volatile int *)&g_selftest_flag != 0) return;
    if ((int64_t)(globaltimer_ns() - t0) >= limit_ns) {
      atomicOr(&g_wait_status, 1u);
      return;
    }
    __nanosleep(1000);
  }
}



// ---- rank selection ---------------------------------------------------------
// One CTA per tensor.  ||X|| from the orthogonalized root; per node the rank
// rule; the root pair shares one rank; discarded energy with the root pair
// counted once.
__global__ void ranks_kernel(const RankItem *__restrict__ items) {
  const RankItem it = items[blockIdx.x];
  __shared__ double red[32];
  __shared__ double s_tail2;
  const int tid = threadIdx.x, nt = blockDim.x;
  double part = 0.0;
  for (int64_t e = tid; e < it.root_count; e += nt) {
    double v = it.root_f64 ? static_cast<const double *>(it.root)[e] : (double)reinterpret_cast<const float *>(it.root)[e];
    part += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) s += red[w];
    const double nrm = sqrt(s);
    it.stats[0] = nrm;
    it.stats[3] = 0.0;
    if (!isfinite(nrm)) {
      it.stats[3] = 1.0;
      atomicOr(&g_numeric_status, 1u);
    }
    double tail2 = 0.0;
    if (it.mode == 1) {
      const double e = it.eps_rel ? it.eps * nrm : it.eps;
      const int counted = 2 * it.d - 3;
      tail2 = e * e / (double)(counted > 0 ? counted : 1);
    }
    s_tail2 = tail2;
    it.stats[2] = tail2;
    it.r_out[0] = 1;
  }
  __syncthreads();
  const double tail2 = s_tail2;
  for (int t = 1 + tid; t < it.nn; t += nt) {
    const int avail = it.korth[t];
    const double *lam = it.lam + it.lam_off[t];
    for (int i = 0; i < avail; ++i) {
      if (!isfinite(lam[i])) {  // a non-finite input or Gramian: report, never a silent rank
        it.stats[3] = 1.0;
        atomicOr(&g_numeric_status, 1u);
        break;
      }
    }
    int r;
    if (it.mode == 1) {
      // a dropped eigenvalue is charged its computed value plus the noise
      // floor of the arithmetic that produced it, so that an eigenvalue at
      // rounding level is never taken for a negligible one
      const double nu = it.noise * (lam[0] > 0.0 ? lam[0] : 0.0);
      double tail = 0.0;
      r = avail;
      for (int i = avail - 1; i >= 1; --i) {
        const double l = (lam[i] > 0.0 ? lam[i] : 0.0) + nu;
        if (tail + l <= tail2) {
          tail += l;
          r = i;
        } else {
          break;
        }
      }
    } else {
      r = it.target ? it.target[t] : it.cap;
      if (r <= 0) r = avail;
    }
    if (it.cap > 0 && r > it.cap) r = it.cap;
    if (r > avail) r = avail;
    if (r < 1) r = 1;
    it.r_out[t] = r;
  }
  __syncthreads();
  if (tid == 0) {
    int rr = it.r_out[it.t1];
    if (it.mode == 0 && it.r_out[it.t2] < rr) rr = it.r_out[it.t2];
    if (rr > it.korth[it.t2]) rr = it.korth[it.t2];
    it.r_out[it.t1] = rr;
    it.r_out[it.t2] = rr;
  }
  __syncthreads();
  double disc = 0.0;
  for (int t = 1 + tid; t < it.nn; t += nt) {
    if (t == it.t2) continue;
    const double *lam = it.lam + it.lam_off[t];
    for (int i = it.r_out[t]; i < it.korth[t]; ++i) disc += lam[i] > 0.0 ? lam[i] : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) disc += __shfl_xor_sync(0xffffffffu, disc, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = disc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) s += red[w];
    it.stats[1] = s;
  }
}

// ---- HT addition packing ------------------------------------------------------
// d_desc: per node 12 int64: [kind, a_off, c_off, o_off, n_or_at, ka, kc, a1, a2, c1, c2, count]
// kind 0 leaf: out column-major n x (ka + kc) = [U, V]
// kind 1 inner/root: out (at+ct) x (a1+c1) x (a2+c2) block diagonal; root: at = ct = 1 sharing index 0
// The grid's y dimension walks nodes, x strides over the node's elements.
template <typename T>
__global__ void pack_add_kernel(const T *__restrict__ a, const T *__restrict__ c, T *__restrict__ out,
                                const int64_t *__restrict__ desc) {
  const int64_t *ds = desc + 12 * (int64_t)blockIdx.y;
  const int64_t kind = ds[0];
  const T *A = a + ds[1];
  const T *C = c + ds[2];
  T *O = out + ds[3];
  const int64_t count = ds[11];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (kind == 0) {
    const int64_t n = ds[4], ka = ds[5];
    const int64_t split = n * ka;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += stride)
      O[e] = (e < split) ? A[e] : C[e - split];
  } else {
    const int64_t at = ds[4], ka1 = ds[7], ka2 = ds[8], kc1 = ds[9], kc2 = ds[10];
    const int64_t o1 = ka1 + kc1, o2 = ka2 + kc2;
    const bool root = (ds[5] == 0);  // ka == 0 marks the root (shared single index)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += stride) {
      const int64_t l = e % o2;
      const int64_t ij = e / o2;
      const int64_t j = ij % o1, i = ij / o1;
      T v = T(0);
      const bool ia = root || i < at;
      const bool ic = root || i >= at;
      const int64_t ic_i = root ? 0 : i - at;
      if (ia && j < ka1 && l < ka2) v = A[(i * ka1 + j) * ka2 + l];
      else if (ic && j >= ka1 && l >= ka2) v = C[(ic_i * kc1 + (j - ka1)) * kc2 + (l - ka2)];
      O[e] = v;
    }
  }
}

// ---- Kronecker transfer tensors of an operator application -------------------
// Lemma "operator" (Sec. 3.6): F_t = H_t (x) B_t, F[(p,i),(q,j),(r,l)] =
// H[p,q,r] B[i,j,l], pair (p, i) flattened as p * k_t + i (operator index
// slow).  desc per node (8 int64): H offset, B offset, F offset,
// pt, p1, p2 (operator ranks), it, i1, i2 (tensor ranks) packed as
// [offH, offB, offF, pt | p1 << 20 | p2 << 40, it | i1 << 20 | i2 << 40, count].
template <typename T>
__global__ void kron_kernel(const T *__restrict__ h, const T *__restrict__ b, T *__restrict__ f,
                            const int64_t *__restrict__ desc) {
  const int64_t *ds = desc + 6 * (int64_t)blockIdx.y;
  const T *H = h + ds[0];
  const T *B = b + ds[1];
  T *F = f + ds[2];
  const int64_t pt = ds[3] & 0xFFFFF, p1 = (ds[3] >> 20) & 0xFFFFF, p2 = (ds[3] >> 40) & 0xFFFFF;
  const int64_t it = ds[4] & 0xFFFFF, i1 = (ds[4] >> 20) & 0xFFFFF, i2 = (ds[4] >> 40) & 0xFFFFF;
  (void)pt;
  const int64_t count = ds[5];
  const int64_t o1 = p1 * i1, o2 = p2 * i2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += stride) {
    const int64_t L = e % o2, IJ = e / o2;
    const int64_t J = IJ % o1, I = IJ / o1;
    const int64_t p = I / it, i = I - p * it, q = J / i1, j = J - q * i1, r = L / i2, l = L - r * i2;
    F[e] = H[(p * p1 + q) * p2 + r] * B[(i * i1 + j) * i2 + l];
  }
}

// ---- entry evaluation ---------------------------------------------------------
// d_tree: per node [is_leaf, mode, son1, son2, height]; rows buffer holds u_t
// for every (index, node) at offset e * rows_per + row_off[t].
template <typename T>
__global__ void eval_level_kernel(const T *__restrict__ x, const int64_t *__restrict__ node_off,
                                  const int *__restrict__ ranks, const int *__restrict__ tree, const int64_t *__restrict__ n,
                                  const int64_t *__restrict__ idx, const int64_t *__restrict__ row_off, int64_t rows_per,
                                  const int *__restrict__ level_nodes, int d, double *rows, double *out) {
  const int t = level_nodes[blockIdx.y];
  const int64_t e = blockIdx.x;
  const int *tn = tree + 5 * t;
  double *u = rows + e * rows_per + row_off[t];
  const T *X = x + node_off[t];
  if (tn[0]) {
    const int mu = tn[1];
    const int64_t nm = n[mu], i = idx[e * d + mu];
    const int kt = ranks[t];
    for (int q = threadIdx.x; q < kt; q += blockDim.x) u[q] = (double)X[(int64_t)q * nm + i];
    return;
  }
  const int s1 = tn[2], s2 = tn[3];
  const int kt = (t == 0) ? 1 : ranks[t], k1 = ranks[s1], k2 = ranks[s2];
  const double *u1 = rows + e * rows_per + row_off[s1];
  const double *u2 = rows + e * rows_per + row_off[s2];
  for (int q = threadIdx.x; q < kt; q += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k1; ++j) {
      double sj = 0.0;
      const T *b = X + ((int64_t)q * k1 + j) * k2;
      for (int l = 0; l < k2; ++l) sj += (double)b[l] * u2[l];
      s += sj * u1[j];
    }
    u[q] = s;
    if (t == 0) out[e] = s;
  }
}

template <typename T>
__global__ void sumsq_kernel(const T *__restrict__ x, int64_t count, double *out) {
  __shared__ double red[32];
  double part = 0.0;
  for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
    double v = (double)x[e];
    part += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s;
  }
}

template <typename T>
__global__ void scale_kernel(T *x, int64_t count, double alpha) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = (T)(alpha * (double)x[e]);
}

}  // namespace

cudaError_t launch_copy(const CopyItem *d_items, int n_items, const int *d_ranks, int, cudaStream_t s) {
  for (int base = 0; base < n_items; base += 65535) {
    int cnt = n_items - base < 65535 ? n_items - base : 65535;
    copy_kernel<<<dim3(16, cnt), 256, 0, s>>>(d_items + base, d_ranks);
    count_launch();
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_compact(const CompactItem *d_items, int n_items, const int *d_ranks, cudaStream_t s) {
  for (int base = 0; base < n_items; base += 65535) {
    int cnt = n_items - base < 65535 ? n_items - base : 65535;
    compact_kernel<T><<<dim3(16, cnt), 256, 0, s>>>(d_items + base, d_ranks);
    count_launch();
  }
  return cudaGetLastError();
}
template cudaError_t launch_compact<double>(const CompactItem *, int, const int *, cudaStream_t);
template cudaError_t launch_compact<float>(const CompactItem *, int, const int *, cudaStream_t);

cudaError_t launch_ranks(const RankItem *d_items, int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  ranks_kernel<<<n_items, 256, 0, s>>>(d_items);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_add(const void *a, const void *c, void *out, const int64_t *d_desc, int n_nodes,
                            int64_t max_elems, cudaStream_t s) {
  int gx = (int)((max_elems + 255) / 256);
  if (gx > 64) gx = 64;
  if (gx < 1) gx = 1;
  for (int base = 0; base < n_nodes; base += 65535) {
    int cnt = n_nodes - base < 65535 ? n_nodes - base : 65535;
    pack_add_kernel<T><<<dim3(gx, cnt), 256, 0, s>>>(static_cast<const T *>(a), static_cast<const T *>(c),
                                                      static_cast<T *>(out), d_desc + 12 * (int64_t)base);
    count_launch();
  }
  return cudaGetLastError();
}
template cudaError_t launch_pack_add<double>(const void *, const void *, void *, const int64_t *, int, int64_t, cudaStream_t);
template cudaError_t launch_pack_add<float>(const void *, const void *, void *, const int64_t *, int, int64_t, cudaStream_t);

template <typename T>
cudaError_t launch_kron(const void *h, const void *b, void *f, const int64_t *d_desc, int n_nodes, int64_t max_elems,
                        cudaStream_t s) {
  int gx = (int)((max_elems + 255) / 256);
  if (gx > 256) gx = 256;
  if (gx < 1) gx = 1;
  for (int base = 0; base < n_nodes; base += 65535) {
    const int cnt = n_nodes - base < 65535 ? n_nodes - base : 65535;
    kron_kernel<T><<<dim3(gx, cnt), 256, 0, s>>>(static_cast<const T *>(h), static_cast<const T *>(b),
                                                  static_cast<T *>(f), d_desc + 6 * (int64_t)base);
    count_launch();
  }
  return cudaGetLastError();
}
template cudaError_t launch_kron<double>(const void *, const void *, void *, const int64_t *, int, int64_t, cudaStream_t);
template cudaError_t launch_kron<float>(const void *, const void *, void *, const int64_t *, int, int64_t, cudaStream_t);

template <typename T>
cudaError_t launch_eval_level(const void *x, const int64_t *node_off, const int *ranks, const int *tree, const int64_t *n,
                              const int64_t *idx, const int64_t *row_off, int64_t rows_per, const int *level_nodes,
                              int n_level, int64_t m, int d, double *rows, double *out, cudaStream_t s) {
  // grid.x = m (indices), grid.y = nodes of the level
  eval_level_kernel<T><<<dim3((unsigned)m, n_level), 64, 0, s>>>(static_cast<const T *>(x), node_off, ranks, tree, n, idx,
                                                                 row_off, rows_per, level_nodes, d, rows, out);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_eval_level<double>(const void *, const int64_t *, const int *, const int *, const int64_t *,
                                               const int64_t *, const int64_t *, int64_t, const int *, int, int64_t, int,
                                               double *, double *, cudaStream_t);
template cudaError_t launch_eval_level<float>(const void *, const int64_t *, const int *, const int *, const int64_t *,
                                              const int64_t *, const int64_t *, int64_t, const int *, int, int64_t, int,
                                              double *, double *, cudaStream_t);

template <typename T>
cudaError_t launch_sumsq(const void *x, int64_t count, double *out, cudaStream_t s) {
  sumsq_kernel<T><<<1, 1024, 0, s>>>(static_cast<const T *>(x), count, out);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_sumsq<double>(const void *, int64_t, double *, cudaStream_t);
template cudaError_t launch_sumsq<float>(const void *, int64_t, double *, cudaStream_t);

template <typename T>
cudaError_t launch_scale(void *x, int64_t count, double alpha, cudaStream_t s) {
  int g = (int)((count + 255) / 256);
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  scale_kernel<T><<<g, 256, 0, s>>>(static_cast<T *>(x), count, alpha);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_scale<double>(void *, int64_t, double, cudaStream_t);
template cudaError_t launch_scale<float>(void *, int64_t, double, cudaStream_t);

unsigned misc_take_status() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_numeric_status, sizeof(v)) != cudaSuccess) return ~0u;
  if (v) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_numeric_status, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return v;
}

cudaError_t launch_selftest_wait(int64_t limit_ns, cudaStream_t s) {
  if (limit_ns < 0) limit_ns = 0;
  if (limit_ns > kWaitLimitNs * 5) limit_ns = kWaitLimitNs * 5;
  selftest_wait_kernel<<<1, 1, 0, s>>>(limit_ns);
  count_launch();
  return cudaGetLastError();
}

unsigned wait_take_status() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_wait_status, sizeof(v)) != cudaSuccess) return ~0u;
  if (v) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_wait_status, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return v;
}

}  // namespace htgb
