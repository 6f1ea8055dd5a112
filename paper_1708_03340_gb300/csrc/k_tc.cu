// k_tc.cu -- strided batched contractions of FP32 data on the 5th-generation
// tensor cores (tcgen05, sm_103a).  Same work items and semantics as the SIMT
// kernel in k_gemm.cu (mode products of Lemma "transfer tensor
// transformation", Gramian contractions of eqs. "acctransferSon1/2", leaf
// products, TSQR recombination).
//
// Precision: each FP32 operand x is split exactly into three TF32 pieces
// x = h + m + l (h, m: 11 significant bits, l: the remaining <= 2 bits); the
// tensor core multiplies TF32 pieces exactly and accumulates in FP32, and the
// six products l*h, h*l, m*m, m*h, h*m, h*h (smallest first) carry the
// product to FP32 accuracy (dropped terms are below 2^-33 relative).
//
// Per CTA: one 128 x 64 tile of C, 128 threads.  K is walked in stages of 32
// through two shared-memory stage buffers (each holding the three pieces of
// A and of B in the canonical no-swizzle K-major layout, 8-row x 16-byte core
// matrices).  Per stage the threads split the FP32 values (loaded into
// registers one stage ahead) into their buffer, and one thread issues the 24
// MMAs (6 piece products x 4 k-steps of 8) into two tensor-memory
// accumulators -- the h*h products and the five corrections -- and commits
// them to that buffer's mbarrier.  The MMAs of a stage run while the threads
// split the next one; a buffer is refilled only after its mbarrier reports the
// MMAs that read it complete (bounded waits, error flag).  The accumulators
// cover the CTA's whole reduction, at most kTcMaxK products (the plan splits
// longer reductions across CTAs, whose partial sums are added in FP64 by
// k_gemm.cu), and are read once at the end with tcgen05.ld (warp w owns TMEM
// lanes 32w..32w+31).
//
// Measured on GB300 (opt-in, HTGB_TC=1): 5.5 - 7.5 TFLOP/s on the benchmark
// workloads, below the SIMT kernel (12 - 25), because the per-element split
// and scattered 4-byte shared stores of 128 threads cannot feed the MMAs; and
// the tensor core's FP32 accumulation is biased (errors grow with the number
// of accumulated products instead of like a random walk), which puts ||X|| of
// the d = 256 workload at 7e-5 relative, above the FP32 path's tolerance.
#include <stdint.h>

#include "internal.h"

namespace htgb {

__device__ int g_tc_wait_error = 0;  // set when an mbarrier wait gave up (never expected)

namespace {

constexpr int TCM = 128;          // rows of a tile (MMA M)
constexpr int TCN = 64;           // columns of a tile (MMA N)
constexpr int TCK = 32;           // K elements per stage
constexpr int TC_THREADS = 128;   // 4 warps = the 4 TMEM lane quadrants
constexpr int TMEM_COLS = 128;    // two accumulators of 64 FP32 columns
constexpr uint32_t PIECE_A = TCM * TCK * 4;  // bytes of one split piece of the A stage
constexpr uint32_t PIECE_B = TCN * TCK * 4;
constexpr long long kWaitLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a stage in the canonical K-major layout:
// core matrix (row/8, k/4) of 8 rows x 16 bytes at ((row/8) * (TCK/4) + k/4) * 128
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return ((uint32_t)(row >> 3) * (TCK / 4) + (uint32_t)(k >> 2)) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

// shared memory matrix descriptor: start address, leading-dimension byte
// offset (next core matrix along K = 128 B), stride-dimension byte offset
// (next 8-row group = (TCK/4) * 128 B), version bits 0b001, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (TCK / 4) * 128;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::tf32: D = F32 (1 << 4), A = B = TF32 (2 << 7,
// 2 << 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void split3(float x, float &h, float &m, float &l) {
  h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  const float r = x - h;  // exact
  m = __uint_as_float(__float_as_uint(r) & 0xFFFFE000u);
  l = r - m;  // exact, <= 2 significant bits
}

__device__ __forceinline__ int eff_dim(int lit, int ref, int mult, const int *ranks) {
  if (ref < 0) return lit;
  int v = ranks[ref] * mult;
  return v < lit ? v : lit;
}

__device__ __forceinline__ int find_item(const GemmItem *items, int n, int tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].tc_tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int NT>  // NT: columns of the tile (multiple of 16, <= TCN, 2 NT <= TMEM_COLS)
__global__ void __launch_bounds__(TC_THREADS) gemm_tc_kernel(const GemmItem *__restrict__ items, int n_items,
                                                             const int *__restrict__ ranks) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const GemmItem &it = items[find_item(items, n_items, blockIdx.x)];
  int local = blockIdx.x - it.tc_tile0;
  const int tm = local % it.tc_tiles_m;
  local /= it.tc_tiles_m;
  const int tn = local % it.tc_tiles_n;
  local /= it.tc_tiles_n;
  const int b = local % it.batch;
  const int chunk = local / it.batch;
  const int M = eff_dim(it.M, it.m_ref, 1, ranks);
  const int N = eff_dim(it.N, it.n_ref, it.n_mult, ranks);
  const int batch = eff_dim(it.batch, it.b_ref, it.b_mult, ranks);
  const int m0 = tm * TCM, n0 = tn * NT;
  if (m0 >= M || n0 >= N || b >= batch) return;  // uniform for the CTA, before any TMEM is held
  const int n_here = (N - n0 < NT) ? N - n0 : NT;
  const int K = it.K;
  const int ko_begin = (int)((int64_t)chunk * it.Ko / it.ksplit);
  const int ko_end = (int)((int64_t)(chunk + 1) * it.Ko / it.ksplit);
  const int kt = (K + TCK - 1) / TCK;
  const int ns = (ko_end - ko_begin) * kt;  // stages of this CTA
  const float *A = static_cast<const float *>(it.A) + (int64_t)b * it.sab;
  const float *B = static_cast<const float *>(it.B) + (int64_t)b * it.sbb;
  constexpr uint32_t STAGE = 3 * PIECE_A + 3 * PIECE_B;  // bytes of one stage buffer
  const uint32_t bar0 = smem_addr(&mbar[0]), bar1 = smem_addr(&mbar[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // accumulator columns: [0, NT) the hi*hi products, [NT, 2 NT) the five correction products
  const uint32_t idesc = idesc_tf32(TCM, NT);
  const bool a_mfast = (it.sam == 1);
  const bool b_nfast = (it.sbn == 1) && (it.sbk != 1);
  constexpr int PA = TCM * TCK / TC_THREADS;  // 32 elements of A per thread and stage
  constexpr int PB = NT * TCK / TC_THREADS;   // 16 elements of B
  float xa[PA], xb[PB];
  auto load = [&](int s) {
    const int ko = ko_begin + s / kt, k0 = (s % kt) * TCK;
    const float *Ak = A + (int64_t)ko * it.sako;
    const float *Bk = B + (int64_t)ko * it.sbko;
    const int64_t kflat = (int64_t)ko * K;
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int e = tid + q * TC_THREADS;
      int r, k;
      if (a_mfast) { r = e % TCM; k = e / TCM; } else { k = e % TCK; r = e / TCK; }
      const int gm = m0 + r, gk = k0 + k;
      const bool kin = gk < K && (it.k_total < 0 || kflat + gk < it.k_total);
      xa[q] = (gm < M && kin) ? Ak[(int64_t)gm * it.sam + (int64_t)gk * it.sak] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int e = tid + q * TC_THREADS;
      int nn, k;
      if (b_nfast) { nn = e % NT; k = e / NT; } else { k = e % TCK; nn = e / TCK; }
      const int gn = n0 + nn, gk = k0 + k;
      const bool kin = gk < K && (it.k_total < 0 || kflat + gk < it.k_total);
      xb[q] = (gn < N && kin) ? Bk[(int64_t)gk * it.sbk + (int64_t)gn * it.sbn] : 0.0f;
    }
  };
  auto split_store = [&](unsigned char *buf) {
    unsigned char *As = buf, *Bs = buf + 3 * PIECE_A;
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int e = tid + q * TC_THREADS;
      int r, k;
      if (a_mfast) { r = e % TCM; k = e / TCM; } else { k = e % TCK; r = e / TCK; }
      float h, md, l;
      split3(xa[q], h, md, l);
      const uint32_t o = core_off(r, k);
      *reinterpret_cast<float *>(As + o) = h;
      *reinterpret_cast<float *>(As + PIECE_A + o) = md;
      *reinterpret_cast<float *>(As + 2 * PIECE_A + o) = l;
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int e = tid + q * TC_THREADS;
      int nn, k;
      if (b_nfast) { nn = e % NT; k = e / NT; } else { k = e % TCK; nn = e / TCK; }
      float h, md, l;
      split3(xb[q], h, md, l);
      const uint32_t o = core_off(nn, k);
      *reinterpret_cast<float *>(Bs + o) = h;
      *reinterpret_cast<float *>(Bs + PIECE_B + o) = md;
      *reinterpret_cast<float *>(Bs + 2 * PIECE_B + o) = l;
    }
  };

  if (ns > 0) load(0);
  for (int s = 0; s < ns; ++s) {
    const int bi = s & 1;
    unsigned char *buf = sm + bi * STAGE;
    // the MMAs of stage s - 2 read this buffer: wait for them (use number s/2 - 1 of its barrier)
    if (s >= 2) {
      if (!mbar_wait(bi ? bar1 : bar0, (uint32_t)((s / 2 - 1) & 1))) {
        atomicExch(&g_tc_wait_error, 1);
        abort_flag = 1;
      }
    }
    split_store(buf);
    if (s + 1 < ns) load(s + 1);  // next stage's values in flight during the sync and the MMAs
    // generic-proxy stores must be visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (abort_flag) break;  // uniform: set before the barrier by some thread, read by all after it
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_addr(buf), b0 = smem_addr(buf + 3 * PIECE_A);
      // correction products (smallest first) into columns [NT, 2NT), hi*hi into [0, NT);
      // the first MMA of the CTA into each accumulator overwrites it
      const int pa[6] = {2, 0, 1, 1, 0, 0};
      const int pb[6] = {0, 2, 1, 0, 1, 0};
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const uint32_t dcol = (p == 5) ? 0u : (uint32_t)NT;
#pragma unroll
        for (int st = 0; st < TCK / 8; ++st) {
          const uint64_t da = smem_desc(a0 + pa[p] * PIECE_A + st * 256);
          const uint64_t db = smem_desc(b0 + pb[p] * PIECE_B + st * 256);
          const uint32_t accf = (s == 0 && (p == 0 || p == 5) && st == 0) ? 0u : 1u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + dcol),
              "l"(da), "l"(db), "r"(idesc), "r"(accf)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bi ? bar1 : bar0)
                   : "memory");
    }
  }
  // the last commit tracks every MMA issued before it
  const int last = ns - 1;
  bool ok = !abort_flag && ns > 0;
  if (ns > 0) {
    if (!mbar_wait((last & 1) ? bar1 : bar0, (uint32_t)((last / 2) & 1))) {
      atomicExch(&g_tc_wait_error, 1);
      ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const int row = m0 + warp * 32 + lane;
  float *Cp = static_cast<float *>(it.C) + (int64_t)b * it.scb;
  float *Pp = it.ksplit > 1 ? static_cast<float *>(it.part) + ((int64_t)chunk * it.batch + b) * (int64_t)it.M * it.N
                            : nullptr;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  if (ok || ns == 0) {
#pragma unroll
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t vh[16], vc[16];
      if (ns > 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(vh[0]), "=r"(vh[1]), "=r"(vh[2]), "=r"(vh[3]), "=r"(vh[4]), "=r"(vh[5]), "=r"(vh[6]), "=r"(vh[7]),
              "=r"(vh[8]), "=r"(vh[9]), "=r"(vh[10]), "=r"(vh[11]), "=r"(vh[12]), "=r"(vh[13]), "=r"(vh[14]),
              "=r"(vh[15])
            : "r"(trow + (uint32_t)c0));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(vc[0]), "=r"(vc[1]), "=r"(vc[2]), "=r"(vc[3]), "=r"(vc[4]), "=r"(vc[5]), "=r"(vc[6]), "=r"(vc[7]),
              "=r"(vc[8]), "=r"(vc[9]), "=r"(vc[10]), "=r"(vc[11]), "=r"(vc[12]), "=r"(vc[13]), "=r"(vc[14]),
              "=r"(vc[15])
            : "r"(trow + (uint32_t)(NT + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) vh[j] = vc[j] = 0u;
      }
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (c0 + j >= n_here) continue;
          const int col = n0 + c0 + j;
          const float v = __uint_as_float(vh[j]) + __uint_as_float(vc[j]);
          if (Pp) {
            Pp[(int64_t)col * it.M + row] = v;
          } else {
            float *c = Cp + (int64_t)row * it.scm + (int64_t)col * it.scn;
            float out = (float)it.alpha * v;
            if (it.beta != 0.0) out += (float)it.beta * *c;
            *c = out;
          }
        }
      }
    }
  } else if (ns > 0) {
    // abandoned: let every issued MMA finish (bounded) before the TMEM is released
    mbar_wait(bar0, 0u);
    mbar_wait(bar1, 0u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

size_t gemm_tc_smem_bytes() { return 2 * (3 * (size_t)PIECE_A + 3 * (size_t)PIECE_B) + 1024; }

cudaError_t launch_gemm_tc(const GemmItem *d_items, int n_items, int total_tiles, const int *d_ranks, cudaStream_t s) {
  if (n_items <= 0 || total_tiles <= 0) return cudaSuccess;
  const size_t smem = gemm_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  gemm_tc_kernel<64><<<total_tiles, TC_THREADS, smem, s>>>(d_items, n_items, d_ranks);
  count_launch();
  return cudaGetLastError();
}

int tc_take_wait_error() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_wait_error, sizeof(int)) != cudaSuccess) return -1;
  if (v) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_tc_wait_error, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return v;
}

}  // namespace htgb
