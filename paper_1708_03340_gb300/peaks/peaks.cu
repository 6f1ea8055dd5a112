// peaks.cu -- throughput microbenchmarks of the GB300 units this library's
// kernels are bound by, timed with CUDA events (no clock or power setting is
// touched):
//   fp64_fma   FP64 FMA chains (the FP64 QR blocks and eigensolvers)
//   fp32_fma   FP32 FMA chains (the SIMT contractions of the FP32 path)
//   bf16_mma   tcgen05.mma kind::f16 (BF16 x BF16 -> FP32), M = 128, N = 256, K = 16,
//              operands in shared memory, accumulator in TMEM (the mixed path's
//              contractions issue this instruction with N = 128)
//   tf32_mma   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8
// Output: one JSON line per measurement.  Every wait is bounded by time.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                \
      return 1;                                                               \
    }                                                                         \
  } while (0)

template <typename T, int NACC>
__global__ void __launch_bounds__(256) fma_kernel(T *out, int iters, T x, T y) {
  T a[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) a[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < NACC; ++i) a[i] = fma(a[i], x, y);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < NACC; ++i) s += a[i];
  if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// core-matrix K-major no-swizzle operand descriptor: LBO 128 B, SBO = (k bytes per row / 16) * 128
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// KIND 0: f16 (BF16), K = 16 per MMA; KIND 1: tf32, K = 8 per MMA.  Each row of an
// operand holds 32 bytes of K (two core matrices), so SBO = 256 B.
template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_kernel(int count, unsigned *status) {
  __shared__ __align__(1024) unsigned char A[128 * 32];
  __shared__ __align__(1024) unsigned char B[256 * 32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x;
  for (int i = tid; i < 128 * 32 / 4; i += 128) reinterpret_cast<uint32_t *>(A)[i] = 0x3F803F80u ^ (i * 2654435761u & 0x00FF00FFu);
  for (int i = tid; i < 256 * 32 / 4; i += 128) reinterpret_cast<uint32_t *>(B)[i] = 0x3F803F80u ^ (i * 40503u & 0x00FF00FFu);
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t fmt = KIND == 0 ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint64_t da = desc(smem_u32(A), 256), db = desc(smem_u32(B), 256);
    for (int i = 0; i < count; ++i) {
      const uint32_t en = i ? 1u : 0u;
      if (KIND == 0)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(en)
                     : "memory");
      else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(en)
                     : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    const uint64_t t0 = gtimer();
    for (;;) {
      uint32_t done;
      asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                   "selp.b32 %0, 1, 0, p;\n\t}"
                   : "=r"(done)
                   : "r"(smem_u32(&bar))
                   : "memory");
      if (done) break;
      if (gtimer() - t0 > 2000000000ull) {  // 2 s
        atomicOr(status, 1u);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

template <typename T, int NACC>
static int run_fma(const char *name, int sms) {
  T *out;
  CK(cudaMalloc(&out, sizeof(T) * 256 * sms * 8));
  const int blocks = sms * 8, iters = sizeof(T) == 8 ? 2048 : 16384;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (int w = 0; w < 3; ++w) fma_kernel<T, NACC><<<blocks, 256>>>(out, iters, (T)0.999, (T)0.001);
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    CK(cudaEventRecord(a));
    fma_kernel<T, NACC><<<blocks, 256>>>(out, iters, (T)0.999, (T)0.001);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms;
    CK(cudaEventElapsedTime(&ms, a, b));
    best = ms < best ? ms : best;
  }
  const double flops = 2.0 * NACC * (double)iters * 256.0 * blocks;
  printf("{\"unit_test\": \"%s\", \"tflops\": %.3f, \"ms\": %.4f, \"blocks\": %d, \"threads\": 256, \"chains_per_thread\": %d}\n",
         name, flops / (best * 1e-3) / 1e12, best, blocks, NACC);
  CK(cudaFree(out));
  return 0;
}

template <int KIND>
static int run_mma(const char *name, int sms) {
  unsigned *st;
  CK(cudaMalloc(&st, sizeof(unsigned)));
  CK(cudaMemset(st, 0, sizeof(unsigned)));
  const int count = 8192;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (int w = 0; w < 3; ++w) mma_kernel<KIND><<<sms, 128>>>(count, st);
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    CK(cudaEventRecord(a));
    mma_kernel<KIND><<<sms, 128>>>(count, st);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms;
    CK(cudaEventElapsedTime(&ms, a, b));
    best = ms < best ? ms : best;
  }
  unsigned hs = 0;
  CK(cudaMemcpy(&hs, st, sizeof(unsigned), cudaMemcpyDeviceToHost));
  const double k = KIND == 0 ? 16.0 : 8.0;
  const double flops = 2.0 * 128.0 * 256.0 * k * count * sms;
  printf("{\"unit_test\": \"%s\", \"tflops\": %.3f, \"ms\": %.4f, \"ctas\": %d, \"mma_per_cta\": %d, \"shape\": \"128x256x%d\", "
         "\"wait_gave_up\": %u}\n",
         name, flops / (best * 1e-3) / 1e12, best, sms, count, (int)k, hs);
  CK(cudaFree(st));
  return 0;
}

int main() {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (run_fma<double, 8>("fp64_fma", sms)) return 1;
  if (run_fma<float, 16>("fp32_fma", sms)) return 1;
  if (run_mma<0>("bf16_mma", sms)) return 1;
  if (run_mma<1>("tf32_mma", sms)) return 1;
  return 0;
}
