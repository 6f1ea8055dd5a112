// k_oz.cu -- strided batched contractions of FP64 data on the 5th-generation
// tensor cores (tcgen05, sm_103a) by exact fixed-point slicing.  Same work
// items and semantics as the SIMT kernel (k_gemm.cu): the transfer-tensor
// mode products of Lemma "transfer tensor transformation" (R-apply of Sec. 3.4,
// projection of eq. "transfertransformationtrunc"), the reduced-Gramian
// contractions of eqs. "acctransferSon1/2", the leaf products and the TSQR
// recombination.  Used by the mixed-precision path (F64 storage, FP64 QR and
// eigensolves, contractions here).
//
// Arithmetic (the splitting idea of Ozaki et al., "Error-free transformations
// of matrix multiplication", written here for BF16 tensor-core operands):
//   * Every operand row (a row of A, a column of B) of one reduction chunk of at
//     most kOzChunk products is put on a common grid: with E the exponent of the
//     row's largest magnitude (|x| < 2^E), X = x 2^-E lies in (-1, 1) and is
//     rounded to an integer F = round(|X| 2^(8S)) < 2^(8S) + 1.
//   * F is cut into S signed base-256 digits, F = sum_i d_i 256^(S-1-i), with
//     d_0 in [0, 256] and d_i in [-128, 127] for i > 0 (balanced digits), and
//     slice i of x is sign(x) d_i 2^(-8(i+1)).  Every slice is an integer of at
//     most 9 significant bits times a power of two: a BF16 value, exactly.
//   * The tensor core multiplies BF16 slices exactly (16-bit products) and
//     accumulates in FP32.  Products of slices i and j sit on the grid
//     2^(-8(i+j+2)); summed over <= 256 reduction indices, the diagonals
//     i+j = 0 (|d_0 d_0'| <= 2^16) and i+j = 1 (<= 2^16 per index) stay below
//     2^24 grid units, i.e. their FP32 sums are exact whatever the order of
//     the additions.  With S = 5 all products with i+j >= 2 share a third
//     accumulator, which rounds at most at 2^-24 of its own size, 2^-40 of the
//     result's scale; with S = 6 (the Gramian contractions) i+j = 2 keeps the
//     third and i+j >= 3 share a fourth (rounding at about 2^-48 of the
//     scale).
//   * Products with i+j >= S are dropped; with the rounding of F this leaves a
//     normwise error of about 2^-(8S) |A| |B| per product: S = 5 gives about
//     2^-40 of the row scale, far below what the 1e-6 results of the mixed
//     path need and well beyond FP32 (2^-24).
//   * The three or four accumulators are read from TMEM, summed in
//     double-float FP32 arithmetic and assembled into FP64 (scaled by
//     2^(E_row + E_col)) with integer operations, then written (or written as
//     a split-K partial; the chunks of a long reduction are added in FP64 by
//     the reduction kernel of k_gemm.cu).
//
// Kernels:
//   oz_split_kernel  one CTA per (item, operand, batch, 128-row block, chunk):
//                    every row's exponent over the chunk, then the S BF16
//                    slices written straight into the tensor core's canonical
//                    no-swizzle K-major shared-memory layout (core matrices of
//                    8 rows x 16 bytes), one 8 KB block per slice and 32-wide
//                    reduction stage, so that the GEMM fetches a stage with a
//                    few bulk copies.  Rows contiguous along the reduction are
//                    read once by lane groups (the exponent a group maximum);
//                    rows adjacent in memory are read in two passes.
//   oz_gemm_kernel   persistent, one CTA per SM walking the launch's tiles of
//                    128 rows x 64 columns, 576 threads: warp 16 issues the
//                    bulk copies (cp.async.bulk, mbarrier transaction counts)
//                    into a three-stage ring, one thread of warp 17 issues the
//                    MMAs (tcgen05.mma kind::f16, BF16 x BF16 -> FP32, M = 128,
//                    N = 64, K = 16) into three or four accumulators of one of
//                    two TMEM buffers, and warps 0-15 read a finished tile's
//                    accumulators with tcgen05.ld while the next tile's MMAs
//                    run.  Every mbarrier wait is bounded by time (wait.cuh);
//                    one that gives up sets g_oz_status, lets the issued MMAs
//                    finish (bounded) before the TMEM is freed, and returns.
#include <stdint.h>

#include "internal.h"
#include "dfloat.cuh"
#include "wait.cuh"

namespace htgb {

// Status word of this file's bounded waits: bit 0 set when a wait gave up.
__device__ unsigned g_oz_status = 0;

namespace {

constexpr int OZ_M = 128;                       // rows of a tile (MMA M); also the rows of one split block
constexpr int OZ_N = 128;                       // rows of a B-operand slice block (two 64-column GEMM tiles)
constexpr int OZ_KC = 32;                       // reduction indices per stage
constexpr uint32_t OZ_BLK = OZ_M * OZ_KC * 2;   // bytes of one slice block of one stage (8 KB)
constexpr int OZ_THREADS = 576;                 // warps 0-15 epilogue, 16 producer, 17 MMA
constexpr int OZ_EPI_THREADS = 512;
constexpr int OZ_PROD_WARP = 16, OZ_MMA_WARP = 17;
constexpr int OZ_TMEM_COLS = 512;               // two tile buffers of up to four FP32 accumulators of 64 columns
constexpr int OZ_EXP_NONFINITE = 0x7FF0;        // exponent marking a row with NaN / Inf

__device__ __forceinline__ int eff_dim(int lit, int ref, int mult, const int *ranks) {
  if (ref < 0) return lit;
  int v = ranks[ref] * mult;
  return v < lit ? v : lit;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a 128 x 32 BF16 block: core matrix
// (row / 8, k / 8) of 8 rows x 16 bytes at ((row / 8) * 4 + k / 8) * 128
__device__ __forceinline__ uint32_t oz_off(int row, int k) {
  return ((uint32_t)(row >> 3) * (OZ_KC / 8) + (uint32_t)(k >> 3)) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// shared memory matrix descriptor of a K-major no-swizzle operand: start
// address, leading-dimension byte offset (next core matrix along K: 128 B),
// stride-dimension byte offset (next 8-row group: 4 core matrices = 512 B),
// descriptor version 1 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (OZ_KC / 8) * 128;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D = F32 (1 << 4), A = B = BF16 (1 << 7,
// 1 << 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Waits for the phase of the given parity; false when kWaitLimitNs passed first.
// Each try_wait may suspend the thread for up to kSuspendHintNs (it resumes
// as soon as the phase completes), so waiting warps take few issue slots.
constexpr uint32_t kSuspendHintNs = 1000000;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (done) return true;
    if ((int64_t)(globaltimer_ns() - t0) > kWaitLimitNs) return false;
  }
}

// Chunk c of an item: reduction indices [f0, f1) of the flat index ko * K + k.
__device__ __forceinline__ void chunk_range(const GemmItem &it, int chunk, int64_t &f0, int64_t &f1) {
  const int ko0 = (int)((int64_t)chunk * it.Ko / it.ksplit);
  const int ko1 = (int)((int64_t)(chunk + 1) * it.Ko / it.ksplit);
  f0 = (int64_t)ko0 * it.K;
  f1 = (int64_t)ko1 * it.K;
  if (it.k_total >= 0 && f1 > it.k_total) f1 = it.k_total;
  if (f1 < f0) f1 = f0;
}

// The S slices of x on the grid of exponent E (|x| < 2^E) as FP32 values
// (each exactly a BF16 value): F = round(|x| 2^(8S - E)) written in balanced
// base-256 digits, F = sum_i d_i 256^(S-1-i) with d_0 in [0, 256] and d_i in
// [-128, 127] for i > 0, slice i = sign(x) d_i 2^(-8(i+1)).  Integer
// operations only, no carry chain: adding 128 to every digit position below
// the top (one 64-bit add of 0x80..80) makes byte i of the sum d_i + 128 for
// i > 0 and leaves d_0 above them.  The float of a digit comes from the bits
// of m_i = 1.5 2^(23 - 8(i+1)), whose unit in the last place is 2^(-8(i+1)):
// bits(m_i) + k is the float m_i + k 2^(-8(i+1)), minus m_i exactly; the
// -128 and the sign fold into that integer add.  Zeros and subnormals give
// zero slices.
template <int S>
__device__ __forceinline__ void oz_slice_values(double x, int E, float (&f)[S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long F = 0;
  if (ex != 0) {
    const int sh = 1075 + E - ex - 8 * S;  // |x| 2^(8S - E) = mant 2^(-sh)
    if (sh <= 0) F = mant << (-sh);         // only for S = 7 (then -sh <= 3)
    else if (sh < 60) F = (mant + (1ull << (sh - 1))) >> sh;
  }
  unsigned long long bias = 0;
#pragma unroll
  for (int j = 0; j < S - 1; ++j) bias |= 128ull << (8 * j);
  const unsigned long long G = F + bias;
  const uint32_t lo = (uint32_t)G, hi = (uint32_t)(G >> 32);
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int i = 1; i < S; ++i) {
    const int byte = S - 1 - i;  // byte of G holding digit i + 128 (S <= 6: bytes 0 .. 4)
    const uint32_t raw = ((byte < 4 ? lo : hi) >> (8 * (byte & 3))) & 255u;
    const uint32_t mb = ((uint32_t)(127 + 23 - 8 * (i + 1)) << 23) | 0x400000u;
    f[i] = __fsub_rn(__uint_as_float(neg ? mb + 128u - raw : mb - 128u + raw), __uint_as_float(mb));
  }
  const uint32_t d0 = (uint32_t)(G >> (8 * (S - 1)));  // [0, 256]
  constexpr uint32_t mb0 = ((uint32_t)(127 + 23 - 8) << 23) | 0x400000u;
  f[0] = __fsub_rn(__uint_as_float(neg ? mb0 - d0 : mb0 + d0), __uint_as_float(mb0));
}

// Slices i of neighbouring elements as one 32-bit word of BF16 values: the
// low half a's (the element at the lower address), the high half b's; a
// slice value has at most 9 significant bits, so its BF16 bits are the upper
// half of its FP32 bits.
__device__ __forceinline__ uint32_t bf16_pair(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// The four accumulators D_0 + D_1 + D_2 + D_3 (in grid units) as a
// double-float (h, l), then h + l scaled by 2^E as an FP64 bit pattern built
// with integer operations (df_to_f64_bits).  About 2^-47 relative.
__device__ __forceinline__ unsigned long long combine_to_f64(float d0, float d1, float d2, float d3, int E) {
  float s, e1, e2, h, l;
  two_sum(d0, d1, s, e1);
  two_sum(s, d2, s, e2);
  fast_two_sum(s, __fadd_rn(__fadd_rn(e1, e2), d3), h, l);
  return df_to_f64_bits(h, l, E);
}

// High 32 bits of |x| (sign cleared).  For non-negative doubles the order of
// these words is the order of the exponents, so the largest word of a row
// carries the row's largest exponent; a word >= kHiNonFinite is Inf or NaN.
// Integer operations only: compares and maxima of FP64 values would run on the
// FP64 pipe (about 1/62 of the FP32 rate on this GPU).
constexpr uint32_t kHiNonFinite = 0x7FF00000u;
__device__ __forceinline__ uint32_t abs_hi(double x) {
  return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
}
// Exponent E of a row with largest high word mh: every |x| of the row is
// below 2^E (|x| = 1.f 2^(ex-1023) < 2^(ex-1022)); zero and subnormal rows
// get E = 0 (their digits are zero), rows with Inf / NaN the marker.
__device__ __forceinline__ int row_exponent(uint32_t mh) {
  if (mh >= kHiNonFinite) return OZ_EXP_NONFINITE;
  const int ex = (int)(mh >> 20);
  return ex ? ex - 1022 : 0;
}

__device__ __forceinline__ int find_split(const GemmItem *items, int n, int blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].oz_split0 <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}


// ---------------------------------------------------------------------------
// split: one CTA (256 threads) per (item, operand, batch, 128-row tile, chunk)
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(256) oz_split_kernel(const GemmItem *__restrict__ items, int n_items,
                                                       const int *__restrict__ ranks) {
  __shared__ uint32_t red[2][OZ_M];
  __shared__ int64_t offt[256];
  __shared__ int sexp[OZ_M];
  const GemmItem &it = items[find_split(items, n_items, blockIdx.x)];
  int local = blockIdx.x - it.oz_split0;
  const int bat_a = (it.oz_share & 1) ? 1 : it.batch;  // an operand shared by the batch is sliced once
  const int per_a = (it.oz_pre & 1) ? 0 : bat_a * it.tc_tiles_m * it.ksplit;  // A given: B only
  const int op = local < per_a ? 0 : 1;
  if (op) local -= per_a;
  const int tiles = op ? it.tc_tiles_n : it.tc_tiles_m;
  const int tile = local % tiles;
  local /= tiles;
  const int chunk = local % it.ksplit;
  const int b = local / it.ksplit;
  const int rows = op ? eff_dim(it.N, it.n_ref, it.n_mult, ranks) : eff_dim(it.M, it.m_ref, 1, ranks);
  const int batch = eff_dim(it.batch, it.b_ref, it.b_mult, ranks);
  if (b >= batch) return;  // the GEMM skips these batches as well
  const double *X = static_cast<const double *>(op ? it.B : it.A) + (int64_t)b * (op ? it.sbb : it.sab);
  const int64_t sr = op ? it.sbn : it.sam, sk = op ? it.sbk : it.sak, sko = op ? it.sbko : it.sako;
  int64_t f0, f1;
  chunk_range(it, chunk, f0, f1);
  const int K = it.K > 0 ? it.K : 1;  // K = 0 leaves an empty chunk
  const int tid = threadIdx.x;
  const int nst = it.oz_stages;
  unsigned char *out = static_cast<unsigned char *>(op ? it.ozb : it.oza) +
                       ((((int64_t)b * tiles + tile) * it.ksplit + chunk) * nst) * S * (int64_t)OZ_BLK;
  int *Ex = (op ? it.oeb : it.oea) + ((int64_t)b * tiles * OZ_M + (int64_t)tile * OZ_M) * it.ksplit + chunk;
  const int row0 = op ? 0 : it.oz_row0;  // slicing-only items write their rows at an offset of the block
  // chunks hold at most 256 reduction indices, and a chunk starts at a
  // multiple of K: local index l of the chunk is (ko0 + l / K, l % K)
  const int len = (int)(f1 - f0);
  const int64_t ko0 = f0 / K;
  if (sk == 1) {
    // reduction index contiguous in memory: a group of lpr lanes per row
    // (lpr * 8 >= chunk length), lane i of a group holding the 8 indices
    // 8i .. 8i+7 of the chunk (coalesced loads, read once); the row maximum is
    // a reduction over the group and the digits come from the registers
    int lpr = 4;
    while (lpr * 8 < len) lpr <<= 1;
    const int rpw = 32 / lpr;  // rows a warp takes at a time
    const int warp = tid >> 5, lane = tid & 31;
    const int sub = lane / lpr, li = lane % lpr;
    int64_t off[8];  // element offsets of this lane's indices within a row
    bool in[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int l = li * 8 + e;
      const int qk = l / K;
      in[e] = l < len;
      off[e] = (int64_t)(l - qk * K) + (ko0 + qk) * sko;
    }
    const int q = li >> 2, kk0 = (li & 3) * 8;
    // rows beyond the operand (padding) feed only discarded outputs: not read, left unwritten
    auto load_row = [&](int r0, double (&dst)[8]) {
      const int grow = tile * OZ_M + r0 + sub;
      const bool live = r0 < OZ_M && grow < rows;
#pragma unroll
      for (int e = 0; e < 8; ++e) dst[e] = (live && in[e]) ? X[(int64_t)grow * sr + off[e]] : 0.0;
    };
    double vn[8];  // the next row's values, loaded while the current row is sliced
    load_row(warp * rpw, vn);
    for (int r0 = warp * rpw; r0 < OZ_M; r0 += 8 * rpw) {
      const int r = r0 + sub;
      const int grow = tile * OZ_M + r;
      const bool live = grow < rows;
      double v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = vn[e];
      load_row(r0 + 8 * rpw, vn);
      uint32_t mh = 0u;  // largest high word of |x|: its exponent field is the row's largest exponent
#pragma unroll
      for (int e = 0; e < 8; ++e) mh = max(mh, abs_hi(v[e]));
      for (int o = lpr >> 1; o > 0; o >>= 1) mh = max(mh, __shfl_xor_sync(0xffffffffu, mh, o));
      const bool bad = mh >= kHiNonFinite;
      const int E = row_exponent(mh);
      if (!live) continue;
      if (li == 0) Ex[(int64_t)(r + row0) * it.ksplit] = E;
      if (q >= nst) continue;
      uint32_t w[S][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float fa[S], fb[S];
        oz_slice_values<S>(bad ? 0.0 : v[e], E, fa);
        oz_slice_values<S>(bad ? 0.0 : v[e + 1], E, fb);
#pragma unroll
        for (int i = 0; i < S; ++i) w[i][e >> 1] = bf16_pair(fa[i], fb[i]);
      }
#pragma unroll
      for (int i = 0; i < S; ++i)
        *reinterpret_cast<uint4 *>(out + ((int64_t)q * S + i) * OZ_BLK + oz_off(r + row0, kk0)) =
            make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
    }
    return;
  }
  // element offsets of the chunk's indices within a row, once per block
  offt[tid] = (int64_t)(tid % K) * sk + (ko0 + tid / K) * sko;
  __syncthreads();
  const int r = tid & (OZ_M - 1), h = tid >> 7;
  const int grow = tile * OZ_M + r;
  const bool row_in = grow < rows;
  const double *Xr = X + (int64_t)grow * sr;
  // pass 1: largest high word of |x| over the row's chunk (NaN / Inf: exponent field all ones)
  uint32_t mh = 0u;
  if (row_in) {
    for (int l = h; l < len; l += 2) mh = max(mh, abs_hi(Xr[offt[l]]));
  }
  red[h][r] = mh;
  __syncthreads();
  if (h == 0) {
    const int E = row_exponent(max(red[0][r], red[1][r]));
    sexp[r] = E;
    if (row_in) Ex[(int64_t)(r + row0) * it.ksplit] = E;
  }
  __syncthreads();
  const int E = sexp[r];
  // pass 2: slices, 8 reduction indices of one row per step (16 bytes per slice);
  // padding rows (beyond the operand) feed only discarded outputs and stay unwritten
  if (!row_in) return;
  // the next step's 8 values are loaded while the current step is sliced
  auto load8 = [&](int g, double (&dst)[8]) {
    const int l0 = (g / (OZ_KC / 8)) * OZ_KC + (g % (OZ_KC / 8)) * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      dst[e] = (g < nst * (OZ_KC / 8) && l0 + e < len && E != OZ_EXP_NONFINITE) ? Xr[offt[l0 + e]] : 0.0;
  };
  double vn[8];
  load8(h, vn);
  for (int g = h; g < nst * (OZ_KC / 8); g += 2) {
    const int q = g / (OZ_KC / 8), kk0 = (g % (OZ_KC / 8)) * 8;
    double v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = vn[e];
    load8(g + 2, vn);
    uint32_t w[S][4];
#pragma unroll
    for (int i = 0; i < S; ++i) w[i][0] = w[i][1] = w[i][2] = w[i][3] = 0u;
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float fa[S], fb[S];
      oz_slice_values<S>(v[e], E, fa);
      oz_slice_values<S>(v[e + 1], E, fb);
#pragma unroll
      for (int i = 0; i < S; ++i) w[i][e >> 1] = bf16_pair(fa[i], fb[i]);
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
      *reinterpret_cast<uint4 *>(out + ((int64_t)q * S + i) * OZ_BLK + oz_off(r + row0, kk0)) =
          make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
  }
}

// ---------------------------------------------------------------------------
// GEMM: persistent CTAs (one per SM) walking the launch's tiles of 128 rows x
// 64 columns (per item: row tiles x column tiles x batch x chunk).
// ---------------------------------------------------------------------------
constexpr int OZ_TN = 64;       // columns of a GEMM tile
constexpr int OZ_STAGES = 3;    // stage buffers of the bulk-copy ring
constexpr uint32_t OZ_BLK_B = OZ_TN * OZ_KC * 2;  // bytes of a 64-row half of a slice block

struct TileInfo {
  const GemmItem *it;
  int tm, tn, b, chunk, nq;
  bool live;
};

__device__ __forceinline__ TileInfo tile_info(const GemmItem *items, const int *tile_item, const int *ranks, int t) {
  TileInfo ti;
  const GemmItem &it = items[tile_item[t]];
  ti.it = &it;
  int local = t - it.tc_tile0;
  const int tiles_n = (it.N + OZ_TN - 1) / OZ_TN;
  ti.tm = local % it.tc_tiles_m;
  local /= it.tc_tiles_m;
  ti.tn = local % tiles_n;
  local /= tiles_n;
  ti.b = local % it.batch;
  ti.chunk = local / it.batch;
  const int M = eff_dim(it.M, it.m_ref, 1, ranks);
  const int N = eff_dim(it.N, it.n_ref, it.n_mult, ranks);
  const int batch = eff_dim(it.batch, it.b_ref, it.b_mult, ranks);
  ti.live = ti.tm * OZ_M < M && ti.tn * OZ_TN < N && ti.b < batch;
  int64_t f0, f1;
  chunk_range(it, ti.chunk, f0, f1);
  ti.nq = (int)((f1 - f0 + OZ_KC - 1) / OZ_KC);
  return ti;
}

// Accumulators per TMEM buffer: D_0, D_1 and D_{>=2} for up to 5 slices (the
// merged sum rounds at about 2^-40 of the scale, the level of the slices
// themselves); D_0, D_1, D_2 and D_{>=3} for 6 slices (about 2^-48).
template <int S>
struct OzAcc {
  static constexpr int n = S >= 6 ? 4 : (S < 3 ? S : 3);
};

template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const GemmItem *__restrict__ items,
                                                                const int *__restrict__ tile_item, int total_tiles,
                                                                const int *__restrict__ ranks) {
  constexpr int NACC = OzAcc<S>::n;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES], bar_acc_full[2], bar_acc_empty[2],
      bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t STA = S * OZ_BLK, STB = S * OZ_BLK_B, STG = STA + STB;  // bytes of one stage
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == OZ_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == OZ_EPI_THREADS) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_empty[i])) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_acc_full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar_acc_empty[i])), "r"(OZ_EPI_THREADS)
                   : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == OZ_PROD_WARP) {
    // ---- producer: the stages of every live tile, through the ring ----
    if (lane == 0) {
      int g = 0;  // stages issued so far
      for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const TileInfo ti = tile_info(items, tile_item, ranks, t);
        if (!ti.live) continue;
        const GemmItem &it = *ti.it;
        const int share = it.oz_share;
        const int ba = (share & 1) ? 0 : ti.b, bb = (share & 2) ? 0 : ti.b;
        const unsigned char *gA = static_cast<const unsigned char *>(it.oza) +
                                  ((((int64_t)ba * it.tc_tiles_m + ti.tm) * it.ksplit + ti.chunk) * it.oz_stages) * (int64_t)STA;
        const unsigned char *gB = static_cast<const unsigned char *>(it.ozb) +
                                  ((((int64_t)bb * it.tc_tiles_n + (ti.tn >> 1)) * it.ksplit + ti.chunk) * it.oz_stages) *
                                      (int64_t)STA +
                                  (ti.tn & 1) * OZ_BLK_B;
        for (int q = 0; q < ti.nq; ++q, ++g) {
          const int slot = g % OZ_STAGES;
          if (*(volatile int *)&abort_flag) break;
          if (g >= OZ_STAGES && !mbar_wait(smem_addr(&bar_empty[slot]), (uint32_t)((g / OZ_STAGES - 1) & 1))) {
            atomicOr(&g_oz_status, 1u);
            atomicExch(&abort_flag, 1);
            break;
          }
          unsigned char *sA = sm + slot * STG;
          const uint32_t fb = smem_addr(&bar_full[slot]);
          asm volatile(
              "{\n\t.reg .b64 st;\n\t"
              "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(fb),
              "r"(STG)
              : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_addr(sA)),
              "l"(gA + (int64_t)q * STA), "r"(STA), "r"(fb)
              : "memory");
#pragma unroll
          for (int i = 0; i < S; ++i)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(sA + STA + i * OZ_BLK_B)),
                "l"(gB + (int64_t)q * STA + i * OZ_BLK), "r"(OZ_BLK_B), "r"(fb)
                : "memory");
        }
        if (*(volatile int *)&abort_flag) break;
      }
    }
  } else if (warp == OZ_MMA_WARP) {
    // ---- MMA issue: per tile, products (i, j), i + j <= S - 1, into accumulator
    // min(i + j, NACC - 1) of the tile's TMEM buffer (two buffers of NACC x 64 columns) ----
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(OZ_M, OZ_TN);
      int g = 0, n = 0;  // stages consumed, live tiles
      for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const TileInfo ti = tile_info(items, tile_item, ranks, t);
        if (!ti.live) continue;
        const int tb = n & 1;
        if (*(volatile int *)&abort_flag) break;
        if (n >= 2 && !mbar_wait(smem_addr(&bar_acc_empty[tb]), (uint32_t)((n / 2 - 1) & 1))) {
          atomicOr(&g_oz_status, 1u);
          atomicExch(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)(tb * NACC * OZ_TN);
        bool ok = true;
        for (int q = 0; q < ti.nq; ++q, ++g) {
          const int slot = g % OZ_STAGES;
          if (*(volatile int *)&abort_flag || !mbar_wait(smem_addr(&bar_full[slot]), (uint32_t)((g / OZ_STAGES) & 1))) {
            atomicOr(&g_oz_status, 1u);
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_addr(sm + slot * STG), b0 = a0 + STA;
#pragma unroll
          for (int ks = 0; ks < OZ_KC / 16; ++ks) {
#pragma unroll
            for (int s = S - 1; s >= 0; --s) {  // smallest products first
#pragma unroll
              for (int i = 0; i <= s; ++i) {
                const int j = s - i;
                const int acc = s < NACC - 1 ? s : NACC - 1;
                const uint64_t da = smem_desc(a0 + i * OZ_BLK + ks * 256);
                const uint64_t db = smem_desc(b0 + j * OZ_BLK_B + ks * 256);
                // the first product into an accumulator of the tile overwrites it
                const bool first = q == 0 && ks == 0 && i == 0 && (acc < NACC - 1 || s == S - 1);
                const uint32_t en = first ? 0u : 1u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dbase + (uint32_t)(acc * OZ_TN)),
                    "l"(da), "l"(db), "r"(idesc), "r"(en)
                    : "memory");
              }
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_addr(&bar_empty[slot]))
                       : "memory");
        }
        if (!ok) break;
        // the tile's accumulators are complete when this commit arrives
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&bar_acc_full[tb]))
                     : "memory");
        ++n;
      }
      // tracks every MMA issued above (also after an abort): the TMEM may be freed once it arrives
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar_done))
                   : "memory");
    }
  } else {
    // ---- epilogue: warps 0-15; warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile
    // rows); the tile's 8-column chunks go to the four warps of a lane quarter
    // in turn, so that a tile with 32 live columns keeps all sixteen busy ----
    const int quad = warp & 3, part = warp >> 2;
    int n = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
      const TileInfo ti = tile_info(items, tile_item, ranks, t);
      if (!ti.live) continue;
      const GemmItem &it = *ti.it;
      const int tb = n & 1;
      bool ok = mbar_wait(smem_addr(&bar_acc_full[tb]), (uint32_t)((n / 2) & 1));
      if (!ok) {
        atomicOr(&g_oz_status, 1u);
        atomicExch(&abort_flag, 1);
      }
      const bool valid = __all_sync(0xffffffffu, ok) && !*(volatile int *)&abort_flag;
      if (!valid) break;  // warp-uniform
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the item's fields in registers
      const int M = eff_dim(it.M, it.m_ref, 1, ranks);
      const int N = eff_dim(it.N, it.n_ref, it.n_mult, ranks);
      const int share = it.oz_share, ksplit = it.ksplit;
      const int ba = (share & 1) ? 0 : ti.b, bb = (share & 2) ? 0 : ti.b;
      const int row = ti.tm * OZ_M + quad * 32 + lane;
      const int n0 = ti.tn * OZ_TN;
      const int ncols = (N - n0 < OZ_TN) ? N - n0 : OZ_TN;  // live columns of the tile
      const int64_t Mpad = (int64_t)it.tc_tiles_m * OZ_M, Npad = (int64_t)it.tc_tiles_n * OZ_N;
      const int ea = it.oea[((int64_t)ba * Mpad + row) * ksplit + ti.chunk];
      // column exponents: lane l holds those of columns n0 + l and n0 + 32 + l
      // (padding columns, below the padded width, hold unused values)
      const int *Eb = it.oeb + ((int64_t)bb * Npad + n0) * ksplit + ti.chunk;
      const int eb_lo = Eb[(int64_t)lane * ksplit], eb_hi = Eb[(int64_t)(lane + 32) * ksplit];
      const double alpha = it.alpha, beta = it.beta;
      const int64_t scm = it.scm, scn = it.scn, ldp = it.M;
      double *Cp = static_cast<double *>(it.C) + (int64_t)ti.b * it.scb;
      double *Pp = ksplit > 1
                       ? static_cast<double *>(it.part) + ((int64_t)ti.chunk * it.batch + ti.b) * (int64_t)it.M * it.N
                       : nullptr;
      const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tb * NACC * OZ_TN);
      // how the results are stored, decided once per tile so that no FP64
      // instruction runs per element where none is needed: 0 split-K partial
      // (alpha and beta are applied by the reduction), 1 C = +-AB (the sign as
      // a bit flip), 2 C = +-AB + beta C (one FP64 FMA), 3 any other alpha
      const bool unit = alpha == 1.0 || alpha == -1.0;
      const int smode = Pp ? 0 : (unit ? (beta == 0.0 ? 1 : 2) : 3);
      const unsigned long long flip = (!Pp && alpha == -1.0) ? 0x8000000000000000ull : 0ull;
      const bool row_ok = row < M;
      double *prow = Pp ? Pp + row : Cp + (int64_t)row * scm;
      const int64_t cstride = Pp ? ldp : scn;
      // chunks of 8 columns (a smaller unrolled body), dealt to the four warps of
      // each TMEM lane quarter in turn
      constexpr int EC = 8;
      for (int c0 = part * EC; c0 < ncols; c0 += 4 * EC) {
        uint32_t v[4][EC];
        if (ti.nq > 0) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (a >= NACC) {
#pragma unroll
              for (int j = 0; j < EC; ++j) v[a][j] = 0u;
              continue;
            }
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3]), "=r"(v[a][4]), "=r"(v[a][5]),
                           "=r"(v[a][6]), "=r"(v[a][7])
                         : "r"(trow + (uint32_t)(a * OZ_TN + c0)));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < EC; ++j) v[a][j] = 0u;
        }
        const int eb_src = c0 < 32 ? eb_lo : eb_hi;
        unsigned long long w[EC];
#pragma unroll
        for (int j = 0; j < EC; ++j) {
          const int eb = __shfl_sync(0xffffffffu, eb_src, (c0 & 31) + j);  // the same column for every lane
          w[j] = (eb == OZ_EXP_NONFINITE || ea == OZ_EXP_NONFINITE)
                     ? 0x7FF8000000000000ull
                     : combine_to_f64(__uint_as_float(v[0][j]), __uint_as_float(v[1][j]),
                                      __uint_as_float(v[2][j]), __uint_as_float(v[3][j]), ea + eb);
        }
        if (!row_ok) continue;
        const int jn = ncols - c0 < EC ? ncols - c0 : EC;
        double *pc = prow + (int64_t)(n0 + c0) * cstride;
        if (smode <= 1) {
#pragma unroll
          for (int j = 0; j < EC; ++j)
            if (j < jn) pc[(int64_t)j * cstride] = __longlong_as_double((long long)(w[j] ^ flip));
        } else {
          // all loads of C before the first store (the stores could alias them
          // for all the compiler knows, which would serialise the loads)
          double cv[EC];
#pragma unroll
          for (int j = 0; j < EC; ++j) cv[j] = j < jn ? pc[(int64_t)j * cstride] : 0.0;
          if (smode == 2) {
#pragma unroll
            for (int j = 0; j < EC; ++j)
              if (j < jn) pc[(int64_t)j * cstride] = fma(beta, cv[j], __longlong_as_double((long long)(w[j] ^ flip)));
          } else {
#pragma unroll
            for (int j = 0; j < EC; ++j) {
              if (j >= jn) continue;
              const double o = alpha * __longlong_as_double((long long)w[j]);
              pc[(int64_t)j * cstride] = beta != 0.0 ? fma(beta, cv[j], o) : o;
            }
          }
        }
      }
      // every load of this tile's buffer has completed (wait::ld above): hand it back
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                       smem_addr(&bar_acc_empty[tb]))
                   : "memory");
      ++n;
    }
  }
  // all MMAs complete (bounded wait) before the TMEM is freed
  if (warp == OZ_MMA_WARP) {
    if (lane == 0 && !mbar_wait(smem_addr(&bar_done), 0u)) atomicOr(&g_oz_status, 1u);
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == OZ_MMA_WARP) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

template <int S>
cudaError_t launch_split_s(const GemmItem *d_items, int n_items, int split_blocks, const int *d_ranks, cudaStream_t s) {
  oz_split_kernel<S><<<split_blocks, 256, 0, s>>>(d_items, n_items, d_ranks);
  count_launch();
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_mma_s(const GemmItem *d_items, const int *tile_item, int tiles, const int *d_ranks, cudaStream_t s) {
  const size_t smem = OZ_STAGES * (size_t)S * (OZ_BLK + OZ_BLK_B) + 1024;
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = kSmCount;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = tiles < sms ? tiles : sms;  // persistent: one CTA per SM (it holds all 512 TMEM columns)
  oz_gemm_kernel<S><<<grid, OZ_THREADS, smem, s>>>(d_items, tile_item, tiles, d_ranks);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int oz_tile_m() { return OZ_M; }
int oz_tile_n() { return OZ_N; }
int oz_gemm_tile_n() { return OZ_TN; }
int oz_stage_k() { return OZ_KC; }
int oz_block_bytes() { return (int)OZ_BLK; }

cudaError_t launch_oz_split(const GemmItem *d_items, int n_items, int split_blocks, const int *d_ranks, int slices,
                            cudaStream_t s) {
  if (n_items <= 0 || split_blocks <= 0) return cudaSuccess;
  switch (slices) {
    case 2: return launch_split_s<2>(d_items, n_items, split_blocks, d_ranks, s);
    case 3: return launch_split_s<3>(d_items, n_items, split_blocks, d_ranks, s);
    case 4: return launch_split_s<4>(d_items, n_items, split_blocks, d_ranks, s);
    case 5: return launch_split_s<5>(d_items, n_items, split_blocks, d_ranks, s);
    case 6: return launch_split_s<6>(d_items, n_items, split_blocks, d_ranks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_oz_gemm(const GemmItem *d_items, const int *tile_item, int n_items, int tiles, const int *d_ranks,
                           bool any_split, int slices, cudaStream_t s) {
  if (n_items <= 0 || tiles <= 0) return cudaSuccess;
  if (!tile_item) return cudaErrorInvalidValue;
  cudaError_t e;
  switch (slices) {
    case 2: e = launch_mma_s<2>(d_items, tile_item, tiles, d_ranks, s); break;
    case 3: e = launch_mma_s<3>(d_items, tile_item, tiles, d_ranks, s); break;
    case 4: e = launch_mma_s<4>(d_items, tile_item, tiles, d_ranks, s); break;
    case 5: e = launch_mma_s<5>(d_items, tile_item, tiles, d_ranks, s); break;
    case 6: e = launch_mma_s<6>(d_items, tile_item, tiles, d_ranks, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  if (any_split) return launch_gemm_reduce_f64(d_items, n_items, d_ranks, s);
  return cudaSuccess;
}

unsigned oz_take_status() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_oz_status, sizeof(v)) != cudaSuccess) return ~0u;
  if (v) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_oz_status, &z, sizeof(z)) != cudaSuccess) return ~0u;
  }
  return v;
}

}  // namespace htgb
