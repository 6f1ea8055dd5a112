// api.cu -- the C-ABI of htgb.h: dimension tree, HT container, HT addition,
// and the plan builder that turns orthogonalization / Gramians / eigen /
// rank selection / projection into a short sequence of batched launches.
//
// A "plan" is built on the host for one call: every launch walks a device
// array of work items (internal.h).  Workspace pointers are recorded as
// tagged offsets while the plan is built, then relocated once the workspace
// is allocated; items and small metadata arrays are uploaded with a single
// copy.  All work is stream-ordered on the tensor's stream.
#include <algorithm>
#include <climits>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "htgb.h"
#include "internal.h"
#include "gemm_tune.h"

using namespace htgb;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static ht_status fail(ht_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

#define HT_CU(call)                                                                           \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(HT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define HT_TRY(expr)                 \
  do {                               \
    ht_status s_ = (expr);           \
    if (s_ != HT_OK) return s_;      \
  } while (0)

// ---------------------------------------------------------------------------
// tracing: launch count and CUDA-event timing per kernel family
// ---------------------------------------------------------------------------
namespace {
std::atomic<int64_t> g_launches{0};
unsigned g_prof_mask = 0;
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double flops;
};
std::vector<ProfRec> g_prof_open, g_prof_done;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t get_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

namespace htgb {
void count_launch(int n) { g_launches += n; }
void prof_begin(int kind, cudaStream_t s) {
  if (!(g_prof_mask & (1u << kind))) return;
  ProfRec r{kind, get_event(), get_event(), 0.0};
  cudaEventRecord(r.a, s);
  g_prof_open.push_back(r);
}
void prof_end(int kind, cudaStream_t s, double flops) {
  if (!(g_prof_mask & (1u << kind))) return;
  for (size_t i = g_prof_open.size(); i-- > 0;) {
    if (g_prof_open[i].kind == kind) {
      cudaEventRecord(g_prof_open[i].b, s);
      g_prof_open[i].flops = flops;
      g_prof_done.push_back(g_prof_open[i]);
      g_prof_open.erase(g_prof_open.begin() + i);
      return;
    }
  }
}
}  // namespace htgb

// ---------------------------------------------------------------------------
// tree (Sec. 2.1)
// ---------------------------------------------------------------------------
struct ht_tree {
  int d = 0, nn = 0, max_depth = 0, max_height = 0;
  std::vector<int> lo, hi, par, s1, s2, depth, height, leaf_node;
};

static int tree_rec(ht_tree *T, int lo, int hi, int parent, int depth) {
  int id = (int)T->lo.size();
  T->lo.push_back(lo);
  T->hi.push_back(hi);
  T->par.push_back(parent);
  T->depth.push_back(depth);
  T->s1.push_back(-1);
  T->s2.push_back(-1);
  T->height.push_back(0);
  if (lo != hi) {
    int last1 = (lo + hi + 1) / 2 - 1;  // eq. "balanced", 0-based
    int a = tree_rec(T, lo, last1, id, depth + 1);
    int b = tree_rec(T, last1 + 1, hi, id, depth + 1);
    T->s1[id] = a;
    T->s2[id] = b;
    T->height[id] = 1 + std::max(T->height[a], T->height[b]);
  }
  return id;
}

static void tree_init(ht_tree *T, int d) {
  T->d = d;
  tree_rec(T, 0, d - 1, -1, 0);
  T->nn = (int)T->lo.size();
  T->leaf_node.assign(d, -1);
  for (int t = 0; t < T->nn; ++t) {
    if (T->s1[t] < 0) T->leaf_node[T->lo[t]] = t;
    T->max_depth = std::max(T->max_depth, T->depth[t]);
  }
  T->max_height = T->height[0];
}

static inline bool is_leaf(const ht_tree &T, int t) { return T.s1[t] < 0; }

// ---------------------------------------------------------------------------
// container (Sec. 2.2)
// ---------------------------------------------------------------------------
struct ht_tensor {
  ht_tree tr;
  std::vector<int64_t> n;
  std::vector<int> k;     // current ranks (host copy, valid if ranks_ok)
  std::vector<int> cap;   // slot capacities
  std::vector<int64_t> slot;  // element offset of each node's slot, nn+1 entries
  int dtype = HT_F64;
  size_t esz = 8;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  int *d_ranks = nullptr;
  bool ranks_ok = true;
  bool orthogonal = false;
};

static int64_t node_elems(const ht_tree &T, const std::vector<int64_t> &n, const std::vector<int> &k, int t) {
  if (is_leaf(T, t)) return n[T.lo[t]] * (int64_t)k[t];
  int64_t kt = (t == 0) ? 1 : k[t];
  return kt * k[T.s1[t]] * k[T.s2[t]];
}

static void *node_ptr(const ht_tensor *x, int t) { return x->arena + x->slot[t] * x->esz; }

static ht_status sync_ranks(ht_tensor *x) {
  if (x->ranks_ok) return HT_OK;
  HT_CU(cudaMemcpyAsync(x->k.data(), x->d_ranks, sizeof(int) * x->tr.nn, cudaMemcpyDeviceToHost, x->stream));
  HT_CU(cudaStreamSynchronize(x->stream));
  x->k[0] = 1;
  x->ranks_ok = true;
  return HT_OK;
}

static void set_pool_threshold() {
  static bool done = false;
  if (done) return;
  done = true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}

static ht_status tensor_alloc(const ht_tree &tr, const int64_t *n, const int *ranks, int dtype, cudaStream_t stream,
                              ht_tensor **out) {
  set_pool_threshold();
  ht_tensor *x = new ht_tensor();
  x->tr = tr;
  x->n.assign(n, n + tr.d);
  x->k.assign(ranks, ranks + tr.nn);
  x->k[0] = 1;
  x->cap = x->k;
  x->dtype = dtype;
  x->esz = (dtype == HT_F64) ? 8 : 4;
  x->stream = stream;
  x->slot.assign(tr.nn + 1, 0);
  int64_t o = 0;
  for (int t = 0; t < tr.nn; ++t) {
    x->slot[t] = o;
    o += node_elems(tr, x->n, x->cap, t);
  }
  x->slot[tr.nn] = o;
  cudaError_t e = cudaMallocAsync((void **)&x->arena, std::max<int64_t>(o, 1) * x->esz, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&x->d_ranks, sizeof(int) * tr.nn, stream);
  if (e != cudaSuccess) {
    if (x->arena) cudaFreeAsync(x->arena, stream);
    delete x;
    return fail(HT_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(x->d_ranks, x->k.data(), sizeof(int) * tr.nn, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  // the host rank vector must stay alive until the copy has been staged
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  *out = x;
  return HT_OK;
}

static ht_status upload_ranks(ht_tensor *x) {
  x->k[0] = 1;
  HT_CU(cudaMemcpyAsync(x->d_ranks, x->k.data(), sizeof(int) * x->tr.nn, cudaMemcpyHostToDevice, x->stream));
  HT_CU(cudaStreamSynchronize(x->stream));
  x->ranks_ok = true;
  return HT_OK;
}

// ---------------------------------------------------------------------------
// plan builder
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t TAG_P = 1ull << 62;  // persistent workspace
constexpr uint64_t TAG_S = 1ull << 61;  // per-phase scratch workspace
constexpr uint64_t TAG_M = 1ull << 60;  // metadata appended to the item upload
constexpr uint64_t TAG_L = 1ull << 59;  // per-launch scratch (split-K partials, tensor-core slices)
constexpr uint64_t TAG_MASK = (1ull << 59) - 1;

enum LKind { L_GEMM, L_QR, L_EIG, L_COPY, L_COMPACT, L_RANKS, L_CHOL };

struct Launch {
  LKind kind;
  size_t off = 0;  // byte offset of the first item in the upload
  int n = 0;       // items
  int tiles = 0;   // GEMM: total tiles
  int max_m = 0, max_n = 0;
  bool split = false;
  int node = -1;
  double flops = 0.0;  // algorithmic flops of the launch (literal, i.e. maximal, dims)
  int tc_tiles = 0;    // GEMM: tiles of the tensor-core kernel (mixed path)
  int oz_split = 0;    // GEMM: CTAs of the tensor-core path's split launch
  int oz_slices = 0;   // GEMM: BF16 slices per operand (mixed path)
  double split_bytes = 0.0;  // GEMM (mixed path): algorithmic bytes of the split (operands read, slices written)
  std::vector<int> tile_item;  // GEMM (mixed path): the launch's item of every tensor-core tile
  const int *tile_tab = nullptr;  // the same, uploaded with the metadata (tagged pointer)
  const void *ranks = nullptr;  // tagged pointer to the rank array used by the launch
  void *scratch = nullptr;      // eig scratch (tagged)
  int variant = 0;              // GEMM: SIMT tile shape (gemm_tile_shape)
  bool comp = true;             // GEMM: compensated FP32 accumulation
  bool df = false;              // GEMM: double-float accumulation, FP64 output (square-root Gramians)
  int uniform = 0;              // GEMM: tiles of every item when all items have the same count (else 0)
};

template <typename P>
inline P *tagp(uint64_t tag, size_t off) {
  return reinterpret_cast<P *>(tag | (uint64_t)off);
}

// Mixed path: products per exactness chunk of the tensor-core kernel (k_oz.cu)
// and its default number of BF16 slices per FP64 operand (5 slices: about
// 2^-40 of the row scale per product).
constexpr int kOzChunk = 256;
constexpr int kOzSlices = 5;
// the reduced-Gramian contractions: 6 slices (about 1e-14 of the row scale).
// Their eigenvalues decide the ranks; the eps cut of the deep workload sits
// at eigenvalues near 1e-15 of the largest, where 5 slices leave noise that
// moves the cut.
constexpr int kOzSlicesGram = 6;

struct Plan {
  std::vector<uint8_t> items;
  std::vector<uint8_t> meta;
  std::vector<Launch> launches;
  size_t p_bytes = 0, s_bytes = 0, s_peak = 0, l_bytes = 0, l_peak = 0;
  bool node_sched = false;
  bool sqrt_gram = false;  // Gramians from square-root factors (HT_PREC_FP32_SQRT)
  bool mixed = false;      // HT_PREC_MIXED: contractions on the tensor cores (k_oz.cu)
  int panel = 64;          // TSQR panel width (columns factored by the Householder blocks at once)
  int oz_slices = kOzSlices;
  int qr_kernel = 0;       // TSQR block kernel choice (ht_trunc_opts.qr_kernel)
  int dtype = HT_F64;
  size_t esz = 8;
  std::string err;  // set by a planning step that cannot handle its input

  // --- workspace ---
  template <typename P>
  P *palloc(size_t count) {
    size_t off = (p_bytes + 255) & ~size_t(255);
    p_bytes = off + count * sizeof(P);
    return tagp<P>(TAG_P, off);
  }
  void *palloc_bytes(size_t bytes) {
    size_t off = (p_bytes + 255) & ~size_t(255);
    p_bytes = off + bytes;
    return tagp<void>(TAG_P, off);
  }
  void *salloc_bytes(size_t bytes) {
    size_t off = (s_bytes + 255) & ~size_t(255);
    s_bytes = off + bytes;
    s_peak = std::max(s_peak, s_bytes);
    return tagp<void>(TAG_S, off);
  }
  void sreset() { s_bytes = 0; }
  // scratch that lives for one launch only (the next launch reuses it)
  void *lalloc_bytes(size_t bytes) {
    size_t off = (l_bytes + 255) & ~size_t(255);
    l_bytes = off + bytes;
    l_peak = std::max(l_peak, l_bytes);
    return tagp<void>(TAG_L, off);
  }
  template <typename P>
  P *mpush(const P *data, size_t count) {
    size_t off = (meta.size() + 15) & ~size_t(15);
    meta.resize(off + count * sizeof(P));
    if (count) memcpy(meta.data() + off, data, count * sizeof(P));
    return tagp<P>(TAG_M, off);
  }

  // --- launches ---
  void begin(LKind kind, const void *ranks = nullptr) {
    Launch L;
    L.kind = kind;
    L.oz_slices = oz_slices;
    l_bytes = 0;
    size_t off = (items.size() + 15) & ~size_t(15);
    items.resize(off);
    L.off = off;
    L.ranks = ranks;
    launches.push_back(L);
  }
  Launch &cur() { return launches.back(); }
  template <typename I>
  void push_item(const I &it, int node) {
    Launch &L = cur();
    if (node_sched && L.n > 0 && L.node != node) {
      LKind k = L.kind;
      const void *r = L.ranks;
      const bool df = L.df;
      const int sl = L.oz_slices;
      begin(k, r);
      cur().df = df;
      cur().oz_slices = sl;
    }
    Launch &M = cur();
    M.node = node;
    size_t off = items.size();
    items.resize(off + sizeof(I));
    memcpy(items.data() + off, &it, sizeof(I));
    M.n++;
  }
  void gemm(GemmItem g, int node) {
    if (g.ksplit < 1) g.ksplit = 1;
    if (g.batch < 1) g.batch = 1;
    if (g.Ko < 1) g.Ko = 1;
    if (g.n_mult < 1) g.n_mult = 1;
    if (g.b_mult < 1) g.b_mult = 1;
    if (g.M <= 0 || g.N <= 0) return;
    {
      // the SIMT kernel keeps a thread's in-tile element offsets in 32 bits
      const int64_t kk = 63;  // largest in-tile k index of any tile shape, with margin
      const int64_t oa = (int64_t)(g.M - 1) * std::llabs(g.sam) + kk * std::llabs(g.sak);
      const int64_t ob = (int64_t)(g.N - 1) * std::llabs(g.sbn) + kk * std::llabs(g.sbk);
      if (oa >= (int64_t)INT32_MAX || ob >= (int64_t)INT32_MAX)
        err = "contraction operand spans 2^31 elements or more within one tile row/column";
    }
    if ((dtype == HT_F32 || mixed) && g.M < 128 && g.N >= 128 && g.m_ref < 0 && g.n_ref < 0) {
      // C^T = B^T A^T puts the long dimension on the 128-row MMA tiles
      std::swap(g.A, g.B);
      const int64_t am = g.sam, ak = g.sak, ako = g.sako, ab = g.sab;
      g.sam = g.sbn; g.sak = g.sbk; g.sako = g.sbko; g.sab = g.sbb;
      g.sbn = am; g.sbk = ak; g.sbko = ako; g.sbb = ab;
      std::swap(g.scm, g.scn);
      std::swap(g.M, g.N);
    }
    if (mixed) {
      // exactness chunks of at most kOzChunk products: split the outer range
      if (g.K > kOzChunk) {
        err = "mixed path: a contraction with more than " + std::to_string(kOzChunk) + " products per outer index";
        return;
      }
      const int per = std::max(1, kOzChunk / g.K);
      g.ksplit = std::max(g.ksplit, (g.Ko + per - 1) / per);
    }
    g.tiles_m = (g.M + 63) / 64;
    g.tiles_n = (g.N + 63) / 64;
    g.tc_tiles_m = (g.M + 127) / 128;
    g.tc_tiles_n = (g.N + 127) / 128;
    if (node_sched && cur().n > 0 && cur().node != node) {
      LKind k = cur().kind;
      const void *r = cur().ranks;
      const bool df = cur().df;
      const int sl = cur().oz_slices;
      begin(k, r);
      cur().df = df;
      cur().oz_slices = sl;
    }
    Launch &L = cur();
    const bool slice_only = mixed && (g.oz_pre & 2);  // operand A's slices only: no tiles, no output
    g.tile0 = L.tiles;
    L.tiles += g.tiles_m * g.tiles_n * g.batch * g.ksplit;
    g.tc_tile0 = L.tc_tiles;
    if (!slice_only)
      L.tc_tiles += g.tc_tiles_m * ((g.N + oz_gemm_tile_n() - 1) / oz_gemm_tile_n()) * g.batch * g.ksplit;
    if (mixed) {
      // BF16 slice blocks (stages of oz_stage_k() reduction indices) and
      // exponents, for this launch only; an operand that every batch entry
      // shares (zero batch stride) is sliced once
      const int max_ko = (g.Ko + g.ksplit - 1) / g.ksplit;
      const int sk = oz_stage_k();
      g.oz_stages = (g.K * max_ko + sk - 1) / sk;
      g.oz_share = (g.batch > 1 && g.sab == 0 ? 1 : 0) | (g.batch > 1 && g.sbb == 0 ? 2 : 0);
      const int ba = (g.oz_share & 1) ? 1 : g.batch, bb = (g.oz_share & 2) ? 1 : g.batch;
      const size_t blk = (size_t)oz_block_bytes() * L.oz_slices * g.oz_stages * g.ksplit;
      // given slices (oz_pre bit 0, made by an earlier slicing-only launch of the
      // same chunk layout) are used as they are; a slicing-only item has no B
      // and writes A's slices to the buffers it brings
      const bool make_a = !(g.oz_pre & 1), make_b = !(g.oz_pre & 2);
      if (make_a && !slice_only) {
        g.oza = lalloc_bytes(blk * ba * g.tc_tiles_m);
        g.oea = static_cast<int *>(lalloc_bytes(sizeof(int) * (size_t)ba * g.tc_tiles_m * oz_tile_m() * g.ksplit));
      }
      if (make_b) {
        g.ozb = lalloc_bytes(blk * bb * g.tc_tiles_n);
        g.oeb = static_cast<int *>(lalloc_bytes(sizeof(int) * (size_t)bb * g.tc_tiles_n * oz_tile_n() * g.ksplit));
      }
      g.oz_split0 = L.oz_split;
      L.oz_split += g.ksplit * ((make_a ? ba * g.tc_tiles_m : 0) + (make_b ? bb * g.tc_tiles_n : 0));
      if (!slice_only) {
        const int tiles_here = g.tc_tiles_m * ((g.N + oz_gemm_tile_n() - 1) / oz_gemm_tile_n()) * g.batch * g.ksplit;
        L.tile_item.insert(L.tile_item.end(), (size_t)tiles_here, L.n);
      }
      // algorithmic bytes: the FP64 operands read once, their slices written once
      const double red = (double)g.K * g.Ko;
      L.split_bytes += red * ((make_a ? (double)ba * g.M : 0.0) + (make_b ? (double)bb * g.N : 0.0)) *
                       (8.0 + 2.0 * L.oz_slices);
    }
    if (slice_only) {
      push_item(g, node);
      return;
    }
    const double fl = 2.0 * g.M * g.N * (double)g.K * g.Ko * g.batch;
    L.flops += fl;
    if (g.ksplit > 1) {
      L.split = true;
      g.part = lalloc_bytes((size_t)g.ksplit * g.batch * g.M * g.N * (L.df ? sizeof(double) : esz));
    }
    push_item(g, node);
  }
  void qr(const QrItem &q, int node) {
    push_item(q, node);
    Launch &L = cur();
    L.max_m = std::max(L.max_m, q.m);
    L.max_n = std::max(L.max_n, q.n);
    // Householder QR with the explicit Q factor: 4 m n^2 - 4 n^3 / 3
    L.flops += 4.0 * q.m * (double)q.n * q.n - 4.0 / 3.0 * (double)q.n * q.n * q.n;
  }
  void eig(const EigItem &e, int node) {
    push_item(e, node);
    cur().max_n = std::max(cur().max_n, e.k);
    cur().flops += 9.0 * (double)e.k * e.k * e.k;  // symmetric eigendecomposition with vectors
  }
  void copy(const CopyItem &c, int node) { push_item(c, node); }
  void compact(const CompactItem &c, int node) { push_item(c, node); }
  void rank(const RankItem &r, int node) { push_item(r, node); }
  void chol(const CholItem &c, int node) { push_item(c, node); }
};

// Launch scratch sits right after the phase scratch; its base is found from
// the phase scratch's base and size (g_lscratch_off, set by prepare_plan).
thread_local size_t g_lscratch_off = 0;
inline void *reloc(const void *p, char *pb, char *sb, char *mb) {
  uint64_t u = (uint64_t)p;
  if (u & TAG_P) return pb + (u & TAG_MASK);
  if (u & TAG_S) return sb + (u & TAG_MASK);
  if (u & TAG_M) return mb + (u & TAG_MASK);
  if (u & TAG_L) return sb + g_lscratch_off + (u & TAG_MASK);
  return const_cast<void *>(p);
}

template <typename I>
void reloc_items(uint8_t *base, int n, char *pb, char *sb, char *mb);

template <>
void reloc_items<GemmItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  GemmItem *it = reinterpret_cast<GemmItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].A = reloc(it[i].A, pb, sb, mb);
    it[i].B = reloc(it[i].B, pb, sb, mb);
    it[i].C = reloc(it[i].C, pb, sb, mb);
    it[i].part = reloc(it[i].part, pb, sb, mb);
    it[i].oza = reloc(it[i].oza, pb, sb, mb);
    it[i].ozb = reloc(it[i].ozb, pb, sb, mb);
    it[i].oea = static_cast<int *>(reloc(it[i].oea, pb, sb, mb));
    it[i].oeb = static_cast<int *>(reloc(it[i].oeb, pb, sb, mb));
  }
}
template <>
void reloc_items<QrItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  QrItem *it = reinterpret_cast<QrItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].A = reloc(it[i].A, pb, sb, mb);
    it[i].Q = reloc(it[i].Q, pb, sb, mb);
    it[i].R = reloc(it[i].R, pb, sb, mb);
  }
}
template <>
void reloc_items<EigItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  EigItem *it = reinterpret_cast<EigItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].G = (const double *)reloc(it[i].G, pb, sb, mb);
    it[i].V = (double *)reloc(it[i].V, pb, sb, mb);
    it[i].lam = (double *)reloc(it[i].lam, pb, sb, mb);
  }
}
template <>
void reloc_items<CopyItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  CopyItem *it = reinterpret_cast<CopyItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].src = reloc(it[i].src, pb, sb, mb);
    it[i].dst = reloc(it[i].dst, pb, sb, mb);
  }
}
template <>
void reloc_items<CompactItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  CompactItem *it = reinterpret_cast<CompactItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].src = reloc(it[i].src, pb, sb, mb);
    it[i].dst = reloc(it[i].dst, pb, sb, mb);
  }
}
template <>
void reloc_items<CholItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  CholItem *it = reinterpret_cast<CholItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].G = (const double *)reloc(it[i].G, pb, sb, mb);
    it[i].W = (double *)reloc(it[i].W, pb, sb, mb);
    it[i].S = (float *)reloc(it[i].S, pb, sb, mb);
  }
}
template <>
void reloc_items<RankItem>(uint8_t *base, int n, char *pb, char *sb, char *mb) {
  RankItem *it = reinterpret_cast<RankItem *>(base);
  for (int i = 0; i < n; ++i) {
    it[i].lam = (const double *)reloc(it[i].lam, pb, sb, mb);
    it[i].lam_off = (const int64_t *)reloc(it[i].lam_off, pb, sb, mb);
    it[i].korth = (const int *)reloc(it[i].korth, pb, sb, mb);
    it[i].target = (const int *)reloc(it[i].target, pb, sb, mb);
    it[i].r_out = (int *)reloc(it[i].r_out, pb, sb, mb);
    it[i].stats = (double *)reloc(it[i].stats, pb, sb, mb);
    it[i].root = (const double *)reloc(it[i].root, pb, sb, mb);
  }
}

// Execute a plan on a stream: allocate workspace (persistent | scratch |
// upload), relocate, upload, launch.  The workspace is released in stream
// order after the last launch.  `keep` receives the relocated persistent base
// (so that callers can read results) and the caller must free it with
// cudaFreeAsync; if keep is null, everything is freed here.


// Tuning table (gemm_tune.h, written by tune_gemm.py); the autotuner sweeps
// candidates through ht_set_gemm_tuning without rebuilding.
struct GemmTune {
  int tall_m = kTuneTallM;
  double tall_share = kTuneTallShare;
  double square_share = kTuneSquareShare;
};
GemmTune g_gemm_tune;
const GemmTune &gemm_tune() { return g_gemm_tune; }

// Split-K factor of a launch with `tiles` output tiles: as many chunks as
// keep every CTA of the launch resident in one round of two CTAs per SM
// (rounded down: a second, nearly empty round would double the time).
inline int split_for(int tiles, int ko) {
  const int ks = (2 * kSmCount) / std::max(tiles, 1);
  return std::max(1, std::min(ko, ks));
}

// SIMT tile shape of a GEMM launch, and the items' tile grid for it.  Items
// with M >= tall_m are "tall", those also with N >= tall_m "square"; the
// shares of the launch's flops in them pick 128 x 128 (uncompensated
// launches), 128 x 64 or 64 x 64 tiles.
void choose_gemm_variant(Plan &P, Launch &L) {
  const GemmTune &tu = gemm_tune();
  GemmItem *it = reinterpret_cast<GemmItem *>(P.items.data() + L.off);
  double tall = 0.0, square = 0.0, all = 0.0;
  int64_t longest = 0;
  for (int i = 0; i < L.n; ++i) {
    const double fl = 2.0 * it[i].M * it[i].N * (double)it[i].K * it[i].Ko * it[i].batch;
    all += fl;
    if (it[i].M >= tu.tall_m) tall += fl;
    if (it[i].M >= tu.tall_m && it[i].N >= tu.tall_m) square += fl;
    const int64_t per_cta = (int64_t)it[i].K * ((it[i].Ko + it[i].ksplit - 1) / it[i].ksplit);
    longest = std::max(longest, per_cta);
  }
  // compensated accumulation where a CTA sums more than kTuneCompLen products;
  // shorter sums carry at most sqrt(kTuneCompLen) u of rounding (typical)
  L.comp = longest > kTuneCompLen && !L.df;
  L.variant = 0;
  if (L.df) L.variant = 0;  // the double-float kernel exists in the 64 x 64 shape only
  else if (all > 0.0 && !L.comp && square >= tu.square_share * all) L.variant = 2;
  else if (all > 0.0 && tall >= tu.tall_share * all) L.variant = 1;
  int bm = 64, bn = 64;
  gemm_tile_shape(L.variant, &bm, &bn);
  int tiles = 0;
  L.uniform = -1;
  for (int i = 0; i < L.n; ++i) {
    it[i].tiles_m = (it[i].M + bm - 1) / bm;
    it[i].tiles_n = (it[i].N + bn - 1) / bn;
    it[i].tile0 = tiles;
    const int per = it[i].tiles_m * it[i].tiles_n * it[i].batch * it[i].ksplit;
    tiles += per;
    L.uniform = (L.uniform == -1 || L.uniform == per) ? per : 0;
  }
  L.tiles = tiles;
  if (L.uniform < 0) L.uniform = 0;
}

// Tile -> item tables of the tensor-core launches, appended to the metadata
// (once, before the plan's sizes are taken).
void finalize_tables(Plan &P) {
  for (Launch &L : P.launches) {
    if (L.kind != L_GEMM || L.tile_item.empty() || L.tile_tab) continue;
    L.tile_tab = P.mpush(L.tile_item.data(), L.tile_item.size());
  }
}

// Workspace size of a plan: persistent | scratch | metadata | items.
size_t plan_bytes(const Plan &P) {
  const size_t p_sz = (P.p_bytes + 255) & ~size_t(255);
  const size_t s_sz = ((P.s_peak + 255) & ~size_t(255)) + ((P.l_peak + 255) & ~size_t(255));
  const size_t m_off = p_sz + s_sz;
  const size_t i_off = m_off + ((P.meta.size() + 255) & ~size_t(255));
  return i_off + P.items.size();
}

// HTGB_PLAN_DUMP=1: one line per launch of every prepared plan on stderr
// (kind, items, tiles, flops, tile shape; for contractions the items' dims).
void dump_plan(const Plan &P) {
  static const char *names[] = {"gemm", "qr", "eig", "copy", "compact", "ranks", "chol"};
  fprintf(stderr, "plan: %zu launches, dtype %s\n", P.launches.size(), P.dtype == HT_F64 ? "f64" : "f32");
  for (const Launch &L : P.launches) {
    fprintf(stderr, "  %-7s items %4d tiles %5d max_m %5d max_n %4d mflop %9.3f", names[L.kind], L.n, L.tiles, L.max_m,
            L.max_n, L.flops * 1e-6);
    if (L.kind == L_GEMM) {
      fprintf(stderr, " variant %d comp %d df %d split %d |", L.variant, (int)L.comp, (int)L.df, (int)L.split);
      const GemmItem *it = reinterpret_cast<const GemmItem *>(P.items.data() + L.off);
      for (int i = 0; i < L.n && i < 3; ++i)
        fprintf(stderr, " %dx%dx(%dx%d)b%d/s%d[a %lld,%lld,%lld b %lld,%lld,%lld c %lld,%lld]", it[i].M, it[i].N, it[i].K,
                it[i].Ko, it[i].batch, it[i].ksplit, (long long)it[i].sam, (long long)it[i].sak, (long long)it[i].sako,
                (long long)it[i].sbk, (long long)it[i].sbko, (long long)it[i].sbn, (long long)it[i].scm,
                (long long)it[i].scn);
      if (L.n > 3) fprintf(stderr, " ...");
    }
    fprintf(stderr, "\n");
  }
}

// Relocate the plan's tagged pointers into the workspace at base and upload
// the metadata and the work items (stream-ordered copies from host memory
// that stays alive in P).
ht_status prepare_plan(Plan &P, cudaStream_t s, char *base, char **ib_dev_out) {
  const size_t p_sz = (P.p_bytes + 255) & ~size_t(255);
  g_lscratch_off = (P.s_peak + 255) & ~size_t(255);
  const size_t s_sz = g_lscratch_off + ((P.l_peak + 255) & ~size_t(255));
  const size_t m_off = p_sz + s_sz;
  const size_t i_off = m_off + ((P.meta.size() + 255) & ~size_t(255));
  char *pb = base, *sb = base + p_sz, *mb = base + m_off;
  for (Launch &L : P.launches)
    if (L.kind == L_GEMM) choose_gemm_variant(P, L);
  if (getenv("HTGB_PLAN_DUMP")) dump_plan(P);
  for (Launch &L : P.launches) {
    uint8_t *ib = P.items.data() + L.off;
    switch (L.kind) {
      case L_GEMM: reloc_items<GemmItem>(ib, L.n, pb, sb, mb); break;
      case L_QR: reloc_items<QrItem>(ib, L.n, pb, sb, mb); break;
      case L_EIG: reloc_items<EigItem>(ib, L.n, pb, sb, mb); break;
      case L_COPY: reloc_items<CopyItem>(ib, L.n, pb, sb, mb); break;
      case L_COMPACT: reloc_items<CompactItem>(ib, L.n, pb, sb, mb); break;
      case L_RANKS: reloc_items<RankItem>(ib, L.n, pb, sb, mb); break;
      case L_CHOL: reloc_items<CholItem>(ib, L.n, pb, sb, mb); break;
    }
    L.ranks = reloc(L.ranks, pb, sb, mb);
    L.scratch = reloc(L.scratch, pb, sb, mb);
    L.tile_tab = static_cast<const int *>(reloc(L.tile_tab, pb, sb, mb));
  }
  cudaError_t e;
  if (!P.meta.empty()) {
    e = cudaMemcpyAsync(mb, P.meta.data(), P.meta.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  }
  char *ib_dev = base + i_off;
  if (!P.items.empty()) {
    e = cudaMemcpyAsync(ib_dev, P.items.data(), P.items.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  }
  *ib_dev_out = ib_dev;
  return HT_OK;
}

// Enqueue the plan's kernels (items already at ib_dev).  Returns the number
// of kernel launches through n_kernels.
ht_status enqueue_plan(const Plan &P, cudaStream_t s, const char *ib_dev, int *n_kernels) {
  const bool f64 = (P.dtype == HT_F64);
  int kernels = 0;
  for (const Launch &L : P.launches) {
    if (L.n == 0) continue;
    const void *items = ib_dev + L.off;
    const int *rk = static_cast<const int *>(L.ranks);
    const int64_t before = g_launches;
    cudaError_t e = cudaSuccess;
    if (L.kind == L_GEMM && P.mixed) {
      // the split into BF16 slices is its own profiled family (bytes, not flops)
      prof_begin(HT_K_SPLIT, s);
      e = launch_oz_split((const GemmItem *)items, L.n, L.oz_split, rk, L.oz_slices, s);
      prof_end(HT_K_SPLIT, s, L.split_bytes);
      if (e != cudaSuccess) return fail(HT_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    }
    if (L.kind == L_GEMM && P.mixed && L.tc_tiles == 0) {  // slicing-only launch
      kernels += (int)(g_launches - before);
      continue;
    }
    prof_begin((int)L.kind, s);
    switch (L.kind) {
      case L_GEMM: {
        if (P.mixed)
          e = launch_oz_gemm((const GemmItem *)items, L.tile_tab, L.n, L.tc_tiles, rk, L.split, L.oz_slices, s);
        else if (f64)
          e = launch_gemm<double>((const GemmItem *)items, L.n, L.tiles, rk, L.split, 0, s, L.variant, false, false,
                                  L.uniform);
        else
          e = launch_gemm<float>((const GemmItem *)items, L.n, L.tiles, rk, L.split, 0, s, L.variant, L.comp, L.df,
                                 L.uniform);
        break;
      }
      case L_QR:
        if (P.mixed && P.qr_kernel != 3)  // mixed path: double-float blocks on the FP32 pipe
          e = launch_qr_df((const QrItem *)items, L.n, L.max_m, L.max_n, s);
        else
          e = f64 ? launch_qr<double>((const QrItem *)items, L.n, L.max_m, L.max_n, s, P.qr_kernel)
                  : launch_qr<float>((const QrItem *)items, L.n, L.max_m, L.max_n, s, P.qr_kernel);
        break;
      case L_EIG:
        // square-root Gramians carry eigenvalues far below the FP32 solve's resolution,
        // which one refinement step cannot separate (it treats them as one cluster): FP64 QL
        // the mixed path accumulates the eigenvectors in double-float (mode 2); the
        // eigenvalues come from the FP64 QL recurrence in every FP64 mode
        e = launch_eig((const EigItem *)items, L.n, L.max_n, (double *)L.scratch, s,
                       P.mixed ? 2 : ((f64 || P.sqrt_gram) ? 0 : 1));
        break;
      case L_COPY: e = launch_copy((const CopyItem *)items, L.n, rk, 0, s); break;
      case L_COMPACT:
        e = f64 ? launch_compact<double>((const CompactItem *)items, L.n, rk, s)
                : launch_compact<float>((const CompactItem *)items, L.n, rk, s);
        break;
      case L_RANKS: e = launch_ranks((const RankItem *)items, L.n, s); break;
      case L_CHOL: e = launch_chol((const CholItem *)items, L.n, s); break;
    }
    // mixed-path contractions: the BF16 slice products the tensor cores execute,
    // S (S + 1) / 2 per FP64-equivalent product
    const double work = (L.kind == L_GEMM && P.mixed) ? L.flops * (L.oz_slices * (L.oz_slices + 1) / 2) : L.flops;
    prof_end((int)L.kind, s, work);
    kernels += (int)(g_launches - before);
    if (e != cudaSuccess) return fail(HT_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  }
  if (n_kernels) *n_kernels = kernels;
  return HT_OK;
}

// Execute a plan on a stream: allocate the workspace, relocate, upload,
// launch.  The workspace is released in stream order after the last launch.
// keep_base receives the workspace base (so that callers can read results)
// and the caller frees it with cudaFreeAsync; if keep_base is null,
// everything is freed here.  ext_base / ext_cap: run inside caller-provided
// device memory instead of allocating (nothing is allocated or freed then;
// keep_base must be null).
ht_status run_plan(Plan &P, cudaStream_t s, char **keep_base, char *ext_base = nullptr, size_t ext_cap = 0) {
  if (!P.err.empty()) return fail(HT_EUNSUPPORTED, P.err);
  finalize_tables(P);
  const size_t total = plan_bytes(P);
  char *base = nullptr;
  if (ext_base) {
    if (total > ext_cap)
      return fail(HT_ENOMEM, "the call needs " + std::to_string(total) + " bytes of device scratch; the fixed scratch holds " +
                                 std::to_string(ext_cap) + " bytes");
    base = ext_base;
  } else {
    cudaError_t e = cudaMallocAsync((void **)&base, std::max<size_t>(total, 256), s);
    if (e != cudaSuccess) return fail(HT_ENOMEM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
  }
  char *ib_dev = nullptr;
  ht_status st = prepare_plan(P, s, base, &ib_dev);
  if (st == HT_OK) st = enqueue_plan(P, s, ib_dev, nullptr);
  if (st != HT_OK) {
    if (!ext_base) cudaFreeAsync(base, s);
    return st;
  }
  if (ext_base) return HT_OK;
  if (keep_base) {
    *keep_base = base;
  } else {
    cudaError_t e = cudaFreeAsync(base, s);
    if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  }
  return HT_OK;
}

// ---------------------------------------------------------------------------
// per-tensor state of a plan
// ---------------------------------------------------------------------------
struct TState {
  ht_tensor *x = nullptr;
  std::vector<int> kin, ko;       // input ranks, ranks after orthogonalization
  std::vector<void *> R;          // R factors (T), ko[t] x kin[t], column-major, ld = ko[t]
  std::vector<void *> G;          // Gramians (T), ko x ko
  std::vector<void *> Sf;         // square-root Gramian factors (FP32), ko x ko, inner nodes
  std::vector<double *> G64;      // Gramians (FP64)
  std::vector<double *> V64;      // eigenvectors (FP64)
  std::vector<void *> V;          // eigenvectors (T)
  double *lam = nullptr;          // eigenvalues, all nodes
  std::vector<int64_t> lam_off;
  int *r = nullptr;               // truncated ranks (device)
  double *stats = nullptr;        // norm, discarded, tail2
  int node_base = 0;              // global index of node 0 in the plan's rank array
};

inline GemmItem gemm0() {
  GemmItem g;
  memset(&g, 0, sizeof(g));
  g.m_ref = g.n_ref = g.b_ref = -1;
  g.n_mult = g.b_mult = 1;
  g.Ko = 1;
  g.batch = 1;
  g.ksplit = 1;
  g.alpha = 1.0;
  g.beta = 0.0;
  g.k_total = -1;
  return g;
}

inline CopyItem copy0() {
  CopyItem c;
  memset(&c, 0, sizeof(c));
  c.rows_ref = c.cols_ref = -1;
  c.alpha = 1.0;
  return c;
}

// ---- TSQR: reduced QR of tall matrices (m >= n) --------------------------
struct Mat {
  const void *A;
  int64_t lda;
  int m, n;
  void *Q;
  int64_t ldq;
  void *R;
  int64_t ldr;
  int node;
};

void plan_tsqr_narrow(Plan &P, const std::vector<Mat> &mats);

// Panel width of the mixed path: narrower panels move QR work from the FP64
// Householder blocks (4 m w^2 per panel) into the panel projections, which run
// on the tensor cores.
constexpr int kPanelMixed = 32;

// Reduced QR of matrices wider than one panel: columns are taken in panels
// of P.panel (64, or 32 on the mixed path); panel p is projected twice
// against the finished Q columns (block Gram-Schmidt, "twice is enough":
// R[<p, p] = C1 + C2 with
// C = Q_<p^T A_p, A_p -= Q_<p C) and then factored by the TSQR of
// plan_tsqr_narrow.  A (the matrix, overwritten by the projections) and Q
// (the output) may be the same buffer.
void plan_tsqr_panels(Plan &P, const std::vector<Mat> &mats) {
  const size_t esz = P.esz;
  const bool f64 = (P.dtype == HT_F64);
  int max_panels = 0;
  const int pw = P.panel;
  for (const Mat &M : mats) max_panels = std::max(max_panels, (M.n + pw - 1) / pw);
  // R starts as zero below the diagonal blocks
  P.begin(L_COPY);
  for (const Mat &M : mats) {
    CopyItem z = copy0();
    z.dst = M.R;
    z.dr = 1;
    z.dc = M.ldr;
    z.rows = M.n;
    z.cols = M.n;
    z.zero = 1;
    z.dst_f64 = f64;
    P.copy(z, M.node);
  }
  constexpr int kChunk = 256;  // rows per chunk of the long reductions Q^T A
  // Mixed path: the projections C = Q_<p^T A_p take Q's columns as operand A,
  // with one exponent per (column, 256-row chunk), so the slices of a finished
  // panel do not change with the panels after it.  Each panel is sliced once,
  // right after its TSQR, into a per-matrix buffer of the same chunk layout
  // (one block row per 128 columns), and both passes of every later panel use
  // it instead of slicing Q_<p again.
  struct QSlices {
    void *oza = nullptr;
    int *oea = nullptr;
    int ko = 0;
    size_t tile_bytes = 0;
  };
  std::vector<QSlices> qs(mats.size());
  const bool cache_q = P.mixed && max_panels > 1 && oz_tile_m() % pw == 0;
  if (cache_q) {
    for (size_t mi = 0; mi < mats.size(); ++mi) {
      const Mat &M = mats[mi];
      if (M.n <= pw) continue;  // a single panel: nothing to project
      QSlices &c = qs[mi];
      c.ko = (M.m + kChunk - 1) / kChunk;
      const int tm = (M.n + oz_tile_m() - 1) / oz_tile_m();
      c.tile_bytes = (size_t)oz_block_bytes() * P.oz_slices * (kChunk / oz_stage_k()) * c.ko;
      c.oza = P.salloc_bytes(c.tile_bytes * tm);
      c.oea = static_cast<int *>(P.salloc_bytes(sizeof(int) * (size_t)tm * oz_tile_m() * c.ko));
    }
  }
  for (int p = 0; p < max_panels; ++p) {
    struct PJ {
      const Mat *M;
      int c0, w;
      void *C1, *C2;
    };
    std::vector<PJ> pj;
    for (const Mat &M : mats) {
      const int np = (M.n + pw - 1) / pw;
      if (p >= np) continue;
      PJ j;
      j.M = &M;
      j.c0 = p * pw;
      j.w = std::min(pw, M.n - j.c0);
      j.C1 = j.C2 = nullptr;
      if (p > 0) {
        j.C1 = P.salloc_bytes((size_t)j.c0 * j.w * esz);
        j.C2 = P.salloc_bytes((size_t)j.c0 * j.w * esz);
      }
      pj.push_back(j);
    }
    if (p > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        // C = Q_<p^T A_p   ((c0 x w), reduction over the m rows in chunks)
        P.begin(L_GEMM);
        int tiles = 0;
        for (PJ &j : pj) tiles += ((j.c0 + 63) / 64) * ((j.w + 63) / 64);
        for (PJ &j : pj) {
          const Mat &M = *j.M;
          const int ko = (M.m + kChunk - 1) / kChunk;
          GemmItem g = gemm0();
          g.A = M.Q;
          g.sam = M.ldq;
          g.sak = 1;
          g.sako = kChunk;
          g.B = static_cast<const char *>(M.A) + (int64_t)j.c0 * M.lda * esz;
          g.sbk = 1;
          g.sbko = kChunk;
          g.sbn = M.lda;
          g.C = pass == 0 ? j.C1 : j.C2;
          g.scm = 1;
          g.scn = j.c0;
          g.M = j.c0;
          g.N = j.w;
          g.K = kChunk;
          g.Ko = ko;
          g.k_total = M.m;
          g.ksplit = split_for(tiles, ko);
          const QSlices &c = qs[&M - mats.data()];
          if (c.oza) {  // Q_<p's slices from the panels' slicing launches
            g.oz_pre = 1;
            g.oza = c.oza;
            g.oea = c.oea;
            g.ksplit = ko;  // the slicing launches' chunk layout: one chunk per 256 rows
          }
          P.gemm(g, M.node);
        }
        // A_p -= Q_<p C
        P.begin(L_GEMM);
        for (PJ &j : pj) {
          const Mat &M = *j.M;
          GemmItem g = gemm0();
          g.A = M.Q;
          g.sam = 1;
          g.sak = M.ldq;
          g.B = pass == 0 ? j.C1 : j.C2;
          g.sbk = 1;
          g.sbn = j.c0;
          g.C = const_cast<char *>(static_cast<const char *>(M.A)) + (int64_t)j.c0 * M.lda * esz;
          g.scm = 1;
          g.scn = M.lda;
          g.M = M.m;
          g.N = j.w;
          g.K = j.c0;
          g.alpha = -1.0;
          g.beta = 1.0;
          P.gemm(g, M.node);
        }
      }
      // R[0:c0, c0:c0+w] = C1 + C2
      P.begin(L_COPY);
      for (PJ &j : pj) {
        const Mat &M = *j.M;
        CopyItem c = copy0();
        c.src = j.C1;
        c.dst = static_cast<char *>(M.R) + (int64_t)j.c0 * M.ldr * esz;
        c.sr = 1;
        c.sc = j.c0;
        c.dr = 1;
        c.dc = M.ldr;
        c.rows = j.c0;
        c.cols = j.w;
        c.src_f64 = c.dst_f64 = f64;
        P.copy(c, M.node);
      }
      P.begin(L_COPY);
      for (PJ &j : pj) {
        const Mat &M = *j.M;
        CopyItem c = copy0();
        c.src = j.C2;
        c.dst = static_cast<char *>(M.R) + (int64_t)j.c0 * M.ldr * esz;
        c.sr = 1;
        c.sc = j.c0;
        c.dr = 1;
        c.dc = M.ldr;
        c.rows = j.c0;
        c.cols = j.w;
        c.beta = 1.0;
        c.src_f64 = c.dst_f64 = f64;
        P.copy(c, M.node);
      }
    }
    // TSQR of the (projected) panel: Q columns c0.., R diagonal block
    std::vector<Mat> panel;
    for (PJ &j : pj) {
      const Mat &M = *j.M;
      Mat q;
      q.A = static_cast<const char *>(M.A) + (int64_t)j.c0 * M.lda * esz;
      q.lda = M.lda;
      q.m = M.m;
      q.n = j.w;
      q.Q = static_cast<char *>(M.Q) + (int64_t)j.c0 * M.ldq * esz;
      q.ldq = M.ldq;
      q.R = static_cast<char *>(M.R) + ((int64_t)j.c0 * M.ldr + j.c0) * esz;
      q.ldr = M.ldr;
      q.node = M.node;
      panel.push_back(q);
    }
    plan_tsqr_narrow(P, panel);
    if (!cache_q) continue;
    // slices of this panel's Q columns for the later panels' projections
    P.begin(L_GEMM);
    for (PJ &j : pj) {
      const Mat &M = *j.M;
      const QSlices &c = qs[&M - mats.data()];
      if (!c.oza || j.c0 + j.w >= M.n) continue;  // no later panel of this matrix
      GemmItem g = gemm0();
      g.A = static_cast<const char *>(M.Q) + (int64_t)j.c0 * M.ldq * esz;
      g.sam = M.ldq;
      g.sak = 1;
      g.sako = kChunk;
      g.B = g.A;
      g.sbk = 1;
      g.sbn = 1;
      g.M = j.w;
      g.N = 1;
      g.K = kChunk;
      g.Ko = c.ko;
      g.k_total = M.m;
      g.ksplit = c.ko;
      g.oz_pre = 2;
      // the panel's columns sit at rows c0 % 128 .. of block row c0 / 128 (panels
      // are at most 32 wide and start at multiples of 32: never across a block row)
      g.oz_row0 = j.c0 % oz_tile_m();
      g.oza = static_cast<char *>(c.oza) + (size_t)(j.c0 / oz_tile_m()) * c.tile_bytes;
      g.oea = c.oea + (size_t)(j.c0 / oz_tile_m()) * oz_tile_m() * c.ko;
      P.gemm(g, M.node);
    }
  }
}

void plan_tsqr(Plan &P, const std::vector<Mat> &mats) {
  std::vector<Mat> narrow, wide;
  for (const Mat &M : mats) (M.n > P.panel ? wide : narrow).push_back(M);
  if (!narrow.empty()) plan_tsqr_narrow(P, narrow);
  if (!wide.empty()) plan_tsqr_panels(P, wide);
}

void plan_tsqr_narrow(Plan &P, const std::vector<Mat> &mats) {
  struct Blk {
    int64_t r0;
    int m;
  };
  struct Lv {
    const void *A;
    int64_t lda;
    int m;
    void *tgt;
    int64_t ldt;
    void *W;
    void *S;
    void *QS;
    std::vector<Blk> blocks;
    bool top;
  };
  const size_t esz = P.esz;
  std::vector<std::vector<Lv>> lv(mats.size());
  int max_rounds = 0;
  for (size_t i = 0; i < mats.size(); ++i) {
    const Mat &M = mats[i];
    const int rows_max = qr_max_rows(M.n, (int)esz);
    if (rows_max < 2 * M.n && M.m > rows_max) {
      P.err = "QR of a " + std::to_string(M.m) + " x " + std::to_string(M.n) +
              " matrix: rank too large for the shared-memory TSQR in this precision";
      return;
    }
    const void *A = M.A;
    int64_t lda = M.lda;
    int m = M.m;
    void *tgt = M.Q;
    int64_t ldt = M.ldq;
    for (;;) {
      Lv L;
      L.A = A;
      L.lda = lda;
      L.m = m;
      L.tgt = tgt;
      L.ldt = ldt;
      int p = (m + rows_max - 1) / rows_max;
      if (p <= 1) {
        L.top = true;
        L.W = L.S = L.QS = nullptr;
        lv[i].push_back(L);
        break;
      }
      L.top = false;
      L.W = P.salloc_bytes((size_t)m * M.n * esz);
      L.S = P.salloc_bytes((size_t)p * M.n * M.n * esz);
      L.QS = P.salloc_bytes((size_t)p * M.n * M.n * esz);
      int base = m / p, rem = m % p;
      int64_t r0 = 0;
      for (int b = 0; b < p; ++b) {
        int mb = base + (b < rem ? 1 : 0);
        L.blocks.push_back({r0, mb});
        r0 += mb;
      }
      lv[i].push_back(L);
      A = L.S;
      lda = (int64_t)p * M.n;
      m = p * M.n;
      tgt = L.QS;
      ldt = (int64_t)p * M.n;
    }
    max_rounds = std::max(max_rounds, (int)lv[i].size());
  }
  // QR rounds, bottom-up
  for (int r = 0; r < max_rounds; ++r) {
    P.begin(L_QR);
    for (size_t i = 0; i < mats.size(); ++i) {
      if (r >= (int)lv[i].size()) continue;
      const Mat &M = mats[i];
      const Lv &L = lv[i][r];
      if (L.top) {
        QrItem q{L.A, L.tgt, M.R, L.lda, L.ldt, M.ldr, L.m, M.n};
        P.qr(q, M.node);
      } else {
        const int64_t ldS = (int64_t)L.blocks.size() * M.n;
        for (size_t b = 0; b < L.blocks.size(); ++b) {
          const Blk &B = L.blocks[b];
          QrItem q;
          q.A = static_cast<const char *>(L.A) + B.r0 * esz;
          q.lda = L.lda;
          q.Q = static_cast<char *>(L.W) + B.r0 * esz;
          q.ldq = L.m;
          q.R = static_cast<char *>(L.S) + (int64_t)b * M.n * esz;
          q.ldr = ldS;
          q.m = B.m;
          q.n = M.n;
          P.qr(q, M.node);
        }
      }
    }
  }
  // recombination, top-down: tgt_r[block b] = W_r[block b] * QS_r[b*n:(b+1)*n, :]
  for (int r = max_rounds - 2; r >= 0; --r) {
    P.begin(L_GEMM);
    for (size_t i = 0; i < mats.size(); ++i) {
      if (r + 1 >= (int)lv[i].size()) continue;
      const Mat &M = mats[i];
      const Lv &L = lv[i][r];
      const int64_t ldS = (int64_t)L.blocks.size() * M.n;
      for (size_t b = 0; b < L.blocks.size(); ++b) {
        const Blk &B = L.blocks[b];
        GemmItem g = gemm0();
        g.A = static_cast<const char *>(L.W) + B.r0 * esz;
        g.sam = 1;
        g.sak = L.m;
        g.B = static_cast<const char *>(L.QS) + (int64_t)b * M.n * esz;
        g.sbk = 1;
        g.sbn = ldS;
        g.C = static_cast<char *>(L.tgt) + B.r0 * esz;
        g.scm = 1;
        g.scn = L.ldt;
        g.M = B.m;
        g.N = M.n;
        g.K = M.n;
        P.gemm(g, M.node);
      }
    }
  }
}

// ---- orthogonalization (Sec. 3.4) ----------------------------------------
void plan_orthogonalize(Plan &P, std::vector<TState> &TS) {
  const size_t esz = P.esz;
  int max_h = 0;
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    S.kin = S.x->k;
    S.ko = S.kin;
    S.R.assign(T.nn, nullptr);
    max_h = std::max(max_h, T.max_height);
  }
  for (int h = 0; h <= max_h; ++h) {
    P.sreset();
    if (h == 0) {
      // leaves: U = Q R (Sec. 3.4 step 1)
      std::vector<Mat> mats;
      std::vector<CopyItem> rcopies, idfills;
      std::vector<int> rnodes, inodes;
      for (TState &S : TS) {
        const ht_tree &T = S.x->tr;
        for (int t = 0; t < T.nn; ++t) {
          if (!is_leaf(T, t)) continue;
          const int64_t nm = S.x->n[T.lo[t]];
          const int k = S.kin[t];
          void *slot = node_ptr(S.x, t);
          if (nm >= k) {
            S.R[t] = P.palloc_bytes((size_t)k * k * esz);
            mats.push_back({slot, nm, (int)nm, k, slot, nm, S.R[t], k, S.node_base + t});
            S.ko[t] = k;
          } else {
            // n < k: Q = I_n, R = U (n x k)
            S.R[t] = P.palloc_bytes((size_t)nm * k * esz);
            CopyItem c = copy0();
            c.src = slot;
            c.dst = S.R[t];
            c.sr = 1;
            c.sc = nm;
            c.dr = 1;
            c.dc = nm;
            c.rows = (int)nm;
            c.cols = k;
            c.src_f64 = c.dst_f64 = (P.dtype == HT_F64);
            rcopies.push_back(c);
            rnodes.push_back(S.node_base + t);
            CopyItem idc = copy0();
            idc.dst = slot;
            idc.dr = 1;
            idc.dc = nm;
            idc.rows = (int)nm;
            idc.cols = (int)nm;
            idc.dst_f64 = (P.dtype == HT_F64);
            idfills.push_back(idc);
            inodes.push_back(S.node_base + t);
            S.ko[t] = (int)nm;
          }
        }
      }
      if (!rcopies.empty()) {
        P.begin(L_COPY);
        for (size_t i = 0; i < rcopies.size(); ++i) P.copy(rcopies[i], rnodes[i]);
        P.begin(L_COPY);
        for (size_t i = 0; i < idfills.size(); ++i) P.copy(idfills[i], inodes[i]);
      }
      if (!mats.empty()) plan_tsqr(P, mats);
      continue;
    }
    // inner nodes of height h: B <- (I, R_s1, R_s2) o B, then QR of M_{2,3}(B)
    struct Job {
      TState *S;
      int t, K0, k1, k2, p1, p2;
      void *Tbuf, *Bp;
    };
    std::vector<Job> jobs;
    for (TState &S : TS) {
      const ht_tree &T = S.x->tr;
      for (int t = 0; t < T.nn; ++t) {
        if (is_leaf(T, t) || T.height[t] != h) continue;
        Job J;
        J.S = &S;
        J.t = t;
        J.K0 = (t == 0) ? 1 : S.kin[t];
        J.k1 = S.kin[T.s1[t]];
        J.k2 = S.kin[T.s2[t]];
        J.p1 = S.ko[T.s1[t]];
        J.p2 = S.ko[T.s2[t]];
        J.Tbuf = P.salloc_bytes((size_t)J.p2 * J.K0 * J.k1 * esz);
        J.Bp = (t == 0) ? node_ptr(S.x, 0) : P.salloc_bytes((size_t)J.K0 * J.p1 * J.p2 * esz);
        jobs.push_back(J);
      }
    }
    if (jobs.empty()) continue;
    // mode 3: T (p2 x K0*k1) = R2 (p2 x k2) * B_view (k2 x K0*k1)
    P.begin(L_GEMM);
    for (Job &J : jobs) {
      const ht_tree &T = J.S->x->tr;
      GemmItem g = gemm0();
      g.A = J.S->R[T.s2[J.t]];
      g.sam = 1;
      g.sak = J.p2;
      g.B = node_ptr(J.S->x, J.t);
      g.sbk = 1;
      g.sbn = J.k2;
      g.C = J.Tbuf;
      g.scm = 1;
      g.scn = J.p2;
      g.M = J.p2;
      g.N = J.K0 * J.k1;
      g.K = J.k2;
      P.gemm(g, J.S->node_base + J.t);
    }
    // mode 2: per i, Bp[i] (p2 x p1) = T[i] (p2 x k1) * R1^T (k1 x p1)
    P.begin(L_GEMM);
    for (Job &J : jobs) {
      const ht_tree &T = J.S->x->tr;
      GemmItem g = gemm0();
      g.A = J.Tbuf;
      g.sam = 1;
      g.sak = J.p2;
      g.sab = (int64_t)J.k1 * J.p2;
      g.B = J.S->R[T.s1[J.t]];
      g.sbk = J.p1;
      g.sbn = 1;
      g.C = J.Bp;
      g.scm = 1;
      g.scn = J.p2;
      g.scb = (int64_t)J.p1 * J.p2;
      g.M = J.p2;
      g.N = J.p1;
      g.K = J.k1;
      g.batch = J.K0;
      P.gemm(g, J.S->node_base + J.t);
    }
    std::vector<Mat> mats;
    std::vector<CopyItem> rcopies, idfills;
    std::vector<int> cnodes;
    for (Job &J : jobs) {
      if (J.t == 0) continue;
      TState &S = *J.S;
      const int64_t m = (int64_t)J.p1 * J.p2;
      void *slot = node_ptr(S.x, J.t);
      if (m >= J.K0) {
        S.R[J.t] = P.palloc_bytes((size_t)J.K0 * J.K0 * esz);
        mats.push_back({J.Bp, m, (int)m, J.K0, slot, m, S.R[J.t], J.K0, S.node_base + J.t});
        S.ko[J.t] = J.K0;
      } else {
        // k_s1 k_s2 < k_t: Q = I, R = M_{2,3}(B) (eq. "qrtransfer" with k = k_s1 k_s2)
        S.R[J.t] = P.palloc_bytes((size_t)m * J.K0 * esz);
        CopyItem c = copy0();
        c.src = J.Bp;
        c.dst = S.R[J.t];
        c.sr = 1;
        c.sc = m;
        c.dr = 1;
        c.dc = m;
        c.rows = (int)m;
        c.cols = J.K0;
        c.src_f64 = c.dst_f64 = (P.dtype == HT_F64);
        rcopies.push_back(c);
        CopyItem idc = copy0();
        idc.dst = slot;
        idc.dr = 1;
        idc.dc = m;
        idc.rows = (int)m;
        idc.cols = (int)m;
        idc.dst_f64 = (P.dtype == HT_F64);
        idfills.push_back(idc);
        cnodes.push_back(S.node_base + J.t);
        S.ko[J.t] = (int)m;
      }
    }
    if (!rcopies.empty()) {
      P.begin(L_COPY);
      for (size_t i = 0; i < rcopies.size(); ++i) P.copy(rcopies[i], cnodes[i]);
      P.begin(L_COPY);
      for (size_t i = 0; i < idfills.size(); ++i) P.copy(idfills[i], cnodes[i]);
    }
    if (!mats.empty()) plan_tsqr(P, mats);
  }
  for (TState &S : TS) S.ko[0] = 1;
}

// ---- reduced Gramians (Sec. 3.3) -----------------------------------------
// dev_out: optional per-tensor FP64 output blocks (ht_gramians); else P-alloc.
// ---- square-root Gramians (HT_PREC_FP32_SQRT) -------------------------------
// The paper's Gramian recursion squares the singular values; with FP32 data
// that resolves sigma only down to about sqrt(u_32) sigma_max.  Here every
// Gramian is carried as a factor, Ghat_t = S_t S_t^T, top-down:
//   Y[a, p, l] = sum_i S_t[i, a] B_t[i, p, l]            (FP32 contraction)
//   Ghat_s1[p, q] = sum_{a,l} Y[a,p,l] Y[a,q,l],  Ghat_s2[l, l'] = sum_{a,j} Y[a,j,l] Y[a,j,l']
// (eqs. "acctransferSon1/2" with Ghat_t = S_t S_t^T inserted), the Gram
// products accumulated exactly in double-float with FP64 output, and S_s the
// semidefinite Cholesky factor of Ghat_s (FP64, stored FP32) for the next
// level.  Rounding then perturbs the factors, i.e. the singular values
// themselves, by O(u_32) sigma_max.  S_root = 1.
void plan_gramians_sqrt(Plan &P, std::vector<TState> &TS, const std::vector<double *> *dev_out) {
  const size_t esz = P.esz;
  int max_d = 0;
  for (size_t si = 0; si < TS.size(); ++si) {
    TState &S = TS[si];
    const ht_tree &T = S.x->tr;
    S.G.assign(T.nn, nullptr);
    S.G64.assign(T.nn, nullptr);
    S.Sf.assign(T.nn, nullptr);
    int64_t off = 0;
    for (int t = 0; t < T.nn; ++t) {
      const int kt = (t == 0) ? 1 : S.ko[t];
      if (dev_out) {
        S.G64[t] = (*dev_out)[si] + off;
        off += (int64_t)kt * kt;
      } else {
        S.G64[t] = P.palloc<double>((size_t)kt * kt);
      }
      if (!is_leaf(T, t)) S.Sf[t] = P.palloc_bytes((size_t)kt * kt * sizeof(float));
    }
    max_d = std::max(max_d, T.max_depth);
  }
  // S_root = 1, Ghat_root = 1
  P.begin(L_COPY);
  for (TState &S : TS) {
    CopyItem c = copy0();
    c.dst = S.Sf[0];
    c.rows = c.cols = 1;
    c.dr = c.dc = 1;
    c.dst_f64 = 0;
    P.copy(c, S.node_base);
    CopyItem c2 = c;
    c2.dst = S.G64[0];
    c2.dst_f64 = 1;
    P.copy(c2, S.node_base);
  }
  for (int L = 0; L <= max_d; ++L) {
    P.sreset();
    struct Job {
      TState *S;
      int t, K0, k1, k2;
      void *Y;
    };
    std::vector<Job> jobs;
    int tiles = 0;
    for (TState &S : TS) {
      const ht_tree &T = S.x->tr;
      for (int t = 0; t < T.nn; ++t) {
        if (is_leaf(T, t) || T.depth[t] != L) continue;
        Job J;
        J.S = &S;
        J.t = t;
        J.K0 = (t == 0) ? 1 : S.ko[t];
        J.k1 = S.ko[T.s1[t]];
        J.k2 = S.ko[T.s2[t]];
        J.Y = P.salloc_bytes((size_t)J.K0 * J.k1 * J.k2 * esz);
        jobs.push_back(J);
        tiles += ((J.k1 + 63) / 64) * ((J.k1 + 63) / 64) + ((J.k2 + 63) / 64) * ((J.k2 + 63) / 64);
      }
    }
    if (jobs.empty()) continue;
    // Y_mat (k1k2 x K0) = B_mat (k1k2 x K0) * S_t (K0 x K0)
    P.begin(L_GEMM);
    for (Job &J : jobs) {
      GemmItem g = gemm0();
      g.A = node_ptr(J.S->x, J.t);
      g.sam = 1;
      g.sak = (int64_t)J.k1 * J.k2;
      g.B = J.S->Sf[J.t];
      g.sbk = 1;
      g.sbn = J.K0;
      g.C = J.Y;
      g.scm = 1;
      g.scn = (int64_t)J.k1 * J.k2;
      g.M = J.k1 * J.k2;
      g.N = J.K0;
      g.K = J.K0;
      P.gemm(g, J.S->node_base + J.t);
    }
    // Ghat_s1 = sum_{a,l} Y[a,p,l] Y[a,q,l], Ghat_s2 = sum_{a,j} Y[a,j,l] Y[a,j,l'] (double-float, FP64 out)
    const int ksplit = split_for(tiles, 1 << 30);
    P.begin(L_GEMM);
    P.cur().df = true;
    for (Job &J : jobs) {
      const ht_tree &T = J.S->x->tr;
      const int s1 = T.s1[J.t], s2 = T.s2[J.t];
      const int64_t kk = (int64_t)J.k1 * J.k2;
      GemmItem g = gemm0();
      g.A = J.Y;
      g.sam = J.k2;
      g.sak = 1;
      g.sako = kk;
      g.B = J.Y;
      g.sbk = 1;
      g.sbko = kk;
      g.sbn = J.k2;
      g.C = J.S->G64[s1];
      g.scm = 1;
      g.scn = J.k1;
      g.M = J.k1;
      g.N = J.k1;
      g.K = J.k2;
      g.Ko = J.K0;
      g.ksplit = std::min(ksplit, J.K0);
      P.gemm(g, J.S->node_base + J.t);
      GemmItem h = gemm0();
      h.A = J.Y;
      h.sam = 1;
      h.sak = J.k2;
      h.sako = kk;
      h.B = J.Y;
      h.sbk = J.k2;
      h.sbko = kk;
      h.sbn = 1;
      h.C = J.S->G64[s2];
      h.scm = 1;
      h.scn = J.k2;
      h.M = J.k2;
      h.N = J.k2;
      h.K = J.k1;
      h.Ko = J.K0;
      h.ksplit = std::min(ksplit, J.K0);
      P.gemm(h, J.S->node_base + J.t);
    }
    // factors of the inner sons for the next level
    P.begin(L_CHOL);
    for (Job &J : jobs) {
      const ht_tree &T = J.S->x->tr;
      for (int s : {T.s1[J.t], T.s2[J.t]}) {
        if (is_leaf(T, s)) continue;
        const int ks = J.S->ko[s];
        CholItem c;
        c.G = J.S->G64[s];
        c.W = static_cast<double *>(P.salloc_bytes((size_t)ks * ks * sizeof(double)));
        c.S = static_cast<float *>(J.S->Sf[s]);
        c.k = ks;
        P.chol(c, J.S->node_base + s);
      }
    }
  }
}

void plan_gramians(Plan &P, std::vector<TState> &TS, const std::vector<double *> *dev_out) {
  if (P.sqrt_gram) {
    plan_gramians_sqrt(P, TS, dev_out);
    return;
  }
  const size_t esz = P.esz;
  const bool f64 = (P.dtype == HT_F64);
  int max_d = 0;
  for (size_t si = 0; si < TS.size(); ++si) {
    TState &S = TS[si];
    const ht_tree &T = S.x->tr;
    S.G.assign(T.nn, nullptr);
    S.G64.assign(T.nn, nullptr);
    int64_t off = 0;
    for (int t = 0; t < T.nn; ++t) {
      const int kt = (t == 0) ? 1 : S.ko[t];
      if (dev_out) {
        S.G64[t] = (*dev_out)[si] + off;
        off += (int64_t)kt * kt;
      } else {
        S.G64[t] = P.palloc<double>((size_t)kt * kt);
      }
      S.G[t] = f64 ? (void *)S.G64[t] : P.palloc_bytes((size_t)kt * kt * esz);
    }
    max_d = std::max(max_d, T.max_depth);
  }
  // root Gramian = 1 (eq. "acctransferroot" written as eqs. "acctransferSon1/2")
  P.begin(L_COPY);
  for (TState &S : TS) {
    CopyItem c = copy0();
    c.dst = S.G[0];
    c.rows = c.cols = 1;
    c.dr = c.dc = 1;
    c.dst_f64 = f64;
    P.copy(c, S.node_base);
    if (!f64) {
      CopyItem c2 = c;
      c2.dst = S.G64[0];
      c2.dst_f64 = 1;
      P.copy(c2, S.node_base);
    }
  }
  for (int L = 0; L <= max_d; ++L) {
    P.sreset();
    struct Job {
      TState *S;
      int t, K0, k1, k2;
      void *C;
    };
    std::vector<Job> jobs;
    int tiles = 0;
    for (TState &S : TS) {
      const ht_tree &T = S.x->tr;
      for (int t = 0; t < T.nn; ++t) {
        if (is_leaf(T, t) || T.depth[t] != L) continue;
        Job J;
        J.S = &S;
        J.t = t;
        J.K0 = (t == 0) ? 1 : S.ko[t];
        J.k1 = S.ko[T.s1[t]];
        J.k2 = S.ko[T.s2[t]];
        J.C = P.salloc_bytes((size_t)J.K0 * J.k1 * J.k2 * esz);
        jobs.push_back(J);
        tiles += ((J.k1 + 63) / 64) * ((J.k1 + 63) / 64) + ((J.k2 + 63) / 64) * ((J.k2 + 63) / 64);
      }
    }
    if (jobs.empty()) continue;
    // C[i2,p,l] = sum_i1 Bhat_t[i1,i2] B[i1,p,l]:  C_mat (k1k2 x K0) = B_mat (k1k2 x K0) * Bhat_t
    P.begin(L_GEMM);
    P.cur().oz_slices = kOzSlicesGram;
    for (Job &J : jobs) {
      GemmItem g = gemm0();
      g.A = node_ptr(J.S->x, J.t);
      g.sam = 1;
      g.sak = (int64_t)J.k1 * J.k2;
      g.B = J.S->G[J.t];
      g.sbk = 1;
      g.sbn = J.K0;
      g.C = J.C;
      g.scm = 1;
      g.scn = (int64_t)J.k1 * J.k2;
      g.M = J.k1 * J.k2;
      g.N = J.K0;
      g.K = J.K0;
      P.gemm(g, J.S->node_base + J.t);
    }
    // eqs. "acctransferSon1" and "acctransferSon2"; the reduction over the
    // parent index i is split across CTAs when the level has few nodes
    int ksplit = split_for(tiles, 1 << 30);
    P.begin(L_GEMM);
    P.cur().oz_slices = kOzSlicesGram;
    for (Job &J : jobs) {
      const ht_tree &T = J.S->x->tr;
      const int s1 = T.s1[J.t], s2 = T.s2[J.t];
      const int64_t kk = (int64_t)J.k1 * J.k2;
      GemmItem g = gemm0();
      g.A = J.C;
      g.sam = J.k2;
      g.sak = 1;
      g.sako = kk;
      g.B = node_ptr(J.S->x, J.t);
      g.sbk = 1;
      g.sbko = kk;
      g.sbn = J.k2;
      g.C = J.S->G[s1];
      g.scm = 1;
      g.scn = J.k1;
      g.M = J.k1;
      g.N = J.k1;
      g.K = J.k2;
      g.Ko = J.K0;
      g.ksplit = std::min(ksplit, J.K0);
      P.gemm(g, J.S->node_base + J.t);
      GemmItem h = gemm0();
      h.A = J.C;
      h.sam = 1;
      h.sak = J.k2;
      h.sako = kk;
      h.B = node_ptr(J.S->x, J.t);
      h.sbk = J.k2;
      h.sbko = kk;
      h.sbn = 1;
      h.C = J.S->G[s2];
      h.scm = 1;
      h.scn = J.k2;
      h.M = J.k2;
      h.N = J.k2;
      h.K = J.k1;
      h.Ko = J.K0;
      h.ksplit = std::min(ksplit, J.K0);
      P.gemm(h, J.S->node_base + J.t);
    }
    if (!f64) {
      P.begin(L_COPY);
      for (Job &J : jobs) {
        const ht_tree &T = J.S->x->tr;
        for (int s : {T.s1[J.t], T.s2[J.t]}) {
          const int ks = J.S->ko[s];
          CopyItem c = copy0();
          c.src = J.S->G[s];
          c.dst = J.S->G64[s];
          c.sr = c.dr = 1;
          c.sc = c.dc = ks;
          c.rows = c.cols = ks;
          c.src_f64 = 0;
          c.dst_f64 = 1;
          P.copy(c, J.S->node_base + J.t);
        }
      }
    }
  }
}

// ---- eigen + ranks + projection (Sec. 3.3) -------------------------------
void plan_eig_ranks(Plan &P, std::vector<TState> &TS, const ht_trunc_opts &o, int *rank_array) {
  (void)rank_array;
  int max_k = 0;
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    S.V64.assign(T.nn, nullptr);
    S.lam_off.assign(T.nn, 0);
    int64_t off = 0;
    for (int t = 0; t < T.nn; ++t) {
      S.lam_off[t] = off;
      off += (t == 0) ? 1 : S.ko[t];
    }
    S.lam = P.palloc<double>((size_t)off);
    for (int t = 1; t < T.nn; ++t) {
      S.V64[t] = P.palloc<double>((size_t)S.ko[t] * S.ko[t]);
      max_k = std::max(max_k, S.ko[t]);
    }
  }
  P.sreset();
  P.begin(L_EIG);
  size_t n_eig = 0;
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    for (int t = 1; t < T.nn; ++t) {
      EigItem e{S.G64[t], S.V64[t], S.lam + S.lam_off[t], S.ko[t]};
      P.eig(e, S.node_base + t);
      n_eig++;
    }
  }
  if (eig_scratch_needed(max_k, (P.dtype == HT_F64 || P.sqrt_gram) ? 0 : 1, P.node_sched ? 1 : (int)n_eig)) {
    // one scratch slab per item of a launch (node schedule: one item per launch)
    size_t per = 4 * (size_t)max_k * max_k;
    size_t cnt = P.node_sched ? 1 : n_eig;
    void *scr = P.salloc_bytes(per * cnt * sizeof(double));
    for (Launch &L : P.launches)
      if (L.kind == L_EIG && !L.scratch) L.scratch = scr;
  }
  // ranks
  P.begin(L_RANKS);
  for (size_t i = 0; i < TS.size(); ++i) {
    TState &S = TS[i];
    const ht_tree &T = S.x->tr;
    S.stats = P.palloc<double>(4);
    RankItem r;
    memset(&r, 0, sizeof(r));
    r.lam = S.lam;
    r.lam_off = P.mpush(S.lam_off.data(), S.lam_off.size());
    r.korth = P.mpush(S.ko.data(), S.ko.size());
    if (o.mode == HT_TRUNC_RANK && o.ranks) r.target = P.mpush(o.ranks, (size_t)T.nn);
    r.r_out = S.r;
    r.stats = S.stats;
    r.root = static_cast<const double *>(node_ptr(S.x, 0));
    r.root_f64 = (P.dtype == HT_F64);
    r.root_count = (int64_t)S.ko[T.s1[0]] * S.ko[T.s2[0]];
    r.nn = T.nn;
    r.t1 = T.s1[0];
    r.t2 = T.s2[0];
    r.d = T.d;
    r.mode = o.mode;
    r.eps_rel = o.eps_relative;
    r.cap = o.tensor_caps ? o.tensor_caps[i] : o.rank_cap;
    r.eps = o.eps;
    // FP64 storage: the plain rule on the computed tail (as the oracle).  FP32
    // storage: every dropped eigenvalue is also charged the noise floor of an
    // FP32-computed Gramian eigenvalue, 4 sqrt(2d-1) u_32 lambda_max (every
    // node's rounding perturbs X independently), so that an eps below what the
    // path resolves keeps rank instead of cutting noise; square-root Gramians
    // perturb the singular values, not their squares: the square of that.
    r.noise = 0.0;
    if (P.dtype != HT_F64) {
      r.noise = 4.0 * std::sqrt(2.0 * T.d - 1.0) * 0x1p-24;
      if (P.sqrt_gram) r.noise = r.noise * r.noise;
    }
    P.rank(r, S.node_base);
  }
}

void plan_project(Plan &P, std::vector<TState> &TS, const int *rank_array) {
  const size_t esz = P.esz;
  const bool f64 = (P.dtype == HT_F64);
  P.sreset();
  // eigenvectors in the working precision; the root's "Q" is the 1x1 identity
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    S.V.assign(T.nn, nullptr);
    S.V[0] = P.palloc_bytes(esz);
    for (int t = 1; t < T.nn; ++t) S.V[t] = f64 ? (void *)S.V64[t] : P.palloc_bytes((size_t)S.ko[t] * S.ko[t] * esz);
  }
  P.begin(L_COPY);
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    CopyItem c = copy0();
    c.dst = S.V[0];
    c.rows = c.cols = 1;
    c.dr = c.dc = 1;
    c.dst_f64 = f64;
    P.copy(c, S.node_base);
    if (!f64) {
      for (int t = 1; t < T.nn; ++t) {
        CopyItem v = copy0();
        v.src = S.V64[t];
        v.dst = S.V[t];
        v.sr = v.dr = 1;
        v.sc = v.dc = S.ko[t];
        v.rows = v.cols = S.ko[t];
        v.src_f64 = 1;
        v.dst_f64 = 0;
        P.copy(v, S.node_base + t);
      }
    }
  }
  const void *rk = rank_array;
  // leaves: Out = U Q|_r
  struct LJob {
    TState *S;
    int t;
    int64_t nm;
    void *out;
  };
  std::vector<LJob> lj;
  P.begin(L_GEMM, rk);
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    for (int t = 0; t < T.nn; ++t) {
      if (!is_leaf(T, t)) continue;
      const int64_t nm = S.x->n[T.lo[t]];
      const int ko = S.ko[t];
      LJob J{&S, t, nm, P.salloc_bytes((size_t)nm * ko * esz)};
      lj.push_back(J);
      GemmItem g = gemm0();
      g.A = node_ptr(S.x, t);
      g.sam = 1;
      g.sak = nm;
      g.B = S.V[t];
      g.sbk = 1;
      g.sbn = ko;
      g.C = J.out;
      g.scm = 1;
      g.scn = nm;
      g.M = (int)nm;
      g.N = ko;
      g.n_ref = S.node_base + t;
      g.K = ko;
      P.gemm(g, S.node_base + t);
    }
  }
  // inner nodes and root: (Q_t|_r^T, Q_s1|_r^T, Q_s2|_r^T) o B, mode 1, 2, 3
  struct IJob {
    TState *S;
    int t, K0, k1, k2;
    void *P1, *P2, *P3;
  };
  std::vector<IJob> ij;
  for (TState &S : TS) {
    const ht_tree &T = S.x->tr;
    for (int t = 0; t < T.nn; ++t) {
      if (is_leaf(T, t)) continue;
      IJob J;
      J.S = &S;
      J.t = t;
      J.K0 = (t == 0) ? 1 : S.ko[t];
      J.k1 = S.ko[T.s1[t]];
      J.k2 = S.ko[T.s2[t]];
      const size_t sz = (size_t)J.K0 * J.k1 * J.k2 * esz;
      J.P1 = P.salloc_bytes(sz);
      J.P2 = P.salloc_bytes(sz);
      J.P3 = P.salloc_bytes(sz);
      ij.push_back(J);
    }
  }
  P.begin(L_GEMM, rk);
  for (IJob &J : ij) {  // mode 1: P1 (k1k2 x r0) = B_mat (k1k2 x K0) * Q_t[:, :r0]
    const int64_t kk = (int64_t)J.k1 * J.k2;
    GemmItem g = gemm0();
    g.A = node_ptr(J.S->x, J.t);
    g.sam = 1;
    g.sak = kk;
    g.B = J.S->V[J.t];
    g.sbk = 1;
    g.sbn = J.K0;
    g.C = J.P1;
    g.scm = 1;
    g.scn = kk;
    g.M = (int)kk;
    g.N = J.K0;
    g.n_ref = (J.t == 0) ? -1 : J.S->node_base + J.t;
    g.K = J.K0;
    P.gemm(g, J.S->node_base + J.t);
  }
  P.begin(L_GEMM, rk);
  for (IJob &J : ij) {  // mode 2: per a < r0, P2[a] (k2 x r1) = P1[a] (k2 x k1) * Q_s1[:, :r1]
    const ht_tree &T = J.S->x->tr;
    const int64_t kk = (int64_t)J.k1 * J.k2;
    GemmItem g = gemm0();
    g.A = J.P1;
    g.sam = 1;
    g.sak = J.k2;
    g.sab = kk;
    g.B = J.S->V[T.s1[J.t]];
    g.sbk = 1;
    g.sbn = J.k1;
    g.C = J.P2;
    g.scm = 1;
    g.scn = J.k2;
    g.scb = kk;
    g.M = J.k2;
    g.N = J.k1;
    g.n_ref = J.S->node_base + T.s1[J.t];
    g.K = J.k1;
    g.batch = J.K0;
    g.b_ref = (J.t == 0) ? -1 : J.S->node_base + J.t;
    P.gemm(g, J.S->node_base + J.t);
  }
  P.begin(L_GEMM, rk);
  for (IJob &J : ij) {  // mode 3: P3 (r2 x (a,b)) = Q_s2[:, :r2]^T * P2_view (k2 x (a*k1+b))
    const ht_tree &T = J.S->x->tr;
    GemmItem g = gemm0();
    g.A = J.S->V[T.s2[J.t]];
    g.sam = J.k2;
    g.sak = 1;
    g.B = J.P2;
    g.sbk = 1;
    g.sbn = J.k2;
    g.C = J.P3;
    g.scm = 1;
    g.scn = J.k2;
    g.M = J.k2;
    g.m_ref = J.S->node_base + T.s2[J.t];
    g.N = J.K0 * J.k1;
    if (J.t != 0) {
      g.n_ref = J.S->node_base + J.t;
      g.n_mult = J.k1;
    }
    g.K = J.k2;
    P.gemm(g, J.S->node_base + J.t);
  }
  P.begin(L_COMPACT, rk);
  for (IJob &J : ij) {
    const ht_tree &T = J.S->x->tr;
    CompactItem c;
    c.src = J.P3;
    c.dst = node_ptr(J.S->x, J.t);
    c.ref0 = (J.t == 0) ? -1 : J.S->node_base + J.t;
    c.ref1 = J.S->node_base + T.s1[J.t];
    c.ref2 = J.S->node_base + T.s2[J.t];
    c.ld1 = J.k1;
    c.ld2 = J.k2;
    c.max0 = J.K0;
    c.max1 = J.k1;
    c.max2 = J.k2;
    P.compact(c, J.S->node_base + J.t);
  }
  P.begin(L_COPY, rk);
  for (LJob &J : lj) {
    CopyItem c = copy0();
    c.src = J.out;
    c.dst = node_ptr(J.S->x, J.t);
    c.sr = c.dr = 1;
    c.sc = c.dc = J.nm;
    c.rows = (int)J.nm;
    c.cols = J.S->ko[J.t];
    c.cols_ref = J.S->node_base + J.t;
    c.src_f64 = c.dst_f64 = f64;
    P.copy(c, J.S->node_base + J.t);
  }
}

// ---- inner product <X, Y> (Sec. 3.2, Definition "phi", Lemma "phi") -------
// Phi_t = U_t^T V_t bottom-up: leaves Phi = U^T V; inner nodes
// Phi_t[i, i'] = sum B_t[i, j, l] Phi_s1[j, j'] Phi_s2[l, l'] B'_t[i', j', l'],
// as three contractions per node: T1 = Phi_s1 B'_t (mode 2), T2 = Phi_s2 T1
// (mode 3), Phi_t = M_1(B_t) M_1(T2)^T; the root's 1 x 1 Phi is <X, Y>.
void *plan_inner(Plan &P, const ht_tensor *x, const ht_tensor *y) {
  const ht_tree &T = x->tr;
  const size_t esz = P.esz;
  std::vector<void *> phi(T.nn);
  for (int t = 0; t < T.nn; ++t) {
    const int kx = (t == 0) ? 1 : x->k[t], ky = (t == 0) ? 1 : y->k[t];
    phi[t] = P.palloc_bytes((size_t)kx * ky * esz);
  }
  constexpr int kChunk = 256;
  for (int h = 0; h <= T.max_height; ++h) {
    P.sreset();
    if (h == 0) {
      int tiles = 0;
      for (int t = 0; t < T.nn; ++t)
        if (is_leaf(T, t)) tiles += ((x->k[t] + 63) / 64) * ((y->k[t] + 63) / 64);
      P.begin(L_GEMM);
      for (int t = 0; t < T.nn; ++t) {
        if (!is_leaf(T, t)) continue;
        const int64_t n = x->n[T.lo[t]];
        GemmItem g = gemm0();
        g.A = node_ptr(x, t);  // U^T: element (m, k) = U[k, m]
        g.sam = n;
        g.sak = 1;
        g.sako = kChunk;
        g.B = node_ptr(y, t);
        g.sbk = 1;
        g.sbn = n;
        g.sbko = kChunk;
        g.C = phi[t];
        g.scm = 1;
        g.scn = x->k[t];
        g.M = x->k[t];
        g.N = y->k[t];
        g.K = (int)std::min<int64_t>(n, kChunk);
        g.Ko = (int)((n + kChunk - 1) / kChunk);
        g.k_total = n;
        g.ksplit = split_for(tiles, g.Ko);
        P.gemm(g, t);
      }
      continue;
    }
    struct Job {
      int t, K0, K0y, k1, k2, k1y, k2y;
      void *T1, *T2;
    };
    std::vector<Job> jobs;
    for (int t = 0; t < T.nn; ++t) {
      if (is_leaf(T, t) || T.height[t] != h) continue;
      Job J;
      J.t = t;
      J.K0 = (t == 0) ? 1 : x->k[t];
      J.K0y = (t == 0) ? 1 : y->k[t];
      J.k1 = x->k[T.s1[t]];
      J.k2 = x->k[T.s2[t]];
      J.k1y = y->k[T.s1[t]];
      J.k2y = y->k[T.s2[t]];
      J.T1 = P.salloc_bytes((size_t)J.K0y * J.k1 * J.k2y * esz);
      J.T2 = P.salloc_bytes((size_t)J.K0y * J.k1 * J.k2 * esz);
      jobs.push_back(J);
    }
    // T1[i'][j][l'] = sum_j' Phi_s1[j, j'] B'[i', j', l']
    P.begin(L_GEMM);
    for (Job &J : jobs) {
      GemmItem g = gemm0();
      g.A = phi[T.s1[J.t]];
      g.sam = 1;
      g.sak = J.k1;
      g.B = node_ptr(y, J.t);
      g.sbk = J.k2y;
      g.sbn = 1;
      g.sbb = (int64_t)J.k1y * J.k2y;
      g.C = J.T1;
      g.scm = J.k2y;
      g.scn = 1;
      g.scb = (int64_t)J.k1 * J.k2y;
      g.M = J.k1;
      g.N = J.k2y;
      g.K = J.k1y;
      g.batch = J.K0y;
      P.gemm(g, J.t);
    }
    // T2[i'][j][l] = sum_l' Phi_s2[l, l'] T1[i'][j][l']
    P.begin(L_GEMM);
    for (Job &J : jobs) {
      GemmItem g = gemm0();
      g.A = phi[T.s2[J.t]];
      g.sam = 1;
      g.sak = J.k2;
      g.B = J.T1;
      g.sbk = 1;
      g.sbn = J.k2y;
      g.C = J.T2;
      g.scm = 1;
      g.scn = J.k2;
      g.M = J.k2;
      g.N = J.K0y * J.k1;
      g.K = J.k2y;
      P.gemm(g, J.t);
    }
    // Phi_t[i, i'] = sum_{j,l} B[i][j][l] T2[i'][j][l]
    int tiles = 0;
    for (Job &J : jobs) tiles += ((J.K0 + 63) / 64) * ((J.K0y + 63) / 64);
    P.begin(L_GEMM);
    for (Job &J : jobs) {
      const int64_t red = (int64_t)J.k1 * J.k2;
      GemmItem g = gemm0();
      g.A = node_ptr(x, J.t);
      g.sam = red;
      g.sak = 1;
      g.sako = kChunk;
      g.B = J.T2;
      g.sbk = 1;
      g.sbn = red;
      g.sbko = kChunk;
      g.C = phi[J.t];
      g.scm = 1;
      g.scn = J.K0;
      g.M = J.K0;
      g.N = J.K0y;
      g.K = (int)std::min<int64_t>(red, kChunk);
      g.Ko = (int)((red + kChunk - 1) / kChunk);
      g.k_total = red;
      g.ksplit = split_for(tiles, g.Ko);
      P.gemm(g, J.t);
    }
  }
  return phi[0];
}

ht_status check_prec(const ht_tensor *x, int prec) {
  if ((prec == HT_PREC_FP64 || prec == HT_PREC_MIXED) && x->dtype != HT_F64)
    return fail(HT_EUNSUPPORTED, "HT_PREC_FP64 and HT_PREC_MIXED need an HT_F64 tensor");
  if ((prec == HT_PREC_FP32 || prec == HT_PREC_FP32_SQRT) && x->dtype != HT_F32)
    return fail(HT_EUNSUPPORTED, "HT_PREC_FP32 and HT_PREC_FP32_SQRT need an HT_F32 tensor");
  if (prec != HT_PREC_FP64 && prec != HT_PREC_FP32 && prec != HT_PREC_FP32_SQRT && prec != HT_PREC_MIXED)
    return fail(HT_EINVAL, "unknown precision");
  return HT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *ht_last_error(void) { return g_err.c_str(); }

ht_status ht_profile_set(unsigned mask) {
  g_prof_mask = mask & ((1u << HT_K_COUNT) - 1);
  return HT_OK;
}

ht_status ht_profile_read(int kind, int64_t *launches, double *total_ms, double *flops, int reset) {
  if (kind < 0 || kind >= HT_K_COUNT) return fail(HT_EINVAL, "bad kernel kind");
  int64_t cnt = 0;
  double ms = 0.0, fl = 0.0;
  for (const ProfRec &r : g_prof_done) {
    if (r.kind != kind) continue;
    HT_CU(cudaEventSynchronize(r.b));
    float f = 0.f;
    HT_CU(cudaEventElapsedTime(&f, r.a, r.b));
    ms += f;
    fl += r.flops;
    cnt++;
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  if (flops) *flops = fl;
  if (reset) {
    std::vector<ProfRec> keep;
    for (const ProfRec &r : g_prof_done) {
      if (r.kind == kind) {
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
      } else {
        keep.push_back(r);
      }
    }
    g_prof_done.swap(keep);
  }
  return HT_OK;
}

ht_status ht_device_status(void) {
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  const unsigned t = oz_take_status();
  const unsigned w = wait_take_status();
  const unsigned q = eig_take_status();
  const unsigned m = misc_take_status();
  if (t == ~0u || w == ~0u || q == ~0u || m == ~0u) return fail(HT_ECUDA, "reading a device status word failed");
  if (t) return fail(HT_ETIMEOUT, "a bounded wait of the tensor-core contraction gave up (its results are NaN)");
  if (w) return fail(HT_ETIMEOUT, "a bounded device-side wait gave up");
  if (q) return fail(HT_ENUMERIC, "an eigensolver sweep reached its iteration limit");
  if (m) return fail(HT_ENUMERIC, "||X|| or a Gramian eigenvalue was not finite (NaN or Inf in the input)");
  return HT_OK;
}

ht_status ht_selftest_wait(double limit_ms, void *stream) {
  if (!(limit_ms >= 0.0) || limit_ms > 1000.0) return fail(HT_EINVAL, "limit_ms must lie in [0, 1000]");
  const cudaError_t e = launch_selftest_wait((int64_t)(limit_ms * 1e6), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(HT_ECUDA, std::string("self-test launch failed: ") + cudaGetErrorString(e));
  return HT_OK;
}

ht_status ht_set_gemm_tuning(int tall_m, double tall_share, double square_share) {
  if (tall_m < 0) {
    g_gemm_tune = GemmTune();
    return HT_OK;
  }
  if (!(tall_share >= 0.0) || !(square_share >= 0.0)) return fail(HT_EINVAL, "shares must be >= 0");
  g_gemm_tune.tall_m = tall_m;
  g_gemm_tune.tall_share = tall_share;
  g_gemm_tune.square_share = square_share;
  return HT_OK;
}

ht_status ht_launch_count(int64_t *total) {
  if (!total) return fail(HT_EINVAL, "null argument");
  *total = g_launches.load();
  return HT_OK;
}

ht_status ht_tree_balanced(int d, ht_tree **out) {
  if (!out) return fail(HT_EINVAL, "null output");
  if (d < 2 || d > 1 << 20) return fail(HT_EINVAL, "d must be >= 2");
  ht_tree *T = new ht_tree();
  tree_init(T, d);
  *out = T;
  return HT_OK;
}

void ht_tree_free(ht_tree *tree) { delete tree; }

int ht_tree_num_nodes(const ht_tree *tree) { return tree ? tree->nn : -1; }

ht_status ht_tree_node(const ht_tree *T, int t, int *lo, int *hi, int *parent, int *son1, int *son2, int *depth,
                       int *height) {
  if (!T || t < 0 || t >= T->nn) return fail(HT_EINVAL, "bad node");
  if (lo) *lo = T->lo[t];
  if (hi) *hi = T->hi[t];
  if (parent) *parent = T->par[t];
  if (son1) *son1 = T->s1[t];
  if (son2) *son2 = T->s2[t];
  if (depth) *depth = T->depth[t];
  if (height) *height = T->height[t];
  return HT_OK;
}

ht_status ht_tensor_create(const ht_tree *tree, const int64_t *n, const int *ranks, ht_dtype dtype, void *stream,
                           ht_tensor **out) {
  if (!tree || !n || !ranks || !out) return fail(HT_EINVAL, "null argument");
  if (dtype != HT_F64 && dtype != HT_F32) return fail(HT_EINVAL, "bad dtype");
  for (int m = 0; m < tree->d; ++m)
    if (n[m] < 1) return fail(HT_EINVAL, "mode sizes must be >= 1");
  for (int t = 1; t < tree->nn; ++t)
    if (ranks[t] < 1) return fail(HT_EINVAL, "ranks must be >= 1");
  HT_TRY(tensor_alloc(*tree, n, ranks, dtype, (cudaStream_t)stream, out));
  ht_tensor *x = *out;
  HT_CU(cudaMemsetAsync(x->arena, 0, x->slot[tree->nn] * x->esz, x->stream));
  return HT_OK;
}

ht_status ht_tensor_free(ht_tensor *x) {
  if (!x) return HT_OK;
  cudaFreeAsync(x->arena, x->stream);
  cudaFreeAsync(x->d_ranks, x->stream);
  delete x;
  return HT_OK;
}

ht_status ht_tensor_ranks(ht_tensor *x, int *ranks) {
  if (!x || !ranks) return fail(HT_EINVAL, "null argument");
  HT_TRY(sync_ranks(x));
  memcpy(ranks, x->k.data(), sizeof(int) * x->tr.nn);
  return HT_OK;
}

ht_status ht_tensor_blob_size(ht_tensor *x, int64_t *count) {
  if (!x || !count) return fail(HT_EINVAL, "null argument");
  HT_TRY(sync_ranks(x));
  int64_t s = 0;
  for (int t = 0; t < x->tr.nn; ++t) s += node_elems(x->tr, x->n, x->k, t);
  *count = s;
  return HT_OK;
}

static bool at_capacity(const ht_tensor *x) {
  for (int t = 1; t < x->tr.nn; ++t)
    if (x->k[t] != x->cap[t]) return false;
  return true;
}

// gather / scatter between the slots and a packed blob held in device memory
static ht_status pack_copy(ht_tensor *x, void *packed, bool to_packed) {
  Plan P;
  P.dtype = x->dtype;
  P.esz = x->esz;
  P.begin(L_COPY);
  int64_t o = 0;
  for (int t = 0; t < x->tr.nn; ++t) {
    int64_t c = node_elems(x->tr, x->n, x->k, t);
    CopyItem it = copy0();
    char *pk = static_cast<char *>(packed) + o * x->esz;
    it.src = to_packed ? node_ptr(x, t) : pk;
    it.dst = to_packed ? (void *)pk : node_ptr(x, t);
    it.sr = it.dr = 1;
    it.sc = it.dc = c;
    it.rows = (int)c;
    it.cols = 1;
    it.src_f64 = it.dst_f64 = (x->dtype == HT_F64);
    P.copy(it, t);
    o += c;
  }
  return run_plan(P, x->stream, nullptr);
}

ht_status ht_tensor_upload(ht_tensor *x, const void *host_blob) {
  if (!x || !host_blob) return fail(HT_EINVAL, "null argument");
  HT_TRY(sync_ranks(x));
  int64_t count = 0;
  for (int t = 0; t < x->tr.nn; ++t) count += node_elems(x->tr, x->n, x->k, t);
  if (at_capacity(x)) {
    HT_CU(cudaMemcpyAsync(x->arena, host_blob, count * x->esz, cudaMemcpyHostToDevice, x->stream));
  } else {
    void *tmp = nullptr;
    HT_CU(cudaMallocAsync(&tmp, count * x->esz, x->stream));
    HT_CU(cudaMemcpyAsync(tmp, host_blob, count * x->esz, cudaMemcpyHostToDevice, x->stream));
    HT_TRY(pack_copy(x, tmp, false));
    HT_CU(cudaFreeAsync(tmp, x->stream));
  }
  x->orthogonal = false;
  return HT_OK;
}

ht_status ht_tensor_download(ht_tensor *x, void *host_blob) {
  if (!x || !host_blob) return fail(HT_EINVAL, "null argument");
  HT_TRY(sync_ranks(x));
  int64_t count = 0;
  for (int t = 0; t < x->tr.nn; ++t) count += node_elems(x->tr, x->n, x->k, t);
  if (at_capacity(x)) {
    HT_CU(cudaMemcpyAsync(host_blob, x->arena, count * x->esz, cudaMemcpyDeviceToHost, x->stream));
  } else {
    void *tmp = nullptr;
    HT_CU(cudaMallocAsync(&tmp, count * x->esz, x->stream));
    HT_TRY(pack_copy(x, tmp, true));
    HT_CU(cudaMemcpyAsync(host_blob, tmp, count * x->esz, cudaMemcpyDeviceToHost, x->stream));
    HT_CU(cudaFreeAsync(tmp, x->stream));
  }
  HT_CU(cudaStreamSynchronize(x->stream));
  return HT_OK;
}

ht_status ht_tensor_node_ptr(ht_tensor *x, int t, void **dev, int64_t *count) {
  if (!x || t < 0 || t >= x->tr.nn) return fail(HT_EINVAL, "bad node");
  HT_TRY(sync_ranks(x));
  if (dev) *dev = node_ptr(x, t);
  if (count) *count = node_elems(x->tr, x->n, x->k, t);
  return HT_OK;
}

ht_status ht_scale(ht_tensor *x, double alpha) {
  if (!x) return fail(HT_EINVAL, "null tensor");
  HT_TRY(sync_ranks(x));
  int64_t c = node_elems(x->tr, x->n, x->k, 0);
  cudaError_t e = (x->dtype == HT_F64) ? launch_scale<double>(node_ptr(x, 0), c, alpha, x->stream)
                                       : launch_scale<float>(node_ptr(x, 0), c, alpha, x->stream);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  return HT_OK;
}

static ht_status add_check(const ht_tensor *a, const ht_tensor *c) {
  if (!a || !c) return fail(HT_EINVAL, "null tensor");
  if (a->tr.d != c->tr.d) return fail(HT_EINVAL, "tensors have different d");
  if (a->dtype != c->dtype) return fail(HT_EINVAL, "tensors have different dtype");
  for (int m = 0; m < a->tr.d; ++m)
    if (a->n[m] != c->n[m]) return fail(HT_EINVAL, "tensors have different mode sizes");
  return HT_OK;
}

// Descriptor of the addition packing: 12 int64 per node (kind, the three
// slot offsets, shapes of the two summands, element count of the sum).
static std::vector<int64_t> add_desc(const ht_tensor *a, const ht_tensor *c, const ht_tensor *o, int64_t *max_e) {
  const ht_tree &T = a->tr;
  std::vector<int64_t> desc(12 * (size_t)T.nn, 0);
  *max_e = 0;
  for (int t = 0; t < T.nn; ++t) {
    int64_t *ds = &desc[12 * (size_t)t];
    ds[1] = a->slot[t];
    ds[2] = c->slot[t];
    ds[3] = o->slot[t];
    ds[11] = node_elems(T, o->n, o->k, t);
    *max_e = std::max(*max_e, ds[11]);
    if (is_leaf(T, t)) {
      ds[0] = 0;
      ds[4] = a->n[T.lo[t]];
      ds[5] = a->k[t];
      ds[6] = c->k[t];
    } else {
      ds[0] = 1;
      ds[4] = (t == 0) ? 1 : a->k[t];
      ds[5] = (t == 0) ? 0 : 1;
      ds[7] = a->k[T.s1[t]];
      ds[8] = a->k[T.s2[t]];
      ds[9] = c->k[T.s1[t]];
      ds[10] = c->k[T.s2[t]];
    }
  }
  return desc;
}

static cudaError_t add_launch(const ht_tensor *a, const ht_tensor *c, ht_tensor *o, const int64_t *d_desc, int64_t max_e,
                              cudaStream_t s) {
  prof_begin(HT_K_ADD, s);
  cudaError_t e = (a->dtype == HT_F64) ? launch_pack_add<double>(a->arena, c->arena, o->arena, d_desc, a->tr.nn, max_e, s)
                                       : launch_pack_add<float>(a->arena, c->arena, o->arena, d_desc, a->tr.nn, max_e, s);
  prof_end(HT_K_ADD, s, 0.0);
  return e;
}

static ht_status add_pack(const ht_tensor *a, const ht_tensor *c, ht_tensor *o) {
  int64_t max_e = 0;
  std::vector<int64_t> desc = add_desc(a, c, o, &max_e);
  int64_t *d_desc = nullptr;
  HT_CU(cudaMallocAsync((void **)&d_desc, desc.size() * sizeof(int64_t), o->stream));
  HT_CU(cudaMemcpyAsync(d_desc, desc.data(), desc.size() * sizeof(int64_t), cudaMemcpyHostToDevice, o->stream));
  cudaError_t e = add_launch(a, c, o, d_desc, max_e, o->stream);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  HT_CU(cudaFreeAsync(d_desc, o->stream));
  return HT_OK;
}

ht_status ht_add(const ht_tensor *a, const ht_tensor *c, ht_tensor **out) {
  HT_TRY(add_check(a, c));
  if (!out) return fail(HT_EINVAL, "null output");
  HT_TRY(sync_ranks(const_cast<ht_tensor *>(a)));
  HT_TRY(sync_ranks(const_cast<ht_tensor *>(c)));
  if (a->stream != c->stream) {
    // c's pending work must be visible on a's stream
    HT_CU(cudaStreamSynchronize(c->stream));
  }
  std::vector<int> k(a->tr.nn);
  for (int t = 0; t < a->tr.nn; ++t) k[t] = a->k[t] + c->k[t];
  k[0] = 1;
  HT_TRY(tensor_alloc(a->tr, a->n.data(), k.data(), a->dtype, a->stream, out));
  return add_pack(a, c, *out);
}

ht_status ht_add_into(const ht_tensor *a, const ht_tensor *c, ht_tensor *out) {
  HT_TRY(add_check(a, c));
  if (!out) return fail(HT_EINVAL, "null output");
  HT_TRY(sync_ranks(const_cast<ht_tensor *>(a)));
  HT_TRY(sync_ranks(const_cast<ht_tensor *>(c)));
  if (out->tr.d != a->tr.d || out->dtype != a->dtype) return fail(HT_EINVAL, "output does not match");
  for (int t = 1; t < a->tr.nn; ++t)
    if (out->cap[t] != a->k[t] + c->k[t]) return fail(HT_EINVAL, "output capacity must equal k + kbar");
  out->k = out->cap;
  out->k[0] = 1;
  out->orthogonal = false;
  HT_TRY(upload_ranks(out));
  return add_pack(a, c, out);
}

ht_status ht_apply(const ht_tensor *op, const ht_tensor *x, ht_tensor *out) {
  if (!op || !x || !out) return fail(HT_EINVAL, "null argument");
  if (op->tr.d != x->tr.d || out->tr.d != x->tr.d) return fail(HT_EINVAL, "tensors have different d");
  if (op->dtype != x->dtype || out->dtype != x->dtype) return fail(HT_EINVAL, "tensors have different dtype");
  const ht_tree &T = x->tr;
  for (int mu = 0; mu < T.d; ++mu)
    if (op->n[mu] != out->n[mu] * x->n[mu])
      return fail(HT_EINVAL, "operator mode size must be (output mode size) x (tensor mode size)");
  HT_TRY(sync_ranks(const_cast<ht_tensor *>(op)));
  HT_TRY(sync_ranks(const_cast<ht_tensor *>(x)));
  for (int t = 1; t < T.nn; ++t)
    if (out->cap[t] != op->k[t] * x->k[t]) return fail(HT_EINVAL, "output capacity must equal kbar_t k_t");
  cudaStream_t s = out->stream;
  if (op->stream != s) HT_CU(cudaStreamSynchronize(op->stream));
  if (x->stream != s) HT_CU(cudaStreamSynchronize(x->stream));
  out->k = out->cap;
  out->k[0] = 1;
  out->orthogonal = false;
  HT_TRY(upload_ranks(out));
  // leaves: V[:, r k + l] = W_r U[:, l], W_r the m x n column-major matrix in column r of the operator's leaf
  Plan P;
  P.dtype = x->dtype;
  P.esz = x->esz;
  P.begin(L_GEMM);
  for (int t = 0; t < T.nn; ++t) {
    if (!is_leaf(T, t)) continue;
    const int mu = T.lo[t];
    const int64_t m = out->n[mu], n = x->n[mu];
    const int kb = op->k[t], k = x->k[t];
    GemmItem g = gemm0();
    g.A = node_ptr(op, t);
    g.sam = 1;
    g.sak = m;
    g.sab = m * n;
    g.B = node_ptr(x, t);
    g.sbk = 1;
    g.sbn = n;
    g.sbb = 0;
    g.C = node_ptr(out, t);
    g.scm = 1;
    g.scn = m;
    g.scb = m * k;
    g.M = (int)m;
    g.N = k;
    g.K = (int)n;
    g.batch = kb;
    P.gemm(g, t);
  }
  HT_TRY(run_plan(P, s, nullptr));
  // inner nodes: F_t = H_t (x) B_t
  std::vector<int64_t> desc;
  int64_t max_e = 0;
  int cnt = 0;
  for (int t = 0; t < T.nn; ++t) {
    if (is_leaf(T, t)) continue;
    const int64_t pt = (t == 0) ? 1 : op->k[t], p1 = op->k[T.s1[t]], p2 = op->k[T.s2[t]];
    const int64_t it = (t == 0) ? 1 : x->k[t], i1 = x->k[T.s1[t]], i2 = x->k[T.s2[t]];
    const int64_t count = pt * it * p1 * i1 * p2 * i2;
    desc.push_back(op->slot[t]);
    desc.push_back(x->slot[t]);
    desc.push_back(out->slot[t]);
    desc.push_back(pt | (p1 << 20) | (p2 << 40));
    desc.push_back(it | (i1 << 20) | (i2 << 40));
    desc.push_back(count);
    max_e = std::max(max_e, count);
    ++cnt;
  }
  int64_t *d_desc = nullptr;
  HT_CU(cudaMallocAsync((void **)&d_desc, desc.size() * sizeof(int64_t), s));
  HT_CU(cudaMemcpyAsync(d_desc, desc.data(), desc.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  prof_begin(HT_K_MISC, s);
  cudaError_t e = (x->dtype == HT_F64) ? launch_kron<double>(op->arena, x->arena, out->arena, d_desc, cnt, max_e, s)
                                       : launch_kron<float>(op->arena, x->arena, out->arena, d_desc, cnt, max_e, s);
  prof_end(HT_K_MISC, s, 0.0);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  HT_CU(cudaFreeAsync(d_desc, s));
  // the host copy of desc must outlive the staged copy
  HT_CU(cudaStreamSynchronize(s));
  return HT_OK;
}

ht_status ht_orthogonalize(ht_tensor *x, int prec) {
  if (!x) return fail(HT_EINVAL, "null tensor");
  HT_TRY(check_prec(x, prec));
  HT_TRY(sync_ranks(x));
  Plan P;
  P.dtype = x->dtype;
  P.esz = x->esz;
  P.mixed = (prec == HT_PREC_MIXED);
  if (P.mixed) P.panel = kPanelMixed;
  std::vector<TState> TS(1);
  TS[0].x = x;
  plan_orthogonalize(P, TS);
  HT_TRY(run_plan(P, x->stream, nullptr));
  x->k = TS[0].ko;
  x->orthogonal = true;
  return upload_ranks(x);
}

ht_status ht_gramians(ht_tensor *x, double *dev_out, int prec) {
  if (!x || !dev_out) return fail(HT_EINVAL, "null argument");
  HT_TRY(check_prec(x, prec));
  HT_TRY(sync_ranks(x));
  Plan P;
  P.sqrt_gram = (prec == HT_PREC_FP32_SQRT);
  P.mixed = (prec == HT_PREC_MIXED);
  if (P.mixed) P.panel = kPanelMixed;
  P.dtype = x->dtype;
  P.esz = x->esz;
  std::vector<TState> TS(1);
  TS[0].x = x;
  TS[0].ko = x->k;
  std::vector<double *> outs{dev_out};
  plan_gramians(P, TS, &outs);
  return run_plan(P, x->stream, nullptr);
}

// ---------------------------------------------------------------------------
// ht_gramians_noalloc: the Gramian computation with its workspace (work-item
// lists, Gramian copies, contraction temporaries, split-K partial sums) held
// in one fixed device array instead of memory allocated per call.  The array
// lives for the whole process on every device that loads the library.  In
// host code its name only denotes a host-side shadow, so the device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, and passed to the kernels through the work items.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[HT_NOALLOC_SCRATCH_BYTES];

static ht_status noalloc_scratch(char **out) {
  static std::mutex mu;
  static char *addr[256] = {};
  int dev = 0;
  HT_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(HT_EUNSUPPORTED, "device ordinal out of range for the fixed scratch");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(HT_ECUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") + cudaGetErrorString(e));
    addr[dev] = static_cast<char *>(p);
  }
  *out = addr[dev];
  return HT_OK;
}

ht_status ht_gramians_noalloc(ht_tensor *x, double *dev_out, int prec) {
  if (!x || !dev_out) return fail(HT_EINVAL, "null argument");
  HT_TRY(check_prec(x, prec));
  {
    // the fixed array looked up below is the current device's: the tensor's
    // stream must run on that device
    int cur = -1, sdev = -1;
    HT_CU(cudaGetDevice(&cur));
    HT_CU(cudaStreamGetDevice(x->stream, &sdev));
    if (sdev != cur)
      return fail(HT_EINVAL, "the tensor's stream runs on device " + std::to_string(sdev) + ", the current device is " +
                                 std::to_string(cur) + ": make the stream's device current");
  }
  char *scratch = nullptr;
  HT_TRY(noalloc_scratch(&scratch));
  HT_TRY(sync_ranks(x));
  Plan P;
  P.sqrt_gram = (prec == HT_PREC_FP32_SQRT);
  P.mixed = (prec == HT_PREC_MIXED);
  if (P.mixed) P.panel = kPanelMixed;
  P.dtype = x->dtype;
  P.esz = x->esz;
  std::vector<TState> TS(1);
  TS[0].x = x;
  TS[0].ko = x->k;
  std::vector<double *> outs{dev_out};
  plan_gramians(P, TS, &outs);
  return run_plan(P, x->stream, nullptr, scratch, HT_NOALLOC_SCRATCH_BYTES);
}

static ht_status truncate_many(ht_tensor *const *xs, int count, const ht_trunc_opts *o, ht_trunc_report *rep) {
  if (!xs || count < 1 || !o) return fail(HT_EINVAL, "null argument");
  if (o->mode != HT_TRUNC_RANK && o->mode != HT_TRUNC_EPS) return fail(HT_EINVAL, "bad mode");
  if (o->mode == HT_TRUNC_EPS && !(o->eps >= 0.0)) return fail(HT_EINVAL, "eps must be >= 0");
  if (o->qr_kernel < 0 || o->qr_kernel > 3) return fail(HT_EINVAL, "qr_kernel must be 0, 1, 2 or 3");
  for (int i = 0; i < count; ++i)
    if (!xs[i]) return fail(HT_EINVAL, "null tensor");
  const int dtype = xs[0]->dtype;
  cudaStream_t s = xs[0]->stream;
  for (int i = 0; i < count; ++i) {
    if (xs[i]->dtype != dtype) return fail(HT_EINVAL, "batch mixes dtypes");
    HT_TRY(check_prec(xs[i], o->prec));
    HT_TRY(sync_ranks(xs[i]));
  }
  if (count > 1 && o->ranks) return fail(HT_EINVAL, "per-node target ranks are only accepted for a single tensor");
  Plan P;
  P.dtype = dtype;
  P.esz = (dtype == HT_F64) ? 8 : 4;
  P.node_sched = (o->schedule == HT_SCHED_NODE);
  P.sqrt_gram = (o->prec == HT_PREC_FP32_SQRT);
  P.mixed = (o->prec == HT_PREC_MIXED);
  if (P.mixed) P.panel = kPanelMixed;
  P.qr_kernel = o->qr_kernel;
  std::vector<TState> TS(count);
  int total_nodes = 0;
  for (int i = 0; i < count; ++i) {
    TS[i].x = xs[i];
    TS[i].node_base = total_nodes;
    total_nodes += xs[i]->tr.nn;
  }
  int *rank_array = P.palloc<int>((size_t)total_nodes);
  for (int i = 0; i < count; ++i) TS[i].r = rank_array + TS[i].node_base;
  plan_orthogonalize(P, TS);
  plan_gramians(P, TS, nullptr);
  plan_eig_ranks(P, TS, *o, rank_array);
  plan_project(P, TS, rank_array);
  char *pb = nullptr;
  HT_TRY(run_plan(P, s, &pb));
  // the new ranks live on the device
  const int *d_r = reinterpret_cast<const int *>(reloc(rank_array, pb, nullptr, nullptr));
  for (int i = 0; i < count; ++i) {
    ht_tensor *x = xs[i];
    if (x->stream != s) HT_CU(cudaStreamSynchronize(s));
    HT_CU(cudaMemcpyAsync(x->d_ranks, d_r + TS[i].node_base, sizeof(int) * x->tr.nn, cudaMemcpyDeviceToDevice, s));
    x->ranks_ok = false;
    x->orthogonal = false;
  }
  int nonfinite = -1;  // first tensor whose report flags non-finite values
  bool eig_limit = false;  // an eigensolver sweep hit its iteration limit (any call since the last check)
  if (rep) {
    std::vector<int> r(total_nodes);
    HT_CU(cudaMemcpyAsync(r.data(), d_r, sizeof(int) * total_nodes, cudaMemcpyDeviceToHost, s));
    std::vector<std::vector<double>> stats(count, std::vector<double>(4)), lam(count);
    for (int i = 0; i < count; ++i) {
      const double *st = reinterpret_cast<const double *>(reloc(TS[i].stats, pb, nullptr, nullptr));
      HT_CU(cudaMemcpyAsync(stats[i].data(), st, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
      lam[i].resize(TS[i].lam_off.back() + TS[i].ko.back());
      const double *lp = reinterpret_cast<const double *>(reloc(TS[i].lam, pb, nullptr, nullptr));
      HT_CU(cudaMemcpyAsync(lam[i].data(), lp, lam[i].size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    HT_CU(cudaStreamSynchronize(s));
    const unsigned q = eig_take_status();
    if (q == ~0u) return fail(HT_ECUDA, "reading the eigensolver status word failed");
    if (q) eig_limit = true;
    for (int i = 0; i < count; ++i) {
      if (stats[i][3] != 0.0) nonfinite = i;
      ht_trunc_report &R = rep[i];
      R.norm = stats[i][0];
      R.discarded_sq = stats[i][1];
      R.bound = std::sqrt(std::max(0.0, stats[i][1]));
      const int nn = xs[i]->tr.nn;
      if (R.ranks_out) memcpy(R.ranks_out, r.data() + TS[i].node_base, sizeof(int) * nn);
      if (R.korth_out) memcpy(R.korth_out, TS[i].ko.data(), sizeof(int) * nn);
      if (R.sigma_out) {
        int64_t o2 = 0;
        for (int t = 1; t < nn; ++t)
          for (int q = 0; q < TS[i].ko[t]; ++q) {
            double l = lam[i][TS[i].lam_off[t] + q];
            R.sigma_out[o2++] = std::sqrt(l > 0.0 ? l : 0.0);
          }
      }
    }
  }
  HT_CU(cudaFreeAsync(pb, s));
  if (nonfinite >= 0) {
    misc_take_status();  // this call's non-finite values are reported here
    return fail(HT_ENUMERIC, "tensor " + std::to_string(nonfinite) +
                                 " of the call: ||X|| or a Gramian eigenvalue is not finite (NaN or Inf in the input)");
  }
  if (eig_limit) return fail(HT_ENUMERIC, "an eigensolver sweep reached its iteration limit");
  return HT_OK;
}

ht_status ht_truncate(ht_tensor *x, const ht_trunc_opts *opts, ht_trunc_report *report) {
  return truncate_many(&x, 1, opts, report);
}

ht_status ht_truncate_batch(ht_tensor *const *xs, int count, const ht_trunc_opts *opts, ht_trunc_report *reports) {
  return truncate_many(xs, count, opts, reports);
}

// ---------------------------------------------------------------------------
// CUDA graph of addition + truncation (replayed without host work)
// ---------------------------------------------------------------------------
}  // extern "C"

struct ht_graph {
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  char *work = nullptr;  // plan workspace, addition descriptors, rank vectors
  std::vector<ht_tensor *> outs;
  int kernels = 0;
};

static void graph_destroy(ht_graph *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->work) cudaFree(g->work);
  delete g;
}

extern "C" {

ht_status ht_graph_add_truncate(const ht_tensor *const *a, const ht_tensor *const *c, ht_tensor *const *out, int count,
                                const ht_trunc_opts *o, ht_graph **gout) {
  if (!a || !c || !out || count < 1 || !o || !gout) return fail(HT_EINVAL, "null argument");
  *gout = nullptr;
  if (o->mode != HT_TRUNC_RANK && o->mode != HT_TRUNC_EPS) return fail(HT_EINVAL, "bad mode");
  if (o->mode == HT_TRUNC_EPS && !(o->eps >= 0.0)) return fail(HT_EINVAL, "eps must be >= 0");
  if (count > 1 && o->ranks) return fail(HT_EINVAL, "per-node target ranks are only accepted for a single tensor");
  if (o->qr_kernel < 0 || o->qr_kernel > 3) return fail(HT_EINVAL, "qr_kernel must be 0, 1, 2 or 3");
  cudaStream_t s = out[0] ? out[0]->stream : nullptr;
  for (int i = 0; i < count; ++i) {
    HT_TRY(add_check(a[i], c[i]));
    ht_tensor *x = out[i];
    if (!x) return fail(HT_EINVAL, "null output");
    if (x->stream != s || a[i]->stream != s || c[i]->stream != s)
      return fail(HT_EINVAL, "all tensors of a graph must use one stream");
    if (x->tr.d != a[i]->tr.d || x->dtype != a[i]->dtype || x->dtype != out[0]->dtype)
      return fail(HT_EINVAL, "output does not match");
    for (int m = 0; m < x->tr.d; ++m)
      if (x->n[m] != a[i]->n[m]) return fail(HT_EINVAL, "output mode sizes do not match");
    HT_TRY(check_prec(x, o->prec));
    HT_TRY(sync_ranks(const_cast<ht_tensor *>(a[i])));
    HT_TRY(sync_ranks(const_cast<ht_tensor *>(c[i])));
    for (int t = 1; t < x->tr.nn; ++t)
      if (x->cap[t] != a[i]->k[t] + c[i]->k[t]) return fail(HT_EINVAL, "output capacity must equal k + kbar");
  }
  // the outputs take the ranks of the sums; the plan is built for them
  for (int i = 0; i < count; ++i) {
    ht_tensor *x = out[i];
    HT_TRY(sync_ranks(x));
    x->k = x->cap;
    x->k[0] = 1;
    x->orthogonal = false;
    HT_TRY(upload_ranks(x));
  }
  Plan P;
  P.dtype = out[0]->dtype;
  P.esz = (P.dtype == HT_F64) ? 8 : 4;
  P.node_sched = (o->schedule == HT_SCHED_NODE);
  P.sqrt_gram = (o->prec == HT_PREC_FP32_SQRT);
  P.mixed = (o->prec == HT_PREC_MIXED);
  if (P.mixed) P.panel = kPanelMixed;
  P.qr_kernel = o->qr_kernel;
  std::vector<TState> TS(count);
  int total_nodes = 0;
  for (int i = 0; i < count; ++i) {
    TS[i].x = out[i];
    TS[i].node_base = total_nodes;
    total_nodes += out[i]->tr.nn;
  }
  int *rank_array = P.palloc<int>((size_t)total_nodes);
  for (int i = 0; i < count; ++i) TS[i].r = rank_array + TS[i].node_base;
  plan_orthogonalize(P, TS);
  plan_gramians(P, TS, nullptr);
  plan_eig_ranks(P, TS, *o, rank_array);
  plan_project(P, TS, rank_array);
  if (!P.err.empty()) return fail(HT_EUNSUPPORTED, P.err);
  finalize_tables(P);
  // one device buffer: plan workspace | per tensor: addition descriptor, sum ranks
  const size_t plan_sz = (plan_bytes(P) + 255) & ~size_t(255);
  std::vector<size_t> desc_off(count), rk_off(count);
  std::vector<int64_t> max_e(count);
  std::vector<std::vector<int64_t>> descs(count);
  size_t total = plan_sz;
  for (int i = 0; i < count; ++i) {
    descs[i] = add_desc(a[i], c[i], out[i], &max_e[i]);
    desc_off[i] = total;
    total += (descs[i].size() * sizeof(int64_t) + 255) & ~size_t(255);
    rk_off[i] = total;
    total += (out[i]->tr.nn * sizeof(int) + 255) & ~size_t(255);
  }
  ht_graph *g = new ht_graph();
  g->stream = s;
  g->outs.assign(out, out + count);
  cudaError_t e = cudaMalloc((void **)&g->work, total);
  if (e != cudaSuccess) {
    graph_destroy(g);
    return fail(HT_ENOMEM, std::string("graph workspace allocation failed: ") + cudaGetErrorString(e));
  }
  char *ib_dev = nullptr;
  ht_status st = prepare_plan(P, s, g->work, &ib_dev);
  for (int i = 0; i < count && st == HT_OK; ++i) {
    e = cudaMemcpyAsync(g->work + desc_off[i], descs[i].data(), descs[i].size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->work + rk_off[i], out[i]->k.data(), out[i]->tr.nn * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = fail(HT_ECUDA, cudaGetErrorString(e));
  }
  if (st == HT_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = fail(HT_ECUDA, cudaGetErrorString(e));
  if (st != HT_OK) {
    graph_destroy(g);
    return st;
  }
  // capture (on a private stream: the tensors' stream may be the legacy
  // default stream, which cannot be captured): per tensor the rank reset and
  // the addition, then the truncation plan, then the new ranks into every
  // output's rank vector.  Replays are launched on the tensors' stream.
  const cudaStream_t tensor_stream = s;
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    graph_destroy(g);
    return fail(HT_ECUDA, std::string("stream creation failed: ") + cudaGetErrorString(e));
  }
  s = cs;
  const unsigned prof_saved = g_prof_mask;
  g_prof_mask = 0;
  const int64_t launches_saved = g_launches;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    g_prof_mask = prof_saved;
    cudaStreamDestroy(cs);
    graph_destroy(g);
    return fail(HT_ECUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < count && st == HT_OK; ++i) {
    ht_tensor *x = out[i];
    e = cudaMemcpyAsync(x->d_ranks, g->work + rk_off[i], x->tr.nn * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = add_launch(a[i], c[i], x, reinterpret_cast<const int64_t *>(g->work + desc_off[i]), max_e[i], s);
    if (e != cudaSuccess) st = fail(HT_ECUDA, cudaGetErrorString(e));
  }
  if (st == HT_OK) st = enqueue_plan(P, s, ib_dev, nullptr);
  const int *d_r = reinterpret_cast<const int *>(reloc(rank_array, g->work, nullptr, nullptr));
  for (int i = 0; i < count && st == HT_OK; ++i) {
    e = cudaMemcpyAsync(out[i]->d_ranks, d_r + TS[i].node_base, sizeof(int) * out[i]->tr.nn, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = fail(HT_ECUDA, cudaGetErrorString(e));
  }
  e = cudaStreamEndCapture(s, &g->graph);
  g->kernels = (int)(g_launches - launches_saved);
  g_launches = launches_saved;
  g_prof_mask = prof_saved;
  cudaStreamDestroy(cs);
  s = tensor_stream;
  if (st == HT_OK && e != cudaSuccess) st = fail(HT_ECUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
  if (st == HT_OK && (e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
    st = fail(HT_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
  if (st != HT_OK) {
    graph_destroy(g);
    return st;
  }
  for (ht_tensor *x : g->outs) x->ranks_ok = false;
  *gout = g;
  return HT_OK;
}

ht_status ht_graph_launch(ht_graph *g) {
  if (!g) return fail(HT_EINVAL, "null graph");
  cudaError_t e = cudaGraphLaunch(g->exec, g->stream);
  if (e != cudaSuccess) return fail(HT_ECUDA, std::string("graph launch failed: ") + cudaGetErrorString(e));
  g_launches += g->kernels;
  for (ht_tensor *x : g->outs) {
    x->ranks_ok = false;
    x->orthogonal = false;
  }
  return HT_OK;
}

ht_status ht_graph_kernels(const ht_graph *g, int *kernels) {
  if (!g || !kernels) return fail(HT_EINVAL, "null argument");
  *kernels = g->kernels;
  return HT_OK;
}

ht_status ht_graph_free(ht_graph *g) {
  if (!g) return HT_OK;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  graph_destroy(g);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  return HT_OK;
}

ht_status ht_norm(const ht_tensor *xc, double *out) {
  if (!xc || !out) return fail(HT_EINVAL, "null argument");
  ht_tensor *x = const_cast<ht_tensor *>(xc);
  HT_TRY(sync_ranks(x));
  ht_tensor *y = nullptr;
  HT_TRY(tensor_alloc(x->tr, x->n.data(), x->cap.data(), x->dtype, x->stream, &y));
  HT_CU(cudaMemcpyAsync(y->arena, x->arena, x->slot[x->tr.nn] * x->esz, cudaMemcpyDeviceToDevice, x->stream));
  y->k = x->k;
  ht_status st = upload_ranks(y);
  if (st == HT_OK) st = ht_orthogonalize(y, x->dtype == HT_F64 ? HT_PREC_FP64 : HT_PREC_FP32);
  double *d_s = nullptr;
  if (st == HT_OK) {
    int64_t c = node_elems(y->tr, y->n, y->k, 0);
    cudaError_t e = cudaMallocAsync((void **)&d_s, sizeof(double), y->stream);
    if (e == cudaSuccess)
      e = (y->dtype == HT_F64) ? launch_sumsq<double>(node_ptr(y, 0), c, d_s, y->stream)
                               : launch_sumsq<float>(node_ptr(y, 0), c, d_s, y->stream);
    double h = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_s, sizeof(double), cudaMemcpyDeviceToHost, y->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(y->stream);
    if (d_s) cudaFreeAsync(d_s, y->stream);
    if (e != cudaSuccess) st = fail(HT_ECUDA, cudaGetErrorString(e));
    *out = std::sqrt(h);
  }
  ht_tensor_free(y);
  return st;
}

ht_status ht_inner(const ht_tensor *xc, const ht_tensor *yc, double *out) {
  if (!xc || !yc || !out) return fail(HT_EINVAL, "null argument");
  HT_TRY(add_check(xc, yc));
  ht_tensor *x = const_cast<ht_tensor *>(xc), *y = const_cast<ht_tensor *>(yc);
  HT_TRY(sync_ranks(x));
  HT_TRY(sync_ranks(y));
  if (x->stream != y->stream) HT_CU(cudaStreamSynchronize(y->stream));
  Plan P;
  P.dtype = x->dtype;
  P.esz = x->esz;
  void *root = plan_inner(P, x, y);
  char *pb = nullptr;
  HT_TRY(run_plan(P, x->stream, &pb));
  const void *d_root = reloc(root, pb, nullptr, nullptr);
  double v = 0.0;
  float vf = 0.0f;
  cudaError_t e = (x->dtype == HT_F64) ? cudaMemcpyAsync(&v, d_root, sizeof(double), cudaMemcpyDeviceToHost, x->stream)
                                       : cudaMemcpyAsync(&vf, d_root, sizeof(float), cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  cudaFreeAsync(pb, x->stream);
  if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  *out = (x->dtype == HT_F64) ? v : (double)vf;
  return HT_OK;
}

ht_status ht_eval_entries(const ht_tensor *xc, const int64_t *idx, int64_t m, double *out) {
  if (!xc || (!idx && m > 0) || (!out && m > 0) || m < 0) return fail(HT_EINVAL, "null argument");
  if (m == 0) return HT_OK;
  ht_tensor *x = const_cast<ht_tensor *>(xc);
  HT_TRY(sync_ranks(x));
  const ht_tree &T = x->tr;
  const int d = T.d, nn = T.nn;
  for (int64_t e = 0; e < m; ++e)
    for (int mu = 0; mu < d; ++mu)
      if (idx[e * d + mu] < 0 || idx[e * d + mu] >= x->n[mu]) return fail(HT_EINVAL, "index out of range");
  std::vector<int> tree(5 * (size_t)nn);
  std::vector<int64_t> node_off(nn), row_off(nn);
  int64_t rows_per = 0;
  for (int t = 0; t < nn; ++t) {
    tree[5 * t + 0] = is_leaf(T, t) ? 1 : 0;
    tree[5 * t + 1] = T.lo[t];
    tree[5 * t + 2] = T.s1[t];
    tree[5 * t + 3] = T.s2[t];
    tree[5 * t + 4] = T.height[t];
    node_off[t] = x->slot[t];
    row_off[t] = rows_per;
    rows_per += (t == 0) ? 1 : x->k[t];
  }
  std::vector<int> level_nodes;
  std::vector<int> level_start(T.max_height + 2, 0);
  for (int h = 0; h <= T.max_height; ++h) {
    level_start[h] = (int)level_nodes.size();
    for (int t = 0; t < nn; ++t)
      if (T.height[t] == h) level_nodes.push_back(t);
  }
  level_start[T.max_height + 1] = (int)level_nodes.size();
  // one device block: tree | node_off | row_off | n | idx | level_nodes | rows | out
  size_t b_tree = tree.size() * sizeof(int), b_no = nn * sizeof(int64_t), b_n = d * sizeof(int64_t);
  size_t b_idx = (size_t)m * d * sizeof(int64_t), b_lv = level_nodes.size() * sizeof(int);
  size_t b_rows = (size_t)m * rows_per * sizeof(double), b_out = (size_t)m * sizeof(double);
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  size_t o_tree = 0, o_no = al(b_tree), o_ro = o_no + al(b_no), o_n = o_ro + al(b_no), o_idx = o_n + al(b_n);
  size_t o_lv = o_idx + al(b_idx), o_rows = o_lv + al(b_lv), o_out = o_rows + al(b_rows), total = o_out + al(b_out);
  char *blk = nullptr;
  HT_CU(cudaMallocAsync((void **)&blk, total, x->stream));
  HT_CU(cudaMemcpyAsync(blk + o_tree, tree.data(), b_tree, cudaMemcpyHostToDevice, x->stream));
  HT_CU(cudaMemcpyAsync(blk + o_no, node_off.data(), b_no, cudaMemcpyHostToDevice, x->stream));
  HT_CU(cudaMemcpyAsync(blk + o_ro, row_off.data(), b_no, cudaMemcpyHostToDevice, x->stream));
  HT_CU(cudaMemcpyAsync(blk + o_n, x->n.data(), b_n, cudaMemcpyHostToDevice, x->stream));
  HT_CU(cudaMemcpyAsync(blk + o_idx, idx, b_idx, cudaMemcpyHostToDevice, x->stream));
  HT_CU(cudaMemcpyAsync(blk + o_lv, level_nodes.data(), b_lv, cudaMemcpyHostToDevice, x->stream));
  for (int h = 0; h <= T.max_height; ++h) {
    int cnt = level_start[h + 1] - level_start[h];
    const int *lvp = reinterpret_cast<const int *>(blk + o_lv) + level_start[h];
    cudaError_t e =
        (x->dtype == HT_F64)
            ? launch_eval_level<double>(x->arena, (const int64_t *)(blk + o_no), x->d_ranks, (const int *)(blk + o_tree),
                                        (const int64_t *)(blk + o_n), (const int64_t *)(blk + o_idx),
                                        (const int64_t *)(blk + o_ro), rows_per, lvp, cnt, m, d, (double *)(blk + o_rows),
                                        (double *)(blk + o_out), x->stream)
            : launch_eval_level<float>(x->arena, (const int64_t *)(blk + o_no), x->d_ranks, (const int *)(blk + o_tree),
                                       (const int64_t *)(blk + o_n), (const int64_t *)(blk + o_idx),
                                       (const int64_t *)(blk + o_ro), rows_per, lvp, cnt, m, d, (double *)(blk + o_rows),
                                       (double *)(blk + o_out), x->stream);
    if (e != cudaSuccess) return fail(HT_ECUDA, cudaGetErrorString(e));
  }
  HT_CU(cudaMemcpyAsync(out, blk + o_out, b_out, cudaMemcpyDeviceToHost, x->stream));
  HT_CU(cudaFreeAsync(blk, x->stream));
  HT_CU(cudaStreamSynchronize(x->stream));
  return HT_OK;
}

}  // extern "C"
