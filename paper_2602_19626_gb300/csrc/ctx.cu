// Host side of the nc24 C ABI: context, stream slots, the per-step launch
// sequence (Algorithm 1's loop body), whole-stream encode / decode, and the
// building-block entry points.  See include/nc24.h for the contract.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <map>
#include <unordered_map>
#include <vector>

#include <cuda.h>

#include "coder.h"
#include "internal.h"

using namespace nc;

namespace {

struct Slot {
  bool open = false;
  bool awaiting_update = false;
  int32_t id = -1;
  int64_t n_coded = 0;
  int32_t last_tok = -1;
  int64_t max_len = 0;
  // device buffers owned by the slot (kept across reopen when large enough)
  void* kv = nullptr;
  bool kv_ready = false;     // kv zeroed and its TMA map written
  float* bias = nullptr;
  int32_t* uni = nullptr;
  float* z = nullptr;
  unsigned long long* keys[3] = {nullptr, nullptr, nullptr};
  int32_t* idx[3] = {nullptr, nullptr, nullptr};
  NgEntry* ent[3] = {nullptr, nullptr, nullptr};
  int64_t cap_len = 0;       // tokens the N-gram buffers can hold
  int64_t cap_hash = 0;      // hash index capacity (power of two)
};

// One projection on the tensor-core path: tensor maps of the weights (box of
// 128 rows) and of the batch operand of each forward buffer set (all its
// rows, one map per batch tile bn = 32, 64, 128, 256), and the bn tuned for a decode step (max_streams
// rows) and for prefill forwards of prefill_rows >> k rows, k < kPfBuckets.
constexpr int kPfBuckets = 4;
struct TcMat {
  CUtensorMap a;
  CUtensorMap b[2][4];               // per forward buffer set
  int M = 0, K = 0;
  int kp = 1;                        // 2: 3D maps, two K blocks per pipeline stage (TcGemm::kp)
  int bn_dec = 0, bn_pf[kPfBuckets] = {};
  const float* scale = nullptr;
};
static int bn_index(int bn) { return bn == 32 ? 0 : bn == 64 ? 1 : bn == 128 ? 2 : 3; }

// The weights' map (box of 128 rows) and its stage shape: BF16 with K a
// multiple of 64 takes 3D maps and two K blocks per stage.
static bool tc_encode_weights(TcMat& t, const void* w, int esz) {
  t.kp = (esz == 2 && t.K % 64 == 0) ? 2 : 1;
  return t.kp == 2 ? tc_encode_tmap3(&t.a, w, esz, t.K, t.M, 128) : tc_encode_tmap(&t.a, w, esz, t.K, t.M, 128);
}
// An operand map of `rows` rows with a box of bn rows, in the weights' shape.
static bool tc_encode_operand(const TcMat& t, CUtensorMap* m, const void* x, int esz, int rows, int bn) {
  return t.kp == 2 ? tc_encode_tmap3(m, x, esz, t.K, rows, bn) : tc_encode_tmap(m, x, esz, t.K, rows, bn);
}

}  // namespace

// Sets of the buffers a prefill chunk's forward hands to its vocabulary
// passes (logits, tokens, N-gram states).
constexpr int kCodeSets = 3;

struct nc_ctx {
  nc_config cfg{};
  Dims D{};
  int fmt = NC_BF16;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool poisoned = false;
  std::string err = "ok";
  std::vector<void*> allocs;   // weight buffers

  // weights
  const void* embed = nullptr;
  const float* embed_scale = nullptr;
  std::vector<LayerW> layers;
  const float* g_final = nullptr;

  // activations for up to max(max_streams, prefill_rows) rows
  float* x = nullptr;
  float* qkv = nullptr;
  float* attn_out = nullptr;         // [rows][hq * 64]
  float* h = nullptr;
  // encoder prefill (P = prefill_rows rows per forward pass)
  int P = 0;
  int32_t* f_slots = nullptr;        // [P] slot, position and input token of each forward row
  int32_t* f_pos = nullptr;
  int32_t* f_tok = nullptr;
  int32_t* d_nB_fwd = nullptr;       // forward rows
  // what a chunk's forward hands to its vocabulary passes (its coding set):
  // chunk c uses set c & 1 while the passes of chunk c - 1 still read the
  // other; with two forward buffer sets, set c mod 3, so that chunk c + 2's
  // forward need not wait for chunk c's passes
  int32_t* d_zidx[kCodeSets] = {};   // [max_streams] first forward row of each stream
  int32_t* f_obs[kCodeSets] = {};    // [P] observed token of (position, stream)
  int32_t* f_nb[kCodeSets] = {};     // [P] active streams per position
  float* zrows[kCodeSets] = {};      // [P][V] logits of the forward rows
  NgSnap* snap[kCodeSets] = {};      // [P] N-gram state of each (stream, position) prediction
  int32_t* d_p0 = nullptr;           // [4]: [0..2] first position of each set's chunk; [3] the next chunk's
  cudaStream_t side = nullptr;       // the N-gram pass of a chunk runs here beside its forward
  cudaStream_t vstream = nullptr;    // the vocabulary passes, beside the next chunk's forward
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_done = nullptr;
  cudaEvent_t ev_fwd[kCodeSets] = {}, ev_voc[kCodeSets] = {};
  uint32_t* cdf = nullptr;
  int32_t* d_slots = nullptr;
  int32_t* d_nB = nullptr;
  int32_t* d_obs = nullptr;
  uint32_t* d_target = nullptr;
  uint32_t* d_lohi = nullptr;
  int32_t* d_status = nullptr;       // scratch status for building blocks
  int64_t* d_meta = nullptr;         // [3 max_streams] an encoder call's row offsets, lengths, caller rows
  // nc_encode's device tokens and intervals, kept (grown as needed) so that
  // repeated calls reuse the same buffers and the captured pass
  int32_t* enc_tok = nullptr;
  size_t enc_tok_cap = 0;
  uint32_t* enc_iv = nullptr;
  size_t enc_iv_cap = 0;
  // pinned host staging
  int32_t* h_i32 = nullptr;          // 3 * max_streams + 1
  uint32_t* h_u32 = nullptr;         // 3 * max_streams: targets, then (lo, hi) pairs
  int32_t* h_status = nullptr;       // max_streams

  // tensor-core path
  std::vector<TcMat> tc;             // per layer: qkv, o, gate/up, down; then the LM head
  void* opnd = nullptr;              // [rows][max(d, F)] BF16 / E4M3 GEMM operand
  void* opnd2 = nullptr;             // BF16: [rows][F] the down projection's operand, written by the
                                     // gate/up epilogue while that GEMM still reads opnd
  float* opnd_scale = nullptr;       // [rows] E4M3 row scales

  // The buffers one forward writes.  Set 0 is the fields above; with a
  // second set (encoder prefill on the tensor-core path) chunk c + 1's
  // forward runs on stream s2 beside chunk c's.
  struct FwdSet {
    float *x = nullptr, *qkv = nullptr, *attn_out = nullptr, *h = nullptr;
    void *opnd = nullptr, *opnd2 = nullptr;
    float* opnd_scale = nullptr;
    void* q16 = nullptr;
    float* attn_part = nullptr;
    int32_t *f_slots = nullptr, *f_pos = nullptr, *f_tok = nullptr, *nB_fwd = nullptr;
  } fs[2];
  int n_fs = 1;
  cudaStream_t s2 = nullptr;
  std::vector<cudaEvent_t> ev_layer[2];     // [set][layer]: that set's chunk has finished layer l's attention
  cudaEvent_t ev_prep[2] = {};              // [set]: that set's chunk has taken its first position
  // the encoder's captured pass of every chunk (two forward sets), kept for
  // the next call with the same chunk plan and buffers
  std::vector<int64_t> pass_key;
  cudaGraphExec_t pass_graph = nullptr;

  StreamDev* d_st = nullptr;
  std::vector<StreamDev> h_st;
  std::vector<Slot> slots;
  std::unordered_map<int32_t, int> id2slot;
};

#define NC_TRY(call)                                                               \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return fail_cuda(ctx, e_, #call);                       \
  } while (0)

static int fail(nc_ctx* ctx, int st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}
static int fail_cuda(nc_ctx* ctx, cudaError_t e, const char* what) {
  if (ctx) {
    ctx->err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return NC_ENOMEM;
    }
    ctx->poisoned = true;
  }
  return NC_ECUDA;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

extern "C" void nc_config_default(nc_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->n_layers = 30;
  c->d_model = 576;
  c->n_heads = 9;
  c->n_kv_heads = 3;
  c->d_ffn = 1536;
  c->vocab = 49152;
  c->rope_theta = 1e5f;
  c->rms_eps = 1e-5f;
  c->ctx_len = 2048;
  c->slide = 512;
  c->ngram_order = 3;
  c->use_head = 1;
  c->cdf_log2_total = 24;
  c->floor = 1;
  c->bias_lr = 1e-3f;
  c->mix_eta = 1.0f;
  c->w_llm_init = 0.85f;
  c->temperature = 1.0f;
  c->warmup = 100;
  c->weight_fmt = NC_BF16;
  c->update_rule = NC_RULE_PAPER;
  c->path = NC_PATH_GEMV;
  c->max_streams = 1;
  c->device = 0;
  c->cuda_stream = nullptr;
  c->prefill_rows = 0;
  c->skip = 0;
  c->coder = NC_CODER_ARITH;
}

extern "C" const char* nc_status_str(int s) {
  switch (s) {
    case NC_OK: return "NC_OK";
    case NC_EINVAL: return "NC_EINVAL";
    case NC_ENOMEM: return "NC_ENOMEM";
    case NC_ECUDA: return "NC_ECUDA";
    case NC_ETIMEOUT: return "NC_ETIMEOUT";
    case NC_ECORRUPT: return "NC_ECORRUPT";
    case NC_ESTATE: return "NC_ESTATE";
    case NC_ENUMERIC: return "NC_ENUMERIC";
  }
  return "NC_UNKNOWN";
}

extern "C" const char* nc_last_error(const nc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

static std::string validate(const nc_config& c) {
  if (c.n_layers < 1 || c.d_model < 16 || c.d_model % 16) return "d_model must be a positive multiple of 16";
  if (c.n_heads < 1 || c.d_model != c.n_heads * kHeadDim) return "d_model / n_heads must be 64";
  if (c.n_kv_heads < 1 || c.n_heads % c.n_kv_heads || c.n_heads / c.n_kv_heads > kMaxGroup)
    return "n_heads must be a multiple of n_kv_heads (at most 4 per KV head)";
  if (c.d_ffn < 16 || c.d_ffn % 16) return "d_ffn must be a positive multiple of 16";
  if (c.d_model > 4096 || c.d_ffn > 4096) return "d_model and d_ffn must be at most 4096";
  if (c.vocab < 2 || c.vocab > 65535) return "vocab must be in [2, 65535]";
  if (c.ctx_len < 2 || (c.ctx_len & (c.ctx_len - 1)) || c.slide < 1 || c.slide >= c.ctx_len)
    return "ctx_len must be a power of two > slide > 0";
  if (c.ctx_len > 2048) return "ctx_len must be at most 2048 (8 attention CTAs of 256 positions)";
  if (c.ngram_order < 0 || c.ngram_order > kMaxOrder) return "ngram_order must be 0..3";
  if (c.cdf_log2_total < 16 || c.cdf_log2_total > 24) return "cdf_log2_total must be 16..24";
  if (c.floor < 1 || (uint64_t)c.vocab * c.floor >= (1ull << c.cdf_log2_total))
    return "floor * vocab must stay below the CDF total";
  if (!(c.temperature > 0.f)) return "temperature must be positive";
  if (c.w_llm_init <= 0.f || c.w_llm_init >= 1.f) return "w_llm_init must be in (0, 1)";
  if (c.weight_fmt < NC_FP32 || c.weight_fmt > NC_FP8E4M3) return "unknown weight_fmt";
  if (c.update_rule != NC_RULE_PAPER && c.update_rule != NC_RULE_MIXED_NLL) return "unknown update_rule";
  if (c.path != NC_PATH_GEMV && c.path != NC_PATH_TC) return "unknown path";
  if (c.path == NC_PATH_TC && c.weight_fmt == NC_FP32) return "the tensor-core path needs BF16 or FP8 weights";
  if (c.max_streams < 1 || c.max_streams > 4096) return "max_streams must be 1..4096";
  if (c.warmup < 0) return "warmup must be >= 0";
  if (c.prefill_rows < 0 || c.prefill_rows > 32768) return "prefill_rows must be 0..32768";
  if (c.coder != NC_CODER_ARITH && c.coder != NC_CODER_RANS) return "unknown coder";
  return "";
}

static size_t n_params(const nc_config& c) {
  const size_t d = c.d_model, qd = (size_t)c.n_heads * kHeadDim, kvd = (size_t)c.n_kv_heads * kHeadDim;
  const size_t per = d + qd * d + 2 * kvd * d + d * qd + d + 3 * (size_t)c.d_ffn * d;
  return (size_t)c.vocab * d + c.n_layers * per + d;
}

// Device allocations of the library go through dev_malloc.  Test hook: with
// NC24_FAIL_ALLOC_AFTER=n in the environment when a context is created, the
// allocations after the first n (counted from that nc_ctx_create on) fail as
// an out-of-memory device would, so that tests can check that every error
// path returns NC_ENOMEM and releases what it holds.
static std::atomic<long> g_alloc_budget{-1};

template <typename T>
static cudaError_t dev_malloc(T** p, size_t bytes) {
  long b = g_alloc_budget.load();
  while (b > 0 && !g_alloc_budget.compare_exchange_weak(b, b - 1)) {
  }
  if (b == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

template <typename T>
static cudaError_t dalloc(nc_ctx* ctx, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = dev_malloc(&q, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    ctx->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

static size_t fmt_bytes(int fmt) { return fmt == NC_FP32 ? 4 : fmt == NC_BF16 ? 2 : 1; }

// Convert one [rows][cols] FP32 device matrix into the storage format.
static int make_mat(nc_ctx* ctx, const float* src, int rows, int cols, Mat* m) {
  void* w = nullptr;
  float* sc = nullptr;
  NC_TRY(dalloc(ctx, &w, (size_t)rows * cols * fmt_bytes(ctx->fmt)));
  if (ctx->fmt == NC_FP8E4M3) NC_TRY(dalloc(ctx, &sc, (size_t)rows * sizeof(float)));
  NC_TRY(launch_convert_weights(src, w, sc, rows, cols, ctx->fmt, ctx->stream));
  m->w = w;
  m->scale = sc;
  m->rows = rows;
  m->cols = cols;
  return NC_OK;
}

static void free_slot(Slot& s) {
  cudaFree(s.kv);
  cudaFree(s.bias);
  cudaFree(s.uni);
  cudaFree(s.z);
  for (int k = 0; k < 3; ++k) {
    cudaFree(s.keys[k]);
    cudaFree(s.idx[k]);
    cudaFree(s.ent[k]);
  }
  s = Slot();
}

extern "C" void nc_ctx_destroy(nc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& s : ctx->slots) free_slot(s);
  for (void* p : ctx->allocs) cudaFree(p);
  cudaFreeHost(ctx->h_i32);
  cudaFreeHost(ctx->h_u32);
  cudaFreeHost(ctx->h_status);
  if (ctx->pass_graph) cudaGraphExecDestroy(ctx->pass_graph);
  cudaFree(ctx->enc_tok);
  cudaFree(ctx->enc_iv);
  for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_join, ctx->ev_done, ctx->ev_fwd[0], ctx->ev_fwd[1], ctx->ev_fwd[2],
                        ctx->ev_voc[0], ctx->ev_voc[1], ctx->ev_voc[2], ctx->ev_prep[0], ctx->ev_prep[1]})
    if (e) cudaEventDestroy(e);
  for (auto& v : ctx->ev_layer)
    for (cudaEvent_t e : v)
      if (e) cudaEventDestroy(e);
  if (ctx->s2) cudaStreamDestroy(ctx->s2);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->vstream) cudaStreamDestroy(ctx->vstream);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static int tc_bn_candidates(int Bmax, int* out) {
  int n = 0;
  for (int bn : {32, 64, 128, 256}) {
    out[n++] = bn;
    if (bn >= Bmax) break;
  }
  return n;
}

// Tensor maps of every projection on the tensor-core path, and the autotuned
// batch tile bn per projection shape: each candidate is timed on the real
// weights, with the epilogue that projection runs, with max_streams rows and
// again with prefill_rows rows for the encoder's prefill forward (the batch
// tile does not change the arithmetic of any output element, so the choice
// never changes results).
static int tc_setup(nc_ctx* ctx) {
  const Dims& D = ctx->D;
  const int B = ctx->cfg.max_streams;
  const int R = std::max(B, ctx->P);                 // operand rows
  const int kb = ctx->fmt == NC_BF16;
  const int esz = kb ? 2 : 1;
  const int Kmax = std::max(std::max(D.d, D.hq * kHeadDim), D.F);
  if (dalloc(ctx, &ctx->opnd, (size_t)R * Kmax * esz) || dalloc(ctx, &ctx->opnd_scale, (size_t)R * 4))
    return fail(ctx, NC_ENOMEM, "tensor-core operand allocation");
  NC_TRY(cudaMemset(ctx->opnd, 0, (size_t)R * Kmax * esz));
  NC_TRY(cudaMemset(ctx->opnd_scale, 0, (size_t)R * 4));
  if (kb) {
    if (dalloc(ctx, &ctx->opnd2, (size_t)R * D.F * 2)) return fail(ctx, NC_ENOMEM, "tensor-core operand allocation");
    NC_TRY(cudaMemset(ctx->opnd2, 0, (size_t)R * D.F * 2));
  }
  // forward buffer sets: set 0 is the context's own; an encoder prefill over
  // a BF16 cache gets a second one (P rows), its stream and its events
  nc_ctx::FwdSet& f0 = ctx->fs[0];
  f0.x = ctx->x;
  f0.qkv = ctx->qkv;
  f0.attn_out = ctx->attn_out;
  f0.h = ctx->h;
  f0.opnd = ctx->opnd;
  f0.opnd2 = ctx->opnd2;
  f0.opnd_scale = ctx->opnd_scale;
  f0.q16 = D.q16;
  f0.attn_part = D.attn_part;
  f0.f_slots = ctx->f_slots;
  f0.f_pos = ctx->f_pos;
  f0.f_tok = ctx->f_tok;
  f0.nB_fwd = ctx->d_nB_fwd;
  if (ctx->P > 0 && D.kv_bf16) {
    nc_ctx::FwdSet& f1 = ctx->fs[1];
    const size_t P = ctx->P;
    if (dalloc(ctx, &f1.x, P * D.d * 4) || dalloc(ctx, &f1.qkv, P * D.qkv_rows * 4) ||
        dalloc(ctx, &f1.attn_out, P * D.hq * kHeadDim * 4) || dalloc(ctx, &f1.h, P * D.F * 4) ||
        dalloc(ctx, &f1.opnd, P * Kmax * esz) || dalloc(ctx, &f1.opnd_scale, P * 4) ||
        (kb && dalloc(ctx, &f1.opnd2, P * D.F * 2)) || dalloc(ctx, &f1.q16, P * D.hq * kHeadDim * 2) ||
        dalloc(ctx, &f1.attn_part, D.attn_part_cap * 4) || dalloc(ctx, &f1.f_slots, P * 4) ||
        dalloc(ctx, &f1.f_pos, P * 4) || dalloc(ctx, &f1.f_tok, P * 4) || dalloc(ctx, &f1.nB_fwd, 16))
      return fail(ctx, NC_ENOMEM, "second forward buffer set");
    NC_TRY(cudaMemset(f1.opnd, 0, P * Kmax * esz));
    NC_TRY(cudaMemset(f1.opnd_scale, 0, P * 4));
    if (kb) NC_TRY(cudaMemset(f1.opnd2, 0, P * D.F * 2));
    NC_TRY(cudaStreamCreateWithFlags(&ctx->s2, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      NC_TRY(cudaEventCreateWithFlags(&ctx->ev_prep[k], cudaEventDisableTiming));
      ctx->ev_layer[k].assign(D.n_layers, nullptr);
      for (auto& e : ctx->ev_layer[k]) NC_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // the third coding set
    if (dalloc(ctx, &ctx->d_zidx[2], (size_t)ctx->cfg.max_streams * 4) ||
        dalloc(ctx, &ctx->zrows[2], P * D.V * 4) || dalloc(ctx, &ctx->f_obs[2], P * 4) ||
        dalloc(ctx, &ctx->f_nb[2], P * 4) || (D.order > 0 && dalloc(ctx, &ctx->snap[2], P * sizeof(NgSnap))))
      return fail(ctx, NC_ENOMEM, "third coding set");
    NC_TRY(cudaEventCreateWithFlags(&ctx->ev_fwd[2], cudaEventDisableTiming));
    NC_TRY(cudaEventCreateWithFlags(&ctx->ev_voc[2], cudaEventDisableTiming));
    ctx->n_fs = 2;
  }
  auto add = [&](const Mat& m) {
    TcMat t;
    t.M = m.rows;
    t.K = m.cols;
    t.scale = m.scale;
    if (!tc_encode_weights(t, m.w, esz)) return false;
    ctx->tc.push_back(t);
    return true;
  };
  for (const LayerW& L : ctx->layers)
    if (!add(L.qkv) || !add(L.o) || !add(L.gu) || !add(L.down)) return fail(ctx, NC_ECUDA, "tensor map encoding failed");
  Mat head{ctx->embed, ctx->embed_scale, D.V, D.d};
  if (!add(head)) return fail(ctx, NC_ECUDA, "tensor map encoding failed");
  // autotune bn per distinct shape (layer 0's matrices and the LM head), for
  // a decode step (B rows) and for prefill forwards of P, P / 2, P / 4, P / 8 rows
  float* scratch = nullptr;
  size_t maxM = 0;
  for (const TcMat& t : ctx->tc) maxM = std::max(maxM, (size_t)t.M);
  NC_TRY(dev_malloc(&scratch, maxM * R * 4));
  int32_t* nB = nullptr;
  NC_TRY(dev_malloc(&nB, 4));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int probe_idx[5] = {0, 1, 2, 3, (int)ctx->tc.size() - 1};
  const int probe_epi[5] = {EPI_STORE, EPI_RESID, EPI_SWIGLU, EPI_RESID, EPI_LOGITS};
  auto tune = [&](int rows, int* chosen) -> int {
    int cands[4];
    const int nc = tc_bn_candidates(rows, cands);
    NC_TRY(cudaMemcpy(nB, &rows, 4, cudaMemcpyHostToDevice));
    for (int q = 0; q < 5; ++q) {
      TcMat& t = ctx->tc[probe_idx[q]];
      float best = 1e30f;
      chosen[q] = cands[0];
      for (int ci = 0; ci < nc; ++ci) {
        TcMat tt = t;
        if (!tc_encode_operand(tt, &tt.b[0][0], ctx->opnd, esz, rows, cands[ci]))
          return fail(ctx, NC_ECUDA, "tensor map encoding failed");
        TcGemm g{};
        g.tmap_a = &tt.a;
        g.tmap_b = &tt.b[0][0];
        g.M = t.M;
        g.K = t.K;
        g.Bmax = rows;
        g.bn = cands[ci];
        g.kp = tt.kp;
        g.kind_bf16 = kb;
        g.nB = nB;
        g.w_scale = t.scale;
        g.x_scale = ctx->opnd_scale;
        g.y = scratch;                              // the residual too: its values do not matter here
        g.h_out = scratch;
        g.h16 = kb ? scratch : nullptr;             // the forward's SwiGLU output format
        g.zrows = scratch;
        g.status = ctx->d_status;
        // the best of four samples of five back-to-back launches (the first
        // sample also loads the kernel)
        float ms_best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
          cudaEventRecord(e0, ctx->stream);
          cudaError_t e = cudaSuccess;
          for (int k = 0; k < 5 && e == cudaSuccess; ++k) e = launch_gemm_tc(g, probe_epi[q], ctx->stream, false);
          cudaEventRecord(e1, ctx->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) return fail_cuda(ctx, e, "tensor-core autotune");
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep) ms_best = std::min(ms_best, ms);
        }
        if (ms_best < best) {
          best = ms_best;
          chosen[q] = cands[ci];
        }
      }
    }
    return NC_OK;
  };
  int chosen[5] = {0, 0, 0, 0, 0}, chosen_p[kPfBuckets][5] = {};
  int st = tune(B, chosen);
  for (int k = 0; k < kPfBuckets && st == NC_OK && ctx->P > 0; ++k)
    st = tune(std::max(ctx->P >> k, 1), chosen_p[k]);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  cudaFree(nB);
  if (st != NC_OK) return st;
  for (size_t i = 0; i < ctx->tc.size(); ++i) {
    TcMat& t = ctx->tc[i];
    const int q = (i + 1 == ctx->tc.size()) ? 4 : (int)(i % 4);
    const void* src = (kb && q == 3) ? ctx->opnd2 : ctx->opnd;   // BF16: the down projection reads opnd2
    t.bn_dec = chosen[q];
    for (int k = 0; k < kPfBuckets; ++k) t.bn_pf[k] = ctx->P > 0 ? chosen_p[k][q] : chosen[q];
    for (int bi = 0; bi < 4; ++bi)
      if (!tc_encode_operand(t, &t.b[0][bi], src, esz, R, 32 << bi))
        return fail(ctx, NC_ECUDA, "tensor map encoding failed");
    if (ctx->n_fs == 2) {
      const void* src1 = (kb && q == 3) ? ctx->fs[1].opnd2 : ctx->fs[1].opnd;
      for (int bi = 0; bi < 4; ++bi)
        if (!tc_encode_operand(t, &t.b[1][bi], src1, esz, ctx->P, 32 << bi))
          return fail(ctx, NC_ECUDA, "tensor map encoding failed");
    }
  }
  return NC_OK;
}

extern "C" int nc_ctx_create(const nc_config* cfg, const void* weights, size_t nbytes, nc_ctx** out) {
  if (!out) return NC_EINVAL;
  *out = nullptr;
  if (!cfg || !weights) return NC_EINVAL;
  const std::string why = validate(*cfg);
  if (!why.empty()) return NC_EINVAL;
  if (nbytes != n_params(*cfg) * sizeof(float)) return NC_EINVAL;
  {
    const char* e = std::getenv("NC24_FAIL_ALLOC_AFTER");
    g_alloc_budget.store(e && e[0] ? std::atol(e) : -1);
  }
  nc_ctx* ctx = new (std::nothrow) nc_ctx();
  if (!ctx) return NC_ENOMEM;
  cudaGetLastError();                              // a stale error of an earlier call is not ours
  ctx->cfg = *cfg;
  ctx->fmt = cfg->weight_fmt;
  const nc_config& c = *cfg;
  auto bail = [&](int st) {
    nc_ctx_destroy(ctx);
    return st;
  };
  if (cudaSetDevice(c.device) != cudaSuccess) return bail(NC_ECUDA);
  if (c.cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(c.cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(NC_ECUDA);
    ctx->own_stream = true;
  }
  Dims& D = ctx->D;
  {
    const char* e = std::getenv("NC24_PDL");     // NC24_PDL=0 launches without PDL
    D.pdl = (e && e[0] == '0') ? 0 : 1;
  }
  D.n_layers = c.n_layers;
  D.d = c.d_model;
  D.hq = c.n_heads;
  D.hkv = c.n_kv_heads;
  D.F = c.d_ffn;
  D.V = c.vocab;
  D.L = c.ctx_len;
  D.C = c.slide;
  D.qkv_rows = (c.n_heads + 2 * c.n_kv_heads) * kHeadDim;
  {
    // RoPE table: (cos, sin) of v * 256^k * theta^(-2j/64), FP64 then rounded
    std::vector<float2> tab((size_t)kRopeLevels * 256 * 32);
    for (int k = 0; k < kRopeLevels; ++k)
      for (int v = 0; v < 256; ++v)
        for (int jf = 0; jf < 32; ++jf) {
          const double inv = std::pow((double)c.rope_theta, -2.0 * jf / (double)kHeadDim);
          const double ang = (double)v * std::ldexp(1.0, 8 * k) * inv;
          tab[((size_t)k * 256 + v) * 32 + jf] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
    float2* dtab = nullptr;
    if (dalloc(ctx, &dtab, tab.size() * sizeof(float2)) != cudaSuccess ||
        cudaMemcpy(dtab, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(NC_ENOMEM);
    D.rope_tab = dtab;
  }
  D.eps = c.rms_eps;
  D.theta = c.rope_theta;
  D.tau = c.temperature;
  D.kv_bf16 = c.weight_fmt != NC_FP32;
  {
    // CUDA-core attention over an FP32 cache: CTAs per (stream, KV head) are
    // picked per launch from its rows (results do not depend on them);
    // NC24_ATTN_CLUSTER=1|2|4|8 fixes them.  The tensor-core attention over a
    // BF16 cache always takes one CTA per 256-position chunk of the window.
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess || nsm <= 0)
      return bail(NC_ECUDA);
    D.n_sm = nsm;
    D.attn_cluster = 0;                            // by the rows of each launch
    const char* e = std::getenv("NC24_ATTN_CLUSTER");
    if (e && (e[0] == '1' || e[0] == '2' || e[0] == '4' || e[0] == '8') && e[1] == 0) D.attn_cluster = e[0] - '0';
  }
  D.order = c.ngram_order;
  D.skip = c.skip && c.ngram_order > 0;
  D.use_head = c.use_head;
  D.warmup = c.warmup;
  D.rule = c.update_rule;
  D.log2T = c.cdf_log2_total;
  D.floor = c.floor;
  D.alpha = c.bias_lr;
  D.eta = c.mix_eta;

  // ---- weights: upload the FP32 buffer once, convert tensor by tensor
  float* src = nullptr;
  if (dev_malloc(&src, nbytes) != cudaSuccess) return bail(NC_ENOMEM);
  int st = NC_OK;
  do {
    if (cudaMemcpy(src, weights, nbytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      st = NC_ECUDA;
      break;
    }
    const size_t d = D.d, F = D.F;
    const size_t qd = (size_t)D.hq * kHeadDim;
    size_t off = 0;
    Mat emb;
    if ((st = make_mat(ctx, src + off, D.V, D.d, &emb)) != NC_OK) break;
    ctx->embed = emb.w;
    ctx->embed_scale = emb.scale;
    off += (size_t)D.V * d;
    float* tmp = nullptr;   // interleaved gate/up in FP32
    if (dalloc(ctx, &tmp, 2 * F * d * sizeof(float)) != cudaSuccess) {
      st = NC_ENOMEM;
      break;
    }
    ctx->layers.resize(D.n_layers);
    for (int l = 0; l < D.n_layers && st == NC_OK; ++l) {
      LayerW& L = ctx->layers[l];
      float* g1 = nullptr;
      float* g2 = nullptr;
      if (dalloc(ctx, &g1, d * 4) != cudaSuccess || dalloc(ctx, &g2, d * 4) != cudaSuccess) {
        st = NC_ENOMEM;
        break;
      }
      cudaMemcpyAsync(g1, src + off, d * 4, cudaMemcpyDeviceToDevice, ctx->stream);
      off += d;
      // wq, wk, wv are adjacent: together they are the [qkv_rows][d] matrix
      if ((st = make_mat(ctx, src + off, D.qkv_rows, D.d, &L.qkv)) != NC_OK) break;
      off += (size_t)D.qkv_rows * d;
      if ((st = make_mat(ctx, src + off, D.d, (int)qd, &L.o)) != NC_OK) break;
      off += d * qd;
      cudaMemcpyAsync(g2, src + off, d * 4, cudaMemcpyDeviceToDevice, ctx->stream);
      off += d;
      if (launch_interleave_f32(src + off, src + off + F * d, tmp, F, d, ctx->stream) != cudaSuccess) {
        st = NC_ECUDA;
        break;
      }
      if ((st = make_mat(ctx, tmp, 2 * D.F, D.d, &L.gu)) != NC_OK) break;
      off += 2 * F * d;
      if ((st = make_mat(ctx, src + off, D.d, D.F, &L.down)) != NC_OK) break;
      off += d * F;
      L.g_attn = g1;
      L.g_ffn = g2;
      cudaStreamSynchronize(ctx->stream);   // tmp is reused by the next layer
    }
    if (st != NC_OK) break;
    float* gf = nullptr;
    if (dalloc(ctx, &gf, d * 4) != cudaSuccess) {
      st = NC_ENOMEM;
      break;
    }
    cudaMemcpyAsync(gf, src + off, d * 4, cudaMemcpyDeviceToDevice, ctx->stream);
    ctx->g_final = gf;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = NC_ECUDA;
  } while (0);
  cudaFree(src);
  if (st != NC_OK) return bail(st);

  // ---- activations and per-step buffers
  const size_t B = c.max_streams;
  ctx->P = c.prefill_rows >= 2 ? c.prefill_rows : 0;
  const size_t RA = std::max(B, (size_t)ctx->P);     // activation rows
  if (ctx->P > 0 &&
      (dalloc(ctx, &ctx->f_slots, (size_t)ctx->P * 4) || dalloc(ctx, &ctx->f_pos, (size_t)ctx->P * 4) ||
       dalloc(ctx, &ctx->f_tok, (size_t)ctx->P * 4) || dalloc(ctx, &ctx->d_nB_fwd, 16) ||
       dalloc(ctx, &ctx->d_p0, 16)))
    return bail(NC_ENOMEM);
  for (int k = 0; k < 2 && ctx->P > 0; ++k) {
    if (dalloc(ctx, &ctx->d_zidx[k], B * 4) || dalloc(ctx, &ctx->zrows[k], (size_t)ctx->P * D.V * 4) ||
        dalloc(ctx, &ctx->f_obs[k], (size_t)ctx->P * 4) || dalloc(ctx, &ctx->f_nb[k], (size_t)ctx->P * 4) ||
        (D.order > 0 && dalloc(ctx, &ctx->snap[k], (size_t)ctx->P * sizeof(NgSnap))))
      return bail(NC_ENOMEM);
  }
  if (ctx->P > 0) {
    bool ok = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&ctx->vstream, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&ctx->ev_fork, &ctx->ev_join, &ctx->ev_done, &ctx->ev_fwd[0], &ctx->ev_fwd[1],
                           &ctx->ev_voc[0], &ctx->ev_voc[1]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return bail(NC_ECUDA);
  }
  if (dalloc(ctx, &ctx->x, RA * D.d * 4) || dalloc(ctx, &ctx->qkv, RA * D.qkv_rows * 4) ||
      dalloc(ctx, &ctx->attn_out, RA * D.hq * kHeadDim * 4) ||
      dalloc(ctx, &ctx->h, RA * D.F * 4) || dalloc(ctx, &ctx->cdf, B * (D.V + 1) * 4) ||
      dalloc(ctx, &ctx->d_slots, B * 4) || dalloc(ctx, &ctx->d_nB, 16) ||
      dalloc(ctx, &ctx->d_obs, B * 4) || dalloc(ctx, &ctx->d_target, B * 4) ||
      dalloc(ctx, &ctx->d_lohi, B * 8) || dalloc(ctx, &ctx->d_status, B * 4) || dalloc(ctx, &ctx->d_meta, B * 24) ||
      dalloc(ctx, &ctx->d_st, B * sizeof(StreamDev)))
    return bail(NC_ENOMEM);
  if (D.kv_bf16) {
    attn_t5_scratch(D, (int)B, ctx->P, &D.attn_part_cap, &D.attn_tickets);
    if (dalloc(ctx, &D.attn_part, D.attn_part_cap * 4) || dalloc(ctx, &D.attn_ticket, (size_t)D.attn_tickets * 4))
      return bail(NC_ENOMEM);
    if (cudaMemset(D.attn_ticket, 0, (size_t)D.attn_tickets * 4) != cudaSuccess) return bail(NC_ECUDA);
    if (ctx->P > 0 && dalloc(ctx, &D.q16, (size_t)ctx->P * D.hq * kHeadDim * 2)) return bail(NC_ENOMEM);
    // the attention loads 64-row boxes of the KV rings through one TMA map per slot
    void* maps = nullptr;
    if (D.L >= 64) {
      if (dalloc(ctx, &maps, B * kTmapBytes)) return bail(NC_ENOMEM);
      D.kv_tmap = maps;
    }
  }
  if (cudaMallocHost(&ctx->h_i32, (3 * B + 4) * 4) != cudaSuccess ||
      cudaMallocHost(&ctx->h_u32, 3 * B * 4) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, B * 4) != cudaSuccess)
    return bail(NC_ENOMEM);
  ctx->h_st.assign(B, StreamDev{});
  ctx->slots.assign(B, Slot{});
  if (cudaMemset(ctx->d_st, 0, B * sizeof(StreamDev)) != cudaSuccess) return bail(NC_ECUDA);
  if (cudaMemset(ctx->d_status, 0, B * 4) != cudaSuccess) return bail(NC_ECUDA);
  if (prepare_model_kernels(D, ctx->fmt) != cudaSuccess || prepare_vocab_kernels(D) != cudaSuccess ||
      (c.path == NC_PATH_TC && prepare_tc_kernels() != cudaSuccess))
    return bail(NC_ECUDA);
  if (c.path == NC_PATH_TC) {
    const int st2 = tc_setup(ctx);
    if (st2 != NC_OK) return bail(st2);
  }
  *out = ctx;
  return NC_OK;
}

// ---------------------------------------------------------------- streams

static_assert(sizeof(CUtensorMap) == kTmapBytes, "one TMA map per slot");

static int slot_alloc(nc_ctx* ctx, Slot& s, int64_t max_len) {
  const Dims& D = ctx->D;
  if (!s.kv) {
    const size_t kvb = (size_t)D.n_layers * 2 * D.hkv * D.L * kHeadDim * (D.kv_bf16 ? 2 : 4);
    NC_TRY(dev_malloc(&s.kv, kvb));
    NC_TRY(dev_malloc(&s.bias, (size_t)D.V * 4));
    NC_TRY(dev_malloc(&s.uni, (size_t)D.V * 4));
    NC_TRY(dev_malloc(&s.z, (size_t)D.V * 4));
  }
  if (!s.kv_ready) {
    // every ring entry finite from the start: the tensor-core attention
    // multiplies the entries past a row's position by zero probabilities
    const size_t kvb = (size_t)D.n_layers * 2 * D.hkv * D.L * kHeadDim * (D.kv_bf16 ? 2 : 4);
    NC_TRY(cudaMemset(s.kv, 0, kvb));
    if (D.kv_tmap) {
      CUtensorMap map;
      if (!tc_encode_tmap(&map, s.kv, 2, kHeadDim, (int64_t)D.n_layers * 2 * D.hkv * D.L, 64))
        return fail(ctx, NC_ECUDA, "KV tensor map encoding failed");
      const int si = (int)(&s - ctx->slots.data());
      NC_TRY(cudaMemcpy(static_cast<unsigned char*>(const_cast<void*>(D.kv_tmap)) + (size_t)si * kTmapBytes, &map,
                        kTmapBytes, cudaMemcpyHostToDevice));
    }
    s.kv_ready = true;
  }
  if (D.order > 0 && s.cap_len < max_len) {
    for (int k = 0; k < 3; ++k) {
      cudaFree(s.keys[k]);
      cudaFree(s.idx[k]);
      cudaFree(s.ent[k]);
      s.keys[k] = nullptr;
      s.idx[k] = nullptr;
      s.ent[k] = nullptr;
    }
    s.cap_len = 0;
    const int64_t cap = next_pow2(std::max<int64_t>(2 * max_len, 16));
    for (int k = 0; k < D.order; ++k) {
      NC_TRY(dev_malloc(&s.keys[k], (size_t)cap * 8));
      NC_TRY(dev_malloc(&s.idx[k], (size_t)cap * 4));
      NC_TRY(dev_malloc(&s.ent[k], (size_t)max_len * sizeof(NgEntry)));
    }
    s.cap_len = max_len;
    s.cap_hash = cap;
  }
  return NC_OK;
}

static int open_slot(nc_ctx* ctx, int32_t id, int64_t max_len, int* slot_out) {
  int si = -1;
  for (int i = 0; i < (int)ctx->slots.size(); ++i)
    if (!ctx->slots[i].open) {
      si = i;
      break;
    }
  if (si < 0) return fail(ctx, NC_EINVAL, "no free stream slot");
  if (max_len >= kMaxPosition) return fail(ctx, NC_EINVAL, "stream longer than 2^24 - 1 tokens");
  Slot& s = ctx->slots[si];
  int st = slot_alloc(ctx, s, max_len);
  if (st != NC_OK) return st;
  const Dims& D = ctx->D;
  cudaStream_t cs = ctx->stream;
  NC_TRY(cudaMemsetAsync(s.bias, 0, (size_t)D.V * 4, cs));
  NC_TRY(cudaMemsetAsync(s.uni, 0, (size_t)D.V * 4, cs));
  for (int k = 0; k < D.order; ++k) NC_TRY(cudaMemsetAsync(s.keys[k], 0xFF, (size_t)s.cap_hash * 8, cs));
  StreamDev sd{};
  sd.n_coded = 0;
  sd.last_tok = 0;   // BOS
  sd.kv_start = 0;
  sd.N = 0;
  for (int k = 0; k < 3; ++k) {
    sd.hist[k] = 0;
    sd.ctx_ent[k] = -1;
    sd.n_ent[k] = 0;
    sd.keys[k] = s.keys[k];
    sd.idx[k] = s.idx[k];
    sd.ent[k] = s.ent[k];
  }
  sd.max_len = (int32_t)max_len;
  sd.status = 0;
  sd.cap_mask = (int32_t)(s.cap_hash - 1);
  sd.theta[0] = logf(ctx->cfg.w_llm_init);
  sd.theta[1] = logf(1.0f - ctx->cfg.w_llm_init);
  sd.bias = s.bias;
  sd.uni = s.uni;
  sd.z = s.z;
  sd.kv = s.kv;
  ctx->h_st[si] = sd;
  NC_TRY(cudaMemcpyAsync(ctx->d_st + si, &ctx->h_st[si], sizeof(StreamDev), cudaMemcpyHostToDevice, cs));
  NC_TRY(cudaStreamSynchronize(cs));
  s.open = true;
  s.awaiting_update = false;
  s.id = id;
  s.n_coded = 0;
  s.last_tok = -1;
  s.max_len = max_len;
  ctx->id2slot[id] = si;
  *slot_out = si;
  return NC_OK;
}

extern "C" int nc_stream_open(nc_ctx* ctx, int32_t stream_id, int64_t expected_len) {
  if (!ctx) return NC_EINVAL;
  if (ctx->poisoned) return NC_ESTATE;
  if (stream_id < 0 || expected_len < 1 || expected_len >= kMaxPosition)
    return fail(ctx, NC_EINVAL, "bad stream id or length (at most 2^24 - 1 tokens)");
  if (ctx->id2slot.count(stream_id)) return fail(ctx, NC_EINVAL, "stream id already open");
  cudaSetDevice(ctx->cfg.device);
  int si;
  return open_slot(ctx, stream_id, expected_len, &si);
}

extern "C" int nc_stream_close(nc_ctx* ctx, int32_t stream_id) {
  if (!ctx) return NC_EINVAL;
  auto it = ctx->id2slot.find(stream_id);
  if (it == ctx->id2slot.end()) return fail(ctx, NC_EINVAL, "unknown stream id");
  Slot& s = ctx->slots[it->second];
  s.open = false;
  s.id = -1;
  ctx->id2slot.erase(it);
  return NC_OK;
}

// ------------------------------------------------------------- step pieces

static Batch make_batch(nc_ctx* ctx) {
  Batch b{};
  b.slots = ctx->d_slots;
  b.nB = ctx->d_nB;
  b.obs = ctx->d_obs;
  b.st = ctx->d_st;
  b.Bmax = ctx->cfg.max_streams;
  return b;
}

// Kernel kinds reported by nc_trace.
enum TraceKind { TK_PREPARE, TK_EMBED, TK_QKV, TK_ATTN, TK_O, TK_GU, TK_DOWN, TK_LMHEAD, TK_VOCAB,
                 TK_NGRAM, TK_COUNT };
static const char* kTraceNames[TK_COUNT] = {"prepare", "embed", "gemv_qkv", "attn", "gemv_o",
                                            "gemv_gate_up", "gemv_down", "lm_head", "vocab", "ngram_update"};

// Records a CUDA event after every launch of a step (when on) so that the
// device time of each kernel is the gap between consecutive events.
struct StepMarks {
  bool on = false;
  bool capturing = false;        // inside stream capture: record external event nodes
  std::vector<cudaEvent_t> ev;   // ev[0] before the first kernel
  std::vector<int> kind;
  int n = 0;
  cudaError_t begin(cudaStream_t s) {
    n = 0;
    kind.clear();
    if (!on) return cudaSuccess;
    return record(ev[0], s);
  }
  cudaError_t record(cudaEvent_t e, cudaStream_t s) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
  }
  cudaError_t mark(cudaStream_t s, int k) {
    if (!on) return cudaSuccess;
    if (n + 1 >= (int)ev.size()) return cudaErrorInvalidValue;
    kind.push_back(k);
    return record(ev[++n], s);
  }
};

// Ordering of a prefill forward with the other buffer set's: before layer
// l's append it waits for wait[l] (the other chunk has finished layer l's
// attention, so no ring entry it reads is overwritten, and the entries it
// appended are in); after layer l's attention it records rec[l].
struct LayerSync {
  const cudaEvent_t* wait = nullptr;
  const cudaEvent_t* rec = nullptr;
  bool no_pdl = false;      // launch without programmatic dependent launch
};

// Model forward of every active row: logits into each stream's z.
static cudaError_t launch_model_tc(nc_ctx* ctx, const Batch& b, StepMarks& m, int set = 0, cudaStream_t st = nullptr,
                                   LayerSync sync = {});

static cudaError_t launch_model(nc_ctx* ctx, const Batch& b, StepMarks* mk = nullptr) {
  const Dims& D = ctx->D;
  cudaStream_t s = ctx->stream;
  StepMarks none;
  StepMarks& m = mk ? *mk : none;
  if (ctx->cfg.path == NC_PATH_TC) return launch_model_tc(ctx, b, m);
  cudaError_t e = launch_embed(D, b, ctx->embed, ctx->embed_scale, ctx->fmt, ctx->x, s);
  if (e == cudaSuccess) e = m.mark(s, TK_EMBED);
  for (int l = 0; l < D.n_layers && e == cudaSuccess; ++l) {
    const LayerW& L = ctx->layers[l];
    GemvIO io{};
    io.x = ctx->x;
    io.g = L.g_attn;
    io.y = ctx->qkv;
    e = launch_gemv(D, b, L.qkv, ctx->fmt, PRO_RMSNORM, EPI_STORE, io, s);
    if (e == cudaSuccess && b.pos) e = launch_kv_append(D, b, l, ctx->qkv, s);
    if (e == cudaSuccess) e = m.mark(s, TK_QKV);
    if (e == cudaSuccess) e = launch_attn(D, b, l, ctx->qkv, ctx->attn_out, s);
    if (e == cudaSuccess) e = m.mark(s, TK_ATTN);
    if (e == cudaSuccess) {
      io = GemvIO{};
      io.x = ctx->attn_out;
      io.y = ctx->x;
      e = launch_gemv(D, b, L.o, ctx->fmt, PRO_PLAIN, EPI_RESID, io, s);
      if (e == cudaSuccess) e = m.mark(s, TK_O);
    }
    if (e == cudaSuccess) {
      io = GemvIO{};
      io.x = ctx->x;
      io.g = L.g_ffn;
      io.y = ctx->h;
      e = launch_gemv(D, b, L.gu, ctx->fmt, PRO_RMSNORM, EPI_SWIGLU, io, s);
      if (e == cudaSuccess) e = m.mark(s, TK_GU);
    }
    if (e == cudaSuccess) {
      io = GemvIO{};
      io.x = ctx->h;
      io.y = ctx->x;
      e = launch_gemv(D, b, L.down, ctx->fmt, PRO_PLAIN, EPI_RESID, io, s);
      if (e == cudaSuccess) e = m.mark(s, TK_DOWN);
    }
  }
  if (e == cudaSuccess) {
    GemvIO io{};
    io.x = ctx->x;
    io.g = ctx->g_final;
    Mat head{ctx->embed, ctx->embed_scale, D.V, D.d};
    e = launch_gemv(D, b, head, ctx->fmt, PRO_RMSNORM, EPI_LOGITS, io, s);
    if (e == cudaSuccess) e = m.mark(s, TK_LMHEAD);
  }
  return e;
}

// Model forward on the tensor-core path: each projection is one tcgen05 GEMM
// over the batch.  Its operand is written by a small kernel (the RMSNorm
// ones; every E4M3 one, for its row scale) or, for BF16, by the producer
// itself: the attention writes the O projection's operand and the gate/up
// epilogue the down projection's (into opnd2).
static cudaError_t launch_model_tc(nc_ctx* ctx, const Batch& b, StepMarks& m, int set, cudaStream_t st,
                                   LayerSync sync) {
  const nc_ctx::FwdSet& F = ctx->fs[set];
  Dims D = ctx->D;
  D.attn_part = F.attn_part;
  D.q16 = F.q16;
  if (sync.no_pdl) D.pdl = 0;
  cudaStream_t s = st ? st : ctx->stream;
  const int kb = ctx->fmt == NC_BF16;
  auto gemm = [&](const TcMat& t, int epi, float* y, float* h, void* h16 = nullptr) {
    // the batch tile tuned for this many rows: a decode step's, or the
    // smallest prefill bucket that holds the forward's rows
    int bn = t.bn_dec;
    if (b.pos) {
      int k = 0;
      while (k + 1 < kPfBuckets && (ctx->P >> (k + 1)) >= b.Bmax) ++k;
      bn = t.bn_pf[k];
    }
    TcGemm g{};
    g.tmap_a = &t.a;
    g.tmap_b = &t.b[set][bn_index(bn)];
    g.M = t.M;
    g.K = t.K;
    g.Bmax = b.Bmax;
    g.bn = bn;
    g.kp = t.kp;
    g.zrows = b.z_out;
    g.kind_bf16 = kb;
    g.nB = b.nB;
    g.w_scale = t.scale;
    g.x_scale = F.opnd_scale;
    g.y = y;
    g.h_out = h;
    g.h16 = h16;
    g.st = b.st;
    g.slots = b.slots;
    g.status = ctx->d_status;
    return launch_gemm_tc(g, epi, s, D.pdl);
  };
  cudaError_t e = launch_embed(D, b, ctx->embed, ctx->embed_scale, ctx->fmt, F.x, s);
  if (e == cudaSuccess) e = m.mark(s, TK_EMBED);
  for (int l = 0; l < D.n_layers && e == cudaSuccess; ++l) {
    const LayerW& L = ctx->layers[l];
    const TcMat* T = &ctx->tc[4 * l];
    e = launch_act_rmsnorm(D, b, F.x, L.g_attn, D.d, kb, F.opnd, F.opnd_scale, s);
    if (e == cudaSuccess) e = gemm(T[0], EPI_STORE, F.qkv, nullptr);
    if (e == cudaSuccess && b.pos && sync.wait) e = cudaStreamWaitEvent(s, sync.wait[l], 0);
    if (e == cudaSuccess && b.pos) e = launch_kv_append(D, b, l, F.qkv, s);
    if (e == cudaSuccess) e = m.mark(s, TK_QKV);
    if (e == cudaSuccess) e = launch_attn(D, b, l, F.qkv, F.attn_out, s, kb ? F.opnd : nullptr);
    if (e == cudaSuccess && sync.rec) e = cudaEventRecord(sync.rec[l], s);
    if (e == cudaSuccess) e = m.mark(s, TK_ATTN);
    if (e == cudaSuccess && !kb)
      e = launch_act_plain(D, b, F.attn_out, D.hq * kHeadDim, kb, F.opnd, F.opnd_scale, s);
    if (e == cudaSuccess) e = gemm(T[1], EPI_RESID, F.x, nullptr);
    if (e == cudaSuccess) e = m.mark(s, TK_O);
    if (e == cudaSuccess) e = launch_act_rmsnorm(D, b, F.x, L.g_ffn, D.d, kb, F.opnd, F.opnd_scale, s);
    if (e == cudaSuccess) e = gemm(T[2], EPI_SWIGLU, nullptr, F.h, kb ? F.opnd2 : nullptr);
    if (e == cudaSuccess) e = m.mark(s, TK_GU);
    if (e == cudaSuccess && !kb) e = launch_act_plain(D, b, F.h, D.F, kb, F.opnd, F.opnd_scale, s);
    if (e == cudaSuccess) e = gemm(T[3], EPI_RESID, F.x, nullptr);
    if (e == cudaSuccess) e = m.mark(s, TK_DOWN);
  }
  if (e == cudaSuccess) e = launch_act_rmsnorm(D, b, F.x, ctx->g_final, D.d, kb, F.opnd, F.opnd_scale, s);
  if (e == cudaSuccess) e = gemm(ctx->tc.back(), EPI_LOGITS, nullptr, nullptr);
  if (e == cudaSuccess) e = m.mark(s, TK_LMHEAD);
  return e;
}

// Algorithmic bytes and arithmetic of one launch of each kind for B active
// rows whose attention windows hold ctx_sum entries in total (the fed tokens
// included), kv_unique of them distinct (a prefill's rows of one stream
// share their window).
static void step_cost(const nc_ctx* ctx, int B, double ctx_sum, double kv_unique, double* out, double* fl) {
  const Dims& D = ctx->D;
  const double esz = ctx->fmt == NC_FP32 ? 4 : ctx->fmt == NC_BF16 ? 2 : 1;
  const double kvsz = D.kv_bf16 ? 2 : 4;
  auto gemv = [&](double rows, double cols, double out_rows, bool resid) {
    double w = rows * cols * esz + (ctx->fmt == NC_FP8E4M3 ? rows * 4 : 0);
    return w + B * cols * 4 + B * out_rows * 4 * (resid ? 2 : 1);
  };
  const double qd = (double)D.hq * kHeadDim;
  for (int k = 0; k < TK_COUNT; ++k) out[k] = fl[k] = 0;
  out[TK_PREPARE] = B * 24.0;
  out[TK_EMBED] = B * D.d * (esz + 4);
  out[TK_QKV] = gemv(D.qkv_rows, D.d, D.qkv_rows, false) + B * D.d * 4;
  out[TK_ATTN] = D.hkv * 2.0 * kHeadDim * kvsz * kv_unique + B * (D.qkv_rows * 4.0 + qd * 4.0);
  out[TK_O] = gemv(D.d, qd, D.d, true);
  out[TK_GU] = gemv(2.0 * D.F, D.d, D.F, false);
  out[TK_DOWN] = gemv(D.d, D.F, D.d, true);
  out[TK_LMHEAD] = gemv(D.V, D.d, D.V, false);
  out[TK_VOCAB] = B * D.V * 16.0 + B * 8.0;
  out[TK_NGRAM] = B * (3.0 * sizeof(NgEntry) + 64.0);
  fl[TK_QKV] = 2.0 * B * D.qkv_rows * D.d;
  fl[TK_ATTN] = 2.0 * 2.0 * qd * ctx_sum;          // scores and weighted values
  fl[TK_O] = 2.0 * B * D.d * qd;
  fl[TK_GU] = 2.0 * B * 2.0 * D.F * D.d;
  fl[TK_DOWN] = 2.0 * B * D.d * D.F;
  fl[TK_LMHEAD] = 2.0 * B * (double)D.V * D.d;
}

// Host-side checks and staging of a batch of open streams.
static int stage_batch(nc_ctx* ctx, int n, const int32_t* ids, std::vector<int>* slot_idx,
                       bool want_awaiting) {
  if (n < 1 || n > ctx->cfg.max_streams || !ids) return fail(ctx, NC_EINVAL, "bad stream count or ids");
  slot_idx->resize(n);
  for (int j = 0; j < n; ++j) {
    auto it = ctx->id2slot.find(ids[j]);
    if (it == ctx->id2slot.end()) return fail(ctx, NC_EINVAL, "unknown stream id");
    (*slot_idx)[j] = it->second;
    const Slot& s = ctx->slots[it->second];
    if (s.awaiting_update != want_awaiting)
      return fail(ctx, NC_ESTATE, want_awaiting ? "stream has no pending step" : "stream awaits nc_update_bias");
    if (!want_awaiting && s.n_coded >= s.max_len) return fail(ctx, NC_ESTATE, "stream longer than its expected_len");
  }
  std::vector<int> sorted(*slot_idx);
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
    return fail(ctx, NC_EINVAL, "duplicate stream id");
  ctx->h_i32[0] = n;
  for (int j = 0; j < n; ++j) ctx->h_i32[1 + j] = (*slot_idx)[j];
  NC_TRY(cudaMemcpyAsync(ctx->d_nB, ctx->h_i32, 4, cudaMemcpyHostToDevice, ctx->stream));
  NC_TRY(cudaMemcpyAsync(ctx->d_slots, ctx->h_i32 + 1, (size_t)n * 4, cudaMemcpyHostToDevice, ctx->stream));
  return NC_OK;
}

// Read and clear the sticky status words of the given slots (and the
// context-wide word of the tensor-core GEMMs).
static int check_status(nc_ctx* ctx, const std::vector<int>& slot_idx) {
  const size_t off = offsetof(StreamDev, status);
  if (ctx->cfg.path == NC_PATH_TC) {
    int32_t w = 0;
    NC_TRY(cudaMemcpyAsync(&w, ctx->d_status, 4, cudaMemcpyDeviceToHost, ctx->stream));
    NC_TRY(cudaStreamSynchronize(ctx->stream));
    if (w) {
      ctx->poisoned = true;
      return fail(ctx, NC_ETIMEOUT, "a tensor-core pipeline wait gave up");
    }
  }
  for (size_t j = 0; j < slot_idx.size(); ++j)
    NC_TRY(cudaMemcpyAsync(ctx->h_status + j, reinterpret_cast<char*>(ctx->d_st + slot_idx[j]) + off, 4,
                           cudaMemcpyDeviceToHost, ctx->stream));
  NC_TRY(cudaStreamSynchronize(ctx->stream));
  int32_t any = 0;
  for (size_t j = 0; j < slot_idx.size(); ++j) any |= ctx->h_status[j];
  if (any) {
    for (size_t j = 0; j < slot_idx.size(); ++j)
      NC_TRY(cudaMemsetAsync(reinterpret_cast<char*>(ctx->d_st + slot_idx[j]) + off, 0, 4, ctx->stream));
    NC_TRY(cudaStreamSynchronize(ctx->stream));
    if (any & ST_TIMEOUT) {
      ctx->poisoned = true;
      return fail(ctx, NC_ETIMEOUT, "a bounded device wait gave up");
    }
    if (any & ST_NUMERIC) return fail(ctx, NC_ENUMERIC, "non-finite probabilities or CDF floor underflow");
    if (any & ST_TABLE_FULL) return fail(ctx, NC_ESTATE, "N-gram tables full (stream longer than expected_len)");
    return fail(ctx, NC_EINVAL, "observed token out of range");
  }
  return NC_OK;
}

static int step_common(nc_ctx* ctx, int n, const int32_t* ids, const int32_t* prev, float* z,
                       float* pt, float* png, float* p, uint32_t* cdf_out) {
  if (!ctx) return NC_EINVAL;
  cudaGetLastError();
  if (ctx->poisoned) return fail(ctx, NC_ESTATE, "context poisoned by an earlier CUDA error");
  cudaSetDevice(ctx->cfg.device);
  std::vector<int> si;
  int st = stage_batch(ctx, n, ids, &si, false);
  if (st != NC_OK) return st;
  if (prev) {
    for (int j = 0; j < n; ++j)
      if (prev[j] != ctx->slots[si[j]].last_tok) return fail(ctx, NC_EINVAL, "prev_tokens differ from the observed history");
  }
  const Dims& D = ctx->D;
  const bool dev_out = cdf_out && is_device_ptr(cdf_out);
  Batch b = make_batch(ctx);
  b.obs = nullptr;
  NC_TRY(launch_model(ctx, b));
  VocabIO io{};
  io.cdf = dev_out ? cdf_out : ctx->cdf;
  io.probe_z = z;
  io.probe_pt = pt;
  io.probe_png = png;
  io.probe_p = p;
  io.predict = 1;
  NC_TRY(launch_vocab(D, b, io, ctx->stream));
  if (cdf_out && !dev_out)
    NC_TRY(cudaMemcpyAsync(cdf_out, ctx->cdf, (size_t)n * (D.V + 1) * 4, cudaMemcpyDeviceToHost, ctx->stream));
  st = check_status(ctx, si);
  if (st != NC_OK) return st;
  for (int j = 0; j < n; ++j) ctx->slots[si[j]].awaiting_update = true;
  return NC_OK;
}

extern "C" int nc_step_cdf(nc_ctx* ctx, int n, const int32_t* stream_ids, const int32_t* prev_tokens,
                           uint32_t* cdf_out) {
  return step_common(ctx, n, stream_ids, prev_tokens, nullptr, nullptr, nullptr, nullptr, cdf_out);
}

extern "C" int nc_step_probe(nc_ctx* ctx, int n, const int32_t* stream_ids, float* z, float* p_tilde,
                             float* p_ng, float* p, uint32_t* cdf_out) {
  for (float* q : {z, p_tilde, p_ng, p})
    if (q && !is_device_ptr(q)) return fail(ctx, NC_EINVAL, "probe buffers must be device memory");
  return step_common(ctx, n, stream_ids, nullptr, z, p_tilde, p_ng, p, cdf_out);
}

extern "C" int nc_update_bias(nc_ctx* ctx, int n, const int32_t* stream_ids, const int32_t* observed) {
  if (!ctx) return NC_EINVAL;
  cudaGetLastError();
  if (ctx->poisoned) return fail(ctx, NC_ESTATE, "context poisoned by an earlier CUDA error");
  if (!observed) return fail(ctx, NC_EINVAL, "observed is NULL");
  cudaSetDevice(ctx->cfg.device);
  for (int j = 0; j < n; ++j)
    if (observed[j] < 0 || observed[j] >= ctx->D.V) return fail(ctx, NC_EINVAL, "observed token out of range");
  std::vector<int> si;
  int st = stage_batch(ctx, n, stream_ids, &si, true);
  if (st != NC_OK) return st;
  std::memcpy(ctx->h_i32 + 1 + ctx->cfg.max_streams, observed, (size_t)n * 4);
  NC_TRY(cudaMemcpyAsync(ctx->d_obs, ctx->h_i32 + 1 + ctx->cfg.max_streams, (size_t)n * 4,
                         cudaMemcpyHostToDevice, ctx->stream));
  Batch b = make_batch(ctx);
  VocabIO io{};
  io.update = 1;
  io.ngram = 1;
  NC_TRY(launch_vocab(ctx->D, b, io, ctx->stream));
  st = check_status(ctx, si);
  if (st != NC_OK) return st;
  for (int j = 0; j < n; ++j) {
    Slot& s = ctx->slots[si[j]];
    s.awaiting_update = false;
    s.n_coded += 1;
    s.last_tok = observed[j];
  }
  return NC_OK;
}

extern "C" int nc_stream_state(nc_ctx* ctx, int32_t stream_id, float* bias, float* mix_logw, int64_t* n_coded) {
  if (!ctx) return NC_EINVAL;
  auto it = ctx->id2slot.find(stream_id);
  if (it == ctx->id2slot.end()) return fail(ctx, NC_EINVAL, "unknown stream id");
  cudaSetDevice(ctx->cfg.device);
  const int si = it->second;
  StreamDev sd;
  NC_TRY(cudaMemcpyAsync(&sd, ctx->d_st + si, sizeof(sd), cudaMemcpyDeviceToHost, ctx->stream));
  if (bias) NC_TRY(cudaMemcpyAsync(bias, ctx->slots[si].bias, (size_t)ctx->D.V * 4, cudaMemcpyDeviceToHost, ctx->stream));
  NC_TRY(cudaStreamSynchronize(ctx->stream));
  if (mix_logw) {
    mix_logw[0] = sd.theta[0];
    mix_logw[1] = sd.theta[1];
  }
  if (n_coded) *n_coded = sd.n_coded;
  return NC_OK;
}

// -------------------------------------------------------- whole streams

static uint8_t flags_byte(const nc_config& c) {
  uint8_t f = 0;
  if (c.ngram_order > 0) f |= 1;
  if (c.use_head) f |= 2;
  if (c.ngram_order > 0 && c.skip) f |= 4;
  if (c.update_rule == NC_RULE_MIXED_NLL) f |= 8;
  if (c.coder == NC_CODER_RANS) f |= 16;
  return f;
}
static uint8_t path_byte(const nc_config& c) { return (uint8_t)(c.weight_fmt | (c.path << 4)); }

// Positions per prefill forward for n streams: the largest power of two m
// with n m <= prefill_rows that divides the window length L and the slide C
// (so no chunk of positions crosses a slide: every row of a forward sees its
// window start fixed), doubling only while m is below the longest stream;
// 0 = no prefill.
static int prefill_chunk(const nc_ctx* ctx, int n, int64_t max_len) {
  const Dims& D = ctx->D;
  if (ctx->P < 2 || n < 1) return 0;
  int m = 1;
  while ((int64_t)2 * m * n <= ctx->P && D.C % (2 * m) == 0 && D.L % (2 * m) == 0 && m < max_len) m *= 2;
  return m >= 2 ? m : 0;
}

// Encoder with prefill: per chunk of m positions, one model forward over the
// n m (stream, position) rows (KV appended for all rows first, logits of
// every row kept), then the m vocabulary passes and updates of each stream
// in order.  Every row's arithmetic is the decode step's, so the intervals
// are those of one position per step.  Streams sorted longest first.
static int encode_prefill(nc_ctx* ctx, int n, int m0, const int32_t* tok_dev, const int64_t* offs_dev,
                          const int64_t* lens_dev, const std::vector<int64_t>& lens_h, uint32_t* intervals,
                          int64_t stride, nc_trace* trace, const VocabIO& probe) {
  const Dims& D = ctx->D;
  cudaStream_t s = ctx->stream;
  int64_t max_len = 0;
  for (int64_t l : lens_h) max_len = std::max(max_len, l);
  // the largest chunk the window allows for one stream
  int m_max = m0;
  while ((int64_t)2 * m_max <= ctx->P && D.C % (2 * m_max) == 0 && D.L % (2 * m_max) == 0 && m_max < max_len)
    m_max *= 2;
  VocabIO io = probe;
  io.predict = 1;
  io.update = 1;
  io.ngram = 1;
  io.intervals = intervals;
  io.interval_stride = stride;
  StepMarks mk;
  mk.on = trace != nullptr;
  const int fwd_marks = 1 + 1 + 5 * D.n_layers + 1;   // prepare, embed, 5 per layer, LM head
  if (mk.on) {
    mk.ev.resize(fwd_marks + 2 + 2);
    for (auto& e : mk.ev) NC_TRY(cudaEventCreate(&e));
  }
  // One chunk of m positions of the first ne streams (the longest; every
  // stream with positions left is among them), with buffer set `par`: the
  // forward (its N-gram pass beside it) and, with_vocab, the vocabulary
  // passes after it on the same stream.
  auto vocab_batch = [&](int ne, int par) {
    Batch br = make_batch(ctx);                   // every stream's m positions, in order
    br.Bmax = ne;
    br.z_idx = ctx->d_zidx[par];
    return br;
  };
  auto one_chunk = [&](int m, int ne, int par, bool with_vocab) -> cudaError_t {
    Batch b = make_batch(ctx);                    // stream rows (slots only)
    b.Bmax = ne;
    Batch f = make_batch(ctx);                    // (stream, position) rows of the forward
    f.slots = ctx->f_slots;
    f.nB = ctx->d_nB_fwd;
    f.obs = nullptr;
    f.Bmax = ne * m;
    f.pos = ctx->f_pos;
    f.tok = ctx->f_tok;
    f.z_out = ctx->zrows[par];
    f.pm = m;
    int32_t* p0 = ctx->d_p0 + par;
    cudaError_t e = mk.begin(s);
    if (e == cudaSuccess) e = launch_chunk_start(ctx->d_p0, par, m, s);
    if (e == cudaSuccess)
      e = launch_prepare_prefill(b, ne, m, D.V, p0, tok_dev, offs_dev, lens_dev, ctx->f_slots, ctx->f_pos,
                                 ctx->f_tok, ctx->d_nB_fwd, ctx->f_obs[par], ctx->f_nb[par], ctx->d_zidx[par], s);
    if (e == cudaSuccess) e = mk.mark(s, TK_PREPARE);
    const Batch br = vocab_batch(ne, par);
    // the N-gram pass needs only the tokens: beside the forward on the side
    // stream (in order on the main stream when each kernel is timed)
    const bool ng = ctx->snap[par] != nullptr;
    const bool side = ng && !mk.on;
    if (side && e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, s);
    if (side && e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    if (side && e == cudaSuccess)
      e = launch_ngram_seq(D, br, m, ctx->f_nb[par], ctx->f_obs[par], p0, ctx->snap[par], ctx->side);
    if (side && e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->side);
    if (e == cudaSuccess) e = launch_model(ctx, f, &mk);
    if (ng && !side && e == cudaSuccess) {
      e = launch_ngram_seq(D, br, m, ctx->f_nb[par], ctx->f_obs[par], p0, ctx->snap[par], s);
      if (e == cudaSuccess) e = mk.mark(s, TK_NGRAM);
    }
    if (side && e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_join, 0);
    if (with_vocab && e == cudaSuccess) {
      e = launch_vocab_seq(D, br, io, m, ctx->zrows[par], ctx->f_nb[par], ctx->f_obs[par], ctx->snap[par], s);
      if (e == cudaSuccess) e = mk.mark(s, TK_VOCAB);
    }
    return e;
  };
  // one captured graph per chunk length and buffer set (captured on first use)
  std::map<int, cudaGraphExec_t> graphs;
  auto graph_for = [&](int m, int ne, int par, bool with_vocab) -> cudaGraphExec_t {
    const int key = 2 * m + par;
    auto it = graphs.find(key);
    if (it != graphs.end()) return it->second;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      mk.capturing = true;
      cudaError_t e = one_chunk(m, ne, par, with_vocab);
      mk.capturing = false;
      cudaError_t e2 = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess || e2 != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
    graphs[key] = ge;
    return ge;
  };
  // chunk c's vocabulary passes run on vstream after its forward, beside
  // chunk c + 1's forward; chunk c + 2 reuses set c & 1 after they are done
  // (timed runs keep every kernel in order on the main stream)
  const bool piped = !mk.on;
  cudaStream_t vs = piped ? ctx->vstream : s;
  NC_TRY(cudaMemsetAsync(ctx->d_p0, 0, 16, s));
  if (trace) {
    std::memset(trace, 0, sizeof(*trace));
    trace->graphed = 1;
    trace->n_kinds = TK_COUNT;
    for (int k = 0; k < TK_COUNT; ++k) std::snprintf(trace->name[k], sizeof(trace->name[k]), "%s", kTraceNames[k]);
  }
  auto start_at = [&](int64_t a) -> int64_t { return a < D.L ? 0 : ((a - D.L) / D.C + 1) * D.C; };
  // Two forward buffer sets: the whole pass is one captured graph.  Chunk
  // c's forward runs on the stream of forward set c & 1 (s, s2) beside chunk
  // c - 1's, each layer's append after chunk c - 1's attention of that layer;
  // the N-gram passes run in chunk order on the side stream and the
  // vocabulary passes in chunk order on vstream.  Chunk c hands its logits,
  // tokens and N-gram states to its passes in coding set c mod 3, which
  // chunk c + 3 reuses after chunk c's vocabulary passes: a forward may run
  // two chunks ahead of the passes.  The graph is kept for the next call with
  // the same chunk plan and buffers.
  if (piped && ctx->n_fs == 2) {
    std::vector<std::pair<int, int>> plan;
    {
      int mm = m0;
      for (int64_t p = 0; p < max_len; p += mm) {
        int live = 0;
        while (live < n && lens_h[live] > p) ++live;
        mm = m_max;
        while (mm > m0 && ((int64_t)live * mm > ctx->P || p % mm != 0)) mm /= 2;
        plan.emplace_back(mm, std::min(n, ctx->P / mm));
      }
    }
    auto ptr = [](const void* q) { return (int64_t)(uintptr_t)q; };
    std::vector<int64_t> key = {n, ptr(tok_dev), ptr(offs_dev), ptr(lens_dev), ptr(intervals), stride,
                                ptr(io.probe_z), ptr(io.probe_pt), ptr(io.probe_png), ptr(io.probe_p), io.probe_tok,
                                ptr(io.probe_row)};
    for (const auto& pc : plan) {
      key.push_back(pc.first);
      key.push_back(pc.second);
    }
    if (!ctx->pass_graph || ctx->pass_key != key) {
      if (ctx->pass_graph) cudaGraphExecDestroy(ctx->pass_graph);
      ctx->pass_graph = nullptr;
      ctx->pass_key.clear();
      cudaStream_t fst[2] = {s, ctx->s2};
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      auto fork = [&](cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
        if (e == cudaSuccess) e = cudaEventRecord(ev, from);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
      };
      fork(s, ctx->s2, ctx->ev_fork);
      fork(s, ctx->side, ctx->ev_fork);
      fork(s, vs, ctx->ev_fork);
      Dims Dv = D;
      Dv.pdl = 0;                                   // the vocabulary passes: see below
      for (size_t c = 0; c < plan.size() && e == cudaSuccess; ++c) {
        const int mc = plan[c].first, ne = plan[c].second, set = (int)(c & 1), cs = (int)(c % kCodeSets);
        cudaStream_t sc = fst[set];
        const nc_ctx::FwdSet& F = ctx->fs[set];
        if (c >= kCodeSets) e = cudaStreamWaitEvent(sc, ctx->ev_voc[cs], 0);   // chunk c - 3's passes read cs
        if (c >= 1 && e == cudaSuccess) e = cudaStreamWaitEvent(sc, ctx->ev_prep[set ^ 1], 0);   // positions in order
        Batch b = make_batch(ctx);
        b.Bmax = ne;
        if (e == cudaSuccess) e = launch_chunk_start(ctx->d_p0, cs, mc, sc);
        int32_t* p0 = ctx->d_p0 + cs;
        if (e == cudaSuccess)
          e = launch_prepare_prefill(b, ne, mc, D.V, p0, tok_dev, offs_dev, lens_dev, F.f_slots, F.f_pos, F.f_tok,
                                     F.nB_fwd, ctx->f_obs[cs], ctx->f_nb[cs], ctx->d_zidx[cs], sc);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_prep[set], sc);
        const Batch br = vocab_batch(ne, cs);
        const bool ng = ctx->snap[cs] != nullptr;
        if (ng && e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_prep[set], 0);
        if (ng && e == cudaSuccess)
          e = launch_ngram_seq(D, br, mc, ctx->f_nb[cs], ctx->f_obs[cs], p0, ctx->snap[cs], ctx->side);
        if (ng && e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->side);
        Batch f = make_batch(ctx);
        f.slots = F.f_slots;
        f.nB = F.nB_fwd;
        f.obs = nullptr;
        f.Bmax = ne * mc;
        f.pos = F.f_pos;
        f.tok = F.f_tok;
        f.z_out = ctx->zrows[cs];
        f.pm = mc;
        LayerSync sync;
        sync.wait = c >= 1 ? ctx->ev_layer[set ^ 1].data() : nullptr;
        sync.rec = ctx->ev_layer[set].data();
        // a kernel launched early would hold its SMs waiting for its
        // predecessor while the other forward could use them
        sync.no_pdl = true;
        StepMarks none;
        if (e == cudaSuccess) e = launch_model_tc(ctx, f, none, set, sc, sync);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fwd[cs], sc);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(vs, ctx->ev_fwd[cs], 0);
        if (ng && e == cudaSuccess) e = cudaStreamWaitEvent(vs, ctx->ev_join, 0);
        // without PDL: it would sit on its SMs while the previous passes run
        if (e == cudaSuccess)
          e = launch_vocab_seq(Dv, br, io, mc, ctx->zrows[cs], ctx->f_nb[cs], ctx->f_obs[cs], ctx->snap[cs], vs);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_voc[cs], vs);
      }
      // join every stream back into s
      fork(ctx->s2, s, ctx->ev_prep[0]);
      fork(ctx->side, s, ctx->ev_join);
      fork(vs, s, ctx->ev_done);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(s, &g);
      if (e == cudaSuccess) e = e2;
      cudaGraphExec_t ge = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail_cuda(ctx, e, "prefill pass capture");
      ctx->pass_graph = ge;
      ctx->pass_key = key;
    }
    const cudaError_t e = cudaGraphLaunch(ctx->pass_graph, s);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "prefill pass");
    for (auto& ev : mk.ev) cudaEventDestroy(ev);
    return NC_OK;
  }
  int st = NC_OK;
  int m = m0;
  int chunk = 0;
  for (int64_t p = 0; p < max_len; p += m, ++chunk) {
    // the largest chunk for the streams still coding, aligned to it (so it
    // never crosses a slide): it only grows as streams end
    int live = 0;
    while (live < n && lens_h[live] > p) ++live;
    m = m_max;
    while (m > m0 && ((int64_t)live * m > ctx->P || p % m != 0)) m /= 2;
    const int ne = std::min(n, ctx->P / m);
    const int par = chunk & 1;
    cudaError_t e = cudaSuccess;
    if (piped && chunk >= 2) e = cudaStreamWaitEvent(s, ctx->ev_voc[par], 0);
    cudaGraphExec_t ge = e == cudaSuccess ? graph_for(m, ne, par, !piped) : nullptr;
    if (trace && !ge) trace->graphed = 0;
    if (e == cudaSuccess) e = ge ? cudaGraphLaunch(ge, s) : one_chunk(m, ne, par, !piped);
    if (piped) {
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fwd[par], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(vs, ctx->ev_fwd[par], 0);
      // without PDL: it would sit on 8 SMs while the previous passes run
      Dims Dv = D;
      Dv.pdl = 0;
      if (e == cudaSuccess)
        e = launch_vocab_seq(Dv, vocab_batch(ne, par), io, m, ctx->zrows[par], ctx->f_nb[par], ctx->f_obs[par],
                             ctx->snap[par], vs);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_voc[par], vs);
    }
    if (e != cudaSuccess) {
      st = fail_cuda(ctx, e, "prefill encode chunk");
      break;
    }
    if (trace) {
      // forward: the live rows and their windows (a stream's rows share the
      // window of its last row); then each position's active streams
      int64_t rows = 0;
      double ctx_sum = 0, kv_unique = 0;
      for (int j = 0; j < n; ++j) {
        const int64_t last = std::min(p + m, lens_h[j]) - 1;
        if (last >= p) kv_unique += (double)(last - start_at(last) + 1);
        for (int64_t a = p; a <= last; ++a) {
          ++rows;
          ctx_sum += (double)(a - start_at(a) + 1);
        }
      }
      double fwd[TK_COUNT], ffl[TK_COUNT];
      step_cost(ctx, (int)rows, ctx_sum, kv_unique, fwd, ffl);
      fwd[TK_PREPARE] = ne * (double)m * 28;
      e = cudaEventSynchronize(mk.ev[mk.n]);
      if (e != cudaSuccess) {
        st = fail_cuda(ctx, e, "trace sync");
        break;
      }
      for (int i = 0; i < mk.n; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, mk.ev[i], mk.ev[i + 1]);
        const int kd = mk.kind[i];
        double by = fwd[kd], fo = ffl[kd];
        if (i >= fwd_marks) {                       // the chunk's vocabulary passes
          by = fo = 0;
          int live = 0;
          for (int64_t a = p; a < p + m; ++a) {
            int act = 0;
            for (int j = 0; j < n; ++j) act += lens_h[j] > a;
            live = std::max(live, act);
            double per[TK_COUNT], pfl[TK_COUNT];
            step_cost(ctx, act, 0.0, 0.0, per, pfl);
            // the loop keeps a stream's bias and unigram counts in registers
            // over the chunk: per position it reads the logits and the
            // N-gram state and writes the interval
            by += kd == TK_VOCAB ? act * (D.V * 4.0 + sizeof(NgSnap) + 8.0) : per[kd];
            fo += pfl[kd];
          }
          if (kd == TK_VOCAB) by += live * D.V * 16.0;   // bias and counts read and written once
        }
        trace->ms[kd] += ms;
        trace->launches[kd] += 1;
        trace->bytes[kd] += by;
        trace->flops[kd] += fo;
      }
    }
  }
  if (piped) {                                    // the caller's stream sees the last passes
    cudaError_t e = cudaEventRecord(ctx->ev_done, vs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_done, 0);
    if (e != cudaSuccess && st == NC_OK) st = fail_cuda(ctx, e, "prefill encode join");
  }
  for (auto& kv : graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  for (auto& e : mk.ev) cudaEventDestroy(e);
  return st;
}

// The device half of nc_encode: tokens resident on the device, one captured
// step replayed until every stream is coded.  Streams must already be open in
// slots slot_of[r] (row order = longest first, so the active rows of every
// step are a prefix).  intervals: DEVICE uint32[n][stride][2].
static int encode_device(nc_ctx* ctx, int n, const std::vector<int>& slot_of, const int32_t* tok_dev,
                         const int64_t* offs_dev, const int64_t* lens_dev, const std::vector<int64_t>& lens_h,
                         uint32_t* intervals, int64_t stride, nc_trace* trace, const VocabIO& probe) {
  const Dims& D = ctx->D;
  cudaStream_t s = ctx->stream;
  int64_t max_len = 0;
  for (int64_t l : lens_h) max_len = std::max(max_len, l);
  for (int j = 0; j < n; ++j) ctx->h_i32[1 + j] = slot_of[j];
  NC_TRY(cudaMemcpyAsync(ctx->d_slots, ctx->h_i32 + 1, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  const int m = prefill_chunk(ctx, n, max_len);
  if (m >= 2) return encode_prefill(ctx, n, m, tok_dev, offs_dev, lens_dev, lens_h, intervals, stride, trace, probe);
  Batch b = make_batch(ctx);
  b.Bmax = n;
  VocabIO io = probe;
  io.predict = 1;
  io.update = 1;
  io.ngram = 1;
  io.intervals = intervals;
  io.interval_stride = stride;
  StepMarks mk;
  mk.on = trace != nullptr;
  if (mk.on) {
    mk.ev.resize(12 + 5 * D.n_layers);
    for (auto& e : mk.ev) NC_TRY(cudaEventCreate(&e));
  }
  auto one_step = [&]() -> cudaError_t {
    cudaError_t e = mk.begin(s);
    if (e == cudaSuccess) e = launch_prepare_encode(b, n, tok_dev, offs_dev, lens_dev, ctx->d_obs, ctx->d_nB, s);
    if (e == cudaSuccess) e = mk.mark(s, TK_PREPARE);
    if (e == cudaSuccess) e = launch_model(ctx, b, &mk);
    if (e == cudaSuccess) e = launch_vocab(D, b, io, s);
    if (e == cudaSuccess) e = mk.mark(s, TK_VOCAB);
    return e;
  };
  // capture one step in a graph (the whole step is device-driven)
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    mk.capturing = true;
    cudaError_t e = one_step();
    mk.capturing = false;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
  }
  if (trace) {
    std::memset(trace, 0, sizeof(*trace));
    trace->graphed = ge != nullptr;
    trace->n_kinds = TK_COUNT;
    for (int k = 0; k < TK_COUNT; ++k) std::snprintf(trace->name[k], sizeof(trace->name[k]), "%s", kTraceNames[k]);
  }
  int st = NC_OK;
  int active = n;
  for (int64_t k = 0; k < max_len; ++k) {
    cudaError_t e = ge ? cudaGraphLaunch(ge, s) : one_step();
    if (e != cudaSuccess) {
      st = fail_cuda(ctx, e, "encode step");
      break;
    }
    if (trace) {
      // every active row has coded k tokens; its window after the step's slide
      while (active > 0 && lens_h[active - 1] <= k) --active;
      int64_t start = 0;
      {
        // kv_start after k steps, from the same recurrence as the kernels
        const int64_t L = D.L, C = D.C;
        if (k >= L) start = ((k - L) / C + 1) * C;
      }
      const int n_ctx = (int)(k - start + 1);
      double bytes[TK_COUNT], flops[TK_COUNT];
      step_cost(ctx, active, (double)active * n_ctx, (double)active * n_ctx, bytes, flops);
      e = cudaEventSynchronize(mk.ev[mk.n]);
      if (e != cudaSuccess) {
        st = fail_cuda(ctx, e, "trace sync");
        break;
      }
      for (int i = 0; i < mk.n; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, mk.ev[i], mk.ev[i + 1]);
        const int kd = mk.kind[i];
        trace->ms[kd] += ms;
        trace->launches[kd] += 1;
        trace->bytes[kd] += bytes[kd];
        trace->flops[kd] += flops[kd];
      }
    }
  }
  if (ge) cudaGraphExecDestroy(ge);
  for (auto& e : mk.ev) cudaEventDestroy(e);
  return st;
}

// Open fresh slots for n streams, longest first; returns the row order.
static int open_rows(nc_ctx* ctx, int n, const int64_t* lens, std::vector<int>* order,
                     std::vector<int>* slot_of, std::vector<int32_t>* ids, int32_t id_base) {
  order->resize(n);
  for (int j = 0; j < n; ++j) (*order)[j] = j;
  std::stable_sort(order->begin(), order->end(), [&](int a, int b) { return lens[a] > lens[b]; });
  slot_of->assign(n, -1);
  ids->assign(n, -1);
  int32_t next_id = id_base;
  for (int r = 0; r < n; ++r) {
    while (ctx->id2slot.count(next_id)) ++next_id;
    (*ids)[r] = next_id++;
    const int st = open_slot(ctx, (*ids)[r], std::max<int64_t>(lens[(*order)[r]], 1), &(*slot_of)[r]);
    if (st != NC_OK) return st;
  }
  return NC_OK;
}

static void close_rows(nc_ctx* ctx, const std::vector<int32_t>& ids) {
  for (int32_t id : ids)
    if (id >= 0 && ctx->id2slot.count(id)) nc_stream_close(ctx, id);
}

// nc_encode_intervals, with the probes of `probe` (probe_tok > 0) written to
// the caller's rows.
static int encode_intervals(nc_ctx* ctx, int n_streams, const int32_t* tokens_dev, const int64_t* offsets,
                            const int64_t* lens, uint32_t* intervals_dev, int64_t stride, nc_trace* trace,
                            VocabIO probe) {
  if (!ctx) return NC_EINVAL;
  if (ctx->poisoned) return fail(ctx, NC_ESTATE, "context poisoned by an earlier CUDA error");
  if (!tokens_dev || !offsets || !lens || !intervals_dev || n_streams < 1) return fail(ctx, NC_EINVAL, "bad arguments");
  if (n_streams > ctx->cfg.max_streams) return fail(ctx, NC_EINVAL, "more streams than max_streams");
  int64_t max_len = 0;
  for (int j = 0; j < n_streams; ++j) {
    if (lens[j] < 0 || offsets[j] < 0) return fail(ctx, NC_EINVAL, "bad stream extent");
    max_len = std::max(max_len, lens[j]);
  }
  if (stride < max_len) return fail(ctx, NC_EINVAL, "stride below the longest stream");
  if (!is_device_ptr(tokens_dev) || !is_device_ptr(intervals_dev)) return fail(ctx, NC_EINVAL, "tokens and intervals must be device memory");
  cudaSetDevice(ctx->cfg.device);
  int free_slots = 0;
  for (auto& s : ctx->slots) free_slots += !s.open;
  if (free_slots < n_streams) return fail(ctx, NC_EINVAL, "not enough free stream slots");
  std::vector<int> order, slot_of;
  std::vector<int32_t> ids;
  int st = open_rows(ctx, n_streams, lens, &order, &slot_of, &ids, 0x60000000);
  int64_t* meta = ctx->d_meta;
  uint32_t* iv_rows = nullptr;
  std::vector<int64_t> lens_h(n_streams);
  do {
    if (st != NC_OK) break;
    // row r reads stream order[r]: offsets in rows, intervals written per row
    // row r reads stream order[r]: offsets, lengths and the probes' rows
    std::vector<int64_t> h_meta(3 * n_streams);
    for (int r = 0; r < n_streams; ++r) {
      h_meta[r] = offsets[order[r]];
      h_meta[n_streams + r] = lens[order[r]];
      h_meta[2 * n_streams + r] = order[r];
      lens_h[r] = lens[order[r]];
    }
    bool identity = true;
    for (int r = 0; r < n_streams; ++r) identity &= order[r] == r;
    if (!identity && dev_malloc(&iv_rows, (size_t)n_streams * stride * 8) != cudaSuccess) {
      st = fail(ctx, NC_ENOMEM, "interval staging allocation");
      break;
    }
    if (cudaMemcpyAsync(meta, h_meta.data(), 3 * n_streams * 8, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
      st = fail_cuda(ctx, cudaErrorUnknown, "meta upload");
      break;
    }
    uint32_t* target = identity ? intervals_dev : iv_rows;
    probe.probe_row = meta + 2 * n_streams;
    st = encode_device(ctx, n_streams, slot_of, tokens_dev, meta, meta + n_streams, lens_h, target, stride, trace,
                       probe);
    if (st != NC_OK) break;
    if (!identity)
      for (int r = 0; r < n_streams; ++r)
        if (cudaMemcpyAsync(intervals_dev + (size_t)order[r] * stride * 2, iv_rows + (size_t)r * stride * 2,
                            (size_t)stride * 8, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
          st = fail_cuda(ctx, cudaErrorUnknown, "interval reorder");
          break;
        }
    if (st == NC_OK) st = check_status(ctx, slot_of);
  } while (0);
  cudaFree(iv_rows);
  close_rows(ctx, ids);
  return st;
}

extern "C" int nc_encode_intervals(nc_ctx* ctx, int n_streams, const int32_t* tokens_dev, const int64_t* offsets,
                                   const int64_t* lens, uint32_t* intervals_dev, int64_t stride, nc_trace* trace) {
  return encode_intervals(ctx, n_streams, tokens_dev, offsets, lens, intervals_dev, stride, trace, VocabIO{});
}

extern "C" int nc_encode_probe(nc_ctx* ctx, int n_streams, const int32_t* tokens_dev, const int64_t* offsets,
                               const int64_t* lens, uint32_t* intervals_dev, int64_t stride, int64_t probe_pos,
                               float* z, float* p_tilde, float* p_ng, float* p) {
  if (!ctx) return NC_EINVAL;
  if (probe_pos < 0) return fail(ctx, NC_EINVAL, "probe position below 0");
  for (float* q : {z, p_tilde, p_ng, p})
    if (q && !is_device_ptr(q)) return fail(ctx, NC_EINVAL, "probe buffers must be device memory");
  VocabIO probe{};
  probe.probe_tok = probe_pos + 1;
  probe.probe_z = z;
  probe.probe_pt = p_tilde;
  probe.probe_png = p_ng;
  probe.probe_p = p;
  return encode_intervals(ctx, n_streams, tokens_dev, offsets, lens, intervals_dev, stride, nullptr, probe);
}

extern "C" int nc_encode(nc_ctx* ctx, int n_streams, const int32_t* const* tokens, const int64_t* lens,
                         uint8_t* out, size_t* inout_nbytes) {
  if (!ctx) return NC_EINVAL;
  if (ctx->poisoned) return fail(ctx, NC_ESTATE, "context poisoned by an earlier CUDA error");
  if (!tokens || !lens || !inout_nbytes || n_streams < 1 || n_streams > 65535)
    return fail(ctx, NC_EINVAL, "bad arguments");
  if (n_streams > ctx->cfg.max_streams) return fail(ctx, NC_EINVAL, "more streams than max_streams");
  const Dims& D = ctx->D;
  int64_t total = 0, max_len = 0;
  for (int j = 0; j < n_streams; ++j) {
    if (lens[j] < 0 || lens[j] > 0x7fffffff || (lens[j] > 0 && !tokens[j])) return fail(ctx, NC_EINVAL, "bad stream");
    total += lens[j];
    max_len = std::max(max_len, lens[j]);
    for (int64_t i = 0; i < lens[j]; ++i)
      if (tokens[j][i] < 0 || tokens[j][i] >= D.V) return fail(ctx, NC_EINVAL, "token out of range");
  }
  // worst case: about 24 bits + 2 per token plus 2 bits per stream
  std::vector<StreamRecord> bound(n_streams);
  for (int j = 0; j < n_streams; ++j) {
    // arithmetic coder: at most log2 T + 2 bits per token; rANS: log2 T plus
    // under 0.02 per token, the 31-bit start and the 64-bit final state
    const uint64_t bits = (uint64_t)lens[j] * (D.log2T + 2) + 192;
    bound[j] = StreamRecord{(uint32_t)lens[j], (uint32_t)bits, (uint32_t)((bits + 7) / 8)};
  }
  if (!out) {
    *inout_nbytes = container_size(bound);
    return NC_OK;
  }
  cudaSetDevice(ctx->cfg.device);
  int free_slots = 0;
  for (auto& s : ctx->slots) free_slots += !s.open;
  if (free_slots < n_streams) return fail(ctx, NC_EINVAL, "not enough free stream slots");
  std::vector<int> order, slot_of;
  std::vector<int32_t> ids;
  int st = open_rows(ctx, n_streams, lens, &order, &slot_of, &ids, 0x40000000);
  auto close_all = [&]() { close_rows(ctx, ids); };
  if (st != NC_OK) {
    close_all();
    return st;
  }
  // tokens, offsets and lengths to the device (row order = longest first)
  int64_t* meta = ctx->d_meta;
  std::vector<int64_t> h_meta(2 * n_streams);
  int64_t off = 0;
  for (int r = 0; r < n_streams; ++r) {
    h_meta[r] = off;
    h_meta[n_streams + r] = lens[order[r]];
    off += lens[order[r]];
  }
  std::vector<uint32_t> h_iv;
  do {
    const size_t need_tok = (size_t)std::max<int64_t>(total, 1);
    const size_t need_iv = (size_t)n_streams * std::max<int64_t>(max_len, 1) * 2;
    if (ctx->enc_tok_cap < need_tok) {
      cudaFree(ctx->enc_tok);
      ctx->enc_tok = nullptr;
      ctx->enc_tok_cap = 0;
      if (dev_malloc(&ctx->enc_tok, need_tok * 4) == cudaSuccess) ctx->enc_tok_cap = need_tok;
    }
    if (ctx->enc_iv_cap < need_iv) {
      cudaFree(ctx->enc_iv);
      ctx->enc_iv = nullptr;
      ctx->enc_iv_cap = 0;
      if (dev_malloc(&ctx->enc_iv, need_iv * 4) == cudaSuccess) ctx->enc_iv_cap = need_iv;
    }
    if (ctx->enc_tok_cap < need_tok || ctx->enc_iv_cap < need_iv) {
      st = fail(ctx, NC_ENOMEM, "device allocation for encode failed");
      break;
    }
    int32_t* tok_dev = ctx->enc_tok;
    uint32_t* iv = ctx->enc_iv;
    for (int r = 0; r < n_streams; ++r)
      if (lens[order[r]] > 0 &&
          cudaMemcpyAsync(tok_dev + h_meta[r], tokens[order[r]], lens[order[r]] * 4, cudaMemcpyHostToDevice,
                          ctx->stream) != cudaSuccess) {
        st = fail_cuda(ctx, cudaErrorUnknown, "token upload");
        break;
      }
    if (st != NC_OK) break;
    if (cudaMemcpyAsync(meta, h_meta.data(), 2 * n_streams * 8, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
      st = fail_cuda(ctx, cudaErrorUnknown, "meta upload");
      break;
    }
    std::vector<int64_t> lens_rows(n_streams);
    for (int r = 0; r < n_streams; ++r) lens_rows[r] = lens[order[r]];
    st = encode_device(ctx, n_streams, slot_of, tok_dev, meta, meta + n_streams, lens_rows, iv, max_len, nullptr,
                       VocabIO{});
    if (st != NC_OK) break;
    h_iv.resize((size_t)n_streams * max_len * 2);
    if (cudaMemcpyAsync(h_iv.data(), iv, h_iv.size() * 4, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) {
      st = fail_cuda(ctx, cudaErrorUnknown, "interval download");
      break;
    }
    st = check_status(ctx, slot_of);
  } while (0);
  close_all();
  if (st != NC_OK) return st;
  // host coder, streams in parallel
  const bool rans = ctx->cfg.coder == NC_CODER_RANS;
  std::vector<AcEncoder> enc;
  enc.reserve(n_streams);
  for (int j = 0; j < n_streams; ++j) enc.emplace_back(D.log2T);
  std::vector<std::vector<uint8_t>> rans_out(n_streams);
  std::vector<int> bad(n_streams, 0);
  auto work = [&](int r0, int r1) {
    std::vector<uint32_t> lo, hi;
    for (int r = r0; r < r1; ++r) {
      const uint32_t* p = h_iv.data() + (size_t)r * max_len * 2;
      const int64_t len = lens[order[r]];
      if (rans) {
        lo.resize(len);
        hi.resize(len);
        for (int64_t i = 0; i < len; ++i) {
          lo[i] = p[2 * i];
          hi[i] = p[2 * i + 1];
        }
        if (!rans_encode(lo.data(), hi.data(), len, D.log2T, &rans_out[order[r]])) bad[order[r]] = 1;
        continue;
      }
      AcEncoder& e = enc[order[r]];
      for (int64_t i = 0; i < len; ++i)
        if (!e.encode(p[2 * i], p[2 * i + 1])) bad[order[r]] = 1;
      e.finish();
    }
  };
  const int nthr = std::max(1, std::min<int>(n_streams, (int)std::thread::hardware_concurrency()));
  if (nthr == 1) {
    work(0, n_streams);
  } else {
    std::vector<std::thread> th;
    const int per = (n_streams + nthr - 1) / nthr;
    for (int t = 0; t < nthr; ++t) {
      const int r0 = t * per, r1 = std::min(n_streams, r0 + per);
      if (r0 < r1) th.emplace_back(work, r0, r1);
    }
    for (auto& t : th) t.join();
  }
  for (int j = 0; j < n_streams; ++j)
    if (bad[j]) return fail(ctx, NC_ENUMERIC, "empty coder interval");
  std::vector<StreamRecord> recs(n_streams);
  std::vector<const std::vector<uint8_t>*> pays(n_streams);
  for (int j = 0; j < n_streams; ++j) {
    const std::vector<uint8_t>& bytes = rans ? rans_out[j] : enc[j].bytes();
    const uint64_t nbits = rans ? 8ull * bytes.size() : enc[j].nbits();
    if (nbits > 0xffffffffull) return fail(ctx, NC_EINVAL, "stream too long for the container");
    recs[j] = StreamRecord{(uint32_t)lens[j], (uint32_t)nbits, (uint32_t)bytes.size()};
    pays[j] = &bytes;
  }
  const size_t need = container_size(recs);
  if (*inout_nbytes < need) {
    *inout_nbytes = need;
    return fail(ctx, NC_EINVAL, "output buffer too small");
  }
  container_write(out, flags_byte(ctx->cfg), ctx->cfg.temperature, path_byte(ctx->cfg), recs, pays);
  *inout_nbytes = need;
  return NC_OK;
}

extern "C" int nc_container_streams(const uint8_t* in, size_t nbytes, int* n_streams) {
  uint8_t flags, pb;
  float tau;
  std::vector<StreamRecord> recs;
  std::vector<const uint8_t*> pays;
  if (!n_streams || !container_read(in, nbytes, &flags, &tau, &pb, &recs, &pays)) return NC_ECORRUPT;
  *n_streams = (int)recs.size();
  return NC_OK;
}

extern "C" int nc_decode(nc_ctx* ctx, const uint8_t* in, size_t nbytes, int32_t* const* tokens_out,
                         int64_t* lens_out) {
  if (!ctx) return NC_EINVAL;
  if (ctx->poisoned) return fail(ctx, NC_ESTATE, "context poisoned by an earlier CUDA error");
  if (!in || !lens_out) return fail(ctx, NC_EINVAL, "bad arguments");
  uint8_t flags, pb;
  float tau;
  std::vector<StreamRecord> recs;
  std::vector<const uint8_t*> pays;
  if (!container_read(in, nbytes, &flags, &tau, &pb, &recs, &pays)) return fail(ctx, NC_ECORRUPT, "malformed container");
  if (flags != flags_byte(ctx->cfg) || pb != path_byte(ctx->cfg) ||
      float_to_half_bits(tau) != float_to_half_bits(ctx->cfg.temperature))
    return fail(ctx, NC_ECORRUPT, "container features or numeric path differ from the context");
  const int n = (int)recs.size();
  for (int j = 0; j < n; ++j) lens_out[j] = recs[j].ntok;
  if (!tokens_out) return NC_OK;
  if (n > ctx->cfg.max_streams) return fail(ctx, NC_EINVAL, "more streams than max_streams");
  if (n == 0) return NC_OK;
  const Dims& D = ctx->D;
  cudaSetDevice(ctx->cfg.device);
  cudaStream_t s = ctx->stream;
  std::vector<int64_t> rlens(n);
  for (int j = 0; j < n; ++j) rlens[j] = recs[j].ntok;
  std::vector<int> order, slot_of;
  std::vector<int32_t> ids;
  int st = open_rows(ctx, n, rlens.data(), &order, &slot_of, &ids, 0x50000000);
  auto close_all = [&]() { close_rows(ctx, ids); };
  if (st != NC_OK) {
    close_all();
    return st;
  }
  // the stream coder the container records (its flags equal the context's)
  const bool rans = (flags & 16) != 0;
  std::vector<AcDecoder> dec;
  std::vector<RansDecoder> rdec;
  dec.reserve(n);
  rdec.reserve(n);
  for (int r = 0; r < n; ++r) {
    dec.emplace_back(pays[order[r]], recs[order[r]].nbits, D.log2T);
    rdec.emplace_back(pays[order[r]], recs[order[r]].nbytes, D.log2T);
    if (rans && !rdec.back().valid()) {
      close_all();
      return fail(ctx, NC_ECORRUPT, "rANS stream length is not 8 + 4k bytes");
    }
  }
  for (int r = 0; r < n; ++r) ctx->h_i32[1 + r] = slot_of[r];
  int64_t max_len = recs[order[0]].ntok;
  Batch b = make_batch(ctx);
  b.Bmax = n;
  do {
    if (cudaMemcpyAsync(ctx->d_slots, ctx->h_i32 + 1, (size_t)n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = fail_cuda(ctx, cudaErrorUnknown, "slot upload");
      break;
    }
    // one decode step (the decoder learns each token from the coder between
    // steps): the active count and the coder targets in from pinned host
    // memory, the model, the CDFs, the search, the updates, the coded
    // intervals and tokens out.  Captured once in a CUDA graph and replayed
    // per position; the copies read and write the same pinned buffers.
    auto one_step = [&]() -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(ctx->d_nB, ctx->h_i32, 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_target, ctx->h_u32, (size_t)n * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = launch_model(ctx, b);
      VocabIO io{};
      io.cdf = ctx->cdf;
      io.predict = 1;
      if (e == cudaSuccess) e = launch_vocab(D, b, io, s);
      if (e == cudaSuccess) e = launch_search(b, D.V, ctx->cdf, ctx->d_target, ctx->d_obs, ctx->d_lohi, s);
      VocabIO up{};
      up.update = 1;
      up.ngram = 1;
      if (e == cudaSuccess) e = launch_vocab(D, b, up, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_u32 + n, ctx->d_lohi, (size_t)n * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_i32 + 1 + 2 * ctx->cfg.max_streams, ctx->d_obs, (size_t)n * 4,
                                                cudaMemcpyDeviceToHost, s);
      return e;
    };
    cudaGraphExec_t ge = nullptr;
    {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const cudaError_t e = one_step();
        const cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
      }
    }
    int active = n;
    for (int64_t k = 0; k < max_len && st == NC_OK; ++k) {
      while (active > 0 && recs[order[active - 1]].ntok <= k) --active;
      ctx->h_i32[0] = active;
      for (int r = 0; r < active; ++r) ctx->h_u32[r] = rans ? rdec[r].target() : dec[r].target();
      cudaError_t e = ge ? cudaGraphLaunch(ge, s) : one_step();
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        st = fail_cuda(ctx, e, "decode step");
        break;
      }
      for (int r = 0; r < active; ++r) {
        const uint32_t lo = ctx->h_u32[n + 2 * r], hi = ctx->h_u32[n + 2 * r + 1];
        if (rans)
          rdec[r].consume(lo, hi);
        else
          dec[r].consume(lo, hi);
        tokens_out[order[r]][k] = ctx->h_i32[1 + 2 * ctx->cfg.max_streams + r];
      }
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (st == NC_OK) st = check_status(ctx, slot_of);
    for (int r = 0; r < n && st == NC_OK && rans; ++r)
      if (!rdec[r].finished()) st = fail(ctx, NC_ECORRUPT, "rANS stream does not end in its initial state");
  } while (0);
  close_all();
  return st;
}

// ------------------------------------------------------ building blocks

extern "C" int nc_selftest_wait(nc_ctx* ctx, uint32_t polls) {
  if (!ctx) return NC_EINVAL;
  if (ctx->poisoned) return fail(ctx, NC_ESTATE, "context poisoned by an earlier CUDA error");
  cudaSetDevice(ctx->cfg.device);
  int32_t w = 0;
  NC_TRY(cudaMemsetAsync(ctx->d_status, 0, 4, ctx->stream));
  NC_TRY(launch_wait_selftest(polls, ctx->d_status, ctx->stream));
  NC_TRY(cudaMemcpyAsync(&w, ctx->d_status, 4, cudaMemcpyDeviceToHost, ctx->stream));
  NC_TRY(cudaStreamSynchronize(ctx->stream));
  if (w & ST_TIMEOUT) {
    ctx->poisoned = true;
    return fail(ctx, NC_ETIMEOUT, "a bounded device wait gave up");
  }
  return NC_OK;
}

extern "C" int nc_launch_chain_floor(int device, int n_links, int blocks, int threads, int reps,
                                    float* us_per_link) {
  if (n_links < 1 || n_links > 4096 || blocks < 1 || blocks > 65535 || threads < 32 || threads > 1024 ||
      threads % 32 || reps < 1 || !us_per_link)
    return NC_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return NC_ECUDA;
  cudaStream_t s = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t el = cudaSuccess;
    for (int i = 0; i < n_links && el == cudaSuccess; ++i) el = launch_chain_link(dim3(blocks), dim3(threads), s);
    e = cudaStreamEndCapture(s, &g);
    if (el != cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaGraphLaunch(ge, s);   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = cudaGraphLaunch(ge, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *us_per_link = ms * 1000.f / ((float)reps * (float)n_links);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return e == cudaSuccess ? NC_OK : NC_ECUDA;
}

extern "C" int nc_probs_to_cdf(const float* p, int n, int V, int log2_total, uint32_t floor_c, uint32_t* cdf,
                               void* stream) {
  if (!p || !cdf || n < 1 || V < 2 || V > 65535 || log2_total < 1 || log2_total > 24 || floor_c < 1 ||
      (uint64_t)V * floor_c >= (1ull << log2_total))
    return NC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* status = nullptr;
  if (dev_malloc(&status, (size_t)n * 4) != cudaSuccess) return NC_ENOMEM;
  int rc = NC_OK;
  std::vector<int32_t> hs(n);
  if (cudaMemsetAsync(status, 0, (size_t)n * 4, s) != cudaSuccess ||
      launch_probs_to_cdf(p, n, V, log2_total, floor_c, cdf, status, s) != cudaSuccess ||
      cudaMemcpyAsync(hs.data(), status, (size_t)n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = NC_ECUDA;
  cudaFree(status);
  if (rc == NC_OK)
    for (int j = 0; j < n; ++j)
      if (hs[j]) rc = NC_ENUMERIC;
  return rc;
}

extern "C" int nc_floor_counts(const float* p, int64_t n, uint32_t K, uint32_t floor_c, uint32_t* c, void* stream) {
  if (!p || !c || n < 0 || K < 1 || K >= (1u << 24)) return NC_EINVAL;
  if (n == 0) return NC_OK;
  return launch_floor_counts(p, n, K, floor_c, c, static_cast<cudaStream_t>(stream)) == cudaSuccess ? NC_OK : NC_ECUDA;
}

extern "C" int nc_gemm_tc(const void* W, const void* X, const float* w_scale, const float* x_scale, int fp8, int M,
                          int N, int K, int bn, float* Y, void* stream) {
  if (!W || !X || !Y || M < 1 || N < 1 || K < 1 || (fp8 && (!w_scale || !x_scale))) return NC_EINVAL;
  cudaGetLastError();                              // a stale error of an earlier call is not ours
  if (prepare_tc_kernels() != cudaSuccess) return NC_ECUDA;
  if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return NC_EINVAL;
  const int esz = fp8 ? 1 : 2;
  if ((K * esz) % 16 || (reinterpret_cast<uintptr_t>(W) | reinterpret_cast<uintptr_t>(X)) % 16) return NC_EINVAL;
  TcMat t;
  t.M = M;
  t.K = K;
  if (!tc_encode_weights(t, W, esz) || !tc_encode_operand(t, &t.b[0][0], X, esz, N, bn)) return NC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* dev = nullptr;
  if (dev_malloc(&dev, 8) != cudaSuccess) return NC_ENOMEM;
  const int32_t h[2] = {N, 0};
  int rc = NC_OK;
  int32_t back[2] = {0, 0};
  TcGemm g{};
  g.tmap_a = &t.a;
  g.tmap_b = &t.b[0][0];
  g.M = M;
  g.K = K;
  g.Bmax = N;
  g.bn = bn;
  g.kp = t.kp;
  g.kind_bf16 = !fp8;
  g.nB = dev;
  g.w_scale = w_scale;
  g.x_scale = x_scale;
  g.y = Y;
  g.status = dev + 1;
  if (cudaMemcpyAsync(dev, h, 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      launch_gemm_tc(g, EPI_STORE, s, false) != cudaSuccess ||
      cudaMemcpyAsync(back, dev, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    rc = NC_ECUDA;
  cudaFree(dev);
  if (rc == NC_OK && back[1]) rc = NC_ETIMEOUT;
  return rc;
}

extern "C" int nc_ac_encode(const uint32_t* lo, const uint32_t* hi, int64_t n, int log2_total, uint8_t* out,
                            size_t* inout_nbytes, uint64_t* nbits) {
  if (!lo || !hi || !inout_nbytes || n < 0 || log2_total < 1 || log2_total > 30) return NC_EINVAL;
  AcEncoder e(log2_total);
  for (int64_t i = 0; i < n; ++i)
    if (!e.encode(lo[i], hi[i])) return NC_EINVAL;
  e.finish();
  const size_t need = e.bytes().size();
  if (nbits) *nbits = e.nbits();
  if (!out || *inout_nbytes < need) {
    *inout_nbytes = need;
    return out ? NC_EINVAL : NC_OK;
  }
  std::memcpy(out, e.bytes().data(), need);
  *inout_nbytes = need;
  return NC_OK;
}

extern "C" int nc_ac_decode(const uint8_t* bits, uint64_t nbits, const uint32_t* cdfs, int V, int64_t n,
                            int log2_total, int32_t* symbols) {
  if ((!bits && nbits) || !cdfs || !symbols || V < 1 || n < 0 || log2_total < 1 || log2_total > 30) return NC_EINVAL;
  const uint64_t T = 1ull << log2_total;
  AcDecoder d(bits, nbits, log2_total);
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t* c = cdfs + (size_t)i * (V + 1);
    if (c[0] != 0 || c[V] != T) return NC_ECORRUPT;
    const uint32_t t = d.target();
    int lo = 0, hi = V - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (c[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (c[lo + 1] <= c[lo]) return NC_ECORRUPT;
    symbols[i] = lo;
    d.consume(c[lo], c[lo + 1]);
  }
  return NC_OK;
}

extern "C" int nc_split_chunks(const int32_t* tokens, int64_t n, const uint8_t* is_boundary, int V, int n_chunks,
                               int64_t* cuts, int* n_chunks_out) {
  if ((!tokens && n > 0) || !is_boundary || !cuts || !n_chunks_out || n < 0 || V < 1 || n_chunks < 1)
    return NC_EINVAL;
  std::vector<int64_t> c;
  if (!split_points(tokens, n, is_boundary, V, n_chunks, &c)) return NC_EINVAL;
  const int m = n == 0 ? 0 : (int)c.size() - 1;
  for (int j = 0; j <= m; ++j) cuts[j] = c[j];
  *n_chunks_out = m;
  return NC_OK;
}

extern "C" int nc_hybrid_segments(const uint8_t* data, int64_t n, uint8_t* kinds, int64_t* lens, int64_t cap,
                                  int64_t* n_runs) {
  if ((!data && n > 0) || n < 0 || !n_runs || cap < 0 || (cap > 0 && (!kinds || !lens))) return NC_EINVAL;
  std::vector<HybridRun> runs;
  hybrid_segments(data, n, &runs);
  *n_runs = (int64_t)runs.size();
  if (cap == 0) return NC_OK;                                  // size query
  if (cap < (int64_t)runs.size()) return NC_EINVAL;
  for (size_t j = 0; j < runs.size(); ++j) {
    kinds[j] = runs[j].kind;
    lens[j] = runs[j].len;
  }
  return NC_OK;
}

extern "C" int nc_hybrid_pack(const uint8_t* kinds, const int64_t* lens, int64_t n_runs, int method,
                              const uint8_t* stored, size_t n_stored, const uint8_t* text, size_t n_text,
                              uint8_t* out, size_t* inout_nbytes) {
  if (!inout_nbytes || n_runs < 0 || n_runs > (int64_t)UINT32_MAX || (n_runs > 0 && (!kinds || !lens)) ||
      method < 0 || method > 2 || n_stored > UINT32_MAX || (n_stored && !stored) || (n_text && !text))
    return NC_EINVAL;
  // the flags byte and temperature of the text runs' container (NC05: bytes 4 and 5..6)
  const bool nc05 = n_text >= kHeaderBytes && std::memcmp(text, "NC05", 4) == 0;
  if (n_text && !nc05) return NC_EINVAL;
  const uint8_t flags = nc05 ? text[4] : 0;
  const uint16_t tau = nc05 ? (uint16_t)(text[5] | (text[6] << 8)) : float_to_half_bits(1.0f);
  std::vector<HybridRun> runs((size_t)n_runs);
  for (int64_t j = 0; j < n_runs; ++j) {
    if (kinds[j] > kRunBinary || lens[j] < 1 || lens[j] > (int64_t)UINT32_MAX) return NC_EINVAL;
    runs[j] = {kinds[j], lens[j]};
  }
  const size_t need = hybrid_size(runs.size(), n_stored, n_text);
  if (!out || *inout_nbytes < need) {
    *inout_nbytes = need;
    return out ? NC_EINVAL : NC_OK;
  }
  hybrid_write(out, flags, tau, runs, (uint8_t)method, stored, n_stored, text, n_text);
  *inout_nbytes = need;
  return NC_OK;
}

extern "C" int nc_hybrid_parse(const uint8_t* buf, size_t n, uint8_t* kinds, int64_t* lens, int64_t cap,
                               int64_t* n_runs, int* method, size_t* stored_off, size_t* stored_len,
                               size_t* text_off) {
  if (!buf || !n_runs || cap < 0 || (cap > 0 && (!kinds || !lens)) || !method || !stored_off || !stored_len ||
      !text_off)
    return NC_EINVAL;
  uint8_t flags = 0, m = 0;
  uint16_t tau = 0;
  std::vector<HybridRun> runs;
  if (!hybrid_read(buf, n, &flags, &tau, &runs, &m, stored_off, stored_len, text_off)) return NC_ECORRUPT;
  *n_runs = (int64_t)runs.size();
  *method = m;
  if (cap == 0) return NC_OK;
  if (cap < (int64_t)runs.size()) return NC_EINVAL;
  for (size_t j = 0; j < runs.size(); ++j) {
    kinds[j] = runs[j].kind;
    lens[j] = runs[j].len;
  }
  return NC_OK;
}

extern "C" int nc_ans_encode(const uint32_t* lo, const uint32_t* hi, int64_t n, int log2_total, uint8_t* out,
                             size_t* inout_nbytes) {
  if ((!lo || !hi) && n > 0) return NC_EINVAL;
  if (!inout_nbytes || n < 0 || log2_total < 1 || log2_total > 31) return NC_EINVAL;
  std::vector<uint8_t> bytes;
  if (!rans_encode(lo, hi, n, log2_total, &bytes)) return NC_EINVAL;
  const size_t need = bytes.size();
  if (!out || *inout_nbytes < need) {
    *inout_nbytes = need;
    return out ? NC_EINVAL : NC_OK;
  }
  std::memcpy(out, bytes.data(), need);
  *inout_nbytes = need;
  return NC_OK;
}

extern "C" int nc_ans_decode(const uint8_t* data, size_t nbytes, const uint32_t* cdfs, int V, int64_t n,
                             int log2_total, int32_t* symbols) {
  if (!data || (n > 0 && (!cdfs || !symbols)) || V < 1 || n < 0 || log2_total < 1 || log2_total > 31)
    return NC_EINVAL;
  const uint64_t T = 1ull << log2_total;
  RansDecoder d(data, nbytes, log2_total);
  if (!d.valid()) return NC_ECORRUPT;
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t* c = cdfs + (size_t)i * (V + 1);
    if (c[0] != 0 || c[V] != T) return NC_ECORRUPT;
    const uint32_t t = d.target();
    int lo = 0, hi = V - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (c[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (c[lo + 1] <= c[lo]) return NC_ECORRUPT;
    symbols[i] = lo;
    d.consume(c[lo], c[lo + 1]);
  }
  return d.finished() ? NC_OK : NC_ECORRUPT;
}

extern "C" int nc_mix_nll_fwd(const float* z, const float* b, const float* p_ng, const float* theta,
                              const int32_t* target, const int32_t* warm, int n, int V, float tau, float* loss,
                              void* stream) {
  if (!z || !b || !p_ng || !theta || !target || !warm || !loss || n < 1 || V < 2 || !(tau > 0.f)) return NC_EINVAL;
  return launch_mix_nll(z, b, p_ng, theta, target, warm, nullptr, n, V, tau, loss, nullptr, nullptr,
                        static_cast<cudaStream_t>(stream)) == cudaSuccess ? NC_OK : NC_ECUDA;
}

extern "C" int nc_mix_nll_bwd(const float* z, const float* b, const float* p_ng, const float* theta,
                              const int32_t* target, const int32_t* warm, const float* gout, int n, int V, float tau,
                              float* db, float* dtheta, void* stream) {
  if (!z || !b || !p_ng || !theta || !target || !warm || n < 1 || V < 2 || !(tau > 0.f)) return NC_EINVAL;
  return launch_mix_nll(z, b, p_ng, theta, target, warm, gout, n, V, tau, nullptr, db, dtheta,
                        static_cast<cudaStream_t>(stream)) == cudaSuccess ? NC_OK : NC_ECUDA;
}
