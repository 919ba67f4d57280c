// Internal declarations shared by the nc24 kernels and the host orchestration.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "nc24.h"

namespace nc {

constexpr int kHeadDim = 64;           // d_head of the supported models (Sec. 3.2)
constexpr int kMaxSlots = 64;          // continuation slots per N-gram context (Sec. 3.4)
constexpr int kMaxOrder = 3;           // N-gram context lengths 1..3
constexpr int kMaxGroup = 4;           // query heads per KV head supported
constexpr int kVocabCluster = 8;       // CTAs per row in the standalone quantiser kernels
constexpr int kVocabThreads = 512;
constexpr float kSkipBits = 1.5f;      // the skip threshold on the N-gram entropy (Sec. 3.7)
constexpr unsigned long long kEmptyKey = ~0ull;

// Status bits a kernel can raise in StreamDev::status (sticky).
enum : int32_t {
  ST_NUMERIC = 1,      // non-finite / out-of-range probability or floor underflow
  ST_TABLE_FULL = 2,   // N-gram tables exhausted (stream longer than expected_len)
  ST_BAD_TOKEN = 4,    // observed token out of range
  ST_TIMEOUT = 8,      // a bounded device wait gave up
};

// One N-gram context: retained continuation slots in arrival / replacement
// order and their count sum n (Sec. 3.4).
struct NgEntry {
  int32_t nslots;
  int32_t n;
  int32_t tok[kMaxSlots];
  int32_t cnt[kMaxSlots];
};

// The N-gram state one prediction reads (Sec. 3.4): per order the context
// entry's slots (ns[k] = 0: no entry) and the closed form's weights
// beta_k / n_k and A / (N + V).  1,584 bytes, a multiple of 16.
struct alignas(16) NgSnap {
  int32_t ns[4];
  float coef[4];
  float cu;
  int32_t pad[3];
  int2 tc[kMaxOrder][kMaxSlots];   // (token, count)
};
static_assert(sizeof(NgSnap) % 16 == 0, "NgSnap is copied in 16-byte pieces");

// Per-stream device state (one per slot).
struct StreamDev {
  int32_t n_coded;          // tokens coded so far; absolute position of the next fed token
  int32_t last_tok;         // token fed at the next step (BOS id 0 first)
  int32_t kv_start;         // absolute position of the oldest cached entry
  int32_t N;                // unigram total
  int32_t hist[3];          // last observed tokens, hist[2] most recent
  int32_t ctx_ent[3];       // entry of the context of order k+1 for the next predict, or -1
  int32_t n_ent[3];         // entries allocated per order
  int32_t max_len;          // tokens this stream may code (sizes the tables)
  int32_t status;           // ST_* bits
  int32_t cap_mask;         // hash index capacity - 1 (power of two)
  float theta[2];           // mixer log-weights (Sec. 3.5)
  float pt_obs, png_obs;    // p_tilde(t*), p_ng(t*) seen by the last update
  unsigned long long* keys[3];
  int32_t* idx[3];
  NgEntry* ent[3];
  float* bias;              // [V] adaptive log-space bias b (Sec. 3.6)
  int32_t* uni;             // [V] unigram counts c(t)
  float* z;                 // [V] logits of the last step
  void* kv;                 // [layers][2][Hkv][L][64], FP32 (FP32 weights) or BF16
};

// RoPE angles: position p = h 2^16 + m 2^8 + l (p < 2^24); rope_tab holds
// (cos, sin) of l w_j, m 2^8 w_j and h 2^16 w_j for the 32 frequencies w_j,
// each computed in FP64 and rounded once; the rotation of p is their product.
constexpr int kRopeLevels = 3;
constexpr int kMaxPosition = 1 << 24;

constexpr int kTmapBytes = 128;             // one CUtensorMap

struct Dims {
  int pdl;                  // launch step kernels with programmatic dependent launch
  const float2* rope_tab;   // [kRopeLevels][256][32]
  int n_layers, d, hq, hkv, F, V, L, C;
  int qkv_rows;             // (hq + 2 hkv) * 64
  float eps, theta, tau;
  int kv_bf16;              // 1: KV cache in BF16
  int attn_cluster;         // CTAs per (stream, KV head) in the FP32-cache attention: 1, 2, 4 or 8; 0 = by batch size
  int n_sm;                 // SMs of the device
  int order;                // N-gram order (0 = off)
  int skip;                 // confidence skip: p = p_ng when H(p_ng) < kSkipBits
  int use_head;
  int warmup;
  int rule;
  int log2T;
  uint32_t floor;
  float alpha, eta;
  // tensor-core attention over a BF16 cache: per (tile, KV head) the chunks'
  // partial results and the ticket that picks the CTA merging them
  const void* kv_tmap;      // [max_streams] TMA maps (kTmapBytes each) of the slots' BF16 KV
                            // rings as 64-wide rows; nullptr: the attention copies rows itself
  void* q16;                // [prefill_rows][hq * 64] BF16 rotated 1/8-scaled queries of a prefill
  float* attn_part;         // attn_part_cap floats
  int32_t* attn_ticket;     // attn_tickets counters, zero between launches
  size_t attn_part_cap;
  int attn_tickets;
};

// Weights of one dense projection in the storage format.
struct Mat {
  const void* w;            // [rows][cols] fp32 / bf16 / e4m3
  const float* scale;       // [rows] per-row scale (FP8) or nullptr
  int rows, cols;
};

struct LayerW {
  Mat qkv, o, gu, down;     // gu rows interleaved: 2j = gate_j, 2j+1 = up_j
  const float* g_attn;
  const float* g_ffn;
};

// Batch description of one step; all pointers are device memory.
struct Batch {
  const int32_t* slots;     // [Bmax] slot of batch row j
  const int32_t* nB;        // active rows (device scalar)
  const int32_t* obs;       // [Bmax] observed token of row j, or nullptr
  StreamDev* st;            // [max_streams]
  int Bmax;
  // Prefill forward (encoder): row j feeds position pos[j] (-1: no position)
  // of stream slots[j] with token tok[j], the KV ring already holds every
  // row's k and v, and the LM head writes row j's logits to z_out + j V.
  // All nullptr in a decode step (position = n_coded, token = last_tok).
  const int32_t* pos;
  const int32_t* tok;
  float* z_out;
  int pm;                   // rows j m .. j m + m - 1 are stream j's consecutive positions
  // Vocabulary pass after a prefill: row j's logits are z_in + z_idx[j] V
  // (nullptr: the stream's own z).  The pass then reads nothing before its
  // wait on the previous kernel.
  const float* z_in;
  const int32_t* z_idx;
};

// (cos, sin) of position a for rotation pair dd from the RoPE table: the
// product of the three table rotations (a split into 8-bit digits), with
// explicit roundings (no multiply-add contraction), so every kernel that
// rotates a position gets the same bits.
__device__ __forceinline__ float2 rope_cs_tab(const float2* tab, int a, int dd) {
  const float2 t1 = tab[(0 * 256 + (a & 255)) * 32 + dd];
  const float2 t2 = tab[(1 * 256 + ((a >> 8) & 255)) * 32 + dd];
  const float2 t3 = tab[(2 * 256 + ((a >> 16) & 255)) * 32 + dd];
  const float c12 = __fsub_rn(__fmul_rn(t1.x, t2.x), __fmul_rn(t1.y, t2.y));
  const float s12 = __fadd_rn(__fmul_rn(t1.x, t2.y), __fmul_rn(t1.y, t2.x));
  return make_float2(__fsub_rn(__fmul_rn(c12, t3.x), __fmul_rn(s12, t3.y)),
                     __fadd_rn(__fmul_rn(c12, t3.y), __fmul_rn(s12, t3.x)));
}
// The rotated pair (x1, x2) -> (x1 c - x2 s, x2 c + x1 s).
__device__ __forceinline__ float2 rope_rotate(float x1, float x2, float2 cs) {
  return make_float2(__fsub_rn(__fmul_rn(x1, cs.x), __fmul_rn(x2, cs.y)),
                     __fadd_rn(__fmul_rn(x2, cs.x), __fmul_rn(x1, cs.y)));
}
// Element offset of plane `which` (K of KV head g: g; V of head g: hkv + g) of
// `layer` in a stream's KV ring [layers][2][hkv][L][64].
__device__ __forceinline__ size_t kv_plane_off(int L, int hkv, int layer, int which) {
  const size_t plane = (size_t)L * kHeadDim;
  return (size_t)layer * 2 * hkv * plane + (size_t)which * plane;
}

// Programmatic dependent launch: a kernel launched with the PDL attribute may
// start while its predecessor still runs.  Each step kernel loads only data
// no in-flight kernel writes (weights, KV entries of earlier tokens, state of
// earlier steps) before pdl_wait(), and signals its own dependents only
// after pdl_wait(); so when a kernel's pdl_wait() returns, every earlier
// kernel of the stream has completed and its writes are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t s, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// The same with a cluster of `cluster_x` CTAs along x chosen at launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel_cluster(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                         cudaStream_t s, bool pdl, int cluster_x, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster_x;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ kernels
enum Prologue { PRO_RMSNORM = 0, PRO_PLAIN = 2 };
enum Epilogue { EPI_STORE = 0, EPI_RESID = 1, EPI_SWIGLU = 2, EPI_LOGITS = 3 };

struct GemvIO {
  const float* x;           // PRO_RMSNORM / PRO_PLAIN input [Bmax][cols]
  const float* g;           // RMSNorm gain (PRO_RMSNORM)
  float* y;                 // EPI_STORE / EPI_SWIGLU output; EPI_RESID residual [Bmax][rows or rows/2]
};

cudaError_t launch_embed(const Dims& D, const Batch& b, const void* E, const float* Escale,
                         int fmt, float* x, cudaStream_t s);
cudaError_t launch_gemv(const Dims& D, const Batch& b, const Mat& m, int fmt, int pro, int epi,
                        const GemvIO& io, cudaStream_t s);
// Decode attention (one cluster per row and KV head) into attn_out
// [Bmax][hq * 64], or (BF16 cache, out16 set) rounded to BF16 into out16.
cudaError_t launch_attn(const Dims& D, const Batch& b, int layer, const float* qkv, float* attn_out,
                        cudaStream_t s, void* out16 = nullptr);

struct VocabIO {
  uint32_t* cdf;            // [Bmax][V+1] or nullptr
  uint32_t* intervals;      // per stream [max_len] x (lo, hi) pairs: base + j * stride, or nullptr
  int64_t interval_stride;  // in uint32 pairs
  float* probe_z;           // optional probes [Bmax][V]
  float* probe_pt;
  float* probe_png;
  float* probe_p;
  int64_t probe_tok;        // 0: probe every step; k > 0: only the stream's k-th token (1-based)
  const int64_t* probe_row; // probe row of batch row j (nullptr: row j)
  int predict;              // quantise (and write cdf / intervals)
  int update;               // apply head + mixer update with b.obs
  int ngram;                // with update: also the N-gram update and the stream's bookkeeping
};
cudaError_t launch_vocab(const Dims& D, const Batch& b, const VocabIO& io, cudaStream_t s);
// The vocabulary passes of a prefill chunk in one launch: stream row j runs
// positions 0 .. m - 1 of the chunk in order while j < nb_step[r], with the
// observed tokens obs_step[r Bmax + j], the logits zrows + (z_idx[j] + r) V
// and (N-gram on) the N-gram state snap[z_idx[j] + r] of each prediction.
cudaError_t launch_vocab_seq(const Dims& D, const Batch& b, const VocabIO& io, int m, const float* zrows,
                             const int32_t* nb_step, const int32_t* obs_step, const NgSnap* snap, cudaStream_t s);
// The N-gram side of the same chunk, ahead of the vocabulary passes (it needs
// only the tokens): for each position of stream row j, in order, the state of
// its prediction into snap[z_idx[j] + r], then the update with the observed
// token (tables, context entries, history, unigram total N).  Leaves the
// unigram counts, the position and the window to the vocabulary passes.
cudaError_t launch_ngram_seq(const Dims& D, const Batch& b, int m, const int32_t* nb_step, const int32_t* obs_step,
                             const int32_t* p0, NgSnap* snap, cudaStream_t s);
cudaError_t launch_prepare_encode(const Batch& b, int n_streams, const int32_t* tok_flat,
                                  const int64_t* offs, const int64_t* lens, int32_t* obs,
                                  int32_t* nB, cudaStream_t s);
// The first position of the next prefill chunk, from a device counter:
// p0s[par] = p0s[2]; p0s[2] += m (so captured chunks replay in order).
cudaError_t launch_chunk_start(int32_t* p0s, int par, int m, cudaStream_t s);
// Encoder prefill of positions p0 .. p0 + m - 1 (p0 = *p0, every live
// stream's position) for n_streams rows: forward row i = j m + r gets the slot of
// stream row j, position p0 + r (or -1 past the stream's end) and its input
// token; *nB_fwd = m x (streams with tokens left).  For the sequential pass
// of position p0 + r: nb_step[r] active rows, observed tokens
// obs_step[r n + j], logits at forward row z_idx[j] + r (z_idx[j] = j m).
cudaError_t launch_prepare_prefill(const Batch& b, int n_streams, int m, int V, const int32_t* p0,
                                   const int32_t* tok_flat, const int64_t* offs, const int64_t* lens,
                                   int32_t* f_slots, int32_t* f_pos, int32_t* f_tok, int32_t* nB_fwd,
                                   int32_t* obs_step, int32_t* nb_step, int32_t* z_idx, cudaStream_t s);
// Attention over a BF16 KV cache on the tcgen05 tensor cores (k_attn_t5.cu):
// decode rows (b.pos null: one row per stream, position n_coded, the fed
// k, v appended by the kernel) or prefill rows (b.pm consecutive positions
// per stream, appended before), into attn_out or, when out16 is set, BF16
// into out16.  A row's result does not depend on the other rows.
// D.attn_part / D.attn_ticket must hold what attn_t5_scratch gives for the
// context's largest batches (tickets zeroed once).
cudaError_t launch_attn_t5(const Dims& D, const Batch& b, int layer, const float* qkv, float* attn_out, void* out16,
                           cudaStream_t s);
void attn_t5_scratch(const Dims& D, int max_streams, int prefill_rows, size_t* part_floats, int* tickets);
// Prefill with a BF16 cache: rotate and append every row's k, v to the ring
// of `layer` and write its rotated, 1/8-scaled BF16 queries to D.q16.
cudaError_t launch_kv_append_t5(const Dims& D, const Batch& b, int layer, const float* qkv, cudaStream_t s);
// Prefill: rotate and append the k, v of every row to the KV ring of `layer`.
cudaError_t launch_kv_append(const Dims& D, const Batch& b, int layer, const float* qkv, cudaStream_t s);
// Decoder: row j's symbol is the s with cdf[s] <= target[j] < cdf[s+1]; writes
// obs[j] = s and lohi[2j..2j+1] = (cdf[s], cdf[s+1]).
cudaError_t launch_search(const Batch& b, int V, const uint32_t* cdf, const uint32_t* target,
                          int32_t* obs, uint32_t* lohi, cudaStream_t s);
cudaError_t launch_convert_weights(const float* src, void* dst, float* scale, int64_t rows,
                                   int64_t cols, int fmt, cudaStream_t s);
cudaError_t launch_interleave_f32(const float* gate, const float* up, float* dst, int64_t rows,
                                  int64_t cols, cudaStream_t s);
// tcgen05 GEMM of one projection: Y[n][m] = sum_k W[m][k] X[n][k] with W the
// weights [M, K] and X the batch operand [Bmax, K] (BF16, or E4M3 with
// per-row scales), FP32 accumulation, fused epilogue.
struct TcGemm {
  const void* tmap_a;       // host copy of the weights' CUtensorMap (box 128 rows)
  const void* tmap_b;       // host copy of the operand's CUtensorMap (box bn rows)
  int M, K, Bmax, bn, kind_bf16;
  int kp;                   // 2: both maps 3D ([K blocks][rows][128 B], tc_encode_tmap3), two K blocks
                            // per stage (BF16, K a multiple of 64); otherwise 2D maps, one per stage
  const int32_t* nB;
  const float* w_scale;     // FP8: [M]
  const float* x_scale;     // FP8: [Bmax]
  float* y;                 // EPI_STORE / EPI_RESID: [Bmax][M]
  float* h_out;             // EPI_SWIGLU: [Bmax][M / 2]
  void* h16;                // EPI_SWIGLU: or, when set, h rounded to BF16 there (the next operand)
  StreamDev* st;            // EPI_LOGITS: each stream's z, or
  float* zrows;             // EPI_LOGITS: [Bmax][M] when set
  const int32_t* slots;
  int32_t* status;          // error word (ST_TIMEOUT)
};
bool tc_encode_tmap(void* tmap, const void* base, int elem_bytes, int64_t inner, int64_t outer, int box_outer);
bool tc_encode_tmap3(void* tmap, const void* base, int elem_bytes, int64_t K, int64_t rows, int box_rows);
cudaError_t launch_gemm_tc(const TcGemm& g, int epi, cudaStream_t s, bool pdl);
// One bounded mbarrier wait on a barrier nothing arrives on (at most `polls`
// polls), recording ST_TIMEOUT in *status when it gives up.
cudaError_t launch_wait_selftest(uint32_t polls, int32_t* status, cudaStream_t s);
cudaError_t launch_chain_link(dim3 grid, dim3 block, cudaStream_t s);
cudaError_t launch_act_rmsnorm(const Dims& D, const Batch& b, const float* x, const float* gain, int cols,
                               int kind_bf16, void* out, float* out_scale, cudaStream_t s);
cudaError_t launch_act_plain(const Dims& D, const Batch& b, const float* x, int cols, int kind_bf16, void* out,
                             float* out_scale, cudaStream_t s);

// Kernel attributes (dynamic shared memory limits) set once, outside any
// stream capture.
cudaError_t prepare_model_kernels(const Dims& D, int fmt);
cudaError_t prepare_vocab_kernels(const Dims& D);
cudaError_t prepare_tc_kernels();

cudaError_t launch_probs_to_cdf(const float* p, int n, int V, int log2T, uint32_t floor,
                                uint32_t* cdf, int32_t* status, cudaStream_t s);
cudaError_t launch_floor_counts(const float* p, int64_t n, uint32_t K, uint32_t floor,
                                uint32_t* c, cudaStream_t s);
cudaError_t launch_mix_nll(const float* z, const float* b, const float* png, const float* theta,
                           const int32_t* target, const int32_t* warm, const float* gout, int n,
                           int V, float tau, float* loss, float* db, float* dtheta,
                           cudaStream_t s);

}  // namespace nc
