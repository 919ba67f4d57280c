// Transformer decode kernels (Sec. 3.2 model, Sec. 3.9 sliding KV window).
//
// One decode step per stream: embedding, per layer RMSNorm -> QKV -> RoPE +
// KV append -> grouped-query attention -> O projection + residual -> RMSNorm
// -> gate/up -> SwiGLU -> down + residual, then the final RMSNorm and the
// tied LM head.  Every reduction has a fixed order that does not depend on
// the batch size, the slot or the grid, so a stream's logits are bit-identical
// whether it runs alone or in a batch.
#include <algorithm>

#include <cooperative_groups.h>

#include "model_dev.cuh"

namespace cg = cooperative_groups;

namespace nc {

namespace {

using namespace dev;

constexpr int kGemvThreads = 128;
constexpr int kGemvWarps = kGemvThreads / 32;

// ----------------------------------------------------------------- embedding
template <int FMT>
__global__ void k_embed(Dims D, Batch b, const void* E, const float* Escale, float* x) {
  const int j = blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (j >= *b.nB) return;
  const int tok = b.tok ? b.tok[j] : b.st[b.slots[j]].last_tok;
  for (int c = threadIdx.x; c < D.d; c += blockDim.x) x[(size_t)j * D.d + c] = embed_at<FMT>(E, Escale, D.d, tok, c);
}

// ---------------------------------------------------------------------- GEMV
// y[j][r] = sum_c W[r][c] * a_j[c] for the active streams j, where a_j is the
// prologue's activation (RMSNorm of the residual, or a plain vector).  Each
// warp owns one row pair (gemv_rowpair).  The activation tile for up to kBT
// streams sits in shared memory; larger batches loop over tiles with the
// warp's weights kept in registers.
template <int FMT, int PRO, int EPI, int HOLD, int BT>
__global__ void __launch_bounds__(kGemvThreads) k_gemv(Dims D, Batch b, Mat m, GemvIO io) {
  extern __shared__ float4 smem4[];
  float* xs = reinterpret_cast<float*>(smem4);   // [kBT][cols]
  __shared__ ProScratch ps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rp = blockIdx.x * kGemvWarps + warp;
  const bool have = 2 * rp < m.rows;
  // Weights do not depend on earlier kernels: fetch this warp's rows before
  // waiting on the predecessor, so the fetch overlaps its execution.
  uint4 h0[HOLD], h1[HOLD];
  if (have) load_rowpair<FMT, HOLD>(m, rp, lane, h0, h1);
  pdl_wait();
  pdl_trigger();
  const int B = *b.nB;
  GemvOut out{io.y, b.st, b.slots, b.z_out};
  const int cols = m.cols;
  auto src = [&](int row, int c) { return __ldcg(io.x + (size_t)row * cols + c); };
  auto sync = [] { __syncthreads(); };
  for (int b0 = 0; b0 < B; b0 += BT) {
    const int nb = min(BT, B - b0);
    prologue<PRO == PRO_RMSNORM>(D, src, io.g, cols, b0, nb, xs, ps, threadIdx.x, kGemvThreads, sync);
    if (have) gemv_rowpair<FMT, EPI, HOLD, BT>(m, rp, xs, b0, nb, h0, h1, lane, out);
    __syncthreads();
  }
}

// ----------------------------------------------------------------- attention
// Merge of a query's nc chunk partials in chunk order into its output dims
// (kDims per head, head h at out + h * 64): M = max of the chunk maxima, then
// sum and accumulator weighted by exp(m_c - M), the factor computed once per
// (head, chunk).  No chunk (a row past a stream's end) writes zeros.
template <typename Sm, int KD>
__device__ void merge_chunks(Sm& sm, const float (*rm)[kMaxGroup], const float (*rl)[kMaxGroup],
                             const float (*racc)[kMaxGroup][KD], int nc, int grp, int tid, float* out) {
  if (tid < grp) {
    const int h = tid;
    float M = -INFINITY;
    for (int c = 0; c < nc; ++c) M = fmaxf(M, rm[c][h]);
    float l = 0.f;
    for (int c = 0; c < nc; ++c) {
      const float f = expf(rm[c][h] - M);
      sm.mf[h][c] = f;
      l = fmaf(rl[c][h], f, l);
    }
    sm.mL[h] = l;
  }
  __syncthreads();
  for (int e = tid; e < grp * KD; e += kAttnThreads) {
    const int h = e / KD, dl = e % KD;
    float o = 0.f;
    for (int c = 0; c < nc; ++c) o = fmaf(racc[c][h][dl], sm.mf[h][c], o);
    out[h * kHeadDim + dl] = nc ? o / sm.mL[h] : 0.f;
  }
  __syncthreads();
}

// One cluster of S CTAs per (stream row, KV head).  CTA `rank` owns chunks
// rank, rank + S, ...; the loads of its first chunk do not depend on the
// QKV projection and are issued before waiting on it.  The owner of a chunk
// stores its (max, sum) and each CTA's 64 / S accumulator dims into that
// CTA's shared memory; after one cluster barrier every CTA merges its dims
// over all chunks in chunk order from local shared memory.
template <int KBF16, int S>
__global__ void __launch_bounds__(kAttnThreads) k_attn(Dims D, Batch b, int layer, AttnIO io) {
  const int rank = S > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int j = blockIdx.z, g = blockIdx.y;
  if (j >= *b.nB) return;                          // uniform across the cluster
  StreamDev& st = b.st[b.slots[j]];
  const int a = b.pos ? b.pos[j] : st.n_coded;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = D.hq / D.hkv;
  if (a < 0) {                                     // prefill row past the stream's end
    pdl_wait();
    pdl_trigger();
    for (int e = tid; e < grp * kHeadDim / S; e += kAttnThreads)
      io.attn_out[(size_t)j * D.hq * kHeadDim + (g * grp + e / (kHeadDim / S)) * kHeadDim +
                  rank * (kHeadDim / S) + e % (kHeadDim / S)] = 0.f;
    return;                                        // uniform across the cluster
  }
  const int start = b.pos ? window_start_at(D, a) : window_start(D, st);
  const int nc = (a - start) / kAttnChunk + 1;     // the last chunk holds position a
  __shared__ AttnSmem<S> sm;
  // every CTA of the cluster must have started before shared memory is
  // written remotely: arrive now, wait before the first remote store
  if (S > 1) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  AttnPre<KBF16> pre;
  attn_rope(D, a, tid, sm);
  // a prefill's ring entries of this chunk of positions were written by the
  // append pass just before: wait for it before loading any of them
  if (b.pos) pdl_wait();
  if (rank < nc) {
    const int c_lo = start + rank * kAttnChunk;
    attn_load<KBF16>(D, st, layer, g, c_lo + warp * 32, min(c_lo + kAttnChunk, a + 1), a, lane, pre);
  }
  pdl_wait();
  pdl_trigger();
  // a prefill appended every row's k, v before this launch
  attn_qkv<KBF16>(D, st, layer, j, g, a, !b.pos && (nc - 1) % S == rank, tid, sm, io);
  auto dst = [&](int r) -> AttnSmem<S>* {
    if (S == 1) return &sm;
    return cg::this_cluster().map_shared_rank(&sm, r);
  };
  if (S > 1) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
  for (int c = rank; c < nc; c += S) {
    const int c_lo = start + c * kAttnChunk;
    const int c_end = min(c_lo + kAttnChunk, a + 1);
    if (c != rank) attn_load<KBF16>(D, st, layer, g, c_lo + warp * 32, c_end, a, lane, pre);
    attn_chunk<KBF16>(D, c_lo, c_end, a, tid, sm, sm, pre, [&](int h, int dd, float o, float M, float l) {
      constexpr int kDims = AttnSmem<S>::kDims;
      AttnSmem<S>* r = dst(dd / kDims);
      r->racc[c][h][dd % kDims] = o;
      if (dd % kDims == 0) {
        r->rm[c][h] = M;
        r->rl[c][h] = l;
      }
    });
  }
  if (S > 1) cg::this_cluster().sync();            // every chunk's partial has arrived
  constexpr int kDims = AttnSmem<S>::kDims;
  merge_chunks(sm, sm.rm, sm.rl, sm.racc, nc, grp, tid,
               io.attn_out + (size_t)j * D.hq * kHeadDim + g * grp * kHeadDim + rank * kDims);
}

// ------------------------------------------------------ prefill attention
// Query side of one prefill row: its rotation, rotated and scaled query
// heads, and the fed token's k and v.
struct RowQ {
  float qs[kMaxGroup][kHeadDim];
  float kn[kHeadDim], vn[kHeadDim];
  float cs[kHeadDim / 2], sn[kHeadDim / 2];
};

constexpr int kRowsMax = 8;                         // query rows per CTA
constexpr int kRowQFloats = sizeof(RowQ) / sizeof(float);

// Shared-memory layout of the multi-row attention, in floats, for rq rows,
// grp query heads per KV head and kd merged dims per CTA.
struct RowsLayout {
  int q, we, wm, wl, wacc, cf, cM, cL, rm, rl, racc, mf, mL, total;
  __host__ __device__ RowsLayout(int rq, int grp, int kd) {
    int o = 0;
    q = o;    o += rq * kRowQFloats;
    we = o;   o += kAttnWarps * grp * 32;
    wm = o;   o += rq * kAttnWarps * grp;
    wl = o;   o += rq * kAttnWarps * grp;
    wacc = o; o += rq * kAttnWarps * grp * kHeadDim;
    cf = o;   o += rq * grp * kAttnWarps;
    cM = o;   o += rq * grp;
    cL = o;   o += rq * grp;
    rm = o;   o += rq * kAttnMaxChunks * grp;
    rl = o;   o += rq * kAttnMaxChunks * grp;
    racc = o; o += rq * kAttnMaxChunks * grp * kd;
    mf = o;   o += grp * kAttnMaxChunks;
    mL = o;   o += grp;
    total = (o + 3) & ~3;
  }
};

// Prefill attention of rq consecutive rows of one stream (consecutive
// positions, one window start) and one KV head.  Per chunk, each warp loads
// the keys and values of its 32 positions once and computes every row's
// block (attn_block, as the decode attention does); then the blocks of all
// rows are combined in block order.  Chunks are split over a cluster of S
// CTAs and merged per row in chunk order, so every row's output equals the
// decode attention's bit for bit.
template <int KBF16, int S>
__global__ void __launch_bounds__(kAttnThreads, 2) k_attn_rows(Dims D, Batch b, int layer, int rq, AttnIO io) {
  extern __shared__ float4 dyn4[];
  float* sm = reinterpret_cast<float*>(dyn4);
  const int rank = S > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int g = blockIdx.y, i0 = blockIdx.z * rq;
  if (i0 >= *b.nB) return;                         // uniform across the cluster
  if (S > 1) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = D.hq / D.hkv;
  constexpr int kd = kHeadDim / S;
  const RowsLayout L(rq, grp, kd);
  RowQ* qv = reinterpret_cast<RowQ*>(sm + L.q);
  StreamDev& st = b.st[b.slots[i0]];
  int a_max = -1;
  for (int r = 0; r < rq; ++r) a_max = max(a_max, b.pos[i0 + r]);
  pdl_wait();                                      // the append pass wrote this chunk of positions
  pdl_trigger();
  const int start = window_start_at(D, max(a_max, 0));
  const int nc_max = a_max < 0 ? 0 : (a_max - start) / kAttnChunk + 1;
  for (int r = 0; r < rq; ++r) {
    const int a = b.pos[i0 + r];
    if (a < 0) continue;                           // uniform across the CTA
    attn_rope(D, a, tid, qv[r]);
    attn_qkv<KBF16>(D, st, layer, i0 + r, g, a, false, tid, qv[r], io);
  }
  auto dst = [&](int rk) -> float* {
    if (S == 1) return sm;
    return cg::this_cluster().map_shared_rank(sm, rk);
  };
  // chunk c of row r exists when position start + 256 c <= a_r
  auto has = [&](int r, int c) {
    const int a = b.pos[i0 + r];
    return a >= 0 && c <= (a - start) / kAttnChunk;
  };
  if (S > 1) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
  for (int c = rank; c < nc_max; c += S) {
    const int c_lo = start + c * kAttnChunk;
    AttnPre<KBF16> pre;
    attn_load<KBF16>(D, st, layer, g, c_lo + warp * 32, min(c_lo + kAttnChunk, a_max + 1), a_max + 1, lane, pre);
    // every row's block of this warp
    for (int r = 0; r < rq; ++r) {
      if (!has(r, c)) continue;                    // uniform across the CTA
      const int a = b.pos[i0 + r];
      float mh[kMaxGroup], lh[kMaxGroup], acc[kMaxGroup][2];
      const int nvalid = attn_block<KBF16>(D, c_lo + warp * 32, min(c_lo + kAttnChunk, a + 1), a, lane, qv[r],
                                           sm + L.we + warp * grp * 32, pre, mh, lh, acc);
      float* wacc = sm + L.wacc + ((r * kAttnWarps + warp) * grp) * kHeadDim;
#pragma unroll
      for (int h = 0; h < kMaxGroup; ++h) {
        if (h < grp) {
          if (lane == 0) {
            sm[L.wm + (r * kAttnWarps + warp) * grp + h] = nvalid > 0 ? mh[h] : -INFINITY;
            sm[L.wl + (r * kAttnWarps + warp) * grp + h] = nvalid > 0 ? lh[h] : 0.f;
          }
          wacc[h * kHeadDim + 2 * lane] = acc[h][0];
          wacc[h * kHeadDim + 2 * lane + 1] = acc[h][1];
        }
      }
    }
    __syncthreads();
    // per (row, head): the block factors exp(m_w - M), M and the sum
    for (int t = tid; t < rq * grp; t += kAttnThreads) {
      const int r = t / grp, h = t % grp;
      if (!has(r, c)) continue;
      const int a = b.pos[i0 + r];
      const int nblk = (min(c_lo + kAttnChunk, a + 1) - c_lo + 31) / 32;
      const float* wm = sm + L.wm + r * kAttnWarps * grp;
      const float* wl = sm + L.wl + r * kAttnWarps * grp;
      float M = -INFINITY;
      for (int w = 0; w < nblk; ++w) M = fmaxf(M, wm[w * grp + h]);
      float l = 0.f;
      for (int w = 0; w < nblk; ++w) {
        const float f = expf(wm[w * grp + h] - M);
        sm[L.cf + t * kAttnWarps + w] = f;
        l = fmaf(wl[w * grp + h], f, l);
      }
      sm[L.cM + t] = M;
      sm[L.cL + t] = l;
    }
    __syncthreads();
    // per (row, head, dim): the chunk accumulator, stored with the chunk's
    // (M, l) into the shared memory of the CTA merging that dim
    for (int e = tid; e < rq * grp * kHeadDim; e += kAttnThreads) {
      const int t = e / kHeadDim, dd = e % kHeadDim, r = t / grp, h = t % grp;
      if (!has(r, c)) continue;
      const int a = b.pos[i0 + r];
      const int nblk = (min(c_lo + kAttnChunk, a + 1) - c_lo + 31) / 32;
      float o = 0.f;
      for (int w = 0; w < nblk; ++w)
        o = fmaf(sm[L.wacc + ((r * kAttnWarps + w) * grp + h) * kHeadDim + dd], sm[L.cf + t * kAttnWarps + w], o);
      float* tgt = dst(dd / kd);
      const int rc = (r * kAttnMaxChunks + c) * grp + h;
      tgt[L.racc + rc * kd + dd % kd] = o;
      if (dd % kd == 0) {
        tgt[L.rm + rc] = sm[L.cM + t];
        tgt[L.rl + rc] = sm[L.cL + t];
      }
    }
    __syncthreads();
  }
  if (S > 1) cg::this_cluster().sync();            // every chunk's partial has arrived
  else __syncthreads();
  // per row: merge its chunks in chunk order
  for (int r = 0; r < rq; ++r) {
    const int a = b.pos[i0 + r];
    const int nc = a < 0 ? 0 : (a - start) / kAttnChunk + 1;
    if (tid < grp) {
      const int h = tid;
      float M = -INFINITY;
      for (int c = 0; c < nc; ++c) M = fmaxf(M, sm[L.rm + (r * kAttnMaxChunks + c) * grp + h]);
      float l = 0.f;
      for (int c = 0; c < nc; ++c) {
        const int rc = (r * kAttnMaxChunks + c) * grp + h;
        const float f = expf(sm[L.rm + rc] - M);
        sm[L.mf + h * kAttnMaxChunks + c] = f;
        l = fmaf(sm[L.rl + rc], f, l);
      }
      sm[L.mL + h] = l;
    }
    __syncthreads();
    float* out = io.attn_out + (size_t)(i0 + r) * D.hq * kHeadDim + g * grp * kHeadDim + rank * kd;
    for (int e = tid; e < grp * kd; e += kAttnThreads) {
      const int h = e / kd, dl = e % kd;
      float o = 0.f;
      for (int c = 0; c < nc; ++c)
        o = fmaf(sm[L.racc + ((r * kAttnMaxChunks + c) * grp + h) * kd + dl], sm[L.mf + h * kAttnMaxChunks + c], o);
      out[h * kHeadDim + dl] = nc ? o / sm[L.mL + h] : 0.f;
    }
    __syncthreads();
  }
}

// Prefill: the k, v of row j (position pos[j]) rotated exactly as the decode
// attention rotates the fed token's, appended to the ring of `layer`.
struct AppendSmem {
  float qs[kMaxGroup][kHeadDim];
  float kn[kHeadDim], vn[kHeadDim];
  float cs[kHeadDim / 2], sn[kHeadDim / 2];
};

template <int KBF16>
__global__ void __launch_bounds__(kAttnThreads) k_kv_append(Dims D, Batch b, int layer, AttnIO io) {
  const int j = blockIdx.y, g = blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (j >= *b.nB) return;
  const int a = b.pos[j];
  if (a < 0) return;
  StreamDev& st = b.st[b.slots[j]];
  __shared__ AppendSmem sm;
  attn_rope(D, a, threadIdx.x, sm);
  attn_qkv<KBF16>(D, st, layer, j, g, a, true, threadIdx.x, sm, io);
}

// ------------------------------------------------------------ weight formats
// One block per row.  BF16: round to nearest even.  FP8: scale = amax / 448
// (IEEE binary32 division), q = e4m3(w / scale) rounded to nearest even,
// saturating; an all-zero row uses scale 1.
__global__ void k_convert(const float* src, void* dst, float* scale, int64_t cols, int fmt) {
  const int64_t r = blockIdx.x;
  const float* s = src + r * cols;
  if (fmt == NC_FP32) {
    float* d = static_cast<float*>(dst) + r * cols;
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) d[c] = s[c];
  } else if (fmt == NC_BF16) {
    __nv_bfloat16* d = static_cast<__nv_bfloat16*>(dst) + r * cols;
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) d[c] = __float2bfloat16_rn(s[c]);
  } else {
    __shared__ float red[32];
    __shared__ float sc;
    float m = 0.f;
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) m = fmaxf(m, fabsf(s[c]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float mm = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
      sc = mm > 0.f ? __fdiv_rn(mm, 448.0f) : 1.0f;
      scale[r] = sc;
    }
    __syncthreads();
    __nv_fp8_storage_t* d = static_cast<__nv_fp8_storage_t*>(dst) + r * cols;
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x)
      d[c] = __nv_cvt_float_to_fp8(__fdiv_rn(s[c], sc), __NV_SATFINITE, __NV_E4M3);
  }
}

__global__ void k_interleave(const float* gate, const float* up, float* dst, int64_t rows,
                             int64_t cols) {
  const int64_t r = blockIdx.x;
  const float* s = (r & 1) ? up + (r >> 1) * cols : gate + (r >> 1) * cols;
  for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) dst[r * cols + c] = s[c];
}

}  // namespace


// One link of an empty chain of dependent launches: it waits for its
// predecessor and lets its successor launch, as the decode step's kernels do
// around their work.
__global__ void k_chain_link() {
  pdl_wait();
  pdl_trigger();
}

cudaError_t launch_chain_link(dim3 grid, dim3 block, cudaStream_t s) {
  return launch_kernel(k_chain_link, grid, block, 0, s, true);
}

cudaError_t launch_embed(const Dims& D, const Batch& b, const void* E, const float* Escale,
                         int fmt, float* x, cudaStream_t s) {
  const int thr = 256;
  auto kern = fmt == NC_FP32 ? k_embed<NC_FP32> : fmt == NC_BF16 ? k_embed<NC_BF16> : k_embed<NC_FP8E4M3>;
  return launch_kernel(kern, dim3(b.Bmax), dim3(thr), 0, s, D.pdl, D, b, E, Escale, x);
}

template <int FMT, int PRO, int EPI>
static cudaError_t gemv_t(const Dims& D, const Batch& b, const Mat& m, const GemvIO& io,
                          cudaStream_t s) {
  const int rows_per_block = kGemvWarps * 2;
  const int grid = (m.rows + rows_per_block - 1) / rows_per_block;
  const size_t smem = (size_t)kBT * m.cols * sizeof(float);
  // rows of at most 96 vectors (3 per lane) hold them all with 3 registers
  // quads; longer rows hold 8 and stream the rest
  // a context of one stream uses the one-stream tile (fewer registers)
  const bool short_row = m.cols / WFmt<FMT>::VW <= 96;
  if (b.Bmax == 1)
    return short_row
               ? launch_kernel(k_gemv<FMT, PRO, EPI, 3, 1>, dim3(grid), dim3(kGemvThreads), smem, s, D.pdl, D, b, m, io)
               : launch_kernel(k_gemv<FMT, PRO, EPI, 8, 1>, dim3(grid), dim3(kGemvThreads), smem, s, D.pdl, D, b, m, io);
  return short_row
             ? launch_kernel(k_gemv<FMT, PRO, EPI, 3, kBT>, dim3(grid), dim3(kGemvThreads), smem, s, D.pdl, D, b, m, io)
             : launch_kernel(k_gemv<FMT, PRO, EPI, 8, kBT>, dim3(grid), dim3(kGemvThreads), smem, s, D.pdl, D, b, m, io);
}

template <int FMT>
static cudaError_t gemv_f(const Dims& D, const Batch& b, const Mat& m, int pro, int epi,
                          const GemvIO& io, cudaStream_t s) {
  if (pro == PRO_RMSNORM && epi == EPI_STORE) return gemv_t<FMT, PRO_RMSNORM, EPI_STORE>(D, b, m, io, s);
  if (pro == PRO_RMSNORM && epi == EPI_SWIGLU) return gemv_t<FMT, PRO_RMSNORM, EPI_SWIGLU>(D, b, m, io, s);
  if (pro == PRO_PLAIN && epi == EPI_RESID) return gemv_t<FMT, PRO_PLAIN, EPI_RESID>(D, b, m, io, s);
  if (pro == PRO_RMSNORM && epi == EPI_LOGITS) return gemv_t<FMT, PRO_RMSNORM, EPI_LOGITS>(D, b, m, io, s);
  return cudaErrorInvalidValue;
}

// The dynamic shared-memory cap is a per-kernel global: set it to the
// largest activation tile any supported model needs (kBT rows of the widest
// projection input, 4,096 columns), not to the current model's, so that
// contexts of different shapes can coexist.
constexpr int kMaxGemvCols = 4096;

template <int FMT>
static cudaError_t prepare_gemv_f(int cmax) {
  const int smem = kBT * (cmax > kMaxGemvCols ? cmax : kMaxGemvCols) * (int)sizeof(float);
  cudaError_t e = cudaSuccess;
  auto set = [&](auto kern) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  };
  set(k_gemv<FMT, PRO_RMSNORM, EPI_STORE, 3, 1>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_SWIGLU, 3, 1>);
  set(k_gemv<FMT, PRO_PLAIN, EPI_RESID, 3, 1>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_LOGITS, 3, 1>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_STORE, 8, 1>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_SWIGLU, 8, 1>);
  set(k_gemv<FMT, PRO_PLAIN, EPI_RESID, 8, 1>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_LOGITS, 8, 1>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_STORE, 3, kBT>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_SWIGLU, 3, kBT>);
  set(k_gemv<FMT, PRO_PLAIN, EPI_RESID, 3, kBT>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_LOGITS, 3, kBT>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_STORE, 8, kBT>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_SWIGLU, 8, kBT>);
  set(k_gemv<FMT, PRO_PLAIN, EPI_RESID, 8, kBT>);
  set(k_gemv<FMT, PRO_RMSNORM, EPI_LOGITS, 8, kBT>);
  return e;
}

static size_t rows_smem(int rq, int grp, int S) { return (size_t)RowsLayout(rq, grp, kHeadDim / S).total * 4; }

template <int S>
static cudaError_t prepare_rows_s(int grp) {
  const int bytes = (int)rows_smem(kRowsMax, grp, S);
  cudaError_t e = cudaFuncSetAttribute(k_attn_rows<1, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_attn_rows<0, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t prepare_model_kernels(const Dims& D, int fmt) {
  const int cmax = std::max(std::max(D.d, D.hq * kHeadDim), D.F);
  cudaError_t e = fmt == NC_FP32 ? prepare_gemv_f<NC_FP32>(cmax)
                  : fmt == NC_BF16 ? prepare_gemv_f<NC_BF16>(cmax)
                                   : prepare_gemv_f<NC_FP8E4M3>(cmax);
  const int grp = D.hq / D.hkv;
  if (e == cudaSuccess) e = prepare_rows_s<1>(grp);
  if (e == cudaSuccess) e = prepare_rows_s<2>(grp);
  if (e == cudaSuccess) e = prepare_rows_s<4>(grp);
  if (e == cudaSuccess) e = prepare_rows_s<8>(grp);
  return e;
}

cudaError_t launch_gemv(const Dims& D, const Batch& b, const Mat& m, int fmt, int pro, int epi,
                        const GemvIO& io, cudaStream_t s) {
  if (fmt == NC_FP32) return gemv_f<NC_FP32>(D, b, m, pro, epi, io, s);
  if (fmt == NC_BF16) return gemv_f<NC_BF16>(D, b, m, pro, epi, io, s);
  return gemv_f<NC_FP8E4M3>(D, b, m, pro, epi, io, s);
}

// CTAs per (row, KV head): the largest of 8, 4, 2, 1 that keeps the launch
// within about two waves of two CTAs per SM.  Results do not depend on it.
static int attn_split(const Dims& D, const Batch& b) {
  if (D.attn_cluster) return D.attn_cluster;
  int S = 8;
  while (S > 1 && (int64_t)D.hkv * b.Bmax * S > 4 * (int64_t)D.n_sm) S /= 2;
  return S;
}

template <int S>
static cudaError_t launch_attn_rows_s(const Dims& D, const Batch& b, int layer, int rq, const AttnIO& io,
                                      cudaStream_t s) {
  dim3 grid(S, D.hkv, b.Bmax / rq);
  return launch_kernel_cluster(D.kv_bf16 ? k_attn_rows<1, S> : k_attn_rows<0, S>, grid, dim3(kAttnThreads),
                               rows_smem(rq, D.hq / D.hkv, S), s, D.pdl, S, D, b, layer, rq, io);
}

// Prefill rows (b.pm consecutive positions per stream): rq rows per CTA
// group, S CTAs per group as for decode.
static cudaError_t launch_attn_rows(const Dims& D, const Batch& b, int layer, const AttnIO& io, cudaStream_t s) {
  int rq = std::min(kRowsMax, b.pm);
  int S = 8;
  if (D.attn_cluster) S = D.attn_cluster;
  else
    while (S > 1 && (int64_t)D.hkv * (b.Bmax / rq) * S > 4 * (int64_t)D.n_sm) S /= 2;
  // one CTA owning every chunk keeps all chunk partials: 4 rows keep two
  // CTAs per SM within shared memory
  if (S == 1) rq = std::min(rq, 4);
  switch (S) {
    case 1: return launch_attn_rows_s<1>(D, b, layer, rq, io, s);
    case 2: return launch_attn_rows_s<2>(D, b, layer, rq, io, s);
    case 4: return launch_attn_rows_s<4>(D, b, layer, rq, io, s);
    case 8: return launch_attn_rows_s<8>(D, b, layer, rq, io, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_attn(const Dims& D, const Batch& b, int layer, const float* qkv, float* attn_out,
                        cudaStream_t s, void* out16) {
  if (D.kv_bf16) return launch_attn_t5(D, b, layer, qkv, attn_out, out16, s);
  if (b.pos && b.pm >= 2 && b.pm % 2 == 0 && b.Bmax % std::min(kRowsMax, b.pm) == 0)
    return launch_attn_rows(D, b, layer, AttnIO{qkv, attn_out}, s);
  const int S = attn_split(D, b);
  dim3 grid(S, D.hkv, b.Bmax);
  AttnIO io{qkv, attn_out};
  auto pick = [&](auto k1, auto k0) { return D.kv_bf16 ? k1 : k0; };
  switch (S) {
    case 1: return launch_kernel_cluster(pick(k_attn<1, 1>, k_attn<0, 1>), grid, dim3(kAttnThreads), 0, s, D.pdl, 1, D, b, layer, io);
    case 2: return launch_kernel_cluster(pick(k_attn<1, 2>, k_attn<0, 2>), grid, dim3(kAttnThreads), 0, s, D.pdl, 2, D, b, layer, io);
    case 4: return launch_kernel_cluster(pick(k_attn<1, 4>, k_attn<0, 4>), grid, dim3(kAttnThreads), 0, s, D.pdl, 4, D, b, layer, io);
    case 8: return launch_kernel_cluster(pick(k_attn<1, 8>, k_attn<0, 8>), grid, dim3(kAttnThreads), 0, s, D.pdl, 8, D, b, layer, io);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_kv_append(const Dims& D, const Batch& b, int layer, const float* qkv, cudaStream_t s) {
  if (D.kv_bf16) return launch_kv_append_t5(D, b, layer, qkv, s);
  AttnIO io{qkv, nullptr};
  return launch_kernel(D.kv_bf16 ? k_kv_append<1> : k_kv_append<0>, dim3(D.hkv, b.Bmax), dim3(kAttnThreads), 0, s,
                       D.pdl, D, b, layer, io);
}

cudaError_t launch_convert_weights(const float* src, void* dst, float* scale, int64_t rows,
                                   int64_t cols, int fmt, cudaStream_t s) {
  k_convert<<<(unsigned)rows, 256, 0, s>>>(src, dst, scale, cols, fmt);
  return cudaGetLastError();
}

cudaError_t launch_interleave_f32(const float* gate, const float* up, float* dst, int64_t rows,
                                  int64_t cols, cudaStream_t s) {
  k_interleave<<<(unsigned)(2 * rows), 256, 0, s>>>(gate, up, dst, 2 * rows, cols);
  return cudaGetLastError();
}

}  // namespace nc
