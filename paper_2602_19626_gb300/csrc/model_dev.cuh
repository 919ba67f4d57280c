// Device building blocks of the decode step, shared by the model kernels
// (k_model.cu) and the tensor-core attention (k_attn_t5.cu), so that every
// kernel computing a value uses the same operations in the same order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"

namespace nc {
namespace dev {

constexpr int kRed = 256;          // threads of the fixed-order RMSNorm reduction
constexpr int kBT = 8;             // streams per activation tile in shared memory
constexpr int kHold = 8;           // 16-byte weight vectors per row held in registers
constexpr int kLoadBatch = 4;      // further vectors per row in flight per lane

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

template <int FMT>
struct WFmt;
template <>
struct WFmt<NC_FP32> {
  static constexpr int VW = 4;
  static constexpr int ESZ = 4;
  __device__ static void deq(const uint4& u, float* f) {
    f[0] = __uint_as_float(u.x);
    f[1] = __uint_as_float(u.y);
    f[2] = __uint_as_float(u.z);
    f[3] = __uint_as_float(u.w);
  }
};
template <>
struct WFmt<NC_BF16> {
  static constexpr int VW = 8;
  static constexpr int ESZ = 2;
  __device__ static void deq(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};
template <>
struct WFmt<NC_FP8E4M3> {
  static constexpr int VW = 16;
  static constexpr int ESZ = 1;
  __device__ static void deq(const uint4& u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFF), __NV_E4M3);
      __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3);
      float2 a = __half22float2(*reinterpret_cast<__half2*>(&lo));
      float2 b = __half22float2(*reinterpret_cast<__half2*>(&hi));
      f[4 * i] = a.x;
      f[4 * i + 1] = a.y;
      f[4 * i + 2] = b.x;
      f[4 * i + 3] = b.y;
    }
  }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Window bookkeeping shared by every kernel of a step: the fed token sits at
// absolute position a = n_coded; a full window (L entries) first drops its
// oldest C entries (Sec. 3.9).  Returns the first cached position.
__device__ __forceinline__ int window_start(const Dims& D, const StreamDev& st) {
  int start = st.kv_start;
  if (st.n_coded - start == D.L) start += D.C;
  return start;
}

// The same window start as a function of the fed position a alone: the
// cache first fills at a = L, then every C positions drops the oldest C.
__device__ __forceinline__ int window_start_at(const Dims& D, int a) {
  return a < D.L ? 0 : ((a - D.L) / D.C + 1) * D.C;
}

__device__ __forceinline__ float silu(float a) { return a / (1.0f + expf(-a)); }

// Embedding value of token `tok`, column c, in the storage format.
template <int FMT>
__device__ __forceinline__ float embed_at(const void* E, const float* Escale, int d, int tok, int c) {
  if (FMT == NC_FP32) return static_cast<const float*>(E)[(size_t)tok * d + c];
  if (FMT == NC_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(E)[(size_t)tok * d + c]);
  __nv_fp8_e4m3 q;
  q.__x = static_cast<const __nv_fp8_storage_t*>(E)[(size_t)tok * d + c];
  return float(q) * Escale[tok];
}

// Shared-memory scratch of a GEMV prologue.
struct ProScratch {
  float red[kRed / 32][kBT];
  float inv[kBT];
};

// Prologue of a GEMV tile: xs[bt][c] = activation of stream b0 + bt, column c.
// RMSNorm sums x^2 over columns c = t, t + 256, ... per virtual thread t,
// then lanes by a fixed xor tree, then the 8 warps in order, whatever the
// block size.  `src` gives the raw value of (row, column); loads that read
// data written by other blocks of the same launch must bypass L1 (the
// callers pass __ldcg-based sources).  `sync` synchronises the block.
template <bool RMS, typename Src, typename Sync>
__device__ void prologue(const Dims& D, Src src, const float* gain, int cols, int b0, int nb, float* xs,
                         ProScratch& ps, int tid, int nthreads, Sync sync) {
  if (RMS) {
    // virtual thread vt (0..255) sums columns vt, vt + 256, ...; a block of
    // fewer threads runs several virtual threads per thread (nthreads is a
    // multiple of 32, so a real warp always holds one virtual warp)
    for (int vt = tid; vt < kRed; vt += nthreads) {
      const int lane = vt & 31, w = vt >> 5;
      for (int bt = 0; bt < nb; ++bt) {
        float ss = 0.f;
        for (int c = vt; c < cols; c += kRed) {
          const float v = src(b0 + bt, c);
          ss = fmaf(v, v, ss);
        }
        ss = warp_sum(ss);
        if (lane == 0) ps.red[w][bt] = ss;
      }
    }
    sync();
    if (tid < nb) {
      float ss = 0.f;
      for (int w = 0; w < kRed / 32; ++w) ss += ps.red[w][tid];
      ps.inv[tid] = 1.0f / sqrtf(ss / (float)cols + D.eps);
    }
    sync();
    for (int bt = 0; bt < nb; ++bt)
      for (int c = tid; c < cols; c += nthreads) xs[bt * cols + c] = src(b0 + bt, c) * ps.inv[bt] * gain[c];
  } else {
    for (int bt = 0; bt < nb; ++bt)
      for (int c = tid; c < cols; c += nthreads) xs[bt * cols + c] = src(b0 + bt, c);
  }
  sync();
}

// Rows of row pair rp (odd row counts duplicate the last row, which is not
// written back).
__device__ __forceinline__ void rowpair_rows(const Mat& m, int rp, int& r0, int& r1, bool& has1) {
  r0 = 2 * rp;
  has1 = r0 + 1 < m.rows;
  r1 = has1 ? r0 + 1 : r0;
}

template <int FMT, int HOLD = kHold>
__device__ __forceinline__ void load_rowpair(const Mat& m, int rp, int lane, uint4 (&h0)[HOLD],
                                             uint4 (&h1)[HOLD]) {
  using W = WFmt<FMT>;
  int r0, r1;
  bool has1;
  rowpair_rows(m, rp, r0, r1, has1);
  const int nvec = m.cols / W::VW;
  const uint4* w0 = reinterpret_cast<const uint4*>(static_cast<const char*>(m.w) + (size_t)r0 * m.cols * W::ESZ);
  const uint4* w1 = reinterpret_cast<const uint4*>(static_cast<const char*>(m.w) + (size_t)r1 * m.cols * W::ESZ);
#pragma unroll
  for (int k = 0; k < HOLD; ++k) {
    const int v = lane + 32 * k;
    if (v < nvec) {
      h0[k] = ld_stream(w0 + v);
      h1[k] = ld_stream(w1 + v);
    }
  }
}

// Where a GEMV writes: EPI_STORE / EPI_RESID into y [B][rows], EPI_SWIGLU
// into y [B][rows / 2], EPI_LOGITS into each stream's logits.
struct GemvOut {
  float* y;
  StreamDev* st;
  const int32_t* slots;
  float* zrows;             // EPI_LOGITS into [B][rows] instead of each stream's z
};

// One row pair for streams b0 .. b0 + nb - 1: lane l accumulates the weight
// vectors l, l + 32, ... of both rows in increasing order (the held ones, then
// the rest of a long row), a fixed xor tree sums the lanes, lane bt writes
// stream b0 + bt.
template <int FMT, int EPI, int HOLD = kHold, int BT = kBT>
__device__ __forceinline__ void gemv_rowpair(const Mat& m, int rp, const float* xs, int b0, int nb,
                                             const uint4 (&h0)[HOLD], const uint4 (&h1)[HOLD], int lane,
                                             const GemvOut& out) {
  using W = WFmt<FMT>;
  constexpr int VW = W::VW;
  int r0, r1;
  bool has1;
  rowpair_rows(m, rp, r0, r1, has1);
  const int cols = m.cols;
  const int nvec = cols / VW;
  const uint4* w0 = reinterpret_cast<const uint4*>(static_cast<const char*>(m.w) + (size_t)r0 * cols * W::ESZ);
  const uint4* w1 = reinterpret_cast<const uint4*>(static_cast<const char*>(m.w) + (size_t)r1 * cols * W::ESZ);
  float acc0[BT], acc1[BT];
#pragma unroll
  for (int bt = 0; bt < BT; ++bt) acc0[bt] = acc1[bt] = 0.f;
  auto fma_vec = [&](const uint4& a0, const uint4& a1, int v) {
    float f0[VW], f1[VW];
    W::deq(a0, f0);
    W::deq(a1, f1);
#pragma unroll
    for (int bt = 0; bt < BT; ++bt) {
      if (bt < nb) {
        const float4* xr = reinterpret_cast<const float4*>(xs + bt * cols + v * VW);
#pragma unroll
        for (int q = 0; q < VW / 4; ++q) {
          const float4 xv = xr[q];
          acc0[bt] = fmaf(f0[4 * q + 0], xv.x, acc0[bt]);
          acc0[bt] = fmaf(f0[4 * q + 1], xv.y, acc0[bt]);
          acc0[bt] = fmaf(f0[4 * q + 2], xv.z, acc0[bt]);
          acc0[bt] = fmaf(f0[4 * q + 3], xv.w, acc0[bt]);
          acc1[bt] = fmaf(f1[4 * q + 0], xv.x, acc1[bt]);
          acc1[bt] = fmaf(f1[4 * q + 1], xv.y, acc1[bt]);
          acc1[bt] = fmaf(f1[4 * q + 2], xv.z, acc1[bt]);
          acc1[bt] = fmaf(f1[4 * q + 3], xv.w, acc1[bt]);
        }
      }
    }
  };
#pragma unroll
  for (int k = 0; k < HOLD; ++k) {
    const int v = lane + 32 * k;
    if (v < nvec) fma_vec(h0[k], h1[k], v);
  }
  for (int v0 = lane + 32 * HOLD; v0 < nvec; v0 += 32 * kLoadBatch) {
    uint4 u0[kLoadBatch], u1[kLoadBatch];
#pragma unroll
    for (int k = 0; k < kLoadBatch; ++k) {
      const int v = v0 + 32 * k;
      if (v < nvec) {
        u0[k] = ld_stream(w0 + v);
        u1[k] = ld_stream(w1 + v);
      }
    }
#pragma unroll
    for (int k = 0; k < kLoadBatch; ++k) {
      const int v = v0 + 32 * k;
      if (v < nvec) fma_vec(u0[k], u1[k], v);
    }
  }
  float s0 = 1.f, s1 = 1.f;
  if (FMT == NC_FP8E4M3) {
    s0 = m.scale[r0];
    s1 = m.scale[r1];
  }
#pragma unroll
  for (int bt = 0; bt < BT; ++bt) {
    if (bt < nb) {
      float y0 = warp_sum(acc0[bt]);
      float y1 = warp_sum(acc1[bt]);
      if (FMT == NC_FP8E4M3) {
        y0 *= s0;
        y1 *= s1;
      }
      if (lane == bt) {
        const int j = b0 + bt;
        if (EPI == EPI_STORE) {
          out.y[(size_t)j * m.rows + r0] = y0;
          if (has1) out.y[(size_t)j * m.rows + r1] = y1;
        } else if (EPI == EPI_RESID) {
          float* p0 = out.y + (size_t)j * m.rows + r0;
          *p0 = __ldcg(p0) + y0;
          if (has1) {
            float* p1 = out.y + (size_t)j * m.rows + r1;
            *p1 = __ldcg(p1) + y1;
          }
        } else if (EPI == EPI_SWIGLU) {
          out.y[(size_t)j * (m.rows / 2) + r0 / 2] = silu(y0) * y1;
        } else {
          float* z = out.zrows ? out.zrows + (size_t)j * m.rows : out.st[out.slots[j]].z;
          z[r0] = y0;
          if (has1) z[r1] = y1;
        }
      }
    }
  }
}

// ----------------------------------------------------------------- attention
// Decode attention of one (stream row j, KV head g).  The window [start, a]
// (a = the fed token's absolute position) is cut into chunks of kAttnChunk
// positions, chunk c = [start + c * 256, ...), and a chunk into 32-position
// blocks, one per warp.  The arithmetic is fixed by the window alone:
// scores, max and P V inside a block (warp shuffles in lane order), the
// blocks of a chunk combined in block order, then the chunks in chunk order.
// Which CTA computes which chunk is a launch choice that does not change a
// bit: a cluster of S CTAs (S = 1, 2, 4 or 8) takes chunks c = rank,
// rank + S, ..., keeps each chunk's (max, sum, accumulator) in its shared
// memory, and the chunk merge reads them through distributed shared memory.
//
// The fed token's q and k are rotated (rotate-half RoPE) at position a;
// cached keys were rotated at their own absolute positions when appended.
// Scores depend only on position differences, so this equals the
// relabelled positions of the sliding window (Sec. 3.9).  The CTA that owns
// the chunk holding position a appends the new k, v at ring index a mod L.
constexpr int kAttnThreads = 256;
constexpr int kAttnWarps = kAttnThreads / 32;
constexpr int kAttnChunk = kAttnWarps * 32;          // positions per chunk
constexpr int kAttnMaxChunks = 2048 / kAttnChunk;    // ctx_len <= 2048

template <int S>
struct __align__(16) AttnSmem {
  static constexpr int kDims = kHeadDim / S;         // output dims merged by one CTA
  float qs[kMaxGroup][kHeadDim];
  float kn[kHeadDim], vn[kHeadDim];
  float cs[kHeadDim / 2], sn[kHeadDim / 2];
  float wm[kAttnWarps][kMaxGroup], wl[kAttnWarps][kMaxGroup];
  float wacc[kAttnWarps][kMaxGroup][kHeadDim];
  float we[kAttnWarps][kMaxGroup][32];               // each warp's softmax numerators
  float cf[kMaxGroup][kAttnWarps], cM[kMaxGroup], cL[kMaxGroup];   // block combine factors
  float mf[kMaxGroup][kAttnMaxChunks], mL[kMaxGroup];              // chunk merge factors
  // every chunk's (max, sum) and this CTA's dims of its accumulator, written
  // by the chunk's owner (a remote store when the owner is another CTA)
  float rm[kAttnMaxChunks][kMaxGroup], rl[kAttnMaxChunks][kMaxGroup];
  float racc[kAttnMaxChunks][kMaxGroup][kDims];
};

struct AttnIO {
  const float* qkv;      // [B][qkv_rows], written by the QKV projection
  float* attn_out;       // [B][hq * 64]
  void* out16;           // or, when set, the output rounded to BF16 there (the tensor-core O operand)
};

// Values of a lane that do not depend on the QKV projection: the cached key
// of its position and the values of its warp's 32 positions.
template <int KBF16>
struct AttnPre {
  float kr[KBF16 ? 1 : kHeadDim];       // FP32 cache: the key
  uint32_t kb[KBF16 ? kHeadDim / 2 : 1];  // BF16 cache: the key as packed pairs
  uint32_t vb[32];
  float2 vf[KBF16 ? 1 : 32];
};

__device__ __forceinline__ float2 rope_cs(const Dims& D, int a, int dd) { return rope_cs_tab(D.rope_tab, a, dd); }

// cos / sin of position a for the 32 rotation pairs.
template <typename Sm>
__device__ __forceinline__ void attn_rope(const Dims& D, int a, int tid, Sm& sm) {
  if (tid < kHeadDim / 2) {
    const float2 cs = rope_cs(D, a, tid);
    sm.cs[tid] = cs.x;
    sm.sn[tid] = cs.y;
  }
}

__device__ __forceinline__ size_t attn_plane_off(const Dims& D, int layer, int which) {
  return kv_plane_off(D.L, D.hkv, layer, which);
}

// Cached K of position p_lo + lane and V of positions p_lo .. p_lo + 31
// (positions >= p_end and position a itself are not loaded).
template <int KBF16>
__device__ __forceinline__ void attn_load(const Dims& D, const StreamDev& st, int layer, int g, int p_lo,
                                          int p_end, int a, int lane, AttnPre<KBF16>& pre) {
  const size_t koff = attn_plane_off(D, layer, g);
  const size_t voff = attn_plane_off(D, layer, D.hkv + g);
  const int p = p_lo + lane;
  if (p < p_end && p < a) {
    const size_t ri = (size_t)(p & (D.L - 1)) * kHeadDim;
    if (KBF16) {
      const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(st.kv) + koff + ri);
#pragma unroll
      for (int q = 0; q < kHeadDim / 8; ++q) {
        const uint4 u = src[q];
        pre.kb[4 * q] = u.x;
        pre.kb[4 * q + 1] = u.y;
        pre.kb[4 * q + 2] = u.z;
        pre.kb[4 * q + 3] = u.w;
      }
    } else {
      const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(st.kv) + koff + ri);
#pragma unroll
      for (int q = 0; q < kHeadDim / 4; ++q) {
        const float4 u = src[q];
        pre.kr[4 * q] = u.x;
        pre.kr[4 * q + 1] = u.y;
        pre.kr[4 * q + 2] = u.z;
        pre.kr[4 * q + 3] = u.w;
      }
    }
  }
  const int nvalid = min(32, min(p_end, a + 1) - p_lo);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int pi = p_lo + i;
    if (i < nvalid && pi != a) {
      const size_t ri = (size_t)(pi & (D.L - 1)) * kHeadDim + 2 * lane;
      if (KBF16)
        pre.vb[i] = *reinterpret_cast<const uint32_t*>(static_cast<const __nv_bfloat16*>(st.kv) + voff + ri);
      else
        pre.vf[KBF16 ? 0 : i] = *reinterpret_cast<const float2*>(static_cast<const float*>(st.kv) + voff + ri);
    }
  }
}

// Once the QKV projection is complete: rotated, pre-scaled q of the group's
// heads and the new k, v into shared memory; the owner of position a
// appends k, v to the ring.
template <int KBF16, typename Sm>
__device__ void attn_qkv(const Dims& D, StreamDev& st, int layer, int j, int g, int a, bool append, int tid,
                         Sm& sm, const AttnIO& io) {
  const int grp = D.hq / D.hkv;
  __syncthreads();
  const float* row = io.qkv + (size_t)j * D.qkv_rows;
  for (int e = tid; e < (grp + 1) * (kHeadDim / 2); e += kAttnThreads) {
    const int h = e / (kHeadDim / 2), dd = e % (kHeadDim / 2);
    const float* src = h < grp ? row + (g * grp + h) * kHeadDim : row + D.hq * kHeadDim + g * kHeadDim;
    const float x1 = __ldcg(src + dd), x2 = __ldcg(src + dd + kHeadDim / 2);
    const float2 rr = rope_rotate(x1, x2, make_float2(sm.cs[dd], sm.sn[dd]));
    const float r1 = rr.x, r2 = rr.y;
    if (h < grp) {   // the 1/sqrt(64) score scale is a power of two: exact
      sm.qs[h][dd] = r1 * 0.125f;
      sm.qs[h][dd + kHeadDim / 2] = r2 * 0.125f;
    } else {
      sm.kn[dd] = r1;
      sm.kn[dd + kHeadDim / 2] = r2;
    }
  }
  if (tid < kHeadDim) sm.vn[tid] = __ldcg(row + (D.hq + D.hkv) * kHeadDim + g * kHeadDim + tid);
  __syncthreads();
  if (append && tid < kHeadDim) {
    const size_t ri = (size_t)(a & (D.L - 1)) * kHeadDim + tid;
    const size_t koff = attn_plane_off(D, layer, g), voff = attn_plane_off(D, layer, D.hkv + g);
    if (KBF16) {
      __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv);
      kv[koff + ri] = __float2bfloat16_rn(sm.kn[tid]);
      kv[voff + ri] = __float2bfloat16_rn(sm.vn[tid]);
    } else {
      float* kv = static_cast<float*>(st.kv);
      kv[koff + ri] = sm.kn[tid];
      kv[voff + ri] = sm.vn[tid];
    }
  }
}

// One warp's block of 32 positions p_lo .. p_lo + 31 of a chunk ending at
// c_end, for the query of position a: scores of the group's heads, the
// warp's softmax numerators (max mh, sum lh) and P V (lane owns output dims
// 2 lane, 2 lane + 1).  `q` holds the rotated, scaled query heads (qs) and
// the fed token's k, v (kn, vn), used in FP32 at position a whatever `pre`
// holds there.  `we` is the warp's [head][32] scratch for the numerators.
// Returns the number of positions of the block (<= 0: none).
template <int KBF16, typename Qv>
__device__ __forceinline__ int attn_block(const Dims& D, int p_lo, int c_end, int a, int lane, const Qv& q,
                                          float* we, const AttnPre<KBF16>& pre, float (&mh)[kMaxGroup],
                                          float (&lh)[kMaxGroup], float (&acc)[kMaxGroup][2]) {
  const int grp = D.hq / D.hkv;
  const int p = p_lo + lane;
  const bool valid = p < c_end && p <= a;
  const int nvalid = min(32, min(c_end, a + 1) - p_lo);
  float sc[kMaxGroup];
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) sc[h] = 0.f;
  if (valid && p != a) {
#pragma unroll
    for (int h = 0; h < kMaxGroup; ++h) {
      if (h < grp) {
        float dot = 0.f;
        if (KBF16) {
#pragma unroll
          for (int i = 0; i < kHeadDim / 2; ++i) {
            const uint32_t w = pre.kb[KBF16 ? i : 0];
            dot = fmaf(q.qs[h][2 * i], __uint_as_float(w << 16), dot);
            dot = fmaf(q.qs[h][2 * i + 1], __uint_as_float(w & 0xFFFF0000u), dot);
          }
        } else {
#pragma unroll
          for (int d = 0; d < kHeadDim; ++d) dot = fmaf(q.qs[h][d], pre.kr[KBF16 ? 0 : d], dot);
        }
        sc[h] = dot;
      }
    }
  } else if (p == a) {   // the new key enters in FP32 from shared memory
#pragma unroll
    for (int h = 0; h < kMaxGroup; ++h) {
      if (h < grp) {
        float dot = 0.f;
#pragma unroll
        for (int d = 0; d < kHeadDim; ++d) dot = fmaf(q.qs[h][d], q.kn[d], dot);
        sc[h] = dot;
      }
    }
  }
  float eh[kMaxGroup];
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) {
    if (h < grp) {
      mh[h] = warp_max(valid ? sc[h] : -INFINITY);
      eh[h] = valid ? expf(sc[h] - mh[h]) : 0.f;
      lh[h] = warp_sum(eh[h]);
    }
  }
  // P V: lane owns output dims 2*lane, 2*lane + 1; the numerators of the
  // warp's 32 positions are read back from shared memory four at a time
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h)
    if (h < grp) we[h * 32 + lane] = eh[h];
  __syncwarp();
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) acc[h][0] = acc[h][1] = 0.f;
#pragma unroll
  for (int i4 = 0; i4 < 32; i4 += 4) {
    if (i4 >= nvalid) break;
    float4 e4[kMaxGroup];
#pragma unroll
    for (int h = 0; h < kMaxGroup; ++h)
      if (h < grp) e4[h] = *reinterpret_cast<const float4*>(we + h * 32 + i4);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i4 + k;
      if (i < nvalid) {
        const int pi = p_lo + i;
        float v0, v1;
        if (pi == a) {
          v0 = q.vn[2 * lane];
          v1 = q.vn[2 * lane + 1];
        } else if (KBF16) {
          v0 = __uint_as_float(pre.vb[i] << 16);
          v1 = __uint_as_float(pre.vb[i] & 0xFFFF0000u);
        } else {
          v0 = pre.vf[KBF16 ? 0 : i].x;
          v1 = pre.vf[KBF16 ? 0 : i].y;
        }
#pragma unroll
        for (int h = 0; h < kMaxGroup; ++h) {
          if (h < grp) {
            const float e = k == 0 ? e4[h].x : k == 1 ? e4[h].y : k == 2 ? e4[h].z : e4[h].w;
            acc[h][0] = fmaf(e, v0, acc[h][0]);
            acc[h][1] = fmaf(e, v1, acc[h][1]);
          }
        }
      }
    }
  }
  __syncwarp();                                    // `we` may be rewritten by the caller
  return nvalid;
}

// One chunk [c_lo, c_end) for the query of position a: every warp's block
// (attn_block), then the blocks combined in block order into the chunk's
// (max M, sum l, accumulator o).  `sm` is the scratch (wm, wl, wacc, we, cf,
// cM, cL).  put(h, dd, o, M, l) receives the accumulator of head h, dim dd.
template <int KBF16, typename Qv, typename Sc, typename Put>
__device__ void attn_chunk(const Dims& D, int c_lo, int c_end, int a, int tid, const Qv& q, Sc& sm,
                           AttnPre<KBF16>& pre, Put put) {
  const int grp = D.hq / D.hkv;
  const int warp = tid >> 5, lane = tid & 31;
  float mh[kMaxGroup], lh[kMaxGroup], acc[kMaxGroup][2];
  const int nvalid = attn_block<KBF16>(D, c_lo + warp * 32, c_end, a, lane, q, &sm.we[warp][0][0], pre, mh, lh, acc);
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) {
    if (h < grp) {
      if (lane == 0) {
        sm.wm[warp][h] = nvalid > 0 ? mh[h] : -INFINITY;
        sm.wl[warp][h] = nvalid > 0 ? lh[h] : 0.f;
      }
      sm.wacc[warp][h][2 * lane] = acc[h][0];
      sm.wacc[warp][h][2 * lane + 1] = acc[h][1];
    }
  }
  __syncthreads();
  // combine the blocks in block order; blocks 0 .. nblk - 1 hold positions.
  // The factor of block w, exp(m_w - M), is computed once per head.
  const int nblk = (min(c_end, a + 1) - c_lo + 31) / 32;
  if (tid < grp) {
    const int h = tid;
    float M = -INFINITY;
    for (int w = 0; w < nblk; ++w) M = fmaxf(M, sm.wm[w][h]);
    float l = 0.f;
    for (int w = 0; w < nblk; ++w) {
      const float f = expf(sm.wm[w][h] - M);
      sm.cf[h][w] = f;
      l = fmaf(sm.wl[w][h], f, l);
    }
    sm.cM[h] = M;
    sm.cL[h] = l;
  }
  __syncthreads();
  for (int e = tid; e < grp * kHeadDim; e += kAttnThreads) {
    const int h = e / kHeadDim, dd = e % kHeadDim;
    float o = 0.f;
    for (int w = 0; w < nblk; ++w) o = fmaf(sm.wacc[w][h][dd], sm.cf[h][w], o);
    put(h, dd, o, sm.cM[h], sm.cL[h]);
  }
  __syncthreads();   // the scratch is rewritten by the next chunk
}

}  // namespace dev
}  // namespace nc
