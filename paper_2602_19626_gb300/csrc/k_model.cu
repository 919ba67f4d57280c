// Transformer decode kernels (Sec. 3.2 model, Sec. 3.9 sliding KV window).
//
// One decode step per stream: embedding, per layer RMSNorm -> QKV -> RoPE +
// KV append -> grouped-query attention -> O projection + residual -> RMSNorm
// -> gate/up -> SwiGLU -> down + residual, then the final RMSNorm and the
// tied LM head.  Every reduction has a fixed order that does not depend on
// the batch size, the slot or the grid, so a stream's logits are bit-identical
// whether it runs alone or in a batch.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"

namespace nc {

namespace {

constexpr int kGemvThreads = 256;
constexpr int kGemvWarps = kGemvThreads / 32;
constexpr int kRowsPerWarp = 2;
constexpr int kGemvBT = 8;        // streams per activation tile held in shared memory
constexpr int kLoadBatch = 4;     // 16-byte loads per row in flight per lane

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

__device__ __forceinline__ float silu(float a) { return a / (1.0f + expf(-a)); }

// ----------------------------------------------------------------- embedding
template <int FMT>
__global__ void k_embed(Dims D, Batch b, const void* E, const float* Escale, float* x) {
  const int j = blockIdx.x;
  pdl_wait();
  pdl_trigger();
  if (j >= *b.nB) return;
  const StreamDev& st = b.st[b.slots[j]];
  const int tok = st.last_tok;
  for (int c = threadIdx.x; c < D.d; c += blockDim.x) {
    float v;
    if (FMT == NC_FP32) {
      v = static_cast<const float*>(E)[(size_t)tok * D.d + c];
    } else if (FMT == NC_BF16) {
      v = __bfloat162float(static_cast<const __nv_bfloat16*>(E)[(size_t)tok * D.d + c]);
    } else {
      __nv_fp8_e4m3 q;
      q.__x = static_cast<const __nv_fp8_storage_t*>(E)[(size_t)tok * D.d + c];
      v = float(q) * Escale[tok];
    }
    x[(size_t)j * D.d + c] = v;
  }
}

// ---------------------------------------------------------------------- GEMV
// y[j][r] = sum_c W[r][c] * a_j[c] for the active streams j, where a_j is the
// prologue's activation (RMSNorm of the residual, merged attention output, or
// a plain vector).  Each warp owns two consecutive rows; lane l accumulates
// the 16-byte weight vectors l, l+32, ... of both rows in order, then a fixed
// xor-shuffle tree sums the lanes.  The activation tile for up to kGemvBT
// streams sits in shared memory; larger batches loop over tiles (the weights
// of a warp's rows are re-read per tile).
template <int FMT, int PRO, int EPI>
__global__ void __launch_bounds__(kGemvThreads) k_gemv(Dims D, Batch b, Mat m, GemvIO io) {
  extern __shared__ float4 smem4[];
  float* xs = reinterpret_cast<float*>(smem4);   // [kGemvBT][cols]
  __shared__ float red[kGemvWarps][kGemvBT];
  __shared__ float inv_rms[kGemvBT];
  using W = WFmt<FMT>;
  constexpr int VW = W::VW;
  constexpr int kHold = 8;                       // 16-byte vectors per row held in registers
  const int cols = m.cols;
  const int nvec = cols / VW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x * kGemvWarps + warp) * kRowsPerWarp;
  const bool have_rows = row0 < m.rows;
  const bool have_row1 = row0 + 1 < m.rows;          // odd row counts (the vocabulary)
  const int row1 = have_row1 ? row0 + 1 : row0;
  const uint4* w0 = reinterpret_cast<const uint4*>(static_cast<const char*>(m.w) +
                                                   (size_t)row0 * cols * W::ESZ);
  const uint4* w1 = reinterpret_cast<const uint4*>(static_cast<const char*>(m.w) +
                                                   (size_t)row1 * cols * W::ESZ);
  // Weights do not depend on earlier kernels: fetch this warp's rows before
  // waiting on the predecessor, so the fetch overlaps its execution.
  uint4 h0[kHold], h1[kHold];
#pragma unroll
  for (int k = 0; k < kHold; ++k) {
    const int v = lane + 32 * k;
    if (have_rows && v < nvec) {
      h0[k] = ld_stream(w0 + v);
      h1[k] = ld_stream(w1 + v);
    }
  }
  pdl_wait();
  pdl_trigger();
  const int B = *b.nB;

  for (int b0 = 0; b0 < B; b0 += kGemvBT) {
    const int nb = min(kGemvBT, B - b0);
    // ---- prologue: activations of streams b0 .. b0+nb-1 into shared memory
    if (PRO == PRO_RMSNORM) {
      for (int bt = 0; bt < nb; ++bt) {
        const float* xr = io.x + (size_t)(b0 + bt) * cols;
        float ss = 0.f;
        for (int c = threadIdx.x; c < cols; c += kGemvThreads) ss = fmaf(xr[c], xr[c], ss);
        ss = warp_sum(ss);
        if (lane == 0) red[warp][bt] = ss;
      }
      __syncthreads();
      if (threadIdx.x < nb) {
        float ss = 0.f;
        for (int w = 0; w < kGemvWarps; ++w) ss += red[w][threadIdx.x];
        inv_rms[threadIdx.x] = 1.0f / sqrtf(ss / (float)cols + D.eps);
      }
      __syncthreads();
      for (int bt = 0; bt < nb; ++bt) {
        const float* xr = io.x + (size_t)(b0 + bt) * cols;
        for (int c = threadIdx.x; c < cols; c += kGemvThreads)
          xs[bt * cols + c] = xr[c] * inv_rms[bt] * io.g[c];
      }
    } else if (PRO == PRO_PLAIN) {
      for (int bt = 0; bt < nb; ++bt) {
        const float* xr = io.x + (size_t)(b0 + bt) * cols;
        for (int c = threadIdx.x; c < cols; c += kGemvThreads) xs[bt * cols + c] = xr[c];
      }
    }
    __syncthreads();

    if (have_rows) {
      float acc0[kGemvBT], acc1[kGemvBT];
#pragma unroll
      for (int bt = 0; bt < kGemvBT; ++bt) acc0[bt] = acc1[bt] = 0.f;
      // lane l accumulates vectors l, l + 32, l + 64, ... in increasing order:
      // first the held ones, then the rest of a long row streamed in batches
      auto fma_vec = [&](const uint4& a0, const uint4& a1, int v) {
        float f0[VW], f1[VW];
        W::deq(a0, f0);
        W::deq(a1, f1);
#pragma unroll
        for (int bt = 0; bt < kGemvBT; ++bt) {
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
      for (int k = 0; k < kHold; ++k) {
        const int v = lane + 32 * k;
        if (v < nvec) fma_vec(h0[k], h1[k], v);
      }
      for (int v0 = lane + 32 * kHold; v0 < nvec; v0 += 32 * kLoadBatch) {
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
        s0 = m.scale[row0];
        s1 = m.scale[row1];
      }
#pragma unroll
      for (int bt = 0; bt < kGemvBT; ++bt) {
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
              io.y[(size_t)j * m.rows + row0] = y0;
              if (have_row1) io.y[(size_t)j * m.rows + row1] = y1;
            } else if (EPI == EPI_RESID) {
              io.y[(size_t)j * m.rows + row0] += y0;
              if (have_row1) io.y[(size_t)j * m.rows + row1] += y1;
            } else if (EPI == EPI_SWIGLU) {
              io.y[(size_t)j * (m.rows / 2) + row0 / 2] = silu(y0) * y1;
            } else {
              float* z = b.st[b.slots[j]].z;
              z[row0] = y0;
              if (have_row1) z[row1] = y1;
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- attention
// Split-KV decode attention for one (stream, KV head, chunk of <= 128 cached
// positions).  The fed token's q and k are rotated (rotate-half RoPE) at its
// absolute position; cached keys were rotated at their own absolute positions
// when appended.  Scores depend only on position differences, so this equals
// the relabelled positions of the sliding window (Sec. 3.9).  The last chunk
// also appends the new k, v at ring index a mod L.  Output per query head:
// running max m, sum l and unnormalised accumulator of the chunk.
template <int KBF16>
__global__ void __launch_bounds__(128) k_attn(Dims D, Batch b, int layer, const float* qkv,
                                              float* part, int* tickets, float* attn_out) {
  const int j = blockIdx.z;
  if (j >= *b.nB) return;
  StreamDev& st = b.st[b.slots[j]];
  const int g = blockIdx.y, s = blockIdx.x;
  const int a = st.n_coded;
  const int start = window_start(D, st);
  const int n = a - start + 1;
  const int ns = (n + kAttnChunk - 1) / kAttnChunk;
  if (s >= ns) return;
  const int grp = D.hq / D.hkv;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  __shared__ float qs[kMaxGroup][kHeadDim];
  __shared__ float kn[kHeadDim], vn[kHeadDim];
  __shared__ float cs[kHeadDim / 2], sn[kHeadDim / 2];
  __shared__ float wm[4][kMaxGroup], wl[4][kMaxGroup];
  __shared__ float wacc[4][kMaxGroup][kHeadDim];

  // ---- before waiting on the QKV projection: rotation angles of position a
  // (FP64 angle, rounded once) and this lane's cached key (earlier tokens)
  if (tid < kHeadDim / 2) {
    const double inv_freq = pow((double)D.theta, -2.0 * tid / (double)kHeadDim);
    double sd, cd;
    sincos((double)a * inv_freq, &sd, &cd);
    cs[tid] = (float)cd;
    sn[tid] = (float)sd;
  }
  const size_t plane = (size_t)D.L * kHeadDim;     // one [L][64] K or V plane
  const size_t layer_off = (size_t)layer * 2 * D.hkv * plane;
  const size_t koff = layer_off + (size_t)g * plane;
  const size_t voff = layer_off + (size_t)(D.hkv + g) * plane;
  const int p_lo = start + s * kAttnChunk + warp * 32;
  const int p = p_lo + lane;
  const bool valid = p <= a;
  float kr[kHeadDim];
  if (valid && p != a) {
    const size_t ri = (size_t)(p & (D.L - 1)) * kHeadDim;
    if (KBF16) {
      const __nv_bfloat16* kvb = static_cast<const __nv_bfloat16*>(st.kv);
      const uint4* src = reinterpret_cast<const uint4*>(kvb + koff + ri);
#pragma unroll
      for (int q = 0; q < kHeadDim / 8; ++q) {
        const uint4 u = src[q];
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          kr[8 * q + 2 * i] = __uint_as_float(w[i] << 16);
          kr[8 * q + 2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
      }
      asm volatile("prefetch.global.L2 [%0];" ::"l"(kvb + voff + ri));
    } else {
      const float* kvf = static_cast<const float*>(st.kv);
      const float4* src = reinterpret_cast<const float4*>(kvf + koff + ri);
#pragma unroll
      for (int q = 0; q < kHeadDim / 4; ++q) {
        const float4 u = src[q];
        kr[4 * q] = u.x;
        kr[4 * q + 1] = u.y;
        kr[4 * q + 2] = u.z;
        kr[4 * q + 3] = u.w;
      }
      asm volatile("prefetch.global.L2 [%0];" ::"l"(kvf + voff + ri));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(kvf + voff + ri + 32));
    }
  }
  // values of the warp's 32 cached positions: lane owns dims 2*lane, 2*lane+1
  const int nvalid = min(32, a - p_lo + 1);
  uint32_t vb[32];        // BF16 pairs
  float2 vf[KBF16 ? 1 : 32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int pi = p_lo + i;
    if (i < nvalid && pi != a) {
      const size_t ri = (size_t)(pi & (D.L - 1)) * kHeadDim + 2 * lane;
      if (KBF16)
        vb[i] = *reinterpret_cast<const uint32_t*>(static_cast<const __nv_bfloat16*>(st.kv) + voff + ri);
      else
        vf[KBF16 ? 0 : i] = *reinterpret_cast<const float2*>(static_cast<const float*>(st.kv) + voff + ri);
    }
  }
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const float* row = qkv + (size_t)j * D.qkv_rows;
  for (int e = tid; e < (grp + 1) * (kHeadDim / 2); e += blockDim.x) {
    const int h = e / (kHeadDim / 2), dd = e % (kHeadDim / 2);
    const float* src = h < grp ? row + (g * grp + h) * kHeadDim : row + D.hq * kHeadDim + g * kHeadDim;
    const float x1 = src[dd], x2 = src[dd + kHeadDim / 2];
    const float r1 = x1 * cs[dd] - x2 * sn[dd];
    const float r2 = x2 * cs[dd] + x1 * sn[dd];
    if (h < grp) {   // the 1/sqrt(64) score scale is a power of two: exact
      qs[h][dd] = r1 * 0.125f;
      qs[h][dd + kHeadDim / 2] = r2 * 0.125f;
    } else {
      kn[dd] = r1;
      kn[dd + kHeadDim / 2] = r2;
    }
  }
  if (tid < kHeadDim) vn[tid] = row[(D.hq + D.hkv) * kHeadDim + g * kHeadDim + tid];
  __syncthreads();

  // the last chunk appends the new key / value at ring index a mod L
  if (s == ns - 1 && tid < kHeadDim) {
    const size_t ri = (size_t)(a & (D.L - 1)) * kHeadDim + tid;
    if (KBF16) {
      __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv);
      kv[koff + ri] = __float2bfloat16_rn(kn[tid]);
      kv[voff + ri] = __float2bfloat16_rn(vn[tid]);
    } else {
      float* kv = static_cast<float*>(st.kv);
      kv[koff + ri] = kn[tid];
      kv[voff + ri] = vn[tid];
    }
  }

  float sc[kMaxGroup];
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) sc[h] = 0.f;
  if (valid) {
    if (p == a) {
#pragma unroll
      for (int d = 0; d < kHeadDim; ++d) kr[d] = kn[d];
    }
#pragma unroll
    for (int h = 0; h < kMaxGroup; ++h) {
      if (h < grp) {
        float acc = 0.f;
#pragma unroll
        for (int d = 0; d < kHeadDim; ++d) acc = fmaf(qs[h][d], kr[d], acc);
        sc[h] = acc;
      }
    }
  }
  float mh[kMaxGroup], eh[kMaxGroup], lh[kMaxGroup];
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) {
    if (h < grp) {
      mh[h] = warp_max(valid ? sc[h] : -INFINITY);
      eh[h] = valid ? expf(sc[h] - mh[h]) : 0.f;
      lh[h] = warp_sum(eh[h]);
    }
  }
  // P V: lane owns output dims 2*lane, 2*lane + 1
  float acc[kMaxGroup][2];
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) acc[h][0] = acc[h][1] = 0.f;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    if (i >= nvalid) break;
    const int pi = p_lo + i;
    float v0, v1;
    if (pi == a) {
      v0 = vn[2 * lane];
      v1 = vn[2 * lane + 1];
    } else if (KBF16) {
      v0 = __uint_as_float(vb[i] << 16);
      v1 = __uint_as_float(vb[i] & 0xFFFF0000u);
    } else {
      v0 = vf[KBF16 ? 0 : i].x;
      v1 = vf[KBF16 ? 0 : i].y;
    }
#pragma unroll
    for (int h = 0; h < kMaxGroup; ++h) {
      if (h < grp) {
        const float e = __shfl_sync(0xffffffffu, eh[h], i);
        acc[h][0] = fmaf(e, v0, acc[h][0]);
        acc[h][1] = fmaf(e, v1, acc[h][1]);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < kMaxGroup; ++h) {
    if (h < grp) {
      if (lane == 0) {
        wm[warp][h] = nvalid > 0 ? mh[h] : -INFINITY;
        wl[warp][h] = nvalid > 0 ? lh[h] : 0.f;
      }
      wacc[warp][h][2 * lane] = acc[h][0];
      wacc[warp][h][2 * lane + 1] = acc[h][1];
    }
  }
  __syncthreads();
  const int nsm = attn_splits_max_dev(D);
  for (int e = tid; e < grp * kHeadDim; e += blockDim.x) {
    const int h = e / kHeadDim, dd = e % kHeadDim;
    float M = -INFINITY;
    for (int w = 0; w < 4; ++w)
      if (start + s * kAttnChunk + w * 32 <= a) M = fmaxf(M, wm[w][h]);
    float l = 0.f, o = 0.f;
    for (int w = 0; w < 4; ++w) {
      if (start + s * kAttnChunk + w * 32 <= a) {
        const float f = expf(wm[w][h] - M);
        l = fmaf(wl[w][h], f, l);
        o = fmaf(wacc[w][h][dd], f, o);
      }
    }
    float* out = part + (((size_t)j * D.hq + g * grp + h) * nsm + s) * (kHeadDim + 2);
    out[dd] = o;
    if (dd == 0) {
      out[kHeadDim] = M;
      out[kHeadDim + 1] = l;
    }
  }
  // The last chunk to finish (atomic ticket) merges the chunks of this
  // (stream, KV head) in chunk order, so the result does not depend on which
  // CTA finished last.
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int t = atomicAdd(tickets + j * D.hkv + g, 1);
    last = (t == ns - 1);
    if (last) tickets[j * D.hkv + g] = 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = tid; e < grp * kHeadDim; e += blockDim.x) {
    const int h = e / kHeadDim, dd = e % kHeadDim;
    const float* ph = part + ((size_t)j * D.hq + g * grp + h) * nsm * (kHeadDim + 2);
    float M = -INFINITY;
    for (int q = 0; q < ns; ++q) M = fmaxf(M, __ldcg(ph + q * (kHeadDim + 2) + kHeadDim));
    float l = 0.f, acc = 0.f;
    for (int q = 0; q < ns; ++q) {
      const float* pq = ph + q * (kHeadDim + 2);
      const float f = expf(__ldcg(pq + kHeadDim) - M);
      l = fmaf(__ldcg(pq + kHeadDim + 1), f, l);
      acc = fmaf(__ldcg(pq + dd), f, acc);
    }
    attn_out[(size_t)j * D.hq * kHeadDim + (g * grp + h) * kHeadDim + dd] = acc / l;
  }
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

int attn_max_splits(const Dims& D) { return (D.L + kAttnChunk - 1) / kAttnChunk; }

cudaError_t launch_embed(const Dims& D, const Batch& b, const void* E, const float* Escale,
                         int fmt, float* x, cudaStream_t s) {
  const int thr = 256;
  auto kern = fmt == NC_FP32 ? k_embed<NC_FP32> : fmt == NC_BF16 ? k_embed<NC_BF16> : k_embed<NC_FP8E4M3>;
  return launch_kernel(kern, dim3(b.Bmax), dim3(thr), 0, s, D.pdl, D, b, E, Escale, x);
}

template <int FMT, int PRO, int EPI>
static cudaError_t gemv_t(const Dims& D, const Batch& b, const Mat& m, const GemvIO& io,
                          cudaStream_t s) {
  const int rows_per_block = kGemvWarps * kRowsPerWarp;
  const int grid = (m.rows + rows_per_block - 1) / rows_per_block;
  const size_t smem = (size_t)kGemvBT * m.cols * sizeof(float);
  auto kern = k_gemv<FMT, PRO, EPI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_kernel(kern, dim3(grid), dim3(kGemvThreads), smem, s, D.pdl, D, b, m, io);
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

cudaError_t launch_gemv(const Dims& D, const Batch& b, const Mat& m, int fmt, int pro, int epi,
                        const GemvIO& io, cudaStream_t s) {
  if (fmt == NC_FP32) return gemv_f<NC_FP32>(D, b, m, pro, epi, io, s);
  if (fmt == NC_BF16) return gemv_f<NC_BF16>(D, b, m, pro, epi, io, s);
  return gemv_f<NC_FP8E4M3>(D, b, m, pro, epi, io, s);
}

cudaError_t launch_attn(const Dims& D, const Batch& b, int layer, const float* qkv, float* part, int* tickets,
                        float* attn_out, cudaStream_t s) {
  dim3 grid(attn_max_splits(D), D.hkv, b.Bmax);
  return launch_kernel(D.kv_bf16 ? k_attn<1> : k_attn<0>, grid, dim3(128), 0, s, D.pdl, D, b, layer, qkv, part,
                       tickets, attn_out);
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
