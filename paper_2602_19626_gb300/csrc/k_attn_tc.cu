// Decode and prefill attention over a BF16 KV cache on the tensor cores
// (Sec. 3.2 model, Sec. 3.9 sliding window).
//
// The window [start, a] of a query row is cut into chunks of 256 positions
// and a chunk into blocks of 32 positions, one per warp, exactly as in the
// CUDA-core attention.  Within a block the scores and the weighted values are
// warp-level BF16 tensor-core products with FP32 accumulation
// (mma.sync m16n8k16): S = Q K^T over the 64 head dims, then O = P V over
// the block's 32 positions, with Q = the rotated, 1/8-scaled query rounded to
// BF16, K and V the cache's BF16 entries (the fed token's own k, v rounded to
// BF16 as the cache stores them) and P = exp(S - m) rounded to BF16; the max
// m and the sum l of exp(S - m) stay in FP32.  The blocks of a chunk, then
// the chunks, are combined in order in FP32 as before.
//
// The rows of the MMA tile are (query row, head) pairs, padding rows zero.
// A row's products do not depend on the other rows of the tile, so a query
// computed alone (decode, one row) and among the rows of a prefill gives the
// same bits.  Two kernels share the per-block code: k_attn_tc (decode, and
// prefill groups of up to 8 rows: block partials in shared memory) and
// k_attn_pf (prefill groups of 32 positions: each warp walks its 16-row tile
// through a chunk's blocks).  A decode step has 3 rows per KV head and must
// give the prefill's bits, which is why the warp-level MMA is used here rather
// than tcgen05 with its 64- or 128-row tiles and its own accumulation order.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "model_dev.cuh"

namespace cg = cooperative_groups;

namespace nc {

namespace {

using namespace dev;

constexpr int kTileStride = kHeadDim + 8;            // BF16 elements per smem row (bank-conflict-free ldmatrix)
constexpr int kTcThreads = 512;                      // 16 warps: one per (block, m-tile)
constexpr int kMaxRowsTc = 8;                        // query rows per CTA (prefill)
constexpr int kMaxTileRows = 32;                     // (row, head) pairs: 8 rows x 4 heads

struct RowQv {
  float qs[kMaxGroup][kHeadDim];
  float kn[kHeadDim], vn[kHeadDim];
  float cs[kHeadDim / 2], sn[kHeadDim / 2];
};

// Shared-memory layout in bytes for rq query rows, grp heads per KV head and
// kd merged dims per CTA.
struct TcLayout {
  int q16, kt, vt, rowq, arow, wm, wl, wacc, cf, cM, cL, rm, rl, racc, mf, mL, total;
  __host__ __device__ TcLayout(int rq, int grp, int kd) {
    const int R = rq * grp;
    int o = 0;
    auto take = [&](int bytes) {
      const int at = o;
      o += (bytes + 15) & ~15;
      return at;
    };
    q16 = take(kMaxTileRows * kTileStride * 2);
    kt = take(kAttnChunk * kTileStride * 2);
    vt = take(kAttnChunk * kTileStride * 2);
    rowq = take(rq * (int)sizeof(RowQv));
    arow = take(kMaxRowsTc * 4);
    wm = take(kAttnWarps * R * 4);
    wl = take(kAttnWarps * R * 4);
    wacc = take(kAttnWarps * R * kHeadDim * 4);
    cf = take(R * kAttnWarps * 4);
    cM = take(R * 4);
    cL = take(R * 4);
    rm = take(rq * kAttnMaxChunks * grp * 4);
    rl = take(rq * kAttnMaxChunks * grp * 4);
    racc = take(rq * kAttnMaxChunks * grp * kd * 4);
    mf = take(R * kAttnMaxChunks * 4);
    mL = take(R * 4);
    total = o;
  }
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr(p)));
}
// D += A B for one m16n8k16 tile: BF16 operands, FP32 accumulator.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// The A fragments of m-tile mt's 16 (row, head) query rows for the 4 k-steps
// of 16 head dims.
__device__ __forceinline__ void q_frags(const __nv_bfloat16* q16, int mt, int lane, uint32_t (&a)[4][4]) {
#pragma unroll
  for (int kk = 0; kk < kHeadDim / 16; ++kk)
    ldsm_x4(a[kk], q16 + (mt * 16 + (lane & 15)) * kTileStride + kk * 16 + (lane >> 4) * 8);
}

// Scores S = Q K^T of a block of 32 positions at tile row pb: 4 n-tiles of 8
// positions, the k-steps in order.
__device__ __forceinline__ void block_scores(const uint32_t (&a)[4][4], const __nv_bfloat16* kt, int pb, int lane,
                                             float (&s)[4][4]) {
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) s[nt][0] = s[nt][1] = s[nt][2] = s[nt][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < kHeadDim / 16; ++kk) {
#pragma unroll
    for (int nt = 0; nt < 4; nt += 2) {
      const int m = lane >> 3;
      uint32_t bk[4];
      ldsm_x4(bk, kt + (pb + 8 * (nt + (m >> 1)) + (lane & 7)) * kTileStride + kk * 16 + (m & 1) * 8);
      mma_bf16(s[nt], a[kk], bk[0], bk[1]);
      mma_bf16(s[nt + 1], a[kk], bk[2], bk[3]);
    }
  }
}

// The block's maxima of this thread's two rows (rA = g, rB = g + 8 of the
// m-tile) over their unmasked positions p <= aA / aB.
__device__ __forceinline__ void block_max(const float (&s)[4][4], int p_lo, int t, int aA, int aB, float& mA,
                                          float& mB) {
  mA = -INFINITY;
  mB = -INFINITY;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int p = p_lo + 8 * nt + 2 * t;
    if (p <= aA) mA = fmaxf(mA, s[nt][0]);
    if (p + 1 <= aA) mA = fmaxf(mA, s[nt][1]);
    if (p <= aB) mB = fmaxf(mB, s[nt][2]);
    if (p + 1 <= aB) mB = fmaxf(mB, s[nt][3]);
  }
  mA = fmaxf(mA, __shfl_xor_sync(0xffffffffu, mA, 1));
  mA = fmaxf(mA, __shfl_xor_sync(0xffffffffu, mA, 2));
  mB = fmaxf(mB, __shfl_xor_sync(0xffffffffu, mB, 1));
  mB = fmaxf(mB, __shfl_xor_sync(0xffffffffu, mB, 2));
}

constexpr float kLog2e = 1.4426950408889634f;
// 2^x (PTX ex2.approx, subnormal results flushed to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exp(S - m) = 2^(S log2 e - m log2 e) in place (masked positions 0) and the
// rows' sums l.
__device__ __forceinline__ void block_exp(float (&s)[4][4], int p_lo, int t, int aA, int aB, float mA, float mB,
                                          float& lA, float& lB) {
  lA = 0.f;
  lB = 0.f;
  const float bA = -__fmul_rn(mA, kLog2e), bB = -__fmul_rn(mB, kLog2e);
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int p = p_lo + 8 * nt + 2 * t;
    s[nt][0] = p <= aA ? ex2_approx(__fmaf_rn(s[nt][0], kLog2e, bA)) : 0.f;
    s[nt][1] = p + 1 <= aA ? ex2_approx(__fmaf_rn(s[nt][1], kLog2e, bA)) : 0.f;
    s[nt][2] = p <= aB ? ex2_approx(__fmaf_rn(s[nt][2], kLog2e, bB)) : 0.f;
    s[nt][3] = p + 1 <= aB ? ex2_approx(__fmaf_rn(s[nt][3], kLog2e, bB)) : 0.f;
    lA = __fadd_rn(lA, s[nt][0]);
    lA = __fadd_rn(lA, s[nt][1]);
    lB = __fadd_rn(lB, s[nt][2]);
    lB = __fadd_rn(lB, s[nt][3]);
  }
  lA += __shfl_xor_sync(0xffffffffu, lA, 1);
  lA += __shfl_xor_sync(0xffffffffu, lA, 2);
  lB += __shfl_xor_sync(0xffffffffu, lB, 1);
  lB += __shfl_xor_sync(0xffffffffu, lB, 2);
}

// Weighted values O = P V of the block: P (BF16) as the A operand, 2
// k-steps of 16 positions.
__device__ __forceinline__ void block_pv(const float (&s)[4][4], const __nv_bfloat16* vt, int pb, int lane,
                                         float (&o)[8][4]) {
#pragma unroll
  for (int nd = 0; nd < 8; ++nd) o[nd][0] = o[nd][1] = o[nd][2] = o[nd][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    uint32_t a[4];
    a[0] = pack_bf16(s[2 * ks][0], s[2 * ks][1]);
    a[1] = pack_bf16(s[2 * ks][2], s[2 * ks][3]);
    a[2] = pack_bf16(s[2 * ks + 1][0], s[2 * ks + 1][1]);
    a[3] = pack_bf16(s[2 * ks + 1][2], s[2 * ks + 1][3]);
#pragma unroll
    for (int nd = 0; nd < 8; nd += 2) {
      const int m = lane >> 3;
      uint32_t bv[4];
      ldsm_x4_t(bv, vt + (pb + 16 * ks + (m & 1) * 8 + (lane & 7)) * kTileStride + 8 * (nd + (m >> 1)));
      mma_bf16(o[nd], a, bv[0], bv[1]);
      mma_bf16(o[nd + 1], a, bv[2], bv[3]);
    }
  }
}

// One warp's block of 32 positions starting at p_lo (tile rows p_lo - c_lo
// ...) for the 16 (row, head) pairs of m-tile mt: S = Q K^T, the block's
// row max m and sum l of exp(S - m), and O = P V, written to the block's
// partials.  a_row[qr] is query row qr's position: positions above it are
// masked.  R real (row, head) pairs; grp heads per row.
__device__ void attn_block_tc(int p_lo, int c_lo, int mt, int R, int grp, const int* a_row,
                              const __nv_bfloat16* q16, const __nv_bfloat16* kt, const __nv_bfloat16* vt, float* wm,
                              float* wl, float* wacc, int warp, int lane) {
  const int t = lane & 3;
  const int pb = p_lo - c_lo;                        // tile row of the block's first position
  uint32_t a[4][4];
  q_frags(q16, mt, lane, a);
  float s[4][4];
  block_scores(a, kt, pb, lane, s);
  // this thread's rows rA = r0 + g and rB = rA + 8, and their positions
  const int rA = mt * 16 + (lane >> 2), rB = rA + 8;
  const int aA = rA < R ? a_row[rA / grp] : -1;
  const int aB = rB < R ? a_row[rB / grp] : -1;
  float mA, mB, lA, lB;
  block_max(s, p_lo, t, aA, aB, mA, mB);
  block_exp(s, p_lo, t, aA, aB, mA, mB, lA, lB);
  float o[8][4];
  block_pv(s, vt, pb, lane, o);
  // partials of this block for the real rows
  if (rA < R) {
    if (t == 0) {
      wm[warp * R + rA] = mA;
      wl[warp * R + rA] = lA;
    }
    float* w = wacc + ((size_t)warp * R + rA) * kHeadDim;
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) *reinterpret_cast<float2*>(w + 8 * nd + 2 * t) = make_float2(o[nd][0], o[nd][1]);
  }
  if (rB < R) {
    if (t == 0) {
      wm[warp * R + rB] = mB;
      wl[warp * R + rB] = lB;
    }
    float* w = wacc + ((size_t)warp * R + rB) * kHeadDim;
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) *reinterpret_cast<float2*>(w + 8 * nd + 2 * t) = make_float2(o[nd][2], o[nd][3]);
  }
}

// One attention output: FP32 into attn_out, or rounded to BF16 into out16.
__device__ __forceinline__ void store_out(const AttnIO& io, size_t i, float v) {
  if (io.out16)
    static_cast<__nv_bfloat16*>(io.out16)[i] = __float2bfloat16_rn(v);
  else
    io.attn_out[i] = v;
}

// The K and V tile rows of positions c_lo .. c_lo + 255: ring entries for
// positions <= last (the fed token's own entry is written separately in
// decode), zeros above.
template <int NT = kTcThreads>
__device__ void load_tile(const Dims& D, const StreamDev& st, int layer, int g, int c_lo, int last,
                          __nv_bfloat16* kt, __nv_bfloat16* vt, int tid, int own) {
  const size_t koff = attn_plane_off(D, layer, g);
  const size_t voff = attn_plane_off(D, layer, D.hkv + g);
  const __nv_bfloat16* kv = static_cast<const __nv_bfloat16*>(st.kv);
  // 256 rows x 8 segments of 16 bytes, for K and for V: every load of this
  // thread is issued before the first store, so they are in flight together
  constexpr int kPer = kAttnChunk * 8 / NT;
  uint4 uk[kPer], uv[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = tid + i * NT;
    const int row = e >> 3, seg = e & 7;
    const int p = c_lo + row;
    uk[i] = uv[i] = make_uint4(0, 0, 0, 0);
    if (p <= last && p != own) {
      const size_t ri = (size_t)(p & (D.L - 1)) * kHeadDim + seg * 8;
      uk[i] = __ldg(reinterpret_cast<const uint4*>(kv + koff + ri));
      uv[i] = __ldg(reinterpret_cast<const uint4*>(kv + voff + ri));
    }
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = tid + i * NT;
    const int row = e >> 3, seg = e & 7;
    *reinterpret_cast<uint4*>(kt + row * kTileStride + seg * 8) = uk[i];
    *reinterpret_cast<uint4*>(vt + row * kTileStride + seg * 8) = uv[i];
  }
}

// Attention of rq query rows (rq = 1: a decode step, position = n_coded; else
// prefill rows with their positions in b.pos, k / v already in the ring) of
// one stream and KV head, by a cluster of S CTAs owning chunks rank,
// rank + S, ...
template <int S>
__global__ void __launch_bounds__(kTcThreads, 1) k_attn_tc(Dims D, Batch b, int layer, int rq, AttnIO io) {
  extern __shared__ float4 dyn4[];
  char* sm = reinterpret_cast<char*>(dyn4);
  const int rank = S > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int g = blockIdx.y, i0 = blockIdx.z * rq;
  if (i0 >= *b.nB) return;                         // uniform across the cluster
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = D.hq / D.hkv, R = rq * grp;
  constexpr int kd = kHeadDim / S;
  const TcLayout L(rq, grp, kd);
  __nv_bfloat16* q16 = reinterpret_cast<__nv_bfloat16*>(sm + L.q16);
  __nv_bfloat16* kt = reinterpret_cast<__nv_bfloat16*>(sm + L.kt);
  __nv_bfloat16* vt = reinterpret_cast<__nv_bfloat16*>(sm + L.vt);
  RowQv* qv = reinterpret_cast<RowQv*>(sm + L.rowq);
  int* a_row = reinterpret_cast<int*>(sm + L.arow);
  float* wm = reinterpret_cast<float*>(sm + L.wm);
  float* wl = reinterpret_cast<float*>(sm + L.wl);
  float* wacc = reinterpret_cast<float*>(sm + L.wacc);
  float* cf = reinterpret_cast<float*>(sm + L.cf);
  float* cM = reinterpret_cast<float*>(sm + L.cM);
  float* cL = reinterpret_cast<float*>(sm + L.cL);
  StreamDev& st = b.st[b.slots[i0]];
  const bool prefill = b.pos != nullptr;
  int a_max = -1;
  for (int r = 0; r < rq; ++r) a_max = max(a_max, prefill ? b.pos[i0 + r] : st.n_coded);
  if (a_max < 0) {                                 // prefill rows past the stream's end
    pdl_wait();
    pdl_trigger();
    for (int e = tid; e < rq * grp * kd; e += kTcThreads) {
      const int r = e / (grp * kd), h = (e / kd) % grp, dl = e % kd;
      store_out(io, (size_t)(i0 + r) * D.hq * kHeadDim + (g * grp + h) * kHeadDim + rank * kd + dl, 0.f);
    }
    return;                                        // uniform across the cluster
  }
  if (S > 1) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  const int start = prefill ? window_start_at(D, a_max) : window_start(D, st);
  const int nc_max = (a_max - start) / kAttnChunk + 1;
  if (tid < rq) a_row[tid] = prefill ? b.pos[i0 + tid] : st.n_coded;
  // decode: the first chunk's cached entries are final before the wait (the
  // fed token's own entry is added after); prefill: the append pass just
  // wrote this chunk of positions, so everything waits
  if (!prefill && rank < nc_max) load_tile(D, st, layer, g, start + rank * kAttnChunk, a_max, kt, vt, tid, a_max);
  pdl_wait();
  pdl_trigger();
  for (int r = 0; r < rq; ++r) {
    const int a = prefill ? b.pos[i0 + r] : st.n_coded;
    if (a < 0) continue;                           // uniform across the CTA
    attn_rope(D, a, tid, qv[r]);
    attn_qkv<1>(D, st, layer, i0 + r, g, a, !prefill && (nc_max - 1) % S == rank, tid, qv[r], io);
  }
  // BF16 query tile: row r * grp + h, padding rows zero
  for (int e = tid; e < kMaxTileRows * kHeadDim; e += kTcThreads) {
    const int row = e / kHeadDim, d = e % kHeadDim;
    float v = 0.f;
    if (row < R) {
      const int r = row / grp;
      if (a_row[r] >= 0) v = qv[r].qs[row % grp][d];
    }
    q16[row * kTileStride + d] = __float2bfloat16_rn(v);
  }
  auto dst = [&](int rk) -> char* {
    if (S == 1) return sm;
    return reinterpret_cast<char*>(cg::this_cluster().map_shared_rank(reinterpret_cast<float4*>(sm), rk));
  };
  if (S > 1) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
  const int nmt = (R + 15) / 16;
  for (int c = rank; c < nc_max; c += S) {
    const int c_lo = start + c * kAttnChunk;
    if (prefill || c != rank) {
      __syncthreads();                             // the previous chunk's tile is no longer read
      load_tile(D, st, layer, g, c_lo, a_max, kt, vt, tid, prefill ? -1 : a_max);
    }
    if (!prefill && a_max >= c_lo && a_max < c_lo + kAttnChunk && tid < kHeadDim) {
      // decode: the fed token's own entry, as the ring stores it
      kt[(a_max - c_lo) * kTileStride + tid] = __float2bfloat16_rn(qv[0].kn[tid]);
      vt[(a_max - c_lo) * kTileStride + tid] = __float2bfloat16_rn(qv[0].vn[tid]);
    }
    __syncthreads();
    {
      const int blk = warp & (kAttnWarps - 1), mt = warp / kAttnWarps;   // block of 32 positions, m-tile
      if (mt < nmt) attn_block_tc(c_lo + blk * 32, c_lo, mt, R, grp, a_row, q16, kt, vt, wm, wl, wacc, blk, lane);
    }
    __syncthreads();
    // per (row, head): the block factors exp(m_w - M), M and the sum, over
    // the blocks holding positions of this row (block order)
    for (int t = tid; t < R; t += kTcThreads) {
      const int a = a_row[t / grp];
      if (a < c_lo) continue;
      const int nblk = (min(c_lo + kAttnChunk, a + 1) - c_lo + 31) / 32;
      float M = -INFINITY;
      for (int w = 0; w < nblk; ++w) M = fmaxf(M, wm[w * R + t]);
      float l = 0.f;
      for (int w = 0; w < nblk; ++w) {
        const float f = expf(wm[w * R + t] - M);
        cf[t * kAttnWarps + w] = f;
        l = fmaf(wl[w * R + t], f, l);
      }
      cM[t] = M;
      cL[t] = l;
    }
    __syncthreads();
    for (int e = tid; e < R * kHeadDim; e += kTcThreads) {
      const int t = e / kHeadDim, dd = e % kHeadDim, r = t / grp, h = t % grp;
      const int a = a_row[r];
      if (a < c_lo) continue;
      const int nblk = (min(c_lo + kAttnChunk, a + 1) - c_lo + 31) / 32;
      float o = 0.f;
      for (int w = 0; w < nblk; ++w) o = fmaf(wacc[((size_t)w * R + t) * kHeadDim + dd], cf[t * kAttnWarps + w], o);
      char* tg = dst(dd / kd);
      const int rc = (r * kAttnMaxChunks + c) * grp + h;
      reinterpret_cast<float*>(tg + L.racc)[rc * kd + dd % kd] = o;
      if (dd % kd == 0) {
        reinterpret_cast<float*>(tg + L.rm)[rc] = cM[t];
        reinterpret_cast<float*>(tg + L.rl)[rc] = cL[t];
      }
    }
  }
  if (S > 1) cg::this_cluster().sync();            // every chunk's partial has arrived
  else __syncthreads();
  const float* rm = reinterpret_cast<const float*>(sm + L.rm);
  const float* rl = reinterpret_cast<const float*>(sm + L.rl);
  const float* racc = reinterpret_cast<const float*>(sm + L.racc);
  float* mf = reinterpret_cast<float*>(sm + L.mf);
  float* mL = reinterpret_cast<float*>(sm + L.mL);
  // every (row, head): the chunk factors, then every output dim
  for (int t = tid; t < R; t += kTcThreads) {
    const int r = t / grp, h = t % grp;
    const int a = a_row[r];
    const int nc = a < 0 ? 0 : (a - start) / kAttnChunk + 1;
    float M = -INFINITY;
    for (int c = 0; c < nc; ++c) M = fmaxf(M, rm[(r * kAttnMaxChunks + c) * grp + h]);
    float l = 0.f;
    for (int c = 0; c < nc; ++c) {
      const int rc = (r * kAttnMaxChunks + c) * grp + h;
      const float f = expf(rm[rc] - M);
      mf[t * kAttnMaxChunks + c] = f;
      l = fmaf(rl[rc], f, l);
    }
    mL[t] = l;
  }
  __syncthreads();
  for (int e = tid; e < R * kd; e += kTcThreads) {
    const int t = e / kd, dl = e % kd, r = t / grp, h = t % grp;
    const int a = a_row[r];
    const int nc = a < 0 ? 0 : (a - start) / kAttnChunk + 1;
    float o = 0.f;
    for (int c = 0; c < nc; ++c)
      o = fmaf(racc[((r * kAttnMaxChunks + c) * grp + h) * kd + dl], mf[t * kAttnMaxChunks + c], o);
    store_out(io, (size_t)(i0 + r) * D.hq * kHeadDim + (g * grp + h) * kHeadDim + rank * kd + dl,
              nc ? o / mL[t] : 0.f);
  }
}

// ----------------------------------------------------------- prefill rows
// Prefill attention of kPfRows consecutive positions of one stream and KV
// head: the arithmetic of k_attn_tc row by row, organised for many rows.
// Each warp owns one m-tile of 16 (row, head) pairs and walks the blocks of
// a chunk itself: a first pass takes every block's masked row maxima (so
// the chunk's maximum M_c); the second recomputes the block's scores, forms
// exp(S - m_w), its sum and P V as k_attn_tc does, and folds the block into
// the chunk's sums in block order with the factors exp(m_w - M_c).  The
// chunk partials then go to the cluster rank owning their output dims, and
// the chunks are merged in order, as in k_attn_tc: a row gets the bits the
// decode kernel gives it alone.  Chunk c of the window is on rank c % kPfS.
constexpr int kPfRows = 32;                          // positions per CTA
constexpr int kPfS = 8;                              // CTAs per cluster
constexpr int kPfThreads = 256;                      // 8 warps: 8 m-tiles of 16 (row, head) pairs
constexpr int kPfKd = kHeadDim / kPfS;               // output dims merged per rank
constexpr int kPfTileRows = kPfThreads / 32 * 16;

// The A fragments of m-tile mt straight from the QKV rows: the rotated,
// 1/8-scaled query of (row, head) pair q = r grp + h rounded to BF16, as
// attn_qkv and the tile of k_attn_tc form it.  The thread holds pairs
// g = lane / 4 and g + 8, dims 16 kk + 2 t (+1) and 16 kk + 8 + 2 t (+1); a
// rotation pair (dd, dd + 32) lands in k-steps kk and kk + 2 of one thread.
__device__ __forceinline__ void q_frags_rows(const Dims& D, const AttnIO& io, int i0, int g, int grp, int R,
                                             const int* a_row, int mt, int lane, uint32_t (&a)[4][4]) {
  const int t = lane & 3;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int q = mt * 16 + (lane >> 2) + 8 * half;
    float v[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) v[kk][0] = v[kk][1] = v[kk][2] = v[kk][3] = 0.f;
    const int r = q / grp, pa = q < R ? a_row[r] : -1;
    if (pa >= 0) {
      const float* src = io.qkv + (size_t)(i0 + r) * D.qkv_rows + (g * grp + q % grp) * kHeadDim;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int dd = 16 * kk + 2 * t + (j & 1) + 8 * (j >> 1);
          const float2 rr = rope_rotate(__ldcg(src + dd), __ldcg(src + dd + kHeadDim / 2), rope_cs(D, pa, dd));
          v[kk][j] = rr.x * 0.125f;
          v[kk + 2][j] = rr.y * 0.125f;
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      a[kk][half] = pack_bf16(v[kk][0], v[kk][1]);
      a[kk][2 + half] = pack_bf16(v[kk][2], v[kk][3]);
    }
  }
}

struct PfLayout {
  int kt, vt, arow, rm, rl, racc, mf, mL, total;
  __host__ __device__ PfLayout(int grp) {
    const int R = kPfRows * grp;
    int o = 0;
    auto take = [&](int bytes) {
      const int at = o;
      o += (bytes + 15) & ~15;
      return at;
    };
    kt = take(kAttnChunk * kTileStride * 2);
    vt = take(kAttnChunk * kTileStride * 2);
    arow = take(kPfRows * 4);
    rm = take(R * kAttnMaxChunks * 4);
    rl = take(R * kAttnMaxChunks * 4);
    racc = take(R * kAttnMaxChunks * kPfKd * 4);
    mf = take(R * kAttnMaxChunks * 4);
    mL = take(R * 4);
    total = o;
  }
};

__global__ void __launch_bounds__(kPfThreads, 2)
    k_attn_pf(Dims D, Batch b, int layer, AttnIO io) {
  extern __shared__ float4 dyn4[];
  char* sm = reinterpret_cast<char*>(dyn4);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int g = blockIdx.y, i0 = blockIdx.z * kPfRows;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = D.hq / D.hkv, R = kPfRows * grp;
  const PfLayout Ly(grp);
  __nv_bfloat16* kt = reinterpret_cast<__nv_bfloat16*>(sm + Ly.kt);
  __nv_bfloat16* vt = reinterpret_cast<__nv_bfloat16*>(sm + Ly.vt);
  int* a_row = reinterpret_cast<int*>(sm + Ly.arow);
  float* rm = reinterpret_cast<float*>(sm + Ly.rm);
  float* rl = reinterpret_cast<float*>(sm + Ly.rl);
  float* racc = reinterpret_cast<float*>(sm + Ly.racc);
  float* mf = reinterpret_cast<float*>(sm + Ly.mf);
  float* mL = reinterpret_cast<float*>(sm + Ly.mL);
  // the append pass just wrote these positions' k, v: everything waits
  pdl_wait();
  pdl_trigger();
  if (i0 >= *b.nB) return;                         // uniform across the cluster
  const StreamDev& st = b.st[b.slots[i0]];
  if (tid < kPfRows) a_row[tid] = b.pos[i0 + tid];
  __syncthreads();
  int a_max = -1;
  for (int r = 0; r < kPfRows; ++r) a_max = max(a_max, a_row[r]);
  auto out_at = [&](int r, int h, int d) -> size_t {
    return (size_t)(i0 + r) * D.hq * kHeadDim + (g * grp + h) * kHeadDim + d;
  };
  if (a_max < 0) {                                 // rows past the stream's end
    for (int e = tid; e < R * kPfKd; e += kPfThreads) {
      const int t = e / kPfKd;
      store_out(io, out_at(t / grp, t % grp, rank * kPfKd + e % kPfKd), 0.f);
    }
    return;                                        // uniform across the cluster
  }
  const int start = window_start_at(D, a_max);
  const int nc_max = (a_max - start) / kAttnChunk + 1;
  const int mt = warp, t4 = lane & 3;
  const int rA = mt * 16 + (lane >> 2), rB = rA + 8;
  const int aA = rA < R ? a_row[rA / grp] : -1;
  const int aB = rB < R ? a_row[rB / grp] : -1;
  int aW = max(aA, aB);                            // the warp's last position
#pragma unroll
  for (int o = 16; o; o >>= 1) aW = max(aW, __shfl_xor_sync(0xffffffffu, aW, o));
  uint32_t qa[4][4];
  q_frags_rows(D, io, i0, g, grp, R, a_row, mt, lane, qa);
  for (int c = rank; c < nc_max; c += kPfS) {
    const int c_lo = start + c * kAttnChunk;
    if (c != rank) __syncthreads();                // the previous chunk's tile is no longer read
    load_tile<kPfThreads>(D, st, layer, g, c_lo, a_max, kt, vt, tid, -1);
    __syncthreads();
    if (aW < c_lo) continue;                       // no row of this warp reaches the chunk
    const int nblk = min(kAttnWarps, (aW - c_lo) / 32 + 1);
    // pass 1: the chunk's maximum of each row over its blocks
    float MA = -INFINITY, MB = -INFINITY;
    for (int w = 0; w < nblk; ++w) {
      const int p_lo = c_lo + 32 * w;
      float s[4][4], mA, mB;
      block_scores(qa, kt, p_lo - c_lo, lane, s);
      block_max(s, p_lo, t4, aA, aB, mA, mB);
      if (p_lo <= aA) MA = fmaxf(MA, mA);
      if (p_lo <= aB) MB = fmaxf(MB, mB);
    }
    // pass 2: every block's partials, folded in block order
    float lcA = 0.f, lcB = 0.f, oc[8][4];
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) oc[nd][0] = oc[nd][1] = oc[nd][2] = oc[nd][3] = 0.f;
    for (int w = 0; w < nblk; ++w) {
      const int p_lo = c_lo + 32 * w;
      float s[4][4], mA, mB, lA, lB, o[8][4];
      block_scores(qa, kt, p_lo - c_lo, lane, s);
      block_max(s, p_lo, t4, aA, aB, mA, mB);
      block_exp(s, p_lo, t4, aA, aB, mA, mB, lA, lB);
      block_pv(s, vt, p_lo - c_lo, lane, o);
      if (p_lo <= aA) {
        const float f = expf(mA - MA);
        lcA = fmaf(lA, f, lcA);
#pragma unroll
        for (int nd = 0; nd < 8; ++nd) {
          oc[nd][0] = fmaf(o[nd][0], f, oc[nd][0]);
          oc[nd][1] = fmaf(o[nd][1], f, oc[nd][1]);
        }
      }
      if (p_lo <= aB) {
        const float f = expf(mB - MB);
        lcB = fmaf(lB, f, lcB);
#pragma unroll
        for (int nd = 0; nd < 8; ++nd) {
          oc[nd][2] = fmaf(o[nd][2], f, oc[nd][2]);
          oc[nd][3] = fmaf(o[nd][3], f, oc[nd][3]);
        }
      }
    }
    // the chunk's partials to the rank owning each output dim (nd = rank)
    static_assert(kPfKd == 8, "one n-tile of 8 dims per rank");
    if (rA < R && c_lo <= aA) {
      const int rc = rA * kAttnMaxChunks + c;
#pragma unroll
      for (int nd = 0; nd < 8; ++nd) {
        char* tg = reinterpret_cast<char*>(cl.map_shared_rank(reinterpret_cast<float4*>(sm), nd));
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(tg + Ly.racc) + rc * kPfKd + 2 * t4) =
            make_float2(oc[nd][0], oc[nd][1]);
        if (t4 == 0) {
          reinterpret_cast<float*>(tg + Ly.rm)[rc] = MA;
          reinterpret_cast<float*>(tg + Ly.rl)[rc] = lcA;
        }
      }
    }
    if (rB < R && c_lo <= aB) {
      const int rc = rB * kAttnMaxChunks + c;
#pragma unroll
      for (int nd = 0; nd < 8; ++nd) {
        char* tg = reinterpret_cast<char*>(cl.map_shared_rank(reinterpret_cast<float4*>(sm), nd));
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(tg + Ly.racc) + rc * kPfKd + 2 * t4) =
            make_float2(oc[nd][2], oc[nd][3]);
        if (t4 == 0) {
          reinterpret_cast<float*>(tg + Ly.rm)[rc] = MB;
          reinterpret_cast<float*>(tg + Ly.rl)[rc] = lcB;
        }
      }
    }
  }
  cl.sync();                                       // every chunk's partial has arrived
  // every (row, head): the chunk factors, then this rank's output dims
  for (int t = tid; t < R; t += kPfThreads) {
    const int a = a_row[t / grp];
    const int nc = a < 0 ? 0 : (a - start) / kAttnChunk + 1;
    float M = -INFINITY;
    for (int c = 0; c < nc; ++c) M = fmaxf(M, rm[t * kAttnMaxChunks + c]);
    float l = 0.f;
    for (int c = 0; c < nc; ++c) {
      const float f = expf(rm[t * kAttnMaxChunks + c] - M);
      mf[t * kAttnMaxChunks + c] = f;
      l = fmaf(rl[t * kAttnMaxChunks + c], f, l);
    }
    mL[t] = l;
  }
  __syncthreads();
  for (int e = tid; e < R * kPfKd; e += kPfThreads) {
    const int t = e / kPfKd, dl = e % kPfKd;
    const int a = a_row[t / grp];
    const int nc = a < 0 ? 0 : (a - start) / kAttnChunk + 1;
    float o = 0.f;
    for (int c = 0; c < nc; ++c) o = fmaf(racc[(t * kAttnMaxChunks + c) * kPfKd + dl], mf[t * kAttnMaxChunks + c], o);
    store_out(io, out_at(t / grp, t % grp, rank * kPfKd + dl), nc ? o / mL[t] : 0.f);
  }
}

template <int S>
cudaError_t launch_tc_s(const Dims& D, const Batch& b, int layer, int rq, const AttnIO& io, cudaStream_t s) {
  const size_t smem = TcLayout(rq, D.hq / D.hkv, kHeadDim / S).total;
  dim3 grid(S, D.hkv, b.Bmax / rq);
  return launch_kernel_cluster(k_attn_tc<S>, grid, dim3(kTcThreads), smem, s, D.pdl, S, D, b, layer, rq, io);
}

template <int S>
cudaError_t prepare_tc_s(int grp) {
  int rq = kMaxRowsTc;
  while (rq > 1 && TcLayout(rq, grp, kHeadDim / S).total > 220 * 1024) rq /= 2;
  return cudaFuncSetAttribute(k_attn_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcLayout(rq, grp, kHeadDim / S).total);
}

}  // namespace

size_t attn_tc_smem(int rq, int grp, int S) { return TcLayout(rq, grp, kHeadDim / S).total; }

cudaError_t prepare_attn_tc(const Dims& D) {
  const int grp = D.hq / D.hkv;
  cudaError_t e = prepare_tc_s<1>(grp);
  if (e == cudaSuccess) e = prepare_tc_s<2>(grp);
  if (e == cudaSuccess) e = prepare_tc_s<4>(grp);
  if (e == cudaSuccess) e = prepare_tc_s<8>(grp);
  return e;
}

bool attn_pf_fits(const Dims& D, const Batch& b) {
  const int grp = D.hq / D.hkv;
  return b.pos && b.pm % kPfRows == 0 && b.Bmax % kPfRows == 0 && kPfRows * grp <= kPfTileRows &&
         PfLayout(grp).total <= 227 * 1024;
}

cudaError_t launch_attn_pf(const Dims& D, const Batch& b, int layer, const float* qkv, float* attn_out,
                           void* out16, cudaStream_t s) {
  const AttnIO io{qkv, attn_out, out16};
  static bool attr = false;                        // the kernel's shared-memory limit: once per process
  const size_t smem = PfLayout(D.hq / D.hkv).total;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_attn_pf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)PfLayout(kMaxGroup).total);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(kPfS, D.hkv, b.Bmax / kPfRows);
  return launch_kernel_cluster(k_attn_pf, grid, dim3(kPfThreads), smem, s, D.pdl, kPfS, D, b, layer, io);
}

cudaError_t launch_attn_tc(const Dims& D, const Batch& b, int layer, int rq, int S, const float* qkv,
                           float* attn_out, void* out16, cudaStream_t s) {
  const AttnIO io{qkv, attn_out, out16};
  switch (S) {
    case 1: return launch_tc_s<1>(D, b, layer, rq, io, s);
    case 2: return launch_tc_s<2>(D, b, layer, rq, io, s);
    case 4: return launch_tc_s<4>(D, b, layer, rq, io, s);
    case 8: return launch_tc_s<8>(D, b, layer, rq, io, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nc
