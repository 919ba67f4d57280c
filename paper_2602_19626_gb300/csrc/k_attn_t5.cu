// Decode and prefill attention over a BF16 KV cache on the tcgen05 tensor
// cores, accumulators in tensor memory (Sec. 3.2 model, Sec. 3.9 sliding
// window).
//
// A tile is up to 128 (query row, head) pairs of one stream and KV head: the
// RT = 128 / grp rows of a group of consecutive positions (one row in a
// decode step) times the grp query heads sharing the KV head, pair
// p = r grp + h.  The pairs are the MMA's M = 128 rows, so each pair's
// products depend on its own query alone: a row computed alone (decode) and
// among the rows of a prefill gives the same bits.
//
// The window [start, a] of a row is cut into chunks of 256 positions (chunk
// c = [start + 256 c, ...)), a chunk into four blocks of 64.  Cluster rank c
// of the tile's S CTAs owns chunk c:
//   - the 256 K and V rows of the chunk go to shared memory in the 128-byte
//     swizzle layout (16-byte asynchronous copies; positions past the tile's
//     last row are zero), the pairs' rotated 1/8-scaled queries, rounded to
//     BF16, beside them;
//   - one thread issues S_b = Q K_b^T for every block b (M 128, N 64, four K
//     steps of 16 head dims) into tensor memory;
//   - the pair's thread reads its scores back (one TMEM lane per pair),
//     masks positions above its row's, and takes the block maximum m_b,
//     e = 2^(s log2 e - m_b log2 e) (PTX ex2.approx), their sum l_b in FP32
//     (eight interleaved partial sums, then a fixed tree) and P_b = BF16(e)
//     into shared memory (two alternating buffers in the K tile's place, which
//     the score products no longer read);
//   - O_b = P_b V_b (M 128, N 64, four K steps of 16 positions, V read
//     MN-major straight from the tile) goes to the columns S_b held;
//   - the chunk's (M_c, l_c, O_c) = (max m_b, sum l_b f_b, sum O_b f_b),
//     f_b = exp(m_b - M_c), blocks in order, a block past the row absent;
//   - after a cluster barrier (every rank done with its query and key tiles)
//     rank k receives, in that memory, every chunk's (O_c, M_c, l_c) of the
//     pairs 128 k / S .. 128 (k + 1) / S - 1 (remote stores), and after a
//     second barrier merges them over the chunks in order:
//     O = sum O_c f_c / sum l_c f_c with f_c = exp(M_c - max M_c).
// The arithmetic of a row is fixed by its window alone.  In a decode step the
// rank of the chunk holding the fed position a rotates the new k at a, rounds
// k and v to BF16, appends them to the ring and to its tile; a prefill's rows
// were appended by k_kv_append (the same rotation code) before this kernel.
// About 92 KB of shared memory and 256 TMEM columns: two CTAs per SM; the
// clusters are launched with the load-balancing placement, so that a
// cluster's CTAs may share SMs (spread placement admits about 15 clusters of
// 8 at a time).
//
// Every wait on an mbarrier is bounded; a wait that gives up raises
// ST_TIMEOUT in the stream's status word, skips the remaining products and,
// before the tensor memory is freed, waits (with the same bound) for the
// products already issued.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "model_dev.cuh"
#include "tc5.cuh"

namespace cg = cooperative_groups;

namespace nc {

namespace {

using namespace dev;
using namespace tc5;

constexpr int kT5Threads = 128;              // 4 warps; warp w reads TMEM lanes 32 w .. 32 w + 31
constexpr int kT5Pairs = 128;                // MMA M: (row, head) pairs per tile
constexpr int kT5Chunk = 256;                // positions per chunk (one CTA)
constexpr int kT5Block = 64;                 // positions per block (N of the scores, K of P V)
constexpr int kT5Blocks = kT5Chunk / kT5Block;
constexpr int kT5MaxRanks = 8;               // chunks of a window of at most 2,048 positions
constexpr int kRowB = 128;                   // bytes of one swizzled row: 64 BF16
constexpr uint32_t kT5Cols = 256;            // TMEM columns: S_b, then O_b, at 64 b

// Shared memory, byte offsets from a 1024-byte aligned base; `cs` holds the
// (cos, sin) of the tile rows' positions, RT rows of 32 pairs.
struct T5Layout {
  int q, k, v, cs, bars, slot, arow, total;
  // the inbox, after the first cluster barrier, in the query and key tiles:
  // [S chunks][128 / S pairs][68] floats (O_c[64], M_c, l_c, padding)
  int inbox;
  __host__ __device__ explicit T5Layout(int rt) {
    q = 0;                                   // [128 pairs][128 B]
    k = q + kT5Pairs * kRowB;                // [256 positions][128 B]; later P_0, P_1 (16 KB each)
    v = k + kT5Chunk * kRowB;                // [256 positions][128 B]
    cs = v + kT5Chunk * kRowB;               // [rt][32] float2
    bars = cs + rt * 32 * 8;                 // 6 mbarriers
    slot = bars + 64;                        // TMEM address
    arow = slot + 16;                        // [128] row positions
    total = arow + kT5Pairs * 4;
    inbox = 0;
  }
};
constexpr int kInboxRow = kHeadDim + 4;      // floats per (chunk, pair) record
static_assert(kT5Pairs * kInboxRow * 4 <= (kT5Pairs + kT5Chunk) * kRowB, "the inbox fits the query and key tiles");

constexpr float kLog2e = 1.4426950408889634f;

// 2^x (PTX ex2.approx, subnormal results flushed to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float exp_fast(float x) { return ex2_approx(__fmul_rn(x, kLog2e)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Byte offset of 16-byte segment `seg` of row `row` in the 128-byte swizzle
// layout (rows of 128 bytes, 8-row atoms at 1024-byte aligned addresses).
__device__ __forceinline__ int swz(int row, int seg) { return row * kRowB + ((seg ^ (row & 7)) << 4); }

__device__ __forceinline__ void cp_async16(uint8_t* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The 256 K and V rows of positions c_lo .. c_lo + 255 from the ring:
// positions <= last (other than `own`, which the caller writes) copied,
// the others zero.
__device__ void load_kv_tile(const Dims& D, const StreamDev& st, int layer, int g, int c_lo, int last, int own,
                             uint8_t* kt, uint8_t* vt, int tid) {
  const __nv_bfloat16* kv = static_cast<const __nv_bfloat16*>(st.kv);
  const __nv_bfloat16* kp = kv + attn_plane_off(D, layer, g);
  const __nv_bfloat16* vp = kv + attn_plane_off(D, layer, D.hkv + g);
  for (int e = tid; e < kT5Chunk * 8; e += kT5Threads) {
    const int row = e >> 3, seg = e & 7;
    const int p = c_lo + row;
    if (p == own) continue;                        // written by the caller
    uint8_t* dk = kt + swz(row, seg);
    uint8_t* dv = vt + swz(row, seg);
    if (p <= last) {
      const size_t ri = (size_t)(p & (D.L - 1)) * kHeadDim + seg * 8;
      cp_async16(dk, kp + ri);
      cp_async16(dv, vp + ri);
    } else {
      *reinterpret_cast<uint4*>(dk) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(dv) = make_uint4(0, 0, 0, 0);
    }
  }
}

// Softmax of one 64-position block for this thread's pair: the block
// maximum m over the first `nvalid` columns of the scores at TMEM column
// `col`, the numerators e = 2^(s log2 e - m log2 e) rounded to BF16 into the
// pair's row of the P tile, and their FP32 sum.  nvalid = 0 writes a zero row
// (an absent block).
__device__ __forceinline__ void block_softmax(uint32_t tmem_lane, uint32_t col, int nvalid, uint8_t* ptile, int pair,
                                              float& m_out, float& l_out) {
  uint32_t r[2][32];
  tmem_ld32_nowait(tmem_lane + col, r[0]);
  tmem_ld32_nowait(tmem_lane + col + 32, r[1]);
  tmem_wait_ld();
  float s[kT5Block];
#pragma unroll
  for (int i = 0; i < kT5Block; ++i) s[i] = __uint_as_float(r[i >> 5][i & 31]);
  float m = -INFINITY;
  if (nvalid == kT5Block) {
#pragma unroll
    for (int i = 0; i < kT5Block; ++i) m = fmaxf(m, s[i]);
  } else {
#pragma unroll
    for (int i = 0; i < kT5Block; ++i)
      if (i < nvalid) m = fmaxf(m, s[i]);
  }
  float acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = 0.f;
  const float mb = nvalid > 0 ? -__fmul_rn(m, kLog2e) : 0.f;
  float e[kT5Block];
  if (nvalid == kT5Block) {
#pragma unroll
    for (int i = 0; i < kT5Block; ++i) e[i] = ex2_approx(__fmaf_rn(s[i], kLog2e, mb));
  } else {
#pragma unroll
    for (int i = 0; i < kT5Block; ++i) e[i] = i < nvalid ? ex2_approx(__fmaf_rn(s[i], kLog2e, mb)) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < kT5Block; ++i) acc[i & 7] = __fadd_rn(acc[i & 7], e[i]);
#pragma unroll
  for (int sg = 0; sg < 8; ++sg) {
    const uint4 u = make_uint4(pack_bf16(e[8 * sg], e[8 * sg + 1]), pack_bf16(e[8 * sg + 2], e[8 * sg + 3]),
                               pack_bf16(e[8 * sg + 4], e[8 * sg + 5]), pack_bf16(e[8 * sg + 6], e[8 * sg + 7]));
    *reinterpret_cast<uint4*>(ptile + swz(pair, sg)) = u;
  }
  m_out = m;
  l_out = __fadd_rn(__fadd_rn(__fadd_rn(acc[0], acc[1]), __fadd_rn(acc[2], acc[3])),
                    __fadd_rn(__fadd_rn(acc[4], acc[5]), __fadd_rn(acc[6], acc[7])));
}

template <int S>
__global__ void __launch_bounds__(kT5Threads, 2) k_attn_t5(Dims D, Batch b, int layer, int tps, AttnIO io) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int grp = D.hq / D.hkv;
  const int RT = kT5Pairs / grp;                   // rows per tile
  const T5Layout Ly(RT);
  uint8_t* qt = sm + Ly.q;
  uint8_t* kt = sm + Ly.k;
  uint8_t* vt = sm + Ly.v;
  float2* cs = reinterpret_cast<float2*>(sm + Ly.cs);
  float* inbox = reinterpret_cast<float*>(sm + Ly.inbox);
  uint64_t* bar_s = reinterpret_cast<uint64_t*>(sm + Ly.bars);    // every score product
  uint64_t* bar_o = bar_s + 1;                                     // [4] P V of block b
  uint64_t* bar_done = bar_s + 5;                                  // every product issued
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Ly.slot);
  int* a_row = reinterpret_cast<int*>(sm + Ly.arow);
  constexpr int kPR = kT5Pairs / S;                // pairs merged by one rank

  const int rank = S > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int g = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool prefill = b.pos != nullptr;
  int row0, nr;
  if (prefill) {
    const int j = blockIdx.z / tps, sub = blockIdx.z % tps;
    row0 = j * b.pm + sub * RT;
    nr = min(RT, b.pm - sub * RT);
  } else {
    row0 = blockIdx.z;
    nr = 1;
  }
  // the row count and the rows' slots and positions were written at least
  // two launches back: read before the wait (uniform across the cluster)
  if (row0 >= *b.nB) return;
  StreamDev& st = b.st[b.slots[row0]];
  if (tid < nr) a_row[tid] = prefill ? b.pos[row0 + tid] : st.n_coded;
  __syncthreads();
  int a_max = -1;
  for (int r = 0; r < nr; ++r) a_max = max(a_max, a_row[r]);
  const int start = a_max < 0 ? 0 : prefill ? window_start_at(D, a_max) : window_start(D, st);
  const int nch = a_max < 0 ? 0 : (a_max - start) / kT5Chunk + 1;
  const bool has_chunk = rank < nch;
  const int c_lo = start + rank * kT5Chunk;
  const int nblk = has_chunk ? min(kT5Blocks, (a_max - c_lo) / kT5Block + 1) : 0;
  const int npairs = nr * grp;
  // this thread's pair and its row's position (-1: padding or past the stream's end)
  const int my_r = tid / grp, my_h = tid % grp;
  const int my_a = tid < npairs ? a_row[my_r] : -1;
  const bool mine = 32 * warp < npairs;            // warp-uniform: the warp holds real pairs

  if (tid == 0) {
    for (int i = 0; i < 6; ++i) mbar_init(bar_s + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (has_chunk && warp == 0) tmem_alloc(tmem_slot, kT5Cols);
  // decode: the cached entries (positions below a) were appended by earlier
  // steps and may be loaded before the wait; a prefill's rows were appended
  // by the launch just before
  if (has_chunk && !prefill) load_kv_tile(D, st, layer, g, c_lo, a_max, a_max, kt, vt, tid);
  pdl_wait();
  pdl_trigger();
  if (has_chunk && prefill) load_kv_tile(D, st, layer, g, c_lo, a_max, -1, kt, vt, tid);

  bool ok = true;
  float Mc = -INFINITY, Lc = 0.f;
  float oc[kHeadDim];
#pragma unroll
  for (int d = 0; d < kHeadDim; ++d) oc[d] = 0.f;
  if (has_chunk) {
    // (cos, sin) of every tile row's position
#pragma unroll 12
    for (int e = tid; e < nr * (kHeadDim / 2); e += kT5Threads) {
      const int r = e / (kHeadDim / 2), dd = e % (kHeadDim / 2);
      if (a_row[r] >= 0) cs[e] = rope_cs(D, a_row[r], dd);
    }
    // decode: the fed token's k (rotated at a) and v, rounded to BF16, into
    // the ring and into this tile (the rank whose chunk holds a)
    if (!prefill && rank == nch - 1 && tid < kHeadDim) {
      const float* row = io.qkv + (size_t)row0 * D.qkv_rows;
      const int a = a_max, R = a - c_lo;
      const size_t ri = (size_t)(a & (D.L - 1)) * kHeadDim;
      if (tid < kHeadDim / 2) {                    // dims tid and tid + 32 of k
        const float* src = row + D.hq * kHeadDim + g * kHeadDim;
        const float2 rr = rope_rotate(__ldcg(src + tid), __ldcg(src + tid + kHeadDim / 2), rope_cs(D, a, tid));
        __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv) + attn_plane_off(D, layer, g) + ri;
        const __nv_bfloat16 k0 = __float2bfloat16_rn(rr.x), k1 = __float2bfloat16_rn(rr.y);
        kv[tid] = k0;
        kv[tid + kHeadDim / 2] = k1;
        *reinterpret_cast<__nv_bfloat16*>(kt + swz(R, tid >> 3) + (tid & 7) * 2) = k0;
        *reinterpret_cast<__nv_bfloat16*>(kt + swz(R, (tid + 32) >> 3) + (tid & 7) * 2) = k1;
      } else {                                     // dims d0, d0 + 1 of v
        const int d0 = 2 * (tid - kHeadDim / 2);
        const float* src = row + (D.hq + D.hkv) * kHeadDim + g * kHeadDim;
        __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv) + attn_plane_off(D, layer, D.hkv + g) + ri;
        const __nv_bfloat16 v0 = __float2bfloat16_rn(__ldcg(src + d0)), v1 = __float2bfloat16_rn(__ldcg(src + d0 + 1));
        kv[d0] = v0;
        kv[d0 + 1] = v1;
        *reinterpret_cast<__nv_bfloat16*>(vt + swz(R, d0 >> 3) + (d0 & 7) * 2) = v0;
        *reinterpret_cast<__nv_bfloat16*>(vt + swz(R, (d0 + 1) >> 3) + ((d0 + 1) & 7) * 2) = v1;
      }
    }
    __syncthreads();                               // the rotation table is complete
    // the pairs' rotated, 1/8-scaled queries in BF16 (padding rows zero)
    if (mine) {
      uint32_t w[kHeadDim / 2];
#pragma unroll
      for (int i = 0; i < kHeadDim / 2; ++i) w[i] = 0u;
      if (my_a >= 0) {
        const float4* src =
            reinterpret_cast<const float4*>(io.qkv + (size_t)(row0 + my_r) * D.qkv_rows + (g * grp + my_h) * kHeadDim);
        float x[kHeadDim];
#pragma unroll
        for (int i = 0; i < kHeadDim / 4; ++i) {
          const float4 u = __ldcg(src + i);
          x[4 * i] = u.x;
          x[4 * i + 1] = u.y;
          x[4 * i + 2] = u.z;
          x[4 * i + 3] = u.w;
        }
        const float2* csr = cs + my_r * (kHeadDim / 2);
        float qv[kHeadDim];
#pragma unroll
        for (int dd = 0; dd < kHeadDim / 2; ++dd) {
          const float2 rr = rope_rotate(x[dd], x[dd + kHeadDim / 2], csr[dd]);
          qv[dd] = rr.x * 0.125f;   // the 1/sqrt(64) score scale is a power of two: exact
          qv[dd + kHeadDim / 2] = rr.y * 0.125f;
        }
#pragma unroll
        for (int i = 0; i < kHeadDim / 2; ++i) w[i] = pack_bf16(qv[2 * i], qv[2 * i + 1]);
      }
#pragma unroll
      for (int seg = 0; seg < 8; ++seg)
        *reinterpret_cast<uint4*>(qt + swz(tid, seg)) = make_uint4(w[4 * seg], w[4 * seg + 1], w[4 * seg + 2], w[4 * seg + 3]);
    }
    cp_async_wait_all();
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
    if (tid == 0) {
      const uint32_t ids = idesc(1, kT5Pairs, kT5Block);
      for (int bb = 0; bb < nblk; ++bb) {
#pragma unroll
        for (int k = 0; k < kHeadDim / 16; ++k)
          mma_issue(1, tmem + kT5Block * bb, sdesc_sw128(smem_u32(qt) + 32 * k),
                    sdesc_sw128(smem_u32(kt + bb * kT5Block * kRowB) + 32 * k), ids, k ? 1u : 0u);
      }
      mma_commit(bar_s);
    }
    __syncwarp();
    // every score product done: the key tile holds the P buffers from here
    ok = __syncthreads_and(mbar_wait(bar_s, 0));
    fence_after_sync();
    float mb[kT5Blocks], lb[kT5Blocks];
    int nv[kT5Blocks];
#pragma unroll
    for (int bb = 0; bb < kT5Blocks; ++bb) {
      mb[bb] = -INFINITY;
      lb[bb] = 0.f;
      const int blo = c_lo + bb * kT5Block;
      nv[bb] = bb < nblk && my_a >= blo ? min(kT5Block, my_a - blo + 1) : 0;
    }
    for (int bb = 0; bb < nblk; ++bb) {
      uint8_t* pt = kt + (bb & 1) * (kT5Pairs * kRowB);
      if (bb >= 2) ok = __syncthreads_and(ok && mbar_wait(bar_o + bb - 2, 0));   // P buffer bb & 1 free
      if (ok && mine) block_softmax(tlane, kT5Block * bb, nv[bb], pt, tid, mb[bb], lb[bb]);
      fence_proxy_async();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid == 0 && ok) {
        // O_b into the columns of S_b (every thread has read S_b)
        const uint32_t ido = idesc(1, kT5Pairs, kHeadDim, 1);
#pragma unroll
        for (int s = 0; s < kT5Block / 16; ++s)
          mma_issue(1, tmem + kT5Block * bb, sdesc_sw128(smem_u32(pt) + 32 * s),
                    sdesc_sw128_mn(smem_u32(vt + (bb * kT5Block + 16 * s) * kRowB)), ido, s ? 1u : 0u);
        mma_commit(bar_o + bb);
      }
      __syncwarp();
    }
    // the chunk's partials: blocks in order, a block past the row absent
#pragma unroll
    for (int bb = 0; bb < kT5Blocks; ++bb)
      if (nv[bb] > 0) Mc = fmaxf(Mc, mb[bb]);
    for (int bb = 0; bb < nblk; ++bb) {
      ok = __syncthreads_and(ok && mbar_wait(bar_o + bb, 0));
      fence_after_sync();
      if (!ok || !mine) continue;
      const bool pres = nv[bb] > 0;
      const float f = pres ? exp_fast(__fsub_rn(mb[bb], Mc)) : 0.f;
      if (pres) Lc = __fmaf_rn(lb[bb], f, Lc);
      uint32_t r[2][32];
      tmem_ld32_nowait(tlane + kT5Block * bb, r[0]);
      tmem_ld32_nowait(tlane + kT5Block * bb + 32, r[1]);
      tmem_wait_ld();
      if (pres) {
#pragma unroll
        for (int d = 0; d < kHeadDim; ++d) oc[d] = __fmaf_rn(__uint_as_float(r[d >> 5][d & 31]), f, oc[d]);
      }
    }
    // give-up path: every product issued has completed before the memory is freed
    if (!ok) {
      if (tid == 0) mma_commit(bar_done);
      __syncwarp();
      mbar_wait(bar_done, 0);
      if (tid == 0) atomicOr(&st.status, ST_TIMEOUT);
    }
  }
  // every rank is done with its query and key tiles: the inbox takes them
  if (S > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
  if (has_chunk && ok && mine && my_a >= c_lo) {
    // the chunk's (O_c, M_c, l_c) of this pair to the rank merging it
    float* dst = inbox + ((size_t)rank * kPR + tid % kPR) * kInboxRow;
    if (S > 1) dst = cg::this_cluster().map_shared_rank(dst, tid / kPR);
#pragma unroll
    for (int d = 0; d < kHeadDim; d += 4)
      *reinterpret_cast<float4*>(dst + d) = make_float4(oc[d], oc[d + 1], oc[d + 2], oc[d + 3]);
    *reinterpret_cast<float4*>(dst + kHeadDim) = make_float4(Mc, Lc, 0.f, 0.f);
  }
  if (S > 1)
    cg::this_cluster().sync();                     // every chunk's partials have arrived
  else
    __syncthreads();
  // merge this rank's pairs over the row's chunks, in chunk order: work item
  // (pair, group of 8 dims)
#pragma unroll 1
  for (int it = tid; it < kPR * (kHeadDim / 8); it += kT5Threads) {
    const int lp = it / (kHeadDim / 8), dg = it % (kHeadDim / 8);
    const int p = rank * kPR + lp;
    if (p >= npairs) continue;
    const int r = p / grp, h = p % grp, a = a_row[r];
    const size_t out = (size_t)(row0 + r) * D.hq * kHeadDim + (g * grp + h) * kHeadDim + dg * 8;
    float o[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) o[d] = 0.f;
    if (a >= 0) {
      const int ncp = (a - start) / kT5Chunk + 1;
      const float* rec = inbox + (size_t)lp * kInboxRow;           // chunk c at + c kPR kInboxRow
      float M = -INFINITY;
      for (int c = 0; c < ncp; ++c) M = fmaxf(M, rec[(size_t)c * kPR * kInboxRow + kHeadDim]);
      float l = 0.f;
      for (int c = 0; c < ncp; ++c) {
        const float* rc = rec + (size_t)c * kPR * kInboxRow;
        const float f = exp_fast(__fsub_rn(rc[kHeadDim], M));
        l = __fmaf_rn(rc[kHeadDim + 1], f, l);
        const float4 u0 = *reinterpret_cast<const float4*>(rc + dg * 8);
        const float4 u1 = *reinterpret_cast<const float4*>(rc + dg * 8 + 4);
        o[0] = __fmaf_rn(u0.x, f, o[0]);
        o[1] = __fmaf_rn(u0.y, f, o[1]);
        o[2] = __fmaf_rn(u0.z, f, o[2]);
        o[3] = __fmaf_rn(u0.w, f, o[3]);
        o[4] = __fmaf_rn(u1.x, f, o[4]);
        o[5] = __fmaf_rn(u1.y, f, o[5]);
        o[6] = __fmaf_rn(u1.z, f, o[6]);
        o[7] = __fmaf_rn(u1.w, f, o[7]);
      }
#pragma unroll
      for (int d = 0; d < 8; ++d) o[d] = __fdiv_rn(o[d], l);
    }
    if (io.out16) {
      *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(io.out16) + out) =
          make_uint4(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]), pack_bf16(o[4], o[5]), pack_bf16(o[6], o[7]));
    } else {
      *reinterpret_cast<float4*>(io.attn_out + out) = make_float4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<float4*>(io.attn_out + out + 4) = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
  if (has_chunk) {
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(*tmem_slot, kT5Cols);
  }
}

size_t t5_smem(int grp) { return (size_t)T5Layout(kT5Pairs / grp).total + 1024; }   // + alignment slack

template <int S>
cudaError_t launch_t5_s(const Dims& D, const Batch& b, int layer, const AttnIO& io, cudaStream_t s) {
  static bool attr = false;                        // the kernel's shared-memory limit, once per process
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_attn_t5<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t5_smem(1));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_attn_t5<S>, cudaFuncAttributeClusterSchedulingPolicyPreference,
                               cudaClusterSchedulingPolicyLoadBalancing);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grp = D.hq / D.hkv;
  const int RT = kT5Pairs / grp;
  int tps = 1, tiles = b.Bmax;
  if (b.pos) {
    tps = (b.pm + RT - 1) / RT;
    tiles = (b.Bmax / b.pm) * tps;
  }
  dim3 grid(S, D.hkv, tiles);
  return launch_kernel_cluster(k_attn_t5<S>, grid, dim3(kT5Threads), t5_smem(grp), s, D.pdl, S, D, b, layer, tps, io);
}

}  // namespace

int attn_t5_ranks(const Dims& D) {
  int S = D.L / kT5Chunk;
  return S < 1 ? 1 : S > kT5MaxRanks ? kT5MaxRanks : S;
}

cudaError_t launch_attn_t5(const Dims& D, const Batch& b, int layer, const float* qkv, float* attn_out, void* out16,
                           cudaStream_t s) {
  const AttnIO io{qkv, attn_out, out16};
  switch (attn_t5_ranks(D)) {
    case 1: return launch_t5_s<1>(D, b, layer, io, s);
    case 2: return launch_t5_s<2>(D, b, layer, io, s);
    case 4: return launch_t5_s<4>(D, b, layer, io, s);
    case 8: return launch_t5_s<8>(D, b, layer, io, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nc
