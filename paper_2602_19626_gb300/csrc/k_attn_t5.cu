// Decode and prefill attention over a BF16 KV cache on the tcgen05 tensor
// cores, accumulators in tensor memory (Sec. 3.2 model, Sec. 3.9 sliding
// window).
//
// A tile is up to 128 (query row, head) pairs of one stream and KV head: the
// grp query heads sharing the KV head of a row of consecutive positions,
// pair p = r grp + h, cut into tiles of 128 consecutive pairs (a tile's
// first and last row may be split with its neighbours); a decode step's tile
// is the grp pairs of its one row.  The pairs are the MMA's M = 128 rows, so
// each pair's products depend on its own query alone: a row computed alone
// (decode) and among the rows of a prefill gives the same bits.
//
// The window [start, a] of a row is cut into chunks of 256 positions (chunk
// c = [start + 256 c, ...)), a chunk into four blocks of 64.  CTA (c, g, t)
// computes chunk c of tile t and KV head g with 8 warps; warp w reads TMEM
// lanes 32 (w mod 4) .. + 31 (one lane per pair) and belongs to warpgroup
// h = w / 4, which takes blocks h and h + 2:
//   - the K and V rows of the chunk's blocks go to shared memory in the
//     128-byte swizzle layout, a block of 64 ring rows per TMA copy (a block
//     that wraps around the ring by 16-byte asynchronous copies); rows past
//     the tile's last position hold whatever the ring holds there (zero from
//     allocation, else finite older entries), which the zero probabilities
//     of masked positions cancel; the pairs' rotated 1/8-scaled queries in
//     BF16 go beside them (a prefill's were written by its append pass, a
//     decode step rotates its own);
//   - one thread issues S_b = Q K_b^T for every block b (M 128, N 64, four K
//     steps of 16 head dims) into tensor-memory columns 64 b .. 64 b + 63;
//   - each pair's chunk maximum M_c over its unmasked scores (positions up
//     to its row's), then e = 2^(s log2 e - M_c log2 e) (PTX ex2.approx),
//     their FP32 sum l_c (per block eight interleaved partial sums and a
//     fixed tree; blocks h, h + 2 added in order per warpgroup, then the two
//     warpgroups' sums) and P_b = BF16(e) into shared memory (the key tile
//     and the query tile hold the P buffers once every score is computed);
//   - O_c = sum_b P_b V_b accumulates in columns 0 .. 63 (block 0's scores,
//     read by then; V read MN-major straight from its tile; blocks past the
//     row carry zero probabilities);
//   - (O_c, M_c, l_c) go to a global partials buffer (O_c as 16 float4
//     planes of the tile's pairs, so that a warp's stores and loads are
//     contiguous), and every output element is merged over the row's chunks
//     in chunk order: O = sum O_c f_c / sum l_c f_c, f_c = exp(M_c - max M_c)
//     by the merge kernel that follows a prefill launch, or, in a decode
//     step, by the CTA that finishes the row's last chunk (an atomic ticket
//     per row and KV head, reset by it).  Both merges are one function of
//     the partials, so the bits do not depend on which one ran.
// In a decode step the CTA of the chunk holding the fed position a rotates
// the new k at a, rounds k and v to BF16, appends them to the ring and to
// its tile; a prefill's rows were appended by k_kv_append_t5 (the same
// arithmetic) before this kernel.  About 84 KB of shared memory and 256 TMEM
// columns: two CTAs per SM.
//
// Every wait on an mbarrier is bounded; a wait that gives up raises
// ST_TIMEOUT in the stream's status word, skips the remaining products and,
// before the tensor memory is freed, waits (with the same bound) for the
// copies and products already issued.
#include <cuda_bf16.h>

#include <algorithm>

#include "model_dev.cuh"
#include "tc5.cuh"

namespace nc {

namespace {

using namespace dev;
using namespace tc5;

constexpr int kT5Threads = 256;              // 8 warps: warpgroup w / 4, TMEM lanes 32 (w % 4) .. + 31
constexpr int kT5Pairs = 128;                // MMA M: (row, head) pairs per tile
constexpr int kT5Chunk = 256;                // positions per chunk (one CTA)
constexpr int kT5Block = 64;                 // positions per block (N of the scores, K of P V)
constexpr int kT5Blocks = kT5Chunk / kT5Block;
constexpr int kT5MaxRanks = 8;               // chunks of a window of at most 2,048 positions
constexpr int kRowB = 128;                   // bytes of one swizzled row: 64 BF16
constexpr uint32_t kT5Cols = 256;            // TMEM columns: S_b at 64 b; O_c at 0
constexpr int kPartRow = kHeadDim + 4;       // floats per (chunk, pair) partial: O_c[64], M_c, l_c, padding
constexpr int kGroups = kHeadDim / 4;        // float4 groups of an output row
constexpr int kMergePairs = 16;              // pairs of one merge CTA (x 16 groups = 256 threads)

// Shared memory, byte offsets from a 1024-byte aligned base.
struct T5Layout {
  static constexpr int q = 0;                              // [128 pairs][128 B]; later P buffer 2
  static constexpr int k = q + kT5Pairs * kRowB;           // [256 positions][128 B]; later P buffers 0, 1
  static constexpr int v = k + kT5Chunk * kRowB;           // [256 positions][128 B]
  static constexpr int cs = v + kT5Chunk * kRowB;          // [32] float2: (cos, sin) of a decode row
  static constexpr int red = cs + (kHeadDim / 2) * 8;      // [2][128] floats: the warpgroups' maxima, then sums
  static constexpr int bars = red + 2 * kT5Pairs * 4;      // 6 mbarriers
  static constexpr int slot = bars + 64;                   // TMEM address
  static constexpr int arow = slot + 16;                   // [128] row positions, then the merge flag
  static constexpr int total = arow + kT5Pairs * 4 + 16;
};
constexpr size_t kT5Smem = T5Layout::total + 1024;         // + alignment slack

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

// The tile of CTA z: pairs pb .. pb + npairs - 1 (pb counted from row0's
// first pair) of rows row0 .. row0 + nr - 1.  A prefill's stream j takes
// tps tiles of 128 consecutive pairs of its pm rows; a decode tile is row z.
struct T5Tile {
  int row0, nr, npairs, pb;
};
__device__ __forceinline__ T5Tile t5_tile(const Batch& b, int grp, int tps, int z) {
  T5Tile t;
  if (b.pos) {
    const int j = z / tps, sub = z % tps;
    const int p0 = sub * kT5Pairs;
    t.npairs = min(kT5Pairs, b.pm * grp - p0);
    const int r_lo = p0 / grp;
    t.nr = (p0 + t.npairs - 1) / grp - r_lo + 1;
    t.row0 = j * b.pm + r_lo;
    t.pb = p0 - r_lo * grp;
  } else {
    t.row0 = z;
    t.nr = 1;
    t.npairs = grp;
    t.pb = 0;
  }
  return t;
}

// Whether block bb of the chunk at c_lo is one TMA box: its 64 ring rows
// contiguous (no wrap) and the slots' tensor maps present.
__device__ __forceinline__ bool kv_block_tma(const Dims& D, int c_lo, int bb) {
  return D.kv_tmap != nullptr && ((c_lo + bb * kT5Block) & (D.L - 1)) + kT5Block <= D.L;
}

// The K and V rows of the chunk's first nblk blocks: TMA boxes of 64 ring
// rows (thread 0; K completes on bar_k, V on bar_v, each arrived on once),
// and the blocks that wrap around the ring by 16-byte copies of the
// positions <= last other than `own` (which the caller writes), zero past
// last (every thread).
__device__ void load_kv(const Dims& D, const StreamDev& st, int slot, int layer, int g, int c_lo, int nblk, int last,
                        int own, uint8_t* kt, uint8_t* vt, uint64_t* bar_k, uint64_t* bar_v, int tid) {
  if (tid == 0) {
    uint32_t n = 0;
    for (int bb = 0; bb < nblk; ++bb) n += kv_block_tma(D, c_lo, bb);
    mbar_expect_tx(bar_k, n * kT5Block * kRowB);
    mbar_expect_tx(bar_v, n * kT5Block * kRowB);
    if (n) {
      const void* map = static_cast<const uint8_t*>(D.kv_tmap) + (size_t)slot * kTmapBytes;
      const int rk = (layer * 2 * D.hkv + g) * D.L, rv = (layer * 2 * D.hkv + D.hkv + g) * D.L;
      for (int bb = 0; bb < nblk; ++bb) {
        if (!kv_block_tma(D, c_lo, bb)) continue;
        const int r = (c_lo + bb * kT5Block) & (D.L - 1);
        tma_load_2d(kt + bb * kT5Block * kRowB, map, bar_k, 0, rk + r);
        tma_load_2d(vt + bb * kT5Block * kRowB, map, bar_v, 0, rv + r);
      }
    }
  }
  const __nv_bfloat16* kv = static_cast<const __nv_bfloat16*>(st.kv);
  const __nv_bfloat16* kp = kv + attn_plane_off(D, layer, g);
  const __nv_bfloat16* vp = kv + attn_plane_off(D, layer, D.hkv + g);
  for (int bb = 0; bb < nblk; ++bb) {
    if (kv_block_tma(D, c_lo, bb)) continue;
    for (int e = tid; e < kT5Block * 8; e += kT5Threads) {
      const int row = bb * kT5Block + (e >> 3), seg = e & 7;
      const int p = c_lo + row;
      if (p == own) continue;                      // written by the caller
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
}

// The maximum of the first nvalid of the 64 scores at TMEM column `col` of
// this thread's lane.
__device__ __forceinline__ float block_max(uint32_t tlane, uint32_t col, int nvalid) {
  uint32_t r[2][32];
  tmem_ld32_nowait(tlane + col, r[0]);
  tmem_ld32_nowait(tlane + col + 32, r[1]);
  tmem_wait_ld();
  float m = -INFINITY;
  if (nvalid == kT5Block) {
#pragma unroll
    for (int i = 0; i < kT5Block; ++i) m = fmaxf(m, __uint_as_float(r[i >> 5][i & 31]));
  } else {
#pragma unroll
    for (int i = 0; i < kT5Block; ++i)
      if (i < nvalid) m = fmaxf(m, __uint_as_float(r[i >> 5][i & 31]));
  }
  return m;
}

// The numerators of one block for this thread's pair: e = 2^(s log2 e + mb)
// (mb = -M_c log2 e) over the first nvalid of the 64 scores at TMEM column
// `col`, zero past them, rounded to BF16 into the pair's row of the P tile;
// returns their FP32 sum.
__device__ __forceinline__ float block_exp(uint32_t tlane, uint32_t col, int nvalid, float mb, uint8_t* ptile,
                                           int pair) {
  float acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t r[32];
    tmem_ld32_nowait(tlane + col + 32 * half, r);
    tmem_wait_ld();
    float e[32];
    if (nvalid == kT5Block) {
#pragma unroll
      for (int i = 0; i < 32; ++i) e[i] = ex2_approx(__fmaf_rn(__uint_as_float(r[i]), kLog2e, mb));
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i)
        e[i] = 32 * half + i < nvalid ? ex2_approx(__fmaf_rn(__uint_as_float(r[i]), kLog2e, mb)) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i & 7] = __fadd_rn(acc[i & 7], e[i]);
#pragma unroll
    for (int sg = 0; sg < 4; ++sg) {
      const uint4 u = make_uint4(pack_bf16(e[8 * sg], e[8 * sg + 1]), pack_bf16(e[8 * sg + 2], e[8 * sg + 3]),
                                 pack_bf16(e[8 * sg + 4], e[8 * sg + 5]), pack_bf16(e[8 * sg + 6], e[8 * sg + 7]));
      *reinterpret_cast<uint4*>(ptile + swz(pair, 4 * half + sg)) = u;
    }
  }
  return __fadd_rn(__fadd_rn(__fadd_rn(acc[0], acc[1]), __fadd_rn(acc[2], acc[3])),
                   __fadd_rn(__fadd_rn(acc[4], acc[5]), __fadd_rn(acc[6], acc[7])));
}

// Partials of tile-and-head tg: O_c of pair p, dims 4 i .. 4 i + 3, at float4
// (c 16 + i) tp + p; (M_c, l_c) at float4 16 kT5MaxRanks tp + c tp + p.
__device__ __forceinline__ float4* part_base(const Dims& D, size_t tg, int tp) {
  return reinterpret_cast<float4*>(D.attn_part) + tg * kT5MaxRanks * tp * (kPartRow / 4);
}

// Dims 4 i .. 4 i + 3 of pair p's output merged over its ncp chunks, in chunk
// order: M = max M_c, f_c = exp(M_c - M), O = sum O_c f_c / sum l_c f_c;
// zero when the row has no chunk.
__device__ __forceinline__ float4 merge_item(const float4* part, int tp, int p, int i, int ncp) {
  const float4* ml = part + (size_t)kT5MaxRanks * kGroups * tp + p;
  float2 v[kT5MaxRanks];
  float4 u[kT5MaxRanks];
#pragma unroll
  for (int c = 0; c < kT5MaxRanks; ++c) {
    if (c < ncp) {
      const float4 w = __ldcg(ml + (size_t)c * tp);
      v[c] = make_float2(w.x, w.y);
      u[c] = __ldcg(part + (size_t)(c * kGroups + i) * tp + p);
    }
  }
  float M = -INFINITY;
#pragma unroll
  for (int c = 0; c < kT5MaxRanks; ++c)
    if (c < ncp) M = fmaxf(M, v[c].x);
  float l = 0.f;
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int c = 0; c < kT5MaxRanks; ++c) {
    if (c < ncp) {
      const float f = exp_fast(__fsub_rn(v[c].x, M));
      l = __fmaf_rn(v[c].y, f, l);
      o.x = __fmaf_rn(u[c].x, f, o.x);
      o.y = __fmaf_rn(u[c].y, f, o.y);
      o.z = __fmaf_rn(u[c].z, f, o.z);
      o.w = __fmaf_rn(u[c].w, f, o.w);
    }
  }
  if (ncp) o = make_float4(__fdiv_rn(o.x, l), __fdiv_rn(o.y, l), __fdiv_rn(o.z, l), __fdiv_rn(o.w, l));
  return o;
}

__device__ __forceinline__ void store_out(const AttnIO& io, size_t off, float4 o) {
  if (io.out16) {
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(io.out16) + off) =
        make_uint2(pack_bf16(o.x, o.y), pack_bf16(o.z, o.w));
  } else {
    *reinterpret_cast<float4*>(io.attn_out + off) = o;
  }
}

__global__ void __launch_bounds__(kT5Threads, 2) k_attn_t5(Dims D, Batch b, int layer, int tps, AttnIO io) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  using Ly = T5Layout;
  const int grp = D.hq / D.hkv;
  uint8_t* qt = sm + Ly::q;
  uint8_t* kt = sm + Ly::k;
  uint8_t* vt = sm + Ly::v;
  float2* cs = reinterpret_cast<float2*>(sm + Ly::cs);
  float* red = reinterpret_cast<float*>(sm + Ly::red);
  uint64_t* bar_k = reinterpret_cast<uint64_t*>(sm + Ly::bars);   // the K boxes
  uint64_t* bar_v = bar_k + 1;                                     // the V boxes
  uint64_t* bar_s = bar_k + 2;                                     // every score product
  uint64_t* bar_o0 = bar_k + 3;                                    // P V of blocks 0, 1
  uint64_t* bar_o1 = bar_k + 4;                                    // P V of blocks 2, 3
  uint64_t* bar_done = bar_k + 5;                                  // every product issued
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + Ly::slot);
  int* a_row = reinterpret_cast<int*>(sm + Ly::arow);
  int* s_last = a_row + kT5Pairs;

  const int rank = blockIdx.x;                     // the chunk of the window
  const int g = blockIdx.y;
  const int tid = threadIdx.x, wg = tid >> 7, p = tid & (kT5Pairs - 1);
  const bool prefill = b.pos != nullptr;
  const T5Tile T = t5_tile(b, grp, tps, blockIdx.z);
  // the row count and the rows' slots and positions were written at least
  // two launches back: read before the wait
  if (T.row0 >= *b.nB) return;
  const int slot = b.slots[T.row0];
  StreamDev& st = b.st[slot];
  if (tid < T.nr) a_row[tid] = prefill ? b.pos[T.row0 + tid] : st.n_coded;
  __syncthreads();
  int a_max = -1;
  for (int r = 0; r < T.nr; ++r) a_max = max(a_max, a_row[r]);
  const int start = a_max < 0 ? 0 : prefill ? window_start_at(D, a_max) : window_start(D, st);
  const int nch = a_max < 0 ? 0 : (a_max - start) / kT5Chunk + 1;
  const bool has_chunk = rank < nch;
  // a decode CTA without a chunk but rank 0 zeroes the rows of no window;
  // a prefill's merge kernel does that
  if (!has_chunk && (prefill || nch > 0 || rank > 0)) return;
  const int c_lo = start + rank * kT5Chunk;
  const int nblk = has_chunk ? min(kT5Blocks, (a_max - c_lo) / kT5Block + 1) : 0;
  // this thread's pair and its row's position (-1: padding or past the stream's end)
  const int my_r = (T.pb + p) / grp, my_h = (T.pb + p) % grp;
  const int my_a = p < T.npairs ? a_row[my_r] : -1;
  const bool mine = 32 * ((tid >> 5) & 3) < T.npairs;   // warp-uniform: the warp's lanes hold real pairs

  bool ok = true;
  if (has_chunk) {
    if (tid == 0) {
      for (int i = 0; i < 6; ++i) mbar_init(bar_k + i, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tmem_alloc(tmem_slot, kT5Cols);
    __syncthreads();                               // the barriers are initialised
    // decode: the cached entries (positions below a) were appended by earlier
    // steps and may be loaded before the wait; a prefill's rows were appended
    // by the launch just before
    if (!prefill) load_kv(D, st, slot, layer, g, c_lo, nblk, a_max, a_max, kt, vt, bar_k, bar_v, tid);
  }
  pdl_wait();
  pdl_trigger();
  if (has_chunk) {
    if (prefill) load_kv(D, st, slot, layer, g, c_lo, nblk, a_max, -1, kt, vt, bar_k, bar_v, tid);
    bool my_ok = true;
    if (!prefill) {
      // (cos, sin) of the decode row's position; the fed token's k (rotated
      // at a) and v, rounded to BF16, into the ring and into this tile (the
      // rank whose chunk holds a), the tile's row after its box has landed
      const int a = a_max;
      if (tid < kHeadDim / 2) cs[tid] = rope_cs(D, a, tid);
      if (rank == nch - 1 && tid >= 64 && tid < 64 + kHeadDim) {
        const int t = tid - 64;
        const float* row = io.qkv + (size_t)T.row0 * D.qkv_rows;
        const int R = a - c_lo;
        const bool boxed = kv_block_tma(D, c_lo, R / kT5Block);
        const size_t ri = (size_t)(a & (D.L - 1)) * kHeadDim;
        if (t < kHeadDim / 2) {                    // dims t and t + 32 of k
          const float* src = row + D.hq * kHeadDim + g * kHeadDim;
          const float2 rr = rope_rotate(__ldcg(src + t), __ldcg(src + t + kHeadDim / 2), rope_cs(D, a, t));
          __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv) + attn_plane_off(D, layer, g) + ri;
          const __nv_bfloat16 k0 = __float2bfloat16_rn(rr.x), k1 = __float2bfloat16_rn(rr.y);
          kv[t] = k0;
          kv[t + kHeadDim / 2] = k1;
          if (boxed) my_ok = mbar_wait(bar_k, 0);
          *reinterpret_cast<__nv_bfloat16*>(kt + swz(R, t >> 3) + (t & 7) * 2) = k0;
          *reinterpret_cast<__nv_bfloat16*>(kt + swz(R, (t + 32) >> 3) + (t & 7) * 2) = k1;
        } else {                                   // dims d0, d0 + 1 of v
          const int d0 = 2 * (t - kHeadDim / 2);
          const float* src = row + (D.hq + D.hkv) * kHeadDim + g * kHeadDim;
          __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv) + attn_plane_off(D, layer, D.hkv + g) + ri;
          const __nv_bfloat16 v0 = __float2bfloat16_rn(__ldcg(src + d0)), v1 = __float2bfloat16_rn(__ldcg(src + d0 + 1));
          kv[d0] = v0;
          kv[d0 + 1] = v1;
          if (boxed) my_ok = mbar_wait(bar_v, 0);
          *reinterpret_cast<__nv_bfloat16*>(vt + swz(R, d0 >> 3) + (d0 & 7) * 2) = v0;
          *reinterpret_cast<__nv_bfloat16*>(vt + swz(R, (d0 + 1) >> 3) + ((d0 + 1) & 7) * 2) = v1;
        }
      }
      __syncthreads();                             // the rotation table is complete
    }
    // the pairs' rotated, 1/8-scaled BF16 queries (zero for padding pairs):
    // warpgroup h writes dims 16 h .. 16 h + 15 and 32 + 16 h .. 32 + 16 h + 15
    if (mine) {
      uint4 s0 = make_uint4(0, 0, 0, 0), s1 = s0, s2 = s0, s3 = s0;
      if (my_a >= 0 && prefill) {
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(D.q16) +
                                                          ((size_t)(T.row0 + my_r) * D.hq + g * grp + my_h) * kHeadDim);
        s0 = __ldcg(src + 2 * wg);
        s1 = __ldcg(src + 2 * wg + 1);
        s2 = __ldcg(src + 4 + 2 * wg);
        s3 = __ldcg(src + 4 + 2 * wg + 1);
      } else if (my_a >= 0) {
        const float* src = io.qkv + (size_t)T.row0 * D.qkv_rows + (g * grp + my_h) * kHeadDim + 16 * wg;
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int dd = 16 * wg + 2 * i;
          const float2 x1 = __ldcg(reinterpret_cast<const float2*>(src + 2 * i));
          const float2 x2 = __ldcg(reinterpret_cast<const float2*>(src + kHeadDim / 2 + 2 * i));
          const float2 r0 = rope_rotate(x1.x, x2.x, cs[dd]);
          const float2 r1 = rope_rotate(x1.y, x2.y, cs[dd + 1]);
          // the 1/sqrt(64) score scale is a power of two: exact
          w[i] = pack_bf16(r0.x * 0.125f, r1.x * 0.125f);
          w[8 + i] = pack_bf16(r0.y * 0.125f, r1.y * 0.125f);
        }
        s0 = make_uint4(w[0], w[1], w[2], w[3]);
        s1 = make_uint4(w[4], w[5], w[6], w[7]);
        s2 = make_uint4(w[8], w[9], w[10], w[11]);
        s3 = make_uint4(w[12], w[13], w[14], w[15]);
      }
      *reinterpret_cast<uint4*>(qt + swz(p, 2 * wg)) = s0;
      *reinterpret_cast<uint4*>(qt + swz(p, 2 * wg + 1)) = s1;
      *reinterpret_cast<uint4*>(qt + swz(p, 4 + 2 * wg)) = s2;
      *reinterpret_cast<uint4*>(qt + swz(p, 4 + 2 * wg + 1)) = s3;
    }
    cp_async_wait_all();
    fence_proxy_async();
    fence_before_sync();
    // the queries, the copied rows and every K box are in place
    ok = __syncthreads_and(my_ok && mbar_wait(bar_k, 0));
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);
    if (tid == 0 && ok) {
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
    // every score product done (the key and query tiles hold the P buffers
    // from here) and every V box in place
    ok = __syncthreads_and(ok && mbar_wait(bar_s, 0) && mbar_wait(bar_v, 0));
    fence_after_sync();
    // the unmasked columns of this pair in each of the warpgroup's blocks
    int nv[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int bb = wg + 2 * k, blo = c_lo + bb * kT5Block;
      nv[k] = bb < nblk && my_a >= blo ? min(kT5Block, my_a - blo + 1) : 0;
    }
    // the chunk maximum: each warpgroup over its blocks, then both (the
    // TMEM loads are warp-collective: every lane of a warp takes them)
    float m = -INFINITY;
    if (ok && mine) {
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (wg + 2 * k < nblk) m = fmaxf(m, block_max(tlane, kT5Block * (wg + 2 * k), nv[k]));
    }
    red[wg * kT5Pairs + p] = m;
    __syncthreads();
    const float Mc = fmaxf(red[p], red[kT5Pairs + p]);
    const float mb = Mc > -INFINITY ? -__fmul_rn(Mc, kLog2e) : 0.f;
    __syncthreads();                               // the maxima are read: the sums take their place
    // stage 0: block h into P buffer h (the key tile); stage 1: block 2 into
    // the query tile, block 3 into P buffer 0 once P V of blocks 0, 1 is done
    float lh = 0.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int bb = wg + 2 * k;
      uint8_t* pt = bb == 2 ? qt : kt + (bb & 1) * (kT5Pairs * kRowB);
      bool wok = true;
      if (ok && bb == 3 && bb < nblk) wok = __all_sync(0xffffffffu, mbar_wait(bar_o0, 0));
      if (ok && wok && mine && bb < nblk) lh = __fadd_rn(lh, block_exp(tlane, kT5Block * bb, nv[k], mb, pt, p));
      fence_proxy_async();
      fence_before_sync();
      ok = __syncthreads_and(ok && wok);
      fence_after_sync();
      if (tid == 0 && ok && 2 * k < nblk) {
        // O_c += P_b V_b for the stage's blocks, into columns 0 .. 63
        const uint32_t ido = idesc(1, kT5Pairs, kHeadDim, 1);
        for (int b2 = 2 * k; b2 < min(2 * k + 2, nblk); ++b2) {
          uint8_t* pt2 = b2 == 2 ? qt : kt + (b2 & 1) * (kT5Pairs * kRowB);
#pragma unroll
          for (int s = 0; s < kT5Block / 16; ++s)
            mma_issue(1, tmem, sdesc_sw128(smem_u32(pt2) + 32 * s),
                      sdesc_sw128_mn(smem_u32(vt + (b2 * kT5Block + 16 * s) * kRowB)), ido, b2 + s ? 1u : 0u);
        }
        mma_commit(k ? bar_o1 : bar_o0);
      }
      __syncwarp();
    }
    red[wg * kT5Pairs + p] = lh;
    // every product done
    ok = __syncthreads_and(ok && mbar_wait(nblk > 2 ? bar_o1 : bar_o0, 0));
    fence_after_sync();
    const float Lc = __fadd_rn(red[p], red[kT5Pairs + p]);
    // the chunk's (O_c, M_c, l_c) of the present pairs: warpgroup h writes
    // dims 32 h .. 32 h + 31
    const int tp = prefill ? min(kT5Pairs, b.pm * grp) : grp;   // pairs a tile can hold
    float4* part = part_base(D, (size_t)blockIdx.z * D.hkv + g, tp);
    if (ok && mine) {
      uint32_t r[32];
      tmem_ld32_nowait(tlane + 32 * wg, r);
      tmem_wait_ld();
      if (p < T.npairs && my_a >= c_lo) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          __stcg(part + (size_t)(rank * kGroups + 8 * wg + i) * tp + p,
                 make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]), __uint_as_float(r[4 * i + 2]),
                             __uint_as_float(r[4 * i + 3])));
        if (wg == 0)
          __stcg(part + (size_t)kT5MaxRanks * kGroups * tp + (size_t)rank * tp + p, make_float4(Mc, Lc, 0.f, 0.f));
      }
    }
    // give-up path: every copy and product issued has completed before the
    // memory is freed
    if (!ok) {
      if (tid == 0) mma_commit(bar_done);
      __syncwarp();
      mbar_wait(bar_done, 0);
      mbar_wait(bar_k, 0);
      mbar_wait(bar_v, 0);
      cp_async_wait_all();
      if (tid == 0) atomicOr(&st.status, ST_TIMEOUT);
    }
    fence_before_sync();
    __syncthreads();
    if (tid < 32) tmem_dealloc(tmem, kT5Cols);
  }
  if (prefill) return;                             // merged by k_attn_merge
  // decode: the CTA that finishes the row's last chunk merges
  const size_t tg = (size_t)blockIdx.z * D.hkv + g;
  if (has_chunk) {
    __threadfence();
    __syncthreads();
    if (tid == 0) *s_last = atomicAdd(D.attn_ticket + tg, 1) == nch - 1;
    __syncthreads();
    if (*s_last == 0) return;
    __threadfence();
    if (tid == 0) D.attn_ticket[tg] = 0;           // for the next launch
  }
  const float4* part = part_base(D, tg, grp);
  for (int it = tid; it < T.npairs * kGroups; it += kT5Threads) {
    const int q = it / kGroups, i = it % kGroups;
    store_out(io, (size_t)T.row0 * D.hq * kHeadDim + (g * grp + q) * kHeadDim + 4 * i, merge_item(part, grp, q, i, nch));
  }
}

// The prefill merge: CTA (t, g, s) merges pairs 16 s .. 16 s + 15 of tile t
// and KV head g; thread (pair, group) = (tid % 16, tid / 16).
__global__ void __launch_bounds__(kT5Threads) k_attn_merge(Dims D, Batch b, int tps, AttnIO io) {
  const int grp = D.hq / D.hkv;
  const int g = blockIdx.y;
  const T5Tile T = t5_tile(b, grp, tps, blockIdx.x);
  const int p = blockIdx.z * kMergePairs + (threadIdx.x % kMergePairs), i = threadIdx.x / kMergePairs;
  if (T.row0 >= *b.nB) return;
  pdl_wait();
  pdl_trigger();
  if (p >= T.npairs) return;
  const int my_r = (T.pb + p) / grp, my_h = (T.pb + p) % grp;
  const int a = b.pos[T.row0 + my_r];
  const int ncp = a < 0 ? 0 : (a - window_start_at(D, a)) / kT5Chunk + 1;
  const int tp = min(kT5Pairs, b.pm * grp);
  const float4* part = part_base(D, (size_t)blockIdx.x * D.hkv + g, tp);
  store_out(io, (size_t)(T.row0 + my_r) * D.hq * kHeadDim + (g * grp + my_h) * kHeadDim + 4 * i,
            merge_item(part, tp, p, i, ncp));
}

// Prefill append: row j's k (rotated at its position a) and v, rounded to
// BF16, into the ring of `layer`, and its grp query heads of KV head g,
// rotated, scaled by 1/8 and rounded to BF16, into q16 (the attention's
// decode step does the same arithmetic for its one row).
__global__ void __launch_bounds__(128) k_kv_append_t5(Dims D, Batch b, int layer, const float* qkv) {
  const int j = blockIdx.y, g = blockIdx.x, tid = threadIdx.x;
  const int grp = D.hq / D.hkv;
  pdl_wait();
  pdl_trigger();
  if (j >= *b.nB) return;
  const int a = b.pos[j];
  if (a < 0) return;
  StreamDev& st = b.st[b.slots[j]];
  const float* row = qkv + (size_t)j * D.qkv_rows;
  const size_t ri = (size_t)(a & (D.L - 1)) * kHeadDim;
  __nv_bfloat16* kv = static_cast<__nv_bfloat16*>(st.kv);
  __nv_bfloat16* q16 = static_cast<__nv_bfloat16*>(D.q16) + (size_t)j * D.hq * kHeadDim;
  for (int e = tid; e < (grp + 1) * (kHeadDim / 2); e += blockDim.x) {
    const int h = e / (kHeadDim / 2), dd = e % (kHeadDim / 2);
    const float2 c = rope_cs(D, a, dd);
    if (h < grp) {
      const float* src = row + (g * grp + h) * kHeadDim;
      const float2 rr = rope_rotate(__ldcg(src + dd), __ldcg(src + dd + kHeadDim / 2), c);
      __nv_bfloat16* dst = q16 + (g * grp + h) * kHeadDim;
      dst[dd] = __float2bfloat16_rn(rr.x * 0.125f);
      dst[dd + kHeadDim / 2] = __float2bfloat16_rn(rr.y * 0.125f);
    } else {
      const float* src = row + D.hq * kHeadDim + g * kHeadDim;
      const float2 rr = rope_rotate(__ldcg(src + dd), __ldcg(src + dd + kHeadDim / 2), c);
      __nv_bfloat16* dst = kv + attn_plane_off(D, layer, g) + ri;
      dst[dd] = __float2bfloat16_rn(rr.x);
      dst[dd + kHeadDim / 2] = __float2bfloat16_rn(rr.y);
    }
  }
  if (tid < kHeadDim)
    kv[attn_plane_off(D, layer, D.hkv + g) + ri + tid] =
        __float2bfloat16_rn(__ldcg(row + (D.hq + D.hkv) * kHeadDim + g * kHeadDim + tid));
}

}  // namespace

void attn_t5_scratch(const Dims& D, int max_streams, int prefill_rows, size_t* part_floats, int* tickets) {
  const int grp = D.hq / D.hkv;
  // a decode tile is one stream's row (grp pairs); a prefill chunk of n
  // streams and m <= prefill_rows / n positions each takes n ceil(m grp / 128)
  // tiles of min(128, m grp) pairs: at most 2 prefill_rows grp pairs (n < 128
  // prefill_rows / (m grp 128) when m grp > 128)
  const size_t pf_pairs = prefill_rows >= 2 ? 2 * (size_t)prefill_rows * grp : 0;
  const size_t per = (size_t)D.hkv * kT5MaxRanks * kPartRow;
  *part_floats = std::max((size_t)max_streams * grp, pf_pairs) * per;
  *tickets = max_streams * D.hkv;                  // decode rows only
}

cudaError_t launch_attn_t5(const Dims& D, const Batch& b, int layer, const float* qkv, float* attn_out, void* out16,
                           cudaStream_t s) {
  if (!D.attn_part || !D.attn_ticket) return cudaErrorInvalidValue;
  static bool attr = false;                        // the kernel's shared-memory limit, once per process
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_attn_t5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT5Smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grp = D.hq / D.hkv;
  if (grp > kT5Pairs) return cudaErrorInvalidValue;
  int tps = 1, tiles = b.Bmax;
  if (b.pos) {
    if (!D.q16) return cudaErrorInvalidValue;
    tps = (b.pm * grp + kT5Pairs - 1) / kT5Pairs;
    tiles = (b.Bmax / b.pm) * tps;
  }
  const size_t tp = b.pos ? std::min(kT5Pairs, b.pm * grp) : grp;
  if ((!b.pos && (size_t)tiles * D.hkv > (size_t)D.attn_tickets) ||
      (size_t)tiles * D.hkv * kT5MaxRanks * tp * kPartRow > D.attn_part_cap)
    return cudaErrorInvalidValue;
  const AttnIO io{qkv, attn_out, out16};
  cudaError_t e = launch_kernel(k_attn_t5, dim3(kT5MaxRanks, D.hkv, tiles), dim3(kT5Threads), kT5Smem, s, D.pdl, D, b,
                                layer, tps, io);
  if (e == cudaSuccess && b.pos)
    e = launch_kernel(k_attn_merge, dim3(tiles, D.hkv, kT5Pairs / kMergePairs), dim3(kT5Threads), 0, s, D.pdl, D, b,
                      tps, io);
  return e;
}

cudaError_t launch_kv_append_t5(const Dims& D, const Batch& b, int layer, const float* qkv, cudaStream_t s) {
  if (!D.q16) return cudaErrorInvalidValue;
  return launch_kernel(k_kv_append_t5, dim3(D.hkv, b.Bmax), dim3(128), 0, s, D.pdl, D, b, layer, qkv);
}

}  // namespace nc
