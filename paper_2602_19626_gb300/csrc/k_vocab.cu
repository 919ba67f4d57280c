// Vocabulary-wide kernels: biased softmax (Sec. 3.6), N-gram distribution
// (Sec. 3.4), linear mix (Sec. 3.5), CDF quantisation with floors and the
// prefix sum (Sec. 3.3), the head / mixer updates, and the N-gram tables.
//
// One stream is handled by a cluster of CTAs (8 or 16 for the per-token
// step, kVocabCluster for the standalone quantiser); each CTA owns a
// contiguous chunk of the vocabulary and each thread a contiguous run of E
// symbols.  The standalone quantiser reduces thread -> warp (fixed xor tree)
// -> CTA (warps in order) -> cluster (ranks in order through distributed
// shared memory); the per-token step goes thread -> warp -> every CTA's inbox
// (one cluster barrier in the step kernel, one exchange round on each CTA's
// mbarrier in the prefill loop) -> the same fixed reduction in every warp.
// Every result is independent of the batch, the slot and the launch.
#include <algorithm>

#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace nc {

namespace {

constexpr int kWarps = kVocabThreads / 32;

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

// floor(p * K) for a binary32 p in [0, 2) and K < 2^24, exactly: p = m 2^(e-150)
// with a 24-bit significand m, so m * K < 2^48 is an exact integer product.
// Sets `bad` (and returns 0) for negative, >= 2, infinite or NaN inputs.
__device__ __forceinline__ uint32_t floor_prod(float p, uint32_t K, bool& bad) {
  const uint32_t u = __float_as_uint(p);
  const uint32_t a = u & 0x7FFFFFFFu;
  const bool out = (u != a && a != 0u) || a >= 0x40000000u;
  bad |= out;
  const uint32_t e = a >> 23;
  const uint32_t m = (a & 0x7FFFFFu) | (e ? 0x800000u : 0u);
  const uint32_t sh = 150u - (e ? e : 1u);            // 23 .. 149 unless out
  const unsigned long long prod = (unsigned long long)m * K;
  const uint32_t q = sh >= 48u ? 0u : (uint32_t)(prod >> sh);
  return out ? 0u : q;
}

// floor(p K) exactly for a binary32 p in [0, 2) and K < 2^24.  Below 2^24 the
// product rounded toward zero has the exact product's integer part (the
// integers there are representable, so floor(x) <= rz(x) <= x); at or above
// 2^24 (p > 2^24 / K > 1 only) the 48-bit integer product decides.  Sets
// `bad` for negative, >= 2 or NaN inputs.
__device__ __forceinline__ uint32_t floor_count(float p, uint32_t K, float Kf, bool& bad) {
  bad |= !(p >= 0.f && p < 2.f);
  const float x = __fmul_rz(p, Kf);
  uint32_t q = __float2uint_rz(x);
  if (x >= 16777216.f) q = floor_prod(p, K, bad);
  return q;
}

struct ArgMax {
  float v;
  int i;
};
__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  // larger value wins; equal values: lower index wins (first maximum)
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

// Shared scratch of one CTA of the standalone kernels: block-reduction
// slots and the values it publishes to the other CTAs of its cluster.
template <int NW>
struct VocabSharedT {
  static constexpr int kNW = NW;
  float wm[NW], wsum[NW];
  unsigned long long wc[NW];
  ArgMax wa[NW];
  uint32_t wscan[NW];
  // published to the cluster
  unsigned long long cl_csum;
  ArgMax cl_arg;
  uint32_t cl_bad;
  uint32_t cl_total;
};
using VocabShared = VocabSharedT<kWarps>;

template <typename Sh>
__device__ float block_max(float v, Sh& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  if (lane == 0) sh.wm[w] = v;
  __syncthreads();
  float r = sh.wm[0];
  for (int i = 1; i < Sh::kNW; ++i) r = fmaxf(r, sh.wm[i]);
  __syncthreads();
  return r;
}
template <typename Sh>
__device__ float block_sum(float v, Sh& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh.wsum[w] = v;
  __syncthreads();
  float r = 0.f;
  for (int i = 0; i < Sh::kNW; ++i) r += sh.wsum[i];
  __syncthreads();
  return r;
}

template <int E>
__device__ __forceinline__ void load_run(const float* src, int v0, int V, float (&out)[E], float fill) {
  if (v0 + E <= V && (reinterpret_cast<uintptr_t>(src + v0) & 15) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src + v0);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
      const float4 u = s4[q];
      out[4 * q] = u.x;
      out[4 * q + 1] = u.y;
      out[4 * q + 2] = u.z;
      out[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) out[i] = (v0 + i < V) ? src[v0 + i] : fill;
  }
}
template <int E>
__device__ __forceinline__ void store_run(float* dst, int v0, int V, const float (&in)[E]) {
  if (v0 + E <= V && (reinterpret_cast<uintptr_t>(dst + v0) & 15) == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst + v0);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) d4[q] = make_float4(in[4 * q], in[4 * q + 1], in[4 * q + 2], in[4 * q + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (v0 + i < V) dst[v0 + i] = in[i];
  }
}

template <int E>
__device__ __forceinline__ void load_counts(const int32_t* src, int v0, int V, int (&out)[E]) {
  if (v0 + E <= V && (reinterpret_cast<uintptr_t>(src + v0) & 15) == 0) {
    const int4* s4 = reinterpret_cast<const int4*>(src + v0);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
      const int4 u = s4[q];
      out[4 * q] = u.x;
      out[4 * q + 1] = u.y;
      out[4 * q + 2] = u.z;
      out[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) out[i] = (v0 + i < V) ? src[v0 + i] : 0;
  }
}
template <int E>
__device__ __forceinline__ void store_counts(int32_t* dst, int v0, int V, const int (&in)[E]) {
  if (v0 + E <= V && (reinterpret_cast<uintptr_t>(dst + v0) & 15) == 0) {
    int4* d4 = reinterpret_cast<int4*>(dst + v0);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) d4[q] = make_int4(in[4 * q], in[4 * q + 1], in[4 * q + 2], in[4 * q + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (v0 + i < V) dst[v0 + i] = in[i];
  }
}

// ------------------------------------------------ standalone quantiser rounds
struct QuantResult {
  long long resid;          // T - sum of floored counts, added to the first maximum
  int argmax;
  bool bad;                 // non-finite / out-of-range probability, or floor underflow
};

// Floor-quantise the thread's E probabilities into c[], reduce the count sum
// and the first argmax over the cluster (thread -> warp -> CTA -> ranks in
// order), and add the residual to the first maximum.
template <int E, int CL, typename Sh>
__device__ QuantResult quantise_round(const float (&p)[E], int v0, int V, int log2T, uint32_t floor_c,
                                      uint32_t (&c)[E], cg::cluster_group& cl, Sh& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t T = 1u << log2T;
  const uint32_t K = T - (uint32_t)V * floor_c;
  bool bad = false;
  unsigned long long csum = 0;
  ArgMax am{-INFINITY, 0x7fffffff};
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int v = v0 + i;
    c[i] = 0;
    if (v < V) {
      const uint32_t q = floor_count(p[i], K, (float)K, bad);
      c[i] = q > floor_c ? q : floor_c;
      csum += c[i];
      if (p[i] > am.v) am = ArgMax{p[i], v};   // strict: keeps the first maximum
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    csum += __shfl_xor_sync(0xffffffffu, csum, o);
    ArgMax b2;
    b2.v = __shfl_xor_sync(0xffffffffu, am.v, o);
    b2.i = __shfl_xor_sync(0xffffffffu, am.i, o);
    am = better(am, b2);
  }
  const unsigned any_bad = __ballot_sync(0xffffffffu, bad);
  if (lane == 0) {
    sh.wc[w] = csum;
    sh.wa[w] = am;
    sh.wscan[w] = any_bad ? 1u : 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tc = 0;
    ArgMax ta{-INFINITY, 0x7fffffff};
    uint32_t tbad = 0;
    for (int i = 0; i < Sh::kNW; ++i) {
      tc += sh.wc[i];
      ta = better(ta, sh.wa[i]);
      tbad |= sh.wscan[i];
    }
    sh.cl_csum = tc;
    sh.cl_arg = ta;
    sh.cl_bad = tbad;
  }
  cl.sync();
  QuantResult r{0, -1, false};
  unsigned long long total = 0;
  ArgMax g{-INFINITY, 0x7fffffff};
  for (int q = 0; q < CL; ++q) {
    const Sh* o = cl.map_shared_rank(&sh, q);
    total += o->cl_csum;
    g = better(g, o->cl_arg);
    r.bad |= o->cl_bad != 0;
  }
  r.resid = (long long)T - (long long)total;
  r.argmax = g.i;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    if (v0 + i == g.i) {
      const long long ci = (long long)c[i] + r.resid;
      if (ci < (long long)floor_c || ci > (long long)T) r.bad = true;
      c[i] = (uint32_t)ci;
    }
  }
  return r;
}

// Exclusive prefix sum of the final counts into cdf_row.
template <int E, typename Sh>
__device__ void scan_round(const uint32_t (&c)[E], int v0, int V, uint32_t T, uint32_t* cdf_row,
                           cg::cluster_group& cl, Sh& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t local[E];
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    local[i] = run;
    run += c[i];
  }
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();                                 // wscan was read by the quantiser round
  if (lane == 31) sh.wscan[w] = inc;
  __syncthreads();
  uint32_t before = 0, total = 0;
  for (int i = 0; i < Sh::kNW; ++i) {
    if (i < w) before += sh.wscan[i];
    total += sh.wscan[i];
  }
  if (threadIdx.x == 0) sh.cl_total = total;
  cl.sync();
  uint32_t off = 0;
  for (int r = 0; r < (int)cl.block_rank(); ++r) off += cl.map_shared_rank(&sh, r)->cl_total;
  const uint32_t base = off + before + inc - run;
#pragma unroll
  for (int i = 0; i < E; ++i)
    if (v0 + i < V) cdf_row[v0 + i] = base + local[i];
  if (v0 <= V - 1 && V - 1 < v0 + E) cdf_row[V] = T;
}

// ======================================================================= step
// The per-token step of one stream (Sec. 3.3-3.7) on a cluster of CL CTAs
// of 4,096 / CL threads (CL = 8 or 16): always 128 warps, global warp
// gw = rank (128 / CL) + w owning the 32 E symbols from wbase = 32 E gw, lane
// l the E symbols from v0 = wbase + E l.  A reduction over the vocabulary
// takes one exchange: every warp sends its partials into every CTA's inbox,
// and once they are all there every warp reads the 128 of them from its own
// CTA's shared memory (lane l the four of global warps 4l .. 4l + 3) and
// reduces them with the same shuffles, so every warp of the cluster holds
// the same result, whatever the batch, the slot, the launch or the cluster
// shape.  The arithmetic is written with explicitly rounded operations and fixed
// approximations, so the single-step and the multi-position kernels below
// compute the same bits.  FULL: the vocabulary fills the cluster's 4,096 E
// symbols exactly (no symbol past V, every run 16-byte aligned).
constexpr int kClusterWarps = 128;               // four warp partials per lane of a reducing warp
template <int CL>
__host__ __device__ constexpr int step_threads() {
  return kClusterWarps * 32 / CL;
}
// A valid warp's count sum is at most T + eps K < 1.5 2^24 (T <= 2^24), so
// 128 clamped warp sums stay below 2^32; larger sums are flagged bad.
constexpr uint32_t kWarpCountCap = 3u << 23;
constexpr float kLog2e = 1.4426950408889634f;

// 2^x (PTX ex2.approx, flushing subnormal results to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// e^x = 2^(x log2 e) for the few scalar exponentials of a step.
__device__ __forceinline__ float exp_fast(float x) { return ex2_approx(__fmul_rn(x, kLog2e)); }

// Every CTA's inbox for one exchange (two alternate): each warp of the
// cluster stores its partials at its global index gw in every CTA's inbox,
// as posted remote stores made visible by a cluster barrier's release (the
// step kernel) or as asynchronous remote stores that complete their bytes on
// the receiving CTA's mbarrier (the prefill loop), so that afterwards every
// warp reduces them from its own CTA's shared memory.
struct StepSlot {
  float4 sm[kClusterWarps];   // softmax: warp maximum m_w, sum of exp(s - m_w), entropy part
  uint4 qn[kClusterWarps];    // quantiser: count sum, first maximum (value bits, index), bad flag
  float4 obs;                             // the observed token's p_tilde(t), p_ng(t), log p_tilde(t)
};

constexpr int kSnapBufs = 3;   // N-gram states in flight in the prefill loop
constexpr int kSeqMax = 1024;  // positions of one prefill chunk at most (a power of two dividing C < L <= 2,048)
struct StepShared {
  StepSlot slot[2];
  NgSnap ng[kSnapBufs];
  uint64_t xbar[2];           // the prefill loop's exchange rounds, by slot
};

// This thread's place in the cluster's split of the vocabulary.
struct Lanes {
  int rank, w, lane, gw, wbase, v0;
};
template <int E, int CL>
__device__ __forceinline__ Lanes lanes_of(int rank) {
  Lanes L;
  L.rank = rank;
  L.w = threadIdx.x >> 5;
  L.lane = threadIdx.x & 31;
  L.gw = rank * (kClusterWarps / CL) + L.w;
  L.wbase = L.gw * 32 * E;
  L.v0 = L.wbase + L.lane * E;
  return L;
}

template <bool FULL>
__device__ __forceinline__ bool in_vocab(int v, int V) {
  return FULL || v < V;
}
template <int E, bool FULL>
__device__ __forceinline__ void load_runf(const float* src, int v0, int V, float (&out)[E], float fill) {
  if (FULL) {
    const float4* s4 = reinterpret_cast<const float4*>(src + v0);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
      const float4 u = s4[q];
      out[4 * q] = u.x;
      out[4 * q + 1] = u.y;
      out[4 * q + 2] = u.z;
      out[4 * q + 3] = u.w;
    }
  } else {
    load_run<E>(src, v0, V, out, fill);
  }
}

// Lanes 0 .. CL - 1 store the warp's (warp-uniform) partial v at its global
// index in the inbox array `mine` of every CTA.
template <int CL, typename T>
__device__ __forceinline__ void push_part(cg::cluster_group& cl, T* mine, const Lanes& L, T v) {
  if (L.lane < CL) cl.map_shared_rank(mine, L.lane)[L.gw] = v;
}
// The observed token's values into every CTA's inbox.
template <int CL>
__device__ __forceinline__ void push_obs(cg::cluster_group& cl, float4* mine, float4 v) {
#pragma unroll
  for (int r = 0; r < CL; ++r) *cl.map_shared_rank(mine, r) = v;
}
// Exchange rounds of the prefill loop without a cluster barrier: each
// value goes to every CTA's inbox as an asynchronous remote store that
// completes its bytes on that CTA's mbarrier of the round's slot; a CTA
// arms its own mbarrier with the round's byte count and waits on it (acquire
// at cluster scope).  Slot s serves rounds s, s + 2, ...: a sender reaches
// round k + 2 only after every CTA's round k + 1 values, sent after each CTA
// finished reading round k.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t remote_addr(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async16(uint32_t raddr, uint32_t rbar, uint4 v) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(raddr),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(rbar)
               : "memory");
}
template <typename T>
__device__ __forceinline__ uint4 as_u4(const T& v) {
  static_assert(sizeof(T) == 16, "16-byte values");
  return *reinterpret_cast<const uint4*>(&v);
}
// Lanes 0 .. CL - 1: the warp's partial v to its global index in the array
// `mine` of CTA `lane`.
template <int CL, typename T>
__device__ __forceinline__ void push_part_async(T* mine, const Lanes& L, T v, uint64_t* bar) {
  if (L.lane < CL) st_async16(remote_addr(smem_addr(mine + L.gw), L.lane), remote_addr(smem_addr(bar), L.lane), as_u4(v));
}
template <int CL>
__device__ __forceinline__ void push_obs_async(float4* mine, float4 v, uint64_t* bar) {
#pragma unroll
  for (int r = 0; r < CL; ++r) st_async16(remote_addr(smem_addr(mine), r), remote_addr(smem_addr(bar), r), as_u4(v));
}
__device__ __forceinline__ void xbar_arm(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Bounded wait (2^22 polls, about 0.2 s) for the round's bytes; false when it gave up.
__device__ __forceinline__ bool xbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  unsigned long long t0 = 0;
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 63) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t0 == 0) t0 = t;
      else if (t - t0 > 200000000ull) return false;
    }
  }
  return false;
}
// Bytes of one round: the softmax partials and / or the quantiser partials
// with the observed token's values.
constexpr uint32_t kRoundSm = kClusterWarps * 16, kRoundQ = kClusterWarps * 16 + 16;

// The inbox entries of global warps 4 lane .. 4 lane + 3.
template <typename T>
__device__ __forceinline__ void local_parts(const T* arr, int lane, T (&v)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = arr[4 * lane + i];
}

// p_ng of the thread's symbols (Sec. 3.4), the closed form
// P(t) = A (c(t) + 1) / (N + V) + sum_k beta_k cnt_k(t) / n_k with the weights
// in g.  Each warp adds the context slots' masses of its own 32 E symbols into
// its region spw of shared memory (order by order, so a symbol's sum is taken
// in the order k = 0, 1, 2); each lane then reads its E sums and zeroes them.
template <int E>
__device__ __forceinline__ void ngram_scatter(const NgSnap& g, float* spw, const Lanes& L) {
  constexpr int kSpan = 32 * E;
  __syncwarp();                                    // the region's last reads and zeroes are done
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) {
    const int ns = g.ns[k];
    const float coef = g.coef[k];
#pragma unroll
    for (int h = 0; h < kMaxSlots / 32; ++h) {
      const int q = L.lane + 32 * h;
      if (q < ns) {
        const int2 tc = g.tc[k][q];
        const int t = tc.x - L.wbase;
        if ((unsigned)t < (unsigned)kSpan) spw[t] = __fadd_rn(spw[t], __fmul_rn(coef, (float)tc.y));
      }
    }
    __syncwarp();
  }
}
template <int E, bool FULL>
__device__ __forceinline__ void ngram_read(float cu, float* spw, const Lanes& L, int V, const int (&cnt)[E],
                                           float (&png)[E]) {
  __syncwarp();                                    // every lane's slot masses are in
  float4* s4 = reinterpret_cast<float4*>(spw + L.lane * E);
#pragma unroll
  for (int q = 0; q < E / 4; ++q) {
    const float4 u = s4[q];
    const float sv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ii = 4 * q + i;
      png[ii] = in_vocab<FULL>(L.v0 + ii, V) ? __fmaf_rn(cu, (float)(cnt[ii] + 1), sv[i]) : 0.f;
    }
    s4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}
template <int E, bool FULL>
__device__ __forceinline__ void ngram_probs(const NgSnap& g, float* spw, const Lanes& L, int V, const int (&cnt)[E],
                                            float (&png)[E]) {
  ngram_scatter<E>(g, spw, L);
  ngram_read<E, FULL>(g.cu, spw, L, V, cnt, png);
}

template <int E>
__device__ __forceinline__ void zero_region(float* spw, int lane) {
  float4* s4 = reinterpret_cast<float4*>(spw + lane * E);
#pragma unroll
  for (int q = 0; q < E / 4; ++q) s4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Biased logits s = z / tau + b (Sec. 3.6); -inf past the vocabulary.
template <int E, bool FULL>
__device__ __forceinline__ void biased_logits(const float (&z)[E], const float (&bias)[E], float inv_tau, int v0,
                                              int V, float (&s)[E]) {
#pragma unroll
  for (int i = 0; i < E; ++i) s[i] = in_vocab<FULL>(v0 + i, V) ? __fmaf_rn(z[i], inv_tau, bias[i]) : -INFINITY;
}

// The thread's part of the N-gram entropy in bits, -sum p log2 p (Sec. 3.7).
template <int E>
__device__ __forceinline__ float entropy_part(const float (&png)[E]) {
  float h = 0.f;
#pragma unroll
  for (int i = 0; i < E; ++i)
    if (png[i] > 0.f) h = __fmaf_rn(-png[i], log2f(png[i]), h);
  return h;
}

// Softmax partials of the warp: its maximum m_w of s, e_i = exp(s_i - m_w)
// = 2^(s_i log2 e - m_w log2 e) and the sum of the e_i; h (a second sum, the
// entropy part of the confidence skip) is reduced alongside when `with_h`.
template <int E>
__device__ __forceinline__ float4 softmax_part(const float (&s)[E], float (&e)[E], float h, bool with_h) {
  float m = -INFINITY;
#pragma unroll
  for (int i = 0; i < E; ++i) m = fmaxf(m, s[i]);
  m = warp_max(m);
  float t = 0.f;
  if (m == -INFINITY) {                           // no symbol of the warp in the vocabulary
#pragma unroll
    for (int i = 0; i < E; ++i) e[i] = 0.f;
  } else {
    const float mb = -__fmul_rn(m, kLog2e);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      e[i] = ex2_approx(__fmaf_rn(s[i], kLog2e, mb));
      t = __fadd_rn(t, e[i]);
    }
  }
  return make_float4(m, warp_sum(t), with_h ? warp_sum(h) : 0.f, 0.f);
}

// The cluster's softmax: M = max m_w, S = sum_w t_w exp(m_w - M), and the
// second sum H.
struct Soft {
  float M, S, H;
};
__device__ __forceinline__ Soft softmax_reduce(const float4 (&v)[4], bool with_h) {
  const float M = warp_max(fmaxf(fmaxf(v[0].x, v[1].x), fmaxf(v[2].x, v[3].x)));
  float s = 0.f, h = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (v[i].y > 0.f) s = __fmaf_rn(v[i].y, exp_fast(__fsub_rn(v[i].x, M)), s);
    h = __fadd_rn(h, v[i].z);
  }
  return Soft{M, warp_sum(s), with_h ? warp_sum(h) : 0.f};
}

// p_tilde of the thread's symbols: e_i exp(m_w - M) / S.
template <int E>
__device__ __forceinline__ void probs_tilde(const float (&e)[E], float m_w, const Soft& sm, float (&pt)[E]) {
  const float f = m_w == -INFINITY ? 0.f : __fdividef(exp_fast(__fsub_rn(m_w, sm.M)), sm.S);
#pragma unroll
  for (int i = 0; i < E; ++i) pt[i] = __fmul_rn(e[i], f);
}

// The step's normaliser, maximum and mixer weights are finite (the quantiser
// then needs no per-symbol range check).
__device__ __forceinline__ bool finite_step(const Soft& sm, float2 w) {
  return isfinite(sm.M) && isfinite(sm.S) && sm.S >= 0.998f && isfinite(w.x) && isfinite(w.y);
}

// The mixer's weights softmax(theta) (Sec. 3.5).
__device__ __forceinline__ float2 mix_weights(float th0, float th1) {
  const float tm = fmaxf(th0, th1);
  const float e0 = exp_fast(__fsub_rn(th0, tm)), e1 = exp_fast(__fsub_rn(th1, tm));
  const float z = __fadd_rn(e0, e1);
  return make_float2(__fdividef(e0, z), __fdividef(e1, z));
}

// The coded distribution: p_ng under the confidence skip (Sec. 3.7), the mix
// w0 p_tilde + w1 p_ng (Sec. 3.5), or p_tilde alone during the warm-up.
template <int E>
__device__ __forceinline__ void coded_probs(const float (&pt)[E], const float (&png)[E], float2 w, bool skipped,
                                            bool mixing, float (&p)[E]) {
  if (skipped) {
#pragma unroll
    for (int i = 0; i < E; ++i) p[i] = png[i];
  } else if (mixing) {
#pragma unroll
    for (int i = 0; i < E; ++i) p[i] = __fmaf_rn(w.x, pt[i], __fmul_rn(w.y, png[i]));
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) p[i] = pt[i];
  }
}

// Quantiser partials (Sec. 3.3): the thread's counts c_i = max(floor(p_i K),
// floor) and the warp's count sum, first maximum and bad flag, packed for
// publication.  scan: also excl = the counts of the warp's lanes below this
// one.  am_i / am_c = the thread's first maximum and its count.
// `sure`: the step's softmax normaliser S >= 0.998 (it is at least the
// maximum's numerator, 1 up to rounding), its maximum and the mixer weights
// are finite (uniform across the cluster), so every p is a finite value in
// [0, 1.0021) (numerators e <= 1 + 2^-22 over S, N-gram probabilities <= 1,
// weights summing to 1): the product p K stays below 2^24, where the
// round-toward-zero product has the exact product's integer part, and no
// per-symbol range check is needed.  Otherwise every value is checked.
template <int E, bool FULL>
__device__ __forceinline__ uint4 quant_part(const float (&p)[E], const Lanes& L, int V, uint32_t K, float Kf,
                                            uint32_t floor_c, bool scan, bool sure, uint32_t (&c)[E], uint32_t& excl,
                                            int& am_i, uint32_t& am_c) {
  bool bad = false;
  uint32_t ts = 0;
  float amv = -INFINITY;
  am_i = 0x7fffffff;
  am_c = 0;
  if (sure) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const bool in = in_vocab<FULL>(L.v0 + i, V);
      const uint32_t q = __float2uint_rz(__fmul_rz(p[i], Kf));
      c[i] = in ? max(q, floor_c) : 0u;
      ts += c[i];
      if (in && p[i] > amv) {                      // strict: keeps the first maximum
        amv = p[i];
        am_i = L.v0 + i;
        am_c = c[i];
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const bool in = in_vocab<FULL>(L.v0 + i, V);
      const uint32_t q = floor_count(p[i], K, Kf, bad);
      c[i] = in ? max(q, floor_c) : 0u;
      ts += c[i];
      if (in && p[i] > amv) {
        amv = p[i];
        am_i = L.v0 + i;
        am_c = c[i];
      }
    }
  }
  if (ts > kWarpCountCap) {                      // invalid: keeps the warp's sum below 2^32
    bad = true;
    ts = kWarpCountCap;
  }
  uint32_t wsum;
  if (scan) {
    uint32_t inc = ts;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (L.lane >= o) inc += t;
    }
    excl = inc - ts;
    wsum = __shfl_sync(0xffffffffu, inc, 31);
  } else {
    wsum = ts;
#pragma unroll
    for (int o = 16; o; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  }
  // first maximum: value bits (p >= 0 orders as unsigned) over the inverted index
  unsigned long long key =
      ((unsigned long long)(amv > 0.f ? __float_as_uint(amv) : 0u) << 32) | (uint32_t)~(uint32_t)am_i;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    key = k2 > key ? k2 : key;
  }
  bad = __any_sync(0xffffffffu, bad) || wsum > kWarpCountCap;
  return make_uint4(bad ? kWarpCountCap : wsum, (uint32_t)(key >> 32), ~(uint32_t)key, bad ? 1u : 0u);
}

// The cluster's quantiser results: the residual T - sum c (added to the first
// maximum), the first maximum, and the counts of the warps before this one.
struct Quant {
  long long resid, woff;
  int argmax;
  bool bad;
};
__device__ __forceinline__ Quant quant_reduce(const uint4 (&v)[4], const Lanes& L, uint32_t T) {
  uint32_t tot = 0, off = 0;
  unsigned long long key = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    tot += v[i].x;
    if (4 * L.lane + i < L.gw) off += v[i].x;
    const unsigned long long k = ((unsigned long long)v[i].y << 32) | (uint32_t)~v[i].z;
    key = k > key ? k : key;
    bad |= v[i].w != 0u;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    off += __shfl_xor_sync(0xffffffffu, off, o);
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    key = k2 > key ? k2 : key;
  }
  Quant q;
  q.resid = (long long)T - (long long)tot;
  q.woff = (long long)off;
  q.argmax = (int)~(uint32_t)key;
  q.bad = __any_sync(0xffffffffu, bad);
  return q;
}

// Mixer update with the observed token (Sec. 3.5): exponential weights with
// rate eta, or one gradient step of the mixed NLL; scale = the head's step
// factor (1, or w0 p_tilde(t) / p(t) under the mixed NLL).
__device__ __forceinline__ void mixer_update(const Dims& D, bool mixing, float2 w, float pts, float pngs, float lpt,
                                             float& th0, float& th1, float& scale) {
  scale = 1.f;
  if (!mixing) return;
  if (D.rule == NC_RULE_MIXED_NLL) {
    const float pm = __fmaf_rn(w.x, pts, __fmul_rn(w.y, pngs));
    const float r0 = __fdividef(__fmul_rn(w.x, pts), pm), r1 = __fdividef(__fmul_rn(w.y, pngs), pm);
    scale = r0;
    th0 = __fsub_rn(th0, __fmul_rn(D.alpha, __fsub_rn(w.x, r0)));
    th1 = __fsub_rn(th1, __fmul_rn(D.alpha, __fsub_rn(w.y, r1)));
  } else {
    const float a0 = __fmaf_rn(D.eta, lpt, th0), a1 = __fmaf_rn(D.eta, __logf(pngs), th1);
    const float am = fmaxf(a0, a1);
    const float lse = __fadd_rn(am, __logf(__fadd_rn(exp_fast(__fsub_rn(a0, am)), exp_fast(__fsub_rn(a1, am)))));
    th0 = __fsub_rn(a0, lse);
    th1 = __fsub_rn(a1, lse);
  }
}

// Head update (Sec. 3.6): b <- b - step (p_tilde - onehot(t)); `own`: t is
// one of the thread's symbols (for the others p_tilde - 0 = p_tilde exactly).
template <int E>
__device__ __forceinline__ void head_update(float (&bias)[E], const float (&pt)[E], float step, int v0, int t,
                                            bool own) {
  if (own) {
#pragma unroll
    for (int i = 0; i < E; ++i) bias[i] = __fmaf_rn(-step, __fsub_rn(pt[i], v0 + i == t ? 1.f : 0.f), bias[i]);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) bias[i] = __fmaf_rn(-step, pt[i], bias[i]);
  }
}

// The owner's value at its symbol t (no dynamic register indexing).
template <int E, typename T>
__device__ __forceinline__ T pick(const T (&a)[E], int v0, int t) {
  T r = T(0);
#pragma unroll
  for (int i = 0; i < E; ++i)
    if (v0 + i == t) r = a[i];
  return r;
}
// Counts of the thread's symbols below t, and t's own.
template <int E>
__device__ __forceinline__ void counts_around(const uint32_t (&c)[E], int v0, int t, uint32_t& below, uint32_t& ct) {
  below = 0;
  ct = 0;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    if (v0 + i < t) below += c[i];
    if (v0 + i == t) ct = c[i];
  }
}

// The coder interval [lo, hi) of t (Sec. 3.3) from the cluster's quantiser
// results and the owner's counts below t within its warp.
__device__ __forceinline__ void write_interval(uint32_t* iv, const Quant& q, int t, uint32_t below, uint32_t ct) {
  const long long lo = q.woff + below + (q.argmax < t ? q.resid : 0);
  const long long hi = lo + ct + (q.argmax == t ? q.resid : 0);
  iv[0] = (uint32_t)lo;
  iv[1] = (uint32_t)hi;
}

// The first maximum's final count must stay within [floor, T].
__device__ __forceinline__ bool final_count_bad(const Quant& q, int am_i, uint32_t am_c, uint32_t floor_c, uint32_t T) {
  if (am_i != q.argmax) return false;
  const long long cf = (long long)am_c + q.resid;
  return cf < (long long)floor_c || cf > (long long)T;
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy one N-gram state into shared memory (asynchronously, 16 bytes per thread).
__device__ __forceinline__ void snap_copy_async(NgSnap* dst, const NgSnap* src) {
  constexpr int kPieces = (int)(sizeof(NgSnap) / 16);
  static_assert(kPieces <= step_threads<16>(), "one piece per thread");
  if ((int)threadIdx.x < kPieces)
    cp_async16(reinterpret_cast<char*>(dst) + 16 * threadIdx.x, reinterpret_cast<const char*>(src) + 16 * threadIdx.x);
  cp_async_commit();
}

__device__ void ngram_update_row(const Dims& D, const Batch& b, int j, int warp, int lane);
__device__ void ng_snapshot(const Dims& D, const StreamDev& st, NgSnap* out, int tid, int nthr);

// One position of stream row j: predict (the coded distribution's CDF and /
// or the coder interval of the observed token) and / or update (head and
// mixer, then the N-gram and the stream's bookkeeping).  The decoder runs
// the two in separate launches (it learns the token in between); the
// arithmetic is the same in either case.
template <int E, bool FULL, int CL>
__global__ void __launch_bounds__(step_threads<CL>(), 1) k_vocab(Dims D, Batch b, VocabIO io) {
  extern __shared__ float4 dyn4[];
  __shared__ StepShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int j = blockIdx.x / CL;
  // after a prefill the previous kernel updated the stream's state: nothing
  // of it may be read before that kernel completed
  if (b.z_in) {
    pdl_wait();
    pdl_trigger();
  }
  if (j >= *b.nB) return;                        // uniform across the cluster
  const Lanes L = lanes_of<E, CL>((int)cl.block_rank());
  StreamDev& st = b.st[b.slots[j]];
  const int V = D.V;
  const bool ngram = D.order > 0;
  float* spw = reinterpret_cast<float*>(dyn4) + L.w * 32 * E;

  // ---- the stream's state of earlier steps, before the wait on the LM head
  float bias[E];
  int cnt[E];
  if (D.use_head) {
    load_runf<E, FULL>(st.bias, L.v0, V, bias, 0.f);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) bias[i] = 0.f;
  }
  if (ngram) {
    load_counts<E>(st.uni, L.v0, V, cnt);
    zero_region<E>(spw, L.lane);
    ng_snapshot(D, st, &sh.ng[0], threadIdx.x, step_threads<CL>());
    __syncthreads();
  }
  const int i_tok = st.n_coded + 1;              // 1-based index of the token being coded
  float th0 = st.theta[0], th1 = st.theta[1];
  float z[E];
  if (b.z_in) load_runf<E, FULL>(b.z_in + (size_t)b.z_idx[j] * V, L.v0, V, z, -INFINITY);
  if (!b.z_in) {
    pdl_wait();
    pdl_trigger();
  }
  const int t = (io.update || io.intervals) ? b.obs[j] : -1;
  if (io.update && (t < 0 || t >= V)) {          // rejected on the host; never index with it
    if (L.rank == 0 && threadIdx.x == 0) atomicOr(&st.status, ST_BAD_TOKEN);
    return;                                      // uniform across the cluster
  }
  if (!b.z_in) load_runf<E, FULL>(st.z, L.v0, V, z, -INFINITY);
  // probes: every step, or only at the stream's probe_tok-th token
  const bool probe = io.probe_tok == 0 || io.probe_tok == (int64_t)i_tok;
  const size_t prow = (size_t)(io.probe_row ? io.probe_row[j] : j) * V;
  if (probe && io.probe_z) store_run<E>(io.probe_z + prow, L.v0, V, z);

  // ---- softmax (Sec. 3.6) and the N-gram distribution
  float png[E];
  if (ngram) {
    ngram_probs<E, FULL>(sh.ng[0], spw, L, V, cnt, png);
    if (probe && io.probe_png) store_run<E>(io.probe_png + prow, L.v0, V, png);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) png[i] = 0.f;
  }
  float s[E], e[E];
  biased_logits<E, FULL>(z, bias, 1.0f / D.tau, L.v0, V, s);
  const bool owner = t >= L.v0 && t < L.v0 + E;
  float s_t = 0.f, png_t = 0.f;
  if (owner) {
    s_t = pick<E>(s, L.v0, t);
    png_t = pick<E>(png, L.v0, t);
  }
  const float4 part = softmax_part<E>(s, e, D.skip ? entropy_part<E>(png) : 0.f, D.skip != 0);
  push_part<CL>(cl, sh.slot[0].sm, L, part);
  cl.sync();
  float4 smv[4];
  local_parts(sh.slot[0].sm, L.lane, smv);
  const Soft sm = softmax_reduce(smv, D.skip != 0);
  const bool skipped = D.skip && sm.H < kSkipBits;
  float pt[E];
  probs_tilde<E>(e, part.x, sm, pt);
  if (probe && io.probe_pt) store_run<E>(io.probe_pt + prow, L.v0, V, pt);

  // ---- the coded distribution and its counts (Sec. 3.3, 3.5)
  const bool mixing = ngram && i_tok > D.warmup;
  const float2 w = mix_weights(th0, th1);
  float p[E];
  coded_probs<E>(pt, png, w, skipped, mixing, p);
  if (probe && io.probe_p) store_run<E>(io.probe_p + prow, L.v0, V, p);
  if (owner)
    push_obs<CL>(cl, &sh.slot[1].obs,
             make_float4(pick<E>(pt, L.v0, t), png_t, __fsub_rn(__fsub_rn(s_t, sm.M), __logf(sm.S)), 0.f));
  const uint32_t T = 1u << D.log2T, K = T - (uint32_t)V * D.floor;
  uint32_t c[E], excl = 0, am_c = 0, below_t = 0, c_t = 0;
  int am_i = 0x7fffffff;
  const bool scan = io.cdf || (t >= L.wbase && t < L.wbase + 32 * E);
  if (io.predict) {
    const uint4 qp = quant_part<E, FULL>(p, L, V, K, (float)K, D.floor, scan, finite_step(sm, w), c, excl, am_i, am_c);
    push_part<CL>(cl, sh.slot[1].qn, L, qp);
    if (owner) {
      counts_around<E>(c, L.v0, t, below_t, c_t);
      below_t += excl;
    }
  }
  cl.sync();
  if (io.predict) {
    uint4 qnv[4];
    local_parts(sh.slot[1].qn, L.lane, qnv);
    const Quant q = quant_reduce(qnv, L, T);
    if (io.intervals && owner)
      write_interval(io.intervals + 2 * ((size_t)j * io.interval_stride + (i_tok - 1)), q, t, below_t, c_t);
    if (io.cdf) {
      uint32_t* row = io.cdf + (size_t)j * (V + 1);
      long long run = q.woff + excl;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int v = L.v0 + i;
        if (in_vocab<FULL>(v, V)) {
          row[v] = (uint32_t)(run + (q.argmax < v ? q.resid : 0));
          run += c[i];
        }
      }
      if (L.v0 <= V - 1 && V - 1 < L.v0 + E) row[V] = T;
    }
    if ((q.bad && L.rank == 0 && threadIdx.x == 0) || final_count_bad(q, am_i, am_c, D.floor, T))
      atomicOr(&st.status, ST_NUMERIC);
  }

  // ---- head and mixer update (a skipped token teaches the N-gram only)
  if (io.update && !skipped) {
    const float4 o = sh.slot[1].obs;
    float scale;
    mixer_update(D, mixing, w, o.x, o.y, o.z, th0, th1, scale);
    if (D.use_head) {
      head_update<E>(bias, pt, __fmul_rn(D.alpha, scale), L.v0, t, owner);
      store_run<E>(st.bias, L.v0, V, bias);
    }
    if (L.rank == 0 && threadIdx.x == 0) {
      st.theta[0] = th0;
      st.theta[1] = th1;
      st.pt_obs = o.x;
      st.png_obs = o.y;
    }
  }
  cl.sync();   // every CTA has read the others' slots and the stream's state
  if (io.update && io.ngram && L.rank == 0) ngram_update_row(D, b, j, L.w, L.lane);
}

// The vocabulary passes of a prefill chunk (encoder): the cluster of stream
// row j runs its positions r = 0 .. m - 1 in order while j < nb_step[r],
// with the bias, the unigram counts, the mixer's log-weights and the position
// kept on chip and the N-gram state of each prediction read from snap (made
// ahead by k_ngram_seq).  Under the log-loss mixer the head's step does not
// wait for the mixer, so position r's quantiser and mixer results share the
// exchange round of position r + 1's softmax: one round per position, with
// no cluster barrier (each CTA waits on its own mbarrier for the round's
// bytes).  The next position's logits, token and activity and the N-gram
// state two positions ahead are fetched while the round's values travel.
template <int E, bool FULL, int CL>
__global__ void __launch_bounds__(step_threads<CL>(), 1)
    k_vocab_seq(Dims D, Batch b, VocabIO io, int m, int n_streams, const float* zrows, const int32_t* nb_step,
                const int32_t* obs_step, const NgSnap* snap) {
  extern __shared__ float4 dyn4[];
  __shared__ StepShared sh;
  __shared__ int32_t s_obs[kSeqMax], s_nb[kSeqMax];   // the chunk's tokens and active rows, per position
  cg::cluster_group cl = cg::this_cluster();
  const int j = blockIdx.x / CL;
  pdl_wait();
  pdl_trigger();
  if (m < 1 || j >= nb_step[0]) return;          // uniform across the cluster
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    s_obs[i] = obs_step[(size_t)i * n_streams + j];
    s_nb[i] = nb_step[i];
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 2; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sh.xbar[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const Lanes L = lanes_of<E, CL>((int)cl.block_rank());
  StreamDev& st = b.st[b.slots[j]];
  const int V = D.V;
  const bool ngram = D.order > 0;
  const bool fused = D.rule != NC_RULE_MIXED_NLL;
  const float inv_tau = 1.0f / D.tau;
  const uint32_t T = 1u << D.log2T, K = T - (uint32_t)V * D.floor;
  const float Kf = (float)K;
  float* spw = reinterpret_cast<float*>(dyn4) + L.w * 32 * E;
  const float* zj = zrows + (size_t)b.z_idx[j] * V;
  const NgSnap* gj = ngram ? snap + b.z_idx[j] : nullptr;

  float bias[E], z[E];
  int cnt[E];
  if (D.use_head) {
    load_runf<E, FULL>(st.bias, L.v0, V, bias, 0.f);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) bias[i] = 0.f;
  }
  __syncthreads();                               // the tokens and active rows are in shared memory
  bool act1 = 1 < m && j < s_nb[1];              // positions r + 1 and r + 2 exist
  bool act2 = act1 && 2 < m && j < s_nb[2];
  if (ngram) {
    load_counts<E>(st.uni, L.v0, V, cnt);
    zero_region<E>(spw, L.lane);
    snap_copy_async(&sh.ng[0], gj);
    if (act1) snap_copy_async(&sh.ng[1], gj + 1);
    if (act2) snap_copy_async(&sh.ng[2], gj + 2);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) cnt[i] = 0;
  }
  load_runf<E, FULL>(zj, L.v0, V, z, -INFINITY);
  int t = s_obs[0];
  float th0 = st.theta[0], th1 = st.theta[1];
  const int n0 = st.n_coded;
  if (ngram) cp_async_wait_all();
  cl.sync();                                     // the first N-gram states are in shared memory, every
                                                 // CTA's exchange barriers initialised
  if (ngram) ngram_scatter<E>(sh.ng[0], spw, L);

  // the previous position's values its quantiser and mixer step need
  bool pend = false, p_skip = false, p_mix = false, p_own = false;
  int p_t = 0, p_pos = 0, p_am_i = 0x7fffffff;
  uint32_t p_below = 0, p_ct = 0, p_am_c = 0;
  float2 p_w = make_float2(0.f, 0.f);
  float last_pts = st.pt_obs, last_pngs = st.png_obs;
  int nb = 0;                                    // exchange rounds taken
  bool xok = true;                               // no exchange wait has given up
  int r = 0, t_last = -1;

  // interval, numeric checks and mixer step of the pending position from its
  // inbox `slot`
  auto finish = [&](const StepSlot& slot, const float (&pt)[E], bool with_head) {
    uint4 qv[4];
    local_parts(slot.qn, L.lane, qv);
    const Quant q = quant_reduce(qv, L, T);
    const float4 o = slot.obs;
    if (p_own)
      write_interval(io.intervals + 2 * ((size_t)j * io.interval_stride + p_pos), q, p_t, p_below, p_ct);
    if ((q.bad && L.rank == 0 && threadIdx.x == 0) || final_count_bad(q, p_am_i, p_am_c, D.floor, T))
      atomicOr(&st.status, ST_NUMERIC);
    if (!p_skip) {
      float scale;
      mixer_update(D, p_mix, p_w, o.x, o.y, o.z, th0, th1, scale);
      if (with_head && D.use_head)
        head_update<E>(bias, pt, __fmul_rn(D.alpha, scale), L.v0, p_t, p_t >= L.v0 && p_t < L.v0 + E);
      last_pts = o.x;
      last_pngs = o.y;
    }
  };

  bool live = true;
  while (live) {
    if (t < 0 || t >= V) {                       // rejected on the host; never index with it
      if (L.rank == 0 && threadIdx.x == 0) atomicOr(&st.status, ST_BAD_TOKEN);
      break;                                     // uniform across the cluster
    }
    const bool more = act1;
    // probes at the stream's probe_tok-th token (uniform across the cluster)
    const bool probe = io.probe_tok == (int64_t)(n0 + r + 1);
    const size_t prow = (size_t)(io.probe_row ? io.probe_row[j] : j) * V;
    if (probe && io.probe_z) store_run<E>(io.probe_z + prow, L.v0, V, z);

    // ---- softmax partials of position r (its slot masses are in spw)
    float png[E];
    if (ngram) {
      ngram_read<E, FULL>(sh.ng[r % kSnapBufs].cu, spw, L, V, cnt, png);
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i) png[i] = 0.f;
    }
    if (probe && io.probe_png) store_run<E>(io.probe_png + prow, L.v0, V, png);
    float s[E], e[E];
    biased_logits<E, FULL>(z, bias, inv_tau, L.v0, V, s);
    const bool owner = t >= L.v0 && t < L.v0 + E;
    float s_t = 0.f, png_t = 0.f;
    if (owner) {
      s_t = pick<E>(s, L.v0, t);
      png_t = pick<E>(png, L.v0, t);
    }
    const float4 part = softmax_part<E>(s, e, D.skip ? entropy_part<E>(png) : 0.f, D.skip != 0);
    StepSlot& in = sh.slot[nb & 1];
    uint64_t* xb = &sh.xbar[nb & 1];
    push_part_async<CL>(in.sm, L, part, xb);
    if (ngram) cp_async_wait_all();              // the state of position r + 2, added after this round
    if (threadIdx.x == 0) xbar_arm(xb, kRoundSm + (pend ? kRoundQ : 0));
    // while the round's values travel: position r + 1's logits, token and
    // slot masses (its state arrived two rounds ago), the activity of r + 3
    int t_n = 0;
    bool act3 = false;
    if (more) {
      load_runf<E, FULL>(zj + (size_t)(r + 1) * V, L.v0, V, z, -INFINITY);
      t_n = s_obs[r + 1];
      act3 = act2 && r + 3 < m && j < s_nb[r + 3];
      if (ngram) ngram_scatter<E>(sh.ng[(r + 1) % kSnapBufs], spw, L);
    }
    if (!__all_sync(0xffffffffu, xbar_wait(xb, (uint32_t)(nb >> 1) & 1u))) {
      xok = false;
      pend = false;
      break;                                     // the other warps give up on their next round
    }
    // every warp of the cluster has added position r's masses (before its
    // partials went out): its buffer takes the state of r + 3
    if (ngram && act3) snap_copy_async(&sh.ng[(r + 3) % kSnapBufs], gj + r + 3);
    ++nb;
    float4 smv[4];
    local_parts(in.sm, L.lane, smv);
    const Soft sm = softmax_reduce(smv, D.skip != 0);
    float pt[E];
    if (pend) {                                  // position r - 1 (log-loss mixer: no head step here)
      finish(in, pt, false);
      pend = false;
    }

    // ---- position r: probabilities, counts, head step
    const bool skipped = D.skip && sm.H < kSkipBits;
    probs_tilde<E>(e, part.x, sm, pt);
    const bool mixing = ngram && n0 + r + 1 > D.warmup;
    const float2 w = mix_weights(th0, th1);
    float p[E];
    coded_probs<E>(pt, png, w, skipped, mixing, p);
    if (probe && io.probe_pt) store_run<E>(io.probe_pt + prow, L.v0, V, pt);
    if (probe && io.probe_p) store_run<E>(io.probe_p + prow, L.v0, V, p);
    StepSlot& nx = sh.slot[nb & 1];
    if (owner)
      push_obs_async<CL>(&nx.obs,
                         make_float4(pick<E>(pt, L.v0, t), png_t, __fsub_rn(__fsub_rn(s_t, sm.M), __logf(sm.S)), 0.f),
                         &sh.xbar[nb & 1]);
    uint32_t c[E], excl = 0;
    const bool scan = io.intervals && t >= L.wbase && t < L.wbase + 32 * E;
    const uint4 qp = quant_part<E, FULL>(p, L, V, K, Kf, D.floor, scan, finite_step(sm, w), c, excl, p_am_i, p_am_c);
    push_part_async<CL>(nx.qn, L, qp, &sh.xbar[nb & 1]);
    p_own = owner && io.intervals;
    if (owner) {
      counts_around<E>(c, L.v0, t, p_below, p_ct);
      p_below += excl;
      if (ngram) {
#pragma unroll
        for (int i = 0; i < E; ++i)
          if (L.v0 + i == t) cnt[i] += 1;
      }
    }
    p_t = t;
    p_pos = n0 + r;                              // the token's index in its stream
    p_skip = skipped;
    p_mix = mixing;
    p_w = w;
    t_last = t;
    if (fused) {
      if (!skipped && D.use_head) head_update<E>(bias, pt, __fmul_rn(D.alpha, 1.f), L.v0, t, owner);
      pend = true;
    } else {
      if (threadIdx.x == 0) xbar_arm(&sh.xbar[nb & 1], kRoundQ);
      if (!__all_sync(0xffffffffu, xbar_wait(&sh.xbar[nb & 1], (uint32_t)(nb >> 1) & 1u))) {
        xok = false;
        break;
      }
      ++nb;
      finish(nx, pt, true);
    }
    ++r;
    t = t_n;
    act1 = act2;
    act2 = act3;
    live = more;
  }
  if (pend) {
    if (threadIdx.x == 0) xbar_arm(&sh.xbar[nb & 1], kRoundQ);
    if (__all_sync(0xffffffffu, xbar_wait(&sh.xbar[nb & 1], (uint32_t)(nb >> 1) & 1u))) {
      ++nb;
      StepSlot& in = sh.slot[(nb - 1) & 1];
      float none[E];
      finish(in, none, false);
    } else {
      xok = false;
    }
  }
  if (!xok && L.lane == 0) atomicOr(&st.status, ST_TIMEOUT);
  if (ngram) cp_async_wait_all();                // no copy outlives the kernel
  cl.sync();   // every CTA is done with the others' shared memory
  if (r == 0) return;

  // ---- the stream's state after the chunk's r positions
  if (D.use_head) store_run<E>(st.bias, L.v0, V, bias);
  if (ngram) store_counts<E>(st.uni, L.v0, V, cnt);
  if (L.rank == 0 && threadIdx.x == 0) {
    st.theta[0] = th0;
    st.theta[1] = th1;
    st.pt_obs = last_pts;
    st.png_obs = last_pngs;
    // the window slides by C whenever it is full before a token is coded
    const int last = n0 + r - 1;
    int start = st.kv_start;
    for (int a = start + D.L; a <= last; a += D.C) start += D.C;
    st.kv_start = start;
    st.n_coded = n0 + r;
    st.last_tok = t_last;
  }
}

// --------------------------------------------------------------- N-gram tables
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// Context of length k ending at the most recent token: ids < 2^16 packed
// injectively into 48 bits.
__device__ __forceinline__ unsigned long long ctx_key(const int32_t* hist, int k) {
  unsigned long long key = 0;
  for (int q = 3 - k; q < 3; ++q) key = (key << 16) | (unsigned long long)(uint32_t)hist[q];
  return key;
}

// Find (insert = false) or find-or-insert a context; returns the entry index
// or -1 (absent, or table full on insert).  Linear probing, bounded by the
// capacity.
__device__ int ng_find(StreamDev& st, int k, unsigned long long key, bool insert) {
  const int cap = st.cap_mask + 1;
  unsigned long long* keys = st.keys[k];
  int h = (int)(mix64(key) & (unsigned long long)st.cap_mask);
  for (int probe = 0; probe < cap; ++probe) {
    const unsigned long long kk = keys[h];
    if (kk == key) return st.idx[k][h];
    if (kk == kEmptyKey) {
      if (!insert) return -1;
      const int ei = st.n_ent[k];
      if (ei >= st.max_len) {
        atomicOr(&st.status, ST_TABLE_FULL);
        return -1;
      }
      st.n_ent[k] = ei + 1;
      keys[h] = key;
      st.idx[k][h] = ei;
      st.ent[k][ei].nslots = 0;
      st.ent[k][ei].n = 0;
      return ei;
    }
    h = (h + 1) & st.cap_mask;
  }
  if (insert) atomicOr(&st.status, ST_TABLE_FULL);
  return -1;
}

// The closed form's weights of the interpolation (Sec. 3.4): lambda_k =
// n_k / (n_k + 5), A = prod (1 - lambda_k), beta_k = lambda_k prod_{j>k}
// (1 - lambda_j), coefficient beta_k / n_k, and cu = A / (N + V).
__device__ void ng_weights(const float (&nk)[kMaxOrder], const bool (&has)[kMaxOrder], int N, int V,
                           float (&coef)[kMaxOrder], float& cu) {
  float lam[kMaxOrder];
  for (int k = 0; k < kMaxOrder; ++k) lam[k] = has[k] ? nk[k] / (nk[k] + 5.0f) : 0.f;
  float A = 1.f;
  for (int k = 0; k < kMaxOrder; ++k) A *= (1.f - lam[k]);
  for (int k = 0; k < kMaxOrder; ++k) {
    float beta = lam[k];
    for (int q = k + 1; q < kMaxOrder; ++q) beta *= (1.f - lam[q]);
    coef[k] = has[k] ? beta / nk[k] : 0.f;
  }
  cu = A / (float)(N + V);
}

// The N-gram state of the stream's next prediction into *out (the context
// entries the last update found), by threads tid = 0 .. nthr - 1.
__device__ void ng_snapshot(const Dims& D, const StreamDev& st, NgSnap* out, int tid, int nthr) {
  for (int e = tid; e < kMaxOrder * kMaxSlots; e += nthr) {
    const int k = e / kMaxSlots, q = e - k * kMaxSlots;
    const int ei = k < D.order ? st.ctx_ent[k] : -1;
    if (ei >= 0) {
      const NgEntry& en = st.ent[k][ei];
      if (q < en.nslots) out->tc[k][q] = make_int2(en.tok[q], en.cnt[q]);
    }
  }
  if (tid == 0) {
    float nk[kMaxOrder], coef[kMaxOrder], cu;
    bool has[kMaxOrder];
    for (int k = 0; k < kMaxOrder; ++k) {
      const int ei = k < D.order ? st.ctx_ent[k] : -1;
      has[k] = ei >= 0;
      nk[k] = has[k] ? (float)st.ent[k][ei].n : 0.f;
      out->ns[k] = has[k] ? st.ent[k][ei].nslots : 0;
    }
    ng_weights(nk, has, st.N, D.V, coef, cu);
    for (int k = 0; k < kMaxOrder; ++k) out->coef[k] = coef[k];
    out->ns[3] = 0;
    out->coef[3] = 0.f;
    out->cu = cu;
  }
}

// Warp k (k < 3) owns order k: it counts the observed token t in the entry of
// the context of length k + 1 (inserting the context if new; a full entry
// evicts its lowest count), then looks up the entry of the next context (t
// appended) for the next prediction.  The orders use separate tables, so the
// warps run concurrently.  n_coded: tokens coded before t.
__device__ void ngram_update_order(const Dims& D, StreamDev& st, int t, int k, int lane, int n_coded) {
  const int nh = min(3, n_coded);                  // contexts before t
  if (k < D.order && k < nh) {
    int ei = 0;
    if (lane == 0) ei = ng_find(st, k, ctx_key(st.hist, k + 1), true);
    ei = __shfl_sync(0xffffffffu, ei, 0);
    if (ei >= 0) {
      NgEntry& en = st.ent[k][ei];
      const int ns = en.nslots;
      int hit = -1;
      for (int q = lane; q < ns; q += 32)
        if (en.tok[q] == t) hit = q;
      unsigned m = __ballot_sync(0xffffffffu, hit >= 0);
      if (m) {
        const int src = __ffs(m) - 1;
        const int q = __shfl_sync(0xffffffffu, hit, src);
        if (lane == 0) {
          en.cnt[q] += 1;
          en.n += 1;
        }
      } else if (ns < kMaxSlots) {
        if (lane == 0) {
          en.tok[ns] = t;
          en.cnt[ns] = 1;
          en.nslots = ns + 1;
          en.n += 1;
        }
      } else {
        // evict the lowest count, lowest slot index on ties
        int bc = 0x7fffffff, bi = 0x7fffffff;
        for (int q = lane; q < kMaxSlots; q += 32) {
          const int cq = en.cnt[q];
          if (cq < bc || (cq == bc && q < bi)) {
            bc = cq;
            bi = q;
          }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (oc < bc || (oc == bc && oi < bi)) {
            bc = oc;
            bi = oi;
          }
        }
        if (lane == 0) {
          en.n += 1 - en.cnt[bi];
          en.tok[bi] = t;
          en.cnt[bi] = 1;
        }
      }
    }
    __syncwarp();
  }
  // the next context: the last k + 1 tokens with t appended
  if (lane == 0) {
    int nhist[3] = {st.hist[1], st.hist[2], t};
    const int nh2 = min(3, n_coded + 1);
    st.ctx_ent[k] = (k < D.order && k < nh2) ? ng_find(st, k, ctx_key(nhist, k + 1), false) : -1;
  }
}

// The N-gram update of row j and the stream's bookkeeping for the next step
// (one position of the step kernel).
__device__ void ngram_update_row(const Dims& D, const Batch& b, int j, int warp, int lane) {
  StreamDev& st = b.st[b.slots[j]];
  const int t = b.obs[j];
  if (t < 0 || t >= D.V) {
    if (warp == 0 && lane == 0) atomicOr(&st.status, ST_BAD_TOKEN);
    return;
  }
  if (warp < kMaxOrder) ngram_update_order(D, st, t, warp, lane, st.n_coded);
  __syncthreads();                                 // every order has read the old history
  if (warp == 0 && lane == 0) {
    if (D.order > 0) {
      st.uni[t] += 1;
      st.N += 1;
    }
    st.hist[0] = st.hist[1];
    st.hist[1] = st.hist[2];
    st.hist[2] = t;
    int start = st.kv_start;
    if (st.n_coded - start == D.L) start += D.C;
    st.kv_start = start;
    st.n_coded += 1;
    st.last_tok = t;
  }
}

// Context of length len ending at a2 (a0, a1 the tokens before it), packed
// as ctx_key packs the history.
__device__ __forceinline__ unsigned long long ctx_key3(int a0, int a1, int a2, int len) {
  unsigned long long key = 0;
  if (len >= 3) key = (unsigned long long)(uint32_t)a0;
  if (len >= 2) key = (key << 16) | (unsigned long long)(uint32_t)a1;
  return (key << 16) | (unsigned long long)(uint32_t)a2;
}

// Lane-parallel step of a linear probe: lane l holds kk, the key of index
// slot home + l (in = false past the capacity).  Returns the first lane, in
// probe order, whose slot holds `key` or is empty (-1: none of the 32), and
// in *hit whether that slot holds the key.
__device__ __forceinline__ int ng_resolve(unsigned long long kk, bool in, unsigned long long key, bool* hit) {
  const unsigned mh = __ballot_sync(0xffffffffu, in && kk == key);
  const unsigned me = __ballot_sync(0xffffffffu, in && kk == kEmptyKey);
  if ((mh | me) == 0) return -1;
  const int f = __ffs(mh | me) - 1;
  *hit = (mh >> f) & 1u;
  return f;
}

// The N-gram side of a prefill chunk, one CTA per stream row: for each
// position in order, the state of its prediction into snap, then the update
// with the observed token (tables, context entries, history and N; the
// unigram counts and the position stay with the vocabulary passes).  It needs
// only the tokens, so it runs beside the chunk's forward pass.
//
// Warp k (k < 3) owns order k, with the history, N and the entry of the
// next prediction's context in registers for the whole chunk:
// - the context a token is counted in is the one its prediction used, so
//   its entry is known from the previous position (the look-up made then);
// - one round of loads per position: that entry's 64 slots (two per lane),
//   the 32 index slots from the home of the context when it has to be
//   inserted, and the keys and entry numbers of the 32 index slots from the
//   home of the next context;
// - a new context goes into the first empty slot of its probe.  The next
//   context's slots are read before that insert: a key found there stays
//   where it is (entries are never removed), one found absent stays absent
//   unless it is the context just counted.
// The counting and eviction are those of ngram_update_order, so the tables,
// and so the coded bits, equal those of one update per step.  Warp 3 forms
// the closed form's weights of each position from the orders' counts.
__global__ void __launch_bounds__(128) k_ngram_seq(Dims D, Batch b, int m, int n_streams, const int32_t* nb_step,
                                                   const int32_t* obs_step, const int32_t* z_idx, const int32_t* p0_at,
                                                   NgSnap* snap) {
  __shared__ int32_t s_obs[kSeqMax], s_nb[kSeqMax];       // the chunk's tokens and active rows, per position
  __shared__ int32_t s_n[2][kMaxOrder], s_ns[2][kMaxOrder];  // by position parity: the orders' n_k (-1: no entry), slots
  const int j = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  StreamDev& st = b.st[b.slots[j]];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    s_obs[i] = obs_step[(size_t)i * n_streams + j];
    s_nb[i] = nb_step[i];
  }
  int n_coded = *p0_at;                            // every live stream is at the chunk's first position
  int h0 = st.hist[0], h1 = st.hist[1], h2 = st.hist[2];
  int N = st.N;
  const int k = warp;                              // order of this warp; warp 3 forms the weights
  const bool ord = k < kMaxOrder && k < D.order;
  const int mask = st.cap_mask, max_len = st.max_len;
  const bool in = lane <= mask;                    // lanes within the index capacity
  unsigned long long* keys = ord ? st.keys[k] : nullptr;
  int32_t* idx = ord ? st.idx[k] : nullptr;
  NgEntry* ent = ord ? st.ent[k] : nullptr;
  int ce = ord ? st.ctx_ent[k] : -1;               // entry of the next prediction's context
  int n_ent = ord ? st.n_ent[k] : 0;
  NgSnap* out = snap + z_idx[j];
  __syncthreads();
  int r = 0;
  for (; r < m; ++r) {
    if (j >= s_nb[r]) break;
    const int t = s_obs[r];
    const bool tok_ok = t >= 0 && t < D.V;
    if (ord) {
      const bool cur = k < min(3, n_coded);        // the context of length k + 1 before t exists
      const bool nxt = k < min(3, n_coded + 1);
      const unsigned long long ckey = ctx_key3(h0, h1, h2, k + 1), nkey = ctx_key3(h1, h2, t, k + 1);
      const int home_c = (int)(mix64(ckey) & (unsigned long long)mask);
      const int home_n = (int)(mix64(nkey) & (unsigned long long)mask);
      const bool ins = tok_ok && cur && ce < 0;    // a new context: inserted below
      const bool probe_n = tok_ok && nxt && !(cur && nkey == ckey);
      // one round of loads
      int tok0 = 0, tok1 = 0, cnt0 = 0, cnt1 = 0, ens = 0, en_n = 0, in_n = -1;
      unsigned long long kc = 0, kn = 0;
      if (ce >= 0) {
        const NgEntry& en = ent[ce];
        tok0 = en.tok[lane];
        tok1 = en.tok[lane + 32];
        cnt0 = en.cnt[lane];
        cnt1 = en.cnt[lane + 32];
        ens = en.nslots;
        en_n = en.n;
      }
      if (ins && in) kc = keys[(home_c + lane) & mask];
      if (probe_n && in) {
        kn = keys[(home_n + lane) & mask];
        in_n = idx[(home_n + lane) & mask];
      }
      // the prediction's state: the entry before t is counted
      NgSnap& o = out[r];
      if (lane < ens) o.tc[k][lane] = make_int2(tok0, cnt0);
      if (lane + 32 < ens) o.tc[k][lane + 32] = make_int2(tok1, cnt1);
      if (lane == 0) {
        s_n[r & 1][k] = ce >= 0 ? en_n : -1;
        s_ns[r & 1][k] = ens;
      }
      if (tok_ok) {
        // count t in the context's entry
        if (ins) {
          bool hit = false;
          const int f = ng_resolve(kc, in, ckey, &hit);
          int ei = -1;
          if (f < 0) {                             // more than 32 probes: the one-slot-at-a-time walk
            if (lane == 0) ei = ng_find(st, k, ckey, true);
            ei = __shfl_sync(0xffffffffu, ei, 0);
            __syncwarp();
            n_ent = st.n_ent[k];
          } else if (hit) {
            ei = idx[(home_c + f) & mask];
          } else if (n_ent >= max_len) {
            if (lane == 0) atomicOr(&st.status, ST_TABLE_FULL);
          } else {                                 // insert into the empty slot, counting t
            const int slot = (home_c + f) & mask;
            ei = n_ent++;
            if (lane == 0) {
              NgEntry& en = ent[ei];
              en.tok[0] = t;
              en.cnt[0] = 1;
              en.nslots = 1;
              en.n = 1;
              keys[slot] = ckey;
              idx[slot] = ei;
              st.n_ent[k] = n_ent;
            }
            ce = ei;
            ens = -1;                              // counted
          }
          if (ei >= 0 && ens == 0) {               // an entry that exists (or the walk made): its slots
            const NgEntry& en = ent[ei];
            tok0 = en.tok[lane];
            tok1 = en.tok[lane + 32];
            cnt0 = en.cnt[lane];
            cnt1 = en.cnt[lane + 32];
            ens = en.nslots;
            en_n = en.n;
            ce = ei;
          }
        }
        if (cur && ce >= 0 && ens >= 0) {
          NgEntry& en = ent[ce];
          const unsigned m0 = __ballot_sync(0xffffffffu, lane < ens && tok0 == t);
          const unsigned m1 = __ballot_sync(0xffffffffu, lane + 32 < ens && tok1 == t);
          if (m0 | m1) {
            const int q = m0 ? __ffs(m0) - 1 : 32 + __ffs(m1) - 1;
            const int cq = __shfl_sync(0xffffffffu, q < 32 ? cnt0 : cnt1, q & 31);
            if (lane == 0) {
              en.cnt[q] = cq + 1;
              en.n = en_n + 1;
            }
          } else if (ens < kMaxSlots) {
            if (lane == 0) {
              en.tok[ens] = t;
              en.cnt[ens] = 1;
              en.nslots = ens + 1;
              en.n = en_n + 1;
            }
          } else {
            // evict the lowest count, lowest slot index on ties
            int bc = cnt0, bi = lane;
            if (cnt1 < bc) {
              bc = cnt1;
              bi = lane + 32;
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
              const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
              const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
              if (oc < bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
              }
            }
            if (lane == 0) {
              en.n = en_n + 1 - bc;
              en.tok[bi] = t;
              en.cnt[bi] = 1;
            }
          }
        }
        // the next prediction's context (t appended)
        int nx = -1;
        if (nxt) {
          if (cur && nkey == ckey) {
            nx = ce;                               // the context just counted (-1: its table is full)
          } else {
            bool hit = false;
            const int f = ng_resolve(kn, in, nkey, &hit);
            if (f < 0) {
              if (lane == 0) nx = ng_find(st, k, nkey, false);
              nx = __shfl_sync(0xffffffffu, nx, 0);
            } else if (hit) {
              nx = __shfl_sync(0xffffffffu, in_n, f);
            }
          }
        }
        ce = nx;
      }
    }
    __syncthreads();                               // the orders' counts of this prediction are in shared memory
    if (warp == 3 && lane == 0) {
      float nk[kMaxOrder], coef[kMaxOrder], cu;
      bool has[kMaxOrder];
      NgSnap& o = out[r];
      for (int q = 0; q < kMaxOrder; ++q) {
        has[q] = q < D.order && s_n[r & 1][q] >= 0;
        nk[q] = has[q] ? (float)s_n[r & 1][q] : 0.f;
        o.ns[q] = has[q] ? s_ns[r & 1][q] : 0;
      }
      ng_weights(nk, has, N, D.V, coef, cu);
      for (int q = 0; q < kMaxOrder; ++q) o.coef[q] = coef[q];
      o.ns[3] = 0;
      o.coef[3] = 0.f;
      o.cu = cu;
    }
    if (!tok_ok) break;                            // flagged by the vocabulary pass
    N += 1;
    h0 = h1;
    h1 = h2;
    h2 = t;
    ++n_coded;
  }
  // the stream's N-gram bookkeeping for the next chunk or step
  if (r > 0) {
    if (k < kMaxOrder && lane == 0) st.ctx_ent[k] = ce;
    if (threadIdx.x == 0) {
      st.N = N;
      st.hist[0] = h0;
      st.hist[1] = h1;
      st.hist[2] = h2;
    }
  }
}

// Encoder driver: row j is active while its stream has tokens left; rows are
// sorted by length (longest first), so the active rows are a prefix.
__global__ void k_prepare_encode(Batch b, int n_streams, const int32_t* tok_flat,
                                 const int64_t* offs, const int64_t* lens, int32_t* obs,
                                 int32_t* nB) {
  __shared__ int cnt[32];
  pdl_wait();
  pdl_trigger();
  int mine = 0;
  for (int j = threadIdx.x; j < n_streams; j += blockDim.x) {
    const int nc = b.st[b.slots[j]].n_coded;
    const bool act = nc < lens[j];
    obs[j] = act ? tok_flat[offs[j] + nc] : 0;
    mine += act;
  }
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += cnt[w];
    *nB = tot;
  }
}

// The next prefill chunk's first position: p0s[par] = p0s[3], p0s[3] += m (par < 3).
__global__ void k_chunk_start(int32_t* p0s, int par, int m) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) {
    const int p0 = p0s[3];
    p0s[par] = p0;
    p0s[3] = p0 + m;
  }
}

// Encoder prefill of positions p0 .. p0 + m - 1 (p0 = *p0_at; rows sorted
// longest first, so the streams with tokens left are a prefix).
// Forward row i = j m + r: slot, position (-1 past the stream's end) and
// input token.  Sequential pass r: active rows nb_step[r], observed tokens
// obs_step[r n + j]; row j's logits sit at forward row z_idx[j] + r.
__global__ void k_prepare_prefill(Batch b, int n_streams, int m, int V, const int32_t* p0_at, const int32_t* tok_flat,
                                  const int64_t* offs, const int64_t* lens, int32_t* f_slots, int32_t* f_pos,
                                  int32_t* f_tok, int32_t* nB_fwd, int32_t* obs_step, int32_t* nb_step,
                                  int32_t* z_idx) {
  pdl_wait();
  pdl_trigger();
  const int p0 = *p0_at;
  const int tid = threadIdx.x + blockIdx.x * blockDim.x, nthr = blockDim.x * gridDim.x;
  for (int i = tid; i < n_streams * m; i += nthr) {
    const int j = i / m, r = i % m;
    const int64_t a = (int64_t)p0 + r;
    const bool live = a < lens[j];
    f_slots[i] = b.slots[j];
    f_pos[i] = live ? (int)a : -1;
    // BOS (id 0) at position 0; an id outside the vocabulary is fed as 0 here
    // and rejected by the vocabulary pass that codes it
    const int t = (live && a > 0) ? tok_flat[offs[j] + a - 1] : 0;
    f_tok[i] = (t >= 0 && t < V) ? t : 0;
    obs_step[r * n_streams + j] = live ? tok_flat[offs[j] + a] : 0;
  }
  for (int r = tid; r < m; r += nthr) {
    int act = 0;
    while (act < n_streams && lens[act] > (int64_t)p0 + r) ++act;
    nb_step[r] = act;
  }
  for (int j = tid; j < n_streams; j += nthr) z_idx[j] = j * m;
  if (tid == 0) {
    int live = 0;
    while (live < n_streams && lens[live] > p0) ++live;
    *nB_fwd = live * m;
  }
}

// Standalone quantiser over rows of binary32 probabilities.
template <int E>
__global__ void __cluster_dims__(kVocabCluster, 1, 1) __launch_bounds__(kVocabThreads)
    k_probs_to_cdf(const float* p, int V, int log2T, uint32_t floor_c, uint32_t* cdf,
                   int32_t* status) {
  __shared__ VocabShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int j = blockIdx.x / kVocabCluster;
  const int rank = (int)cl.block_rank();
  const int v0 = rank * kVocabThreads * E + threadIdx.x * E;
  float pr[E];
  load_run<E>(p + (size_t)j * V, v0, V, pr, 0.f);
  uint32_t c[E];
  const QuantResult q = quantise_round<E, kVocabCluster>(pr, v0, V, log2T, floor_c, c, cl, sh);
  if (q.bad && threadIdx.x == 0 && rank == 0) atomicOr(status + j, ST_NUMERIC);
  scan_round<E>(c, v0, V, 1u << log2T, cdf + (size_t)j * (V + 1), cl, sh);
  cl.sync();
}

__global__ void k_floor_counts(const float* p, int64_t n, uint32_t K, uint32_t floor_c,
                               uint32_t* c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool bad = false;
    const uint32_t q = floor_count(p[i], K, (float)K, bad);
    c[i] = bad ? 0xFFFFFFFFu : (q > floor_c ? q : floor_c);
  }
}

// Mixed-distribution NLL forward / backward, one CTA per row.
__global__ void __launch_bounds__(kVocabThreads)
    k_mix_nll(const float* z, const float* bv, const float* png, const float* theta,
              const int32_t* target, const int32_t* warm, const float* gout, int V, float tau,
              float* loss, float* db, float* dth) {
  __shared__ VocabShared sh;
  const int j = blockIdx.x;
  const float* zr = z + (size_t)j * V;
  const float* br = bv + (size_t)j * V;
  const int t = target[j];
  if (t < 0 || t >= V) {     // out-of-range target: NaN loss and gradients
    for (int v = threadIdx.x; v < V && db; v += kVocabThreads) db[(size_t)j * V + v] = NAN;
    if (threadIdx.x == 0) {
      if (loss) loss[j] = NAN;
      if (dth) dth[2 * j] = dth[2 * j + 1] = NAN;
    }
    return;
  }
  // s = z / tau + b as the coding step forms it (Sec. 3.2, Sec. 3.6): one
  // fused multiply-add by the rounded reciprocal of tau
  const float inv_tau = 1.0f / tau;
  float mx = -INFINITY;
  for (int v = threadIdx.x; v < V; v += kVocabThreads) mx = fmaxf(mx, __fmaf_rn(zr[v], inv_tau, br[v]));
  const float M = block_max(mx, sh);
  float ls = 0.f;
  for (int v = threadIdx.x; v < V; v += kVocabThreads) ls += expf(__fmaf_rn(zr[v], inv_tau, br[v]) - M);
  const float S = block_sum(ls, sh);
  const float pts = __fdiv_rn(expf(__fmaf_rn(zr[t], inv_tau, br[t]) - M), S);
  const float pngs = png[(size_t)j * V + t];
  const float th0 = theta[2 * j], th1 = theta[2 * j + 1];
  const float tm = fmaxf(th0, th1);
  const float e0 = expf(th0 - tm), e1 = expf(th1 - tm);
  const float w0 = e0 / (e0 + e1), w1 = e1 / (e0 + e1);
  const bool wu = warm[j] != 0;
  const float pm = wu ? pts : w0 * pts + w1 * pngs;
  const float g = gout ? gout[j] : 1.f;
  if (loss && threadIdx.x == 0) loss[j] = -logf(pm);
  if (db) {
    const float rho = wu ? 1.f : w0 * pts / pm;
    for (int v = threadIdx.x; v < V; v += kVocabThreads) {
      const float ptv = __fdiv_rn(expf(__fmaf_rn(zr[v], inv_tau, br[v]) - M), S);
      db[(size_t)j * V + v] = g * rho * (ptv - (v == t ? 1.f : 0.f));
    }
  }
  if (dth && threadIdx.x == 0) {
    dth[2 * j] = wu ? 0.f : g * (w0 - w0 * pts / pm);
    dth[2 * j + 1] = wu ? 0.f : g * (w1 - w1 * pngs / pm);
  }
}

// One warp per row: binary search of the decoder's target count in the CDF.
__global__ void k_search(Batch b, int V, const uint32_t* cdf, const uint32_t* target, int32_t* obs,
                         uint32_t* lohi) {
  pdl_wait();
  pdl_trigger();
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= *b.nB || lane != 0) return;
  const uint32_t* row = cdf + (size_t)j * (V + 1);
  const uint32_t t = target[j];
  int lo = 0, hi = V - 1;                // largest s with row[s] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  obs[j] = lo;
  lohi[2 * j] = row[lo];
  lohi[2 * j + 1] = row[lo + 1];
}

}  // namespace

// Elements per thread for a vocabulary of V over `ctas` CTAs of `threads`.
static int vocab_E(int V, int ctas = kVocabCluster, int threads = kVocabThreads) {
  const int per = ctas * threads;
  int e = (V + per - 1) / per;
  e = (e + 3) / 4 * 4;
  return e < 4 ? 4 : e;
}

// FULL: the vocabulary fills the step cluster's 4,096 E symbols exactly.
template <int E>
static bool step_full(int V) {
  return V == kClusterWarps * 32 * E;
}

// 16-CTA clusters (a non-portable size) are used when the device places them.
static bool g_cl16 = false;

// CTAs per stream of a step launch over `rows` streams: 16 while the
// clusters fit in one wave (one stream or a few: the per-position latency
// falls with the work per SM), else 8 (more streams per wave).  Results do
// not depend on it.
static int step_cluster(const Dims& D, int rows) {
  return g_cl16 && rows * 16 <= D.n_sm ? 16 : 8;
}

template <int E, bool FULL, int CL>
static cudaError_t vocab_tfc(const Dims& D, const Batch& b, const VocabIO& io, cudaStream_t s) {
  const size_t smem = (size_t)step_threads<CL>() * E * sizeof(float);
  return launch_kernel_cluster(&k_vocab<E, FULL, CL>, dim3(b.Bmax * CL), dim3(step_threads<CL>()), smem, s, D.pdl,
                               CL, D, b, io);
}
template <int E>
static cudaError_t vocab_t(const Dims& D, const Batch& b, const VocabIO& io, cudaStream_t s) {
  const bool full = step_full<E>(D.V);
  if (step_cluster(D, b.Bmax) == 16)
    return full ? vocab_tfc<E, true, 16>(D, b, io, s) : vocab_tfc<E, false, 16>(D, b, io, s);
  return full ? vocab_tfc<E, true, 8>(D, b, io, s) : vocab_tfc<E, false, 8>(D, b, io, s);
}

template <int E, bool FULL, int CL>
static cudaError_t prepare_vocab_tfc() {
  const int smem = step_threads<CL>() * E * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_vocab<E, FULL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vocab_seq<E, FULL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && CL > 8) {
    e = cudaFuncSetAttribute(k_vocab<E, FULL, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_vocab_seq<E, FULL, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  return e;
}
// Whether clusters of CL CTAs of the loop kernel can be placed on the device.
template <int E, bool FULL, int CL>
static bool clusters_fit() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(step_threads<CL>());
  cfg.dynamicSmemBytes = (size_t)step_threads<CL>() * E * sizeof(float);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&n, &k_vocab_seq<E, FULL, CL>, &cfg) == cudaSuccess && n > 0;
  cudaGetLastError();
  return ok;
}
template <int E, bool FULL>
static cudaError_t prepare_vocab_tf() {
  cudaError_t e = prepare_vocab_tfc<E, FULL, 8>();
  if (e != cudaSuccess) return e;
  g_cl16 = prepare_vocab_tfc<E, FULL, 16>() == cudaSuccess && clusters_fit<E, FULL, 16>();
  cudaGetLastError();
  return cudaSuccess;
}
template <int E>
static cudaError_t prepare_vocab_t(int V) {
  return step_full<E>(V) ? prepare_vocab_tf<E, true>() : prepare_vocab_tf<E, false>();
}

cudaError_t prepare_vocab_kernels(const Dims& D) {
  switch (vocab_E(D.V, 8, step_threads<8>())) {
    case 4: return prepare_vocab_t<4>(D.V);
    case 8: return prepare_vocab_t<8>(D.V);
    case 12: return prepare_vocab_t<12>(D.V);
    case 16: return prepare_vocab_t<16>(D.V);
  }
  return cudaErrorInvalidValue;
}

template <int E, bool FULL, int CL>
static cudaError_t vocab_seq_tfc(const Dims& D, const Batch& b, const VocabIO& io, int m, const float* zrows,
                                 const int32_t* nb_step, const int32_t* obs_step, const NgSnap* snap,
                                 cudaStream_t s) {
  const size_t smem = (size_t)step_threads<CL>() * E * sizeof(float);
  if (m > kSeqMax) return cudaErrorInvalidValue;
  return launch_kernel_cluster(&k_vocab_seq<E, FULL, CL>, dim3(b.Bmax * CL), dim3(step_threads<CL>()), smem, s,
                               D.pdl, CL, D, b, io, m, b.Bmax, zrows, nb_step, obs_step, snap);
}
template <int E>
static cudaError_t vocab_seq_t(const Dims& D, const Batch& b, const VocabIO& io, int m, const float* zrows,
                               const int32_t* nb_step, const int32_t* obs_step, const NgSnap* snap,
                               cudaStream_t s) {
  const bool full = step_full<E>(D.V);
  if (step_cluster(D, b.Bmax) == 16)
    return full ? vocab_seq_tfc<E, true, 16>(D, b, io, m, zrows, nb_step, obs_step, snap, s)
                : vocab_seq_tfc<E, false, 16>(D, b, io, m, zrows, nb_step, obs_step, snap, s);
  return full ? vocab_seq_tfc<E, true, 8>(D, b, io, m, zrows, nb_step, obs_step, snap, s)
              : vocab_seq_tfc<E, false, 8>(D, b, io, m, zrows, nb_step, obs_step, snap, s);
}

cudaError_t launch_vocab_seq(const Dims& D, const Batch& b, const VocabIO& io, int m, const float* zrows,
                             const int32_t* nb_step, const int32_t* obs_step, const NgSnap* snap, cudaStream_t s) {
  if (D.order > 0 && !snap) return cudaErrorInvalidValue;
  switch (vocab_E(D.V, 8, step_threads<8>())) {
    case 4: return vocab_seq_t<4>(D, b, io, m, zrows, nb_step, obs_step, snap, s);
    case 8: return vocab_seq_t<8>(D, b, io, m, zrows, nb_step, obs_step, snap, s);
    case 12: return vocab_seq_t<12>(D, b, io, m, zrows, nb_step, obs_step, snap, s);
    case 16: return vocab_seq_t<16>(D, b, io, m, zrows, nb_step, obs_step, snap, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ngram_seq(const Dims& D, const Batch& b, int m, const int32_t* nb_step, const int32_t* obs_step,
                             const int32_t* p0, NgSnap* snap, cudaStream_t s) {
  if (D.order <= 0 || b.Bmax < 1) return cudaSuccess;
  if (m > kSeqMax) return cudaErrorInvalidValue;
  return launch_kernel(k_ngram_seq, dim3(b.Bmax), dim3(128), 0, s, false, D, b, m, b.Bmax, nb_step, obs_step,
                       b.z_idx, p0, snap);
}

cudaError_t launch_vocab(const Dims& D, const Batch& b, const VocabIO& io, cudaStream_t s) {
  switch (vocab_E(D.V, 8, step_threads<8>())) {
    case 4: return vocab_t<4>(D, b, io, s);
    case 8: return vocab_t<8>(D, b, io, s);
    case 12: return vocab_t<12>(D, b, io, s);
    case 16: return vocab_t<16>(D, b, io, s);
  }
  return cudaErrorInvalidValue;
}


cudaError_t launch_prepare_encode(const Batch& b, int n_streams, const int32_t* tok_flat,
                                  const int64_t* offs, const int64_t* lens, int32_t* obs,
                                  int32_t* nB, cudaStream_t s) {
  return launch_kernel(k_prepare_encode, dim3(1), dim3(1024), 0, s, true, b, n_streams, tok_flat, offs, lens,
                       obs, nB);
}

cudaError_t launch_chunk_start(int32_t* p0s, int par, int m, cudaStream_t s) {
  return launch_kernel(k_chunk_start, dim3(1), dim3(32), 0, s, true, p0s, par, m);
}

cudaError_t launch_prepare_prefill(const Batch& b, int n_streams, int m, int V, const int32_t* p0,
                                   const int32_t* tok_flat, const int64_t* offs, const int64_t* lens,
                                   int32_t* f_slots, int32_t* f_pos, int32_t* f_tok, int32_t* nB_fwd,
                                   int32_t* obs_step, int32_t* nb_step, int32_t* z_idx, cudaStream_t s) {
  const int rows = n_streams * m;
  const int blocks = std::min((rows + 255) / 256, 64);
  return launch_kernel(k_prepare_prefill, dim3(blocks), dim3(256), 0, s, true, b, n_streams, m, V, p0, tok_flat,
                       offs, lens, f_slots, f_pos, f_tok, nB_fwd, obs_step, nb_step, z_idx);
}

template <int E>
static cudaError_t p2c_t(const float* p, int n, int V, int log2T, uint32_t floor_c, uint32_t* cdf,
                         int32_t* status, cudaStream_t s) {
  k_probs_to_cdf<E><<<n * kVocabCluster, kVocabThreads, 0, s>>>(p, V, log2T, floor_c, cdf, status);
  return cudaGetLastError();
}

cudaError_t launch_probs_to_cdf(const float* p, int n, int V, int log2T, uint32_t floor_c,
                                uint32_t* cdf, int32_t* status, cudaStream_t s) {
  switch (vocab_E(V)) {
    case 4: return p2c_t<4>(p, n, V, log2T, floor_c, cdf, status, s);
    case 8: return p2c_t<8>(p, n, V, log2T, floor_c, cdf, status, s);
    case 12: return p2c_t<12>(p, n, V, log2T, floor_c, cdf, status, s);
    case 16: return p2c_t<16>(p, n, V, log2T, floor_c, cdf, status, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_floor_counts(const float* p, int64_t n, uint32_t K, uint32_t floor_c,
                                uint32_t* c, cudaStream_t s) {
  const int64_t blocks = (n + 255) / 256;
  k_floor_counts<<<(unsigned)(blocks < 152 * 64 ? (blocks > 0 ? blocks : 1) : 152 * 64), 256, 0, s>>>(p, n, K, floor_c, c);
  return cudaGetLastError();
}

cudaError_t launch_search(const Batch& b, int V, const uint32_t* cdf, const uint32_t* target,
                          int32_t* obs, uint32_t* lohi, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (b.Bmax * 32 + threads - 1) / threads;
  k_search<<<blocks, threads, 0, s>>>(b, V, cdf, target, obs, lohi);
  return cudaGetLastError();
}

cudaError_t launch_mix_nll(const float* z, const float* b, const float* png, const float* theta,
                           const int32_t* target, const int32_t* warm, const float* gout, int n,
                           int V, float tau, float* loss, float* db, float* dtheta,
                           cudaStream_t s) {
  k_mix_nll<<<n, kVocabThreads, 0, s>>>(z, b, png, theta, target, warm, gout, V, tau, loss, db, dtheta);
  return cudaGetLastError();
}

}  // namespace nc
