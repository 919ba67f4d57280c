// Vocabulary-wide kernels: biased softmax (Sec. 3.6), N-gram distribution
// (Sec. 3.4), linear mix (Sec. 3.5), CDF quantisation with floors and the
// prefix sum (Sec. 3.3), the head / mixer updates, and the N-gram tables.
//
// One stream is handled by a cluster of CTAs (kStepCluster for the per-token
// step, kVocabCluster for the standalone quantiser); each CTA owns a
// contiguous chunk of the vocabulary and each thread a contiguous run of E
// symbols.  Reductions go thread -> warp (fixed xor tree) -> CTA (warps in
// order) -> cluster (ranks in order through distributed shared memory), so
// every result is independent of the batch, the slot and the launch.
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
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// floor(p * K) for a binary32 p in [0, 2) and K < 2^24, exactly: p = m 2^(e-150)
// with a 24-bit significand m, so m * K < 2^48 is an exact integer product.
// Sets `bad` for negative, >= 2, infinite or NaN inputs.
__device__ __forceinline__ uint32_t floor_prod(float p, uint32_t K, bool& bad) {
  const uint32_t u = __float_as_uint(p);
  if (u == 0u || u == 0x80000000u) return 0u;
  if (u >> 31) {
    bad = true;
    return 0u;
  }
  uint32_t e = u >> 23;
  if (e >= 128u) {
    bad = true;
    return 0u;
  }
  uint32_t m = u & 0x7FFFFFu;
  if (e == 0u)
    e = 1u;
  else
    m |= 0x800000u;
  const unsigned long long prod = (unsigned long long)m * K;
  const uint32_t sh = 150u - e;
  return sh >= 64u ? 0u : (uint32_t)(prod >> sh);
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

// Shared scratch of one CTA: block-reduction slots, the values it publishes
// to the other CTAs of its cluster, and the step's N-gram coefficients.
template <int NW>
struct VocabSharedT {
  static constexpr int kNW = NW;
  float wm[NW], wsum[NW], wh[NW];
  unsigned long long wc[NW], wb[NW];
  ArgMax wa[NW];
  uint32_t wscan[NW];
  // published to the cluster
  float cl_m, cl_s, cl_h;
  unsigned long long cl_csum, cl_below;
  ArgMax cl_arg;
  uint32_t cl_bad;
  uint32_t cl_total;
  float cl_obs[3];          // p_tilde(t*), p_ng(t*), log p_tilde(t*) (owner CTA of t*)
  // N-gram coefficients of this step
  float cu, coef[kMaxOrder], nk[kMaxOrder];
  const NgEntry* ent[kMaxOrder];
  // the N-gram state one prediction reads: per order the context entry's
  // (token, count) slots (ns < 0: no entry) and the closed form's weights
  int ng_ns[kMaxOrder];
  int ng_tok[kMaxOrder][kMaxSlots], ng_cnt[kMaxOrder][kMaxSlots];
  float ng_coef[kMaxOrder], ng_cu;
};
using VocabShared = VocabSharedT<kWarps>;                         // standalone quantiser
using StepShared = VocabSharedT<kStepThreads / 32>;               // the per-token step

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

// Softmax statistics: the maximum and the sum of exp(s - max).
struct MS {
  float m, s;
};

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

// Round 1 of the step: the softmax of s over the cluster's vocabulary.
// Each CTA takes its own maximum m_c (exact) and its numerators
// e_i = exp(s_i - m_c) with their sum s_c (thread, i in order -> warp, xor
// tree -> CTA, warps in order); one cluster round then gives
// M = max m_c and S = sum_c s_c exp(m_c - M) (ranks in order), and this
// CTA's factor exp(m_c - M) / S turns e_i into p_i.  A second sum (the
// N-gram entropy terms h_in) is reduced alongside, unscaled.
template <int E, int CL, typename Sh>
__device__ MS softmax_round(const float (&s)[E], float (&e)[E], float h_in, float& h_out, float& scale,
                            cg::cluster_group& cl, Sh& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float m = -INFINITY;
#pragma unroll
  for (int i = 0; i < E; ++i) m = fmaxf(m, s[i]);
  m = warp_max(m);
  if (lane == 0) sh.wm[w] = m;
  __syncthreads();
  float mc = sh.wm[0];
  for (int i = 1; i < Sh::kNW; ++i) mc = fmaxf(mc, sh.wm[i]);
  float t = 0.f;
  if (mc != -INFINITY) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      e[i] = expf(s[i] - mc);
      t += e[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) e[i] = 0.f;
  }
  t = warp_sum(t);
  const float hw = warp_sum(h_in);
  if (lane == 0) {
    sh.wsum[w] = t;
    sh.wh[w] = hw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f, bh = 0.f;
    for (int i = 0; i < Sh::kNW; ++i) {
      b += sh.wsum[i];
      bh += sh.wh[i];
    }
    sh.cl_m = mc;
    sh.cl_s = b;
    sh.cl_h = bh;
  }
  cl.sync();
  float M = -INFINITY;
#pragma unroll
  for (int r = 0; r < CL; ++r) M = fmaxf(M, cl.map_shared_rank(&sh, r)->cl_m);
  float S = 0.f, H = 0.f;
#pragma unroll
  for (int r = 0; r < CL; ++r) {
    const Sh* o = cl.map_shared_rank(&sh, r);
    if (o->cl_m != -INFINITY) S = fmaf(o->cl_s, expf(o->cl_m - M), S);
    H += o->cl_h;
  }
  h_out = H;
  scale = mc != -INFINITY ? expf(mc - M) / S : 0.f;
  return MS{M, S};
}

struct QuantResult {
  long long resid;          // T - sum of floored counts, added to the first maximum
  int argmax;
  unsigned long long below; // sum of floored counts of symbols below `want`
  bool bad;                 // non-finite / out-of-range probability, or floor underflow
};

// Round 2: floor-quantise the thread's E probabilities into c[], reduce the
// count sum, the first argmax and (for `want` >= 0) the count sum below
// `want` over the cluster.  The CTA owning `want` also publishes obs[3]
// (read by every CTA after this round through cl_obs of the owner rank).
template <int E, int CL, typename Sh>
__device__ QuantResult quantise_round(const float (&p)[E], int v0, int V, int log2T, uint32_t floor_c,
                                      bool quantise, int want, const float* obs, uint32_t (&c)[E],
                                      cg::cluster_group& cl, Sh& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t T = 1u << log2T;
  const uint32_t K = T - (uint32_t)V * floor_c;
  bool bad = false;
  unsigned long long csum = 0, below = 0;
  ArgMax am{-INFINITY, 0x7fffffff};
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int v = v0 + i;
    c[i] = 0;
    if (quantise && v < V) {
      const uint32_t q = floor_prod(p[i], K, bad);
      c[i] = q > floor_c ? q : floor_c;
      csum += c[i];
      if (v < want) below += c[i];
      if (p[i] > am.v) am = ArgMax{p[i], v};   // strict: keeps the first maximum
      bad |= !(p[i] == p[i]);
    }
  }
  if (obs && want >= v0 && want < v0 + E) {
    sh.cl_obs[0] = obs[0];
    sh.cl_obs[1] = obs[1];
    sh.cl_obs[2] = obs[2];
  }
  if (quantise) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      csum += __shfl_xor_sync(0xffffffffu, csum, o);
      below += __shfl_xor_sync(0xffffffffu, below, o);
      ArgMax b2;
      b2.v = __shfl_xor_sync(0xffffffffu, am.v, o);
      b2.i = __shfl_xor_sync(0xffffffffu, am.i, o);
      am = better(am, b2);
    }
    const unsigned any_bad = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
      sh.wc[w] = csum;
      sh.wb[w] = below;
      sh.wa[w] = am;
      sh.wscan[w] = any_bad ? 1u : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tc = 0, tb = 0;
      ArgMax ta{-INFINITY, 0x7fffffff};
      uint32_t tbad = 0;
      for (int i = 0; i < Sh::kNW; ++i) {
        tc += sh.wc[i];
        tb += sh.wb[i];
        ta = better(ta, sh.wa[i]);
        tbad |= sh.wscan[i];
      }
      sh.cl_csum = tc;
      sh.cl_below = tb;
      sh.cl_arg = ta;
      sh.cl_bad = tbad;
    }
  }
  cl.sync();
  QuantResult r{0, -1, 0, false};
  if (quantise) {
    unsigned long long total = 0;
    ArgMax g{-INFINITY, 0x7fffffff};
    for (int q = 0; q < CL; ++q) {
      const Sh* o = cl.map_shared_rank(&sh, q);
      total += o->cl_csum;
      r.below += o->cl_below;
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
  }
  return r;
}

// Round 3: exclusive prefix sum of the final counts into cdf_row.
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

// One stream per cluster.  predict: p -> counts -> CDF and / or the coder
// interval of the observed token.  update: head and mixer update with the
// observed token.  Both may run in one pass (encoder) or in two (decoder,
// which learns the token in between); the arithmetic is the same in either
// case.
__device__ void ngram_update_row(const Dims& D, const Batch& b, int j, int warp, int lane, StepShared* push,
                                 cg::cluster_group* cl);

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

// The N-gram state of the next prediction from the stream's tables: the
// context entries' slots and the weights, into shared memory.
template <typename Sh>
__device__ void ng_gather(const Dims& D, const StreamDev& st, Sh& sh) {
  if (threadIdx.x < kMaxOrder) {
    const int k = threadIdx.x;
    const int ei = (k < D.order) ? st.ctx_ent[k] : -1;
    const NgEntry* en = ei >= 0 ? st.ent[k] + ei : nullptr;
    sh.ent[k] = en;
    sh.nk[k] = en ? (float)en->n : 0.f;
    sh.ng_ns[k] = en ? en->nslots : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float nk[kMaxOrder];
    bool has[kMaxOrder];
    for (int k = 0; k < kMaxOrder; ++k) {
      nk[k] = sh.nk[k];
      has[k] = sh.ent[k] != nullptr;
    }
    ng_weights(nk, has, st.N, D.V, sh.ng_coef, sh.ng_cu);
  }
  for (int e = threadIdx.x; e < kMaxOrder * kMaxSlots; e += blockDim.x) {
    const int k = e / kMaxSlots, q = e % kMaxSlots;
    if (q < sh.ng_ns[k]) {
      sh.ng_tok[k][q] = sh.ent[k]->tok[q];
      sh.ng_cnt[k][q] = sh.ent[k]->cnt[q];
    }
  }
  __syncthreads();
}

// One position of stream row j, by the cluster CTA `rank`: predict (biased
// softmax, N-gram, mix, quantise; the coder interval or the CDF) and the
// head and mixer update.  `bias` and `cnt` hold this thread's bias run and
// unigram counts (loaded here unless have_bias / have_cnt; cnt gains the
// coded token); ng_ready: the N-gram context state is already in shared
// memory; `waited`: the caller already waited on the previous kernel.  Returns false when the observed token is out of range (flagged,
// nothing updated).  The caller runs the N-gram update after it.
template <int E>
__device__ bool vocab_pass(const Dims& D, const Batch& b, const VocabIO& io, int j, int rank, cg::cluster_group& cl,
                           StepShared& sh, float* sp, float (&bias)[E], bool have_bias, int (&cnt)[E], bool have_cnt,
                           bool ng_ready, bool waited) {
  StreamDev& st = b.st[b.slots[j]];
  const int V = D.V;
  const int chunk = kStepThreads * E;
  const int base = rank * chunk;
  const int v0 = base + threadIdx.x * E;
  const int i_tok = st.n_coded + 1;              // 1-based index of the token being coded
  const float th0 = st.theta[0], th1 = st.theta[1];

  // ---- before waiting on the LM head: bias and the N-gram distribution
  // (state of earlier steps only)
  if (!have_bias) {
    if (D.use_head) {
      load_run<E>(st.bias, v0, V, bias, 0.f);
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i) bias[i] = 0.f;
    }
  }
  // N-gram: P = A (c + 1) / (N + V) + sum_k beta_k cnt_k / n_k, the closed
  // form of the interpolation recursion with lambda_k = n_k / (n_k + 5).
  float png[E];
  // logits: after a prefill they are final already (the wait came first)
  float s[E];
  if (b.z_in) load_run<E>(b.z_in + (size_t)b.z_idx[j] * V, v0, V, s, -INFINITY);
  const bool ngram = D.order > 0;
  if (ngram) {
    // unigram counts first (unless kept from the previous position):
    // independent of the context entries below
    if (have_cnt) {
    } else if (v0 + E <= V && (reinterpret_cast<uintptr_t>(st.uni + v0) & 15) == 0) {
      const int4* u4 = reinterpret_cast<const int4*>(st.uni + v0);
#pragma unroll
      for (int q = 0; q < E / 4; ++q) {
        const int4 u = u4[q];
        cnt[4 * q] = u.x;
        cnt[4 * q + 1] = u.y;
        cnt[4 * q + 2] = u.z;
        cnt[4 * q + 3] = u.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i) cnt[i] = (v0 + i < V) ? st.uni[v0 + i] : 0;
    }
    if (!ng_ready) ng_gather(D, st, sh);         // else pushed by the previous position
    for (int i = threadIdx.x; i < chunk; i += kStepThreads) sp[i] = 0.f;
    __syncthreads();
    for (int k = 0; k < kMaxOrder; ++k) {
      const int ns = sh.ng_ns[k];
      for (int q = threadIdx.x; q < ns; q += kStepThreads) {
        const int t = sh.ng_tok[k][q] - base;
        if (t >= 0 && t < chunk) sp[t] += sh.ng_coef[k] * (float)sh.ng_cnt[k][q];
      }
      __syncthreads();
    }
    const float cu = sh.ng_cu;
#pragma unroll
    for (int i = 0; i < E; ++i) png[i] = (v0 + i < V) ? cu * (float)(cnt[i] + 1) + sp[threadIdx.x * E + i] : 0.f;
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) png[i] = 0.f;
  }

  if (!waited) {
    pdl_wait();
    pdl_trigger();
  }
  const int t_obs = (io.update || io.intervals) ? b.obs[j] : -1;
  if (io.update && (t_obs < 0 || t_obs >= V)) {   // rejected on the host; never index with it
    if (rank == 0 && threadIdx.x == 0) atomicOr(&st.status, ST_BAD_TOKEN);
    return false;                                 // uniform across the cluster
  }
  if (io.probe_png && ngram) store_run<E>(io.probe_png + (size_t)j * V, v0, V, png);

  // ---- biased logits s = z / tau + b and their softmax (round 1)
  if (!b.z_in) load_run<E>(st.z, v0, V, s, -INFINITY);
  if (io.probe_z) store_run<E>(io.probe_z + (size_t)j * V, v0, V, s);
  const float inv_tau = 1.0f / D.tau;             // exact for tau = 1
#pragma unroll
  for (int i = 0; i < E; ++i) s[i] = (v0 + i < V) ? fmaf(s[i], inv_tau, bias[i]) : -INFINITY;
  // the N-gram entropy in bits (confidence skip, Sec. 3.7), -p log2 p summed
  // with the softmax normaliser
  float h_in = 0.f;
  if (D.skip) {
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (v0 + i < V && png[i] > 0.f) h_in -= png[i] * log2f(png[i]);
  }
  float pt[E], H = 0.f, f_cta = 0.f;
  const MS ms = softmax_round<E, kStepCluster>(s, pt, h_in, H, f_cta, cl, sh);
  const bool skipped = D.skip && H < kSkipBits;
  const float M = ms.m, S = ms.s;
#pragma unroll
  for (int i = 0; i < E; ++i) pt[i] = (v0 + i < V) ? pt[i] * f_cta : 0.f;
  if (io.probe_pt) store_run<E>(io.probe_pt + (size_t)j * V, v0, V, pt);

  // ---- mix (Sec. 3.5): LLM alone during warm-up
  const bool mixing = ngram && i_tok > D.warmup;
  const float tm = fmaxf(th0, th1);
  const float e0 = expf(th0 - tm), e1 = expf(th1 - tm);
  const float w0 = e0 / (e0 + e1), w1 = e1 / (e0 + e1);
  float p[E];
#pragma unroll
  for (int i = 0; i < E; ++i) p[i] = skipped ? png[i] : mixing ? w0 * pt[i] + w1 * png[i] : pt[i];
  if (io.probe_p) store_run<E>(io.probe_p + (size_t)j * V, v0, V, p);

  // ---- round 2: counts, residual, argmax, interval; publish t*'s values
  float obs[3] = {0.f, 0.f, 0.f};
  if (t_obs >= v0 && t_obs < v0 + E) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if (v0 + i == t_obs) {
        obs[0] = pt[i];
        obs[1] = png[i];
        obs[2] = s[i] - M - logf(S);
      }
    }
  }
  uint32_t c[E];
  const QuantResult q = quantise_round<E, kStepCluster>(p, v0, V, D.log2T, D.floor, io.predict != 0, t_obs,
                                          io.update ? obs : nullptr, c, cl, sh);
  if (io.predict) {
    if (q.bad && threadIdx.x == 0 && rank == 0) atomicOr(&st.status, ST_NUMERIC);
    if (io.intervals && t_obs >= v0 && t_obs < v0 + E) {
      const unsigned long long lo = q.below + (q.argmax < t_obs ? (unsigned long long)q.resid : 0ull);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        if (v0 + i == t_obs) {
          uint32_t* iv = io.intervals + 2 * ((size_t)j * io.interval_stride + (i_tok - 1));
          iv[0] = (uint32_t)lo;
          iv[1] = (uint32_t)(lo + c[i]);
        }
      }
    }
    if (io.cdf) scan_round<E>(c, v0, V, 1u << D.log2T, io.cdf + (size_t)j * (V + 1), cl, sh);
  }

  if (io.update && !skipped) {                     // a skipped token teaches the N-gram only
    const StepShared* o = cl.map_shared_rank(&sh, t_obs / chunk);
    const float pts = o->cl_obs[0], pngs = o->cl_obs[1], lpt = o->cl_obs[2];
    float scale = 1.f;
    float nth0 = th0, nth1 = th1;
    if (D.rule == NC_RULE_MIXED_NLL) {
      if (mixing) {
        const float pm = w0 * pts + w1 * pngs;
        scale = w0 * pts / pm;
        nth0 = th0 - D.alpha * (w0 - w0 * pts / pm);
        nth1 = th1 - D.alpha * (w1 - w1 * pngs / pm);
      }
    } else if (mixing) {
      const float a0 = th0 + D.eta * lpt, a1 = th1 + D.eta * logf(pngs);
      const float am = fmaxf(a0, a1);
      const float lse = am + logf(expf(a0 - am) + expf(a1 - am));
      nth0 = a0 - lse;
      nth1 = a1 - lse;
    }
    if (D.use_head) {
      const float step = D.alpha * scale;
#pragma unroll
      for (int i = 0; i < E; ++i) bias[i] = bias[i] - step * (pt[i] - (v0 + i == t_obs ? 1.f : 0.f));
      store_run<E>(st.bias, v0, V, bias);
    }
    if (rank == 0 && threadIdx.x == 0) {
      st.theta[0] = nth0;
      st.theta[1] = nth1;
      st.pt_obs = pts;
      st.png_obs = pngs;
    }
  }
  // the unigram count of the coded token, for a caller that keeps the
  // counts from one position to the next (the N-gram update adds it in memory)
  if (ngram && io.update && t_obs >= v0 && t_obs < v0 + E) {
#pragma unroll
    for (int i = 0; i < E; ++i)
      if (v0 + i == t_obs) cnt[i] += 1;
  }
  return true;
}

template <int E>
__global__ void __launch_bounds__(kStepThreads, 1) k_vocab(Dims D, Batch b, VocabIO io) {
  extern __shared__ float4 dyn4[];
  float* sp = reinterpret_cast<float*>(dyn4);    // sparse N-gram mass of this CTA's chunk
  __shared__ StepShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int j = blockIdx.x / kStepCluster;
  // after a prefill the previous kernel is the N-gram update of the previous
  // position: nothing of the stream's state may be read before it completed
  if (b.z_in) {
    pdl_wait();
    pdl_trigger();
  }
  if (j >= *b.nB) return;                        // uniform across the cluster
  const int rank = (int)cl.block_rank();
  float bias[E];
  int cnt[E];
  if (!vocab_pass<E>(D, b, io, j, rank, cl, sh, sp, bias, false, cnt, false, false, b.z_in != nullptr)) return;
  cl.sync();   // keep this CTA's shared memory alive until the cluster has read it
  // the N-gram update and bookkeeping of this row, once every CTA has read
  // the stream's state
  if (io.update && io.ngram && rank == 0)
    ngram_update_row(D, b, j, threadIdx.x >> 5, threadIdx.x & 31, nullptr, nullptr);
}

// The vocabulary passes of a prefill chunk: the cluster of stream row j runs
// positions p0 .. p0 + m - 1 in order (while the stream has tokens), each
// one vocab_pass and the N-gram update, with the bias kept in registers and
// a cluster barrier between positions.
template <int E>
__global__ void __launch_bounds__(kStepThreads, 1)
    k_vocab_seq(Dims D, Batch b, VocabIO io, int m, int n_streams, const float* zrows, const int32_t* nb_step,
                const int32_t* obs_step) {
  extern __shared__ float4 dyn4[];
  float* sp = reinterpret_cast<float*>(dyn4);
  __shared__ StepShared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int j = blockIdx.x / kStepCluster;
  pdl_wait();
  pdl_trigger();
  const int rank = (int)cl.block_rank();
  float bias[E];
  int cnt[E];
  for (int r = 0; r < m; ++r) {
    if (j >= nb_step[r]) break;                    // uniform across the cluster
    Batch br = b;
    br.obs = obs_step + (size_t)r * n_streams;
    br.z_in = zrows + (size_t)r * D.V;
    if (!vocab_pass<E>(D, br, io, j, rank, cl, sh, sp, bias, r > 0, cnt, r > 0, r > 0, true)) break;
    if (io.ngram && rank == 0) ngram_update_row(D, br, j, threadIdx.x >> 5, threadIdx.x & 31, &sh, &cl);
    cl.sync();   // the stream's state of this position is final for the next
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

// One warp per stream: count the observed token in every context order,
// the unigram counts, then advance the stream (window, history, position) and
// look up the contexts of the next prediction.
// The N-gram update of row j and the stream's bookkeeping for the next step.
// Warp k (k < 3) owns order k: it counts the observed token t in the entry
// of the context of length k + 1 (inserting the context if new), then looks
// up the entry of the next context (t appended) for the next prediction.
// The orders use separate tables, so the warps run concurrently; within an
// order the lookup follows the update.  Warp 0 also updates the unigram
// counts and the stream's position, history and window start.
__device__ void ngram_update_order(const Dims& D, StreamDev& st, int t, int k, int lane) {
  const int nh = min(3, st.n_coded);               // contexts before t
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
    const int nh2 = min(3, st.n_coded + 1);
    st.ctx_ent[k] = (k < D.order && k < nh2) ? ng_find(st, k, ctx_key(nhist, k + 1), false) : -1;
  }
}

// push (the persistent loop): afterwards the N-gram state of the stream's
// next prediction is written into the shared memory of every CTA of the
// cluster (the same values ng_gather would read from the tables).
__device__ void ngram_update_row(const Dims& D, const Batch& b, int j, int warp, int lane, StepShared* push,
                                 cg::cluster_group* cl) {
  StreamDev& st = b.st[b.slots[j]];
  const int t = b.obs[j];
  if (t < 0 || t >= D.V) {
    if (warp == 0 && lane == 0) atomicOr(&st.status, ST_BAD_TOKEN);
    return;
  }
  if (warp < kMaxOrder) ngram_update_order(D, st, t, warp, lane);
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
  if (!push || D.order == 0) return;
  __syncthreads();                                 // every order's lookup and the unigram total are final
  if (warp < kMaxOrder) {
    const int k = warp;
    const int ei = k < D.order ? st.ctx_ent[k] : -1;
    const NgEntry* en = ei >= 0 ? st.ent[k] + ei : nullptr;
    const int ns = en ? en->nslots : 0;
    for (int r = 0; r < kStepCluster; ++r) {
      StepShared* o = cl->map_shared_rank(push, r);
      if (lane == 0) o->ng_ns[k] = ns;
      for (int q = lane; q < ns; q += 32) {
        o->ng_tok[k][q] = en->tok[q];
        o->ng_cnt[k][q] = en->cnt[q];
      }
    }
  } else if (warp == kMaxOrder && lane == 0) {
    float nk[kMaxOrder], coef[kMaxOrder], cu;
    bool has[kMaxOrder];
    for (int k = 0; k < kMaxOrder; ++k) {
      const int ei = k < D.order ? st.ctx_ent[k] : -1;
      has[k] = ei >= 0;
      nk[k] = has[k] ? (float)st.ent[k][ei].n : 0.f;
    }
    ng_weights(nk, has, st.N, D.V, coef, cu);
    for (int r = 0; r < kStepCluster; ++r) {
      StepShared* o = cl->map_shared_rank(push, r);
      for (int k = 0; k < kMaxOrder; ++k) o->ng_coef[k] = coef[k];
      o->ng_cu = cu;
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

// Encoder prefill of positions p0 .. p0 + m - 1 (p0 = n_coded of row 0;
// rows sorted longest first, so the streams with tokens left are a prefix).
// Forward row i = j m + r: slot, position (-1 past the stream's end) and
// input token.  Sequential pass r: active rows nb_step[r], observed tokens
// obs_step[r n + j]; row j's logits sit at forward row z_idx[j] + r.
__global__ void k_prepare_prefill(Batch b, int n_streams, int m, int V, const int32_t* tok_flat, const int64_t* offs,
                                  const int64_t* lens, int32_t* f_slots, int32_t* f_pos, int32_t* f_tok,
                                  int32_t* nB_fwd, int32_t* obs_step, int32_t* nb_step, int32_t* z_idx) {
  pdl_wait();
  pdl_trigger();
  const int p0 = b.st[b.slots[0]].n_coded;
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
  const QuantResult q = quantise_round<E, kVocabCluster>(pr, v0, V, log2T, floor_c, true, -1, nullptr, c, cl, sh);
  if (q.bad && threadIdx.x == 0 && rank == 0) atomicOr(status + j, ST_NUMERIC);
  scan_round<E>(c, v0, V, 1u << log2T, cdf + (size_t)j * (V + 1), cl, sh);
  cl.sync();
}

__global__ void k_floor_counts(const float* p, int64_t n, uint32_t K, uint32_t floor_c,
                               uint32_t* c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool bad = false;
    const uint32_t q = floor_prod(p[i], K, bad);
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
  float mx = -INFINITY;
  for (int v = threadIdx.x; v < V; v += kVocabThreads) mx = fmaxf(mx, __fdiv_rn(zr[v], tau) + br[v]);
  const float M = block_max(mx, sh);
  float ls = 0.f;
  for (int v = threadIdx.x; v < V; v += kVocabThreads) ls += expf(__fdiv_rn(zr[v], tau) + br[v] - M);
  const float S = block_sum(ls, sh);
  const float pts = __fdiv_rn(expf(__fdiv_rn(zr[t], tau) + br[t] - M), S);
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
      const float ptv = __fdiv_rn(expf(__fdiv_rn(zr[v], tau) + br[v] - M), S);
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

template <int E>
static cudaError_t vocab_t(const Dims& D, const Batch& b, const VocabIO& io, cudaStream_t s) {
  const size_t smem = (size_t)kStepThreads * E * sizeof(float);
  return launch_kernel_cluster(k_vocab<E>, dim3(b.Bmax * kStepCluster), dim3(kStepThreads), smem, s, D.pdl,
                               kStepCluster, D, b, io);
}

template <int E>
static cudaError_t prepare_vocab_t() {
  cudaError_t e = cudaFuncSetAttribute(k_vocab<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStepThreads * E * (int)sizeof(float));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vocab_seq<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStepThreads * E * (int)sizeof(float));
  return e;
}

cudaError_t prepare_vocab_kernels(const Dims& D) {
  switch (vocab_E(D.V, kStepCluster, kStepThreads)) {
    case 4: return prepare_vocab_t<4>();
    case 8: return prepare_vocab_t<8>();
    case 12: return prepare_vocab_t<12>();
    case 16: return prepare_vocab_t<16>();
  }
  return cudaErrorInvalidValue;
}

template <int E>
static cudaError_t vocab_seq_t(const Dims& D, const Batch& b, const VocabIO& io, int m, const float* zrows,
                               const int32_t* nb_step, const int32_t* obs_step, cudaStream_t s) {
  const size_t smem = (size_t)kStepThreads * E * sizeof(float);
  return launch_kernel_cluster(k_vocab_seq<E>, dim3(b.Bmax * kStepCluster), dim3(kStepThreads), smem, s, D.pdl,
                               kStepCluster, D, b, io, m, b.Bmax, zrows, nb_step, obs_step);
}

cudaError_t launch_vocab_seq(const Dims& D, const Batch& b, const VocabIO& io, int m, const float* zrows,
                             const int32_t* nb_step, const int32_t* obs_step, cudaStream_t s) {
  switch (vocab_E(D.V, kStepCluster, kStepThreads)) {
    case 4: return vocab_seq_t<4>(D, b, io, m, zrows, nb_step, obs_step, s);
    case 8: return vocab_seq_t<8>(D, b, io, m, zrows, nb_step, obs_step, s);
    case 12: return vocab_seq_t<12>(D, b, io, m, zrows, nb_step, obs_step, s);
    case 16: return vocab_seq_t<16>(D, b, io, m, zrows, nb_step, obs_step, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_vocab(const Dims& D, const Batch& b, const VocabIO& io, cudaStream_t s) {
  switch (vocab_E(D.V, kStepCluster, kStepThreads)) {
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

cudaError_t launch_prepare_prefill(const Batch& b, int n_streams, int m, int V, const int32_t* tok_flat,
                                   const int64_t* offs, const int64_t* lens, int32_t* f_slots, int32_t* f_pos,
                                   int32_t* f_tok, int32_t* nB_fwd, int32_t* obs_step, int32_t* nb_step,
                                   int32_t* z_idx, cudaStream_t s) {
  const int rows = n_streams * m;
  const int blocks = std::min((rows + 255) / 256, 64);
  return launch_kernel(k_prepare_prefill, dim3(blocks), dim3(256), 0, s, true, b, n_streams, m, V, tok_flat, offs,
                       lens, f_slots, f_pos, f_tok, nB_fwd, obs_step, nb_step, z_idx);
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
