// Persistent decode step: the whole transformer forward of a small batch of
// streams (embedding, 30 layers, final norm, LM head) in one cooperative
// launch.  The phases of a layer (QKV, attention, O projection, gate/up,
// down) are separated by a grid-wide barrier instead of kernel boundaries.
// Before arriving at a barrier, each warp loads the weight rows (or the
// cached keys and values) it will need in the next phase, so the loads are
// in flight while the barrier completes.
//
// Work is divided exactly as in the one-kernel-per-phase path and uses the
// same device functions (model_dev.cuh), so every value is bit-identical to
// that path.  The barrier spins are bounded: a barrier that gives up sets
// the error word, and every block leaves at its next barrier.
#include "model_dev.cuh"

namespace nc {

namespace {

using namespace dev;

template <int V>
struct EpiTag {
  static constexpr int value = V;
};
using EStore = EpiTag<EPI_STORE>;
using EResid = EpiTag<EPI_RESID>;
using ESwiglu = EpiTag<EPI_SWIGLU>;
using ELogits = EpiTag<EPI_LOGITS>;

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;
constexpr int kGroups = kStepThreads / 128;        // attention units per block at a time
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on a monotonically increasing arrival counter (reset to zero
// before each launch).  Returns false when the step must stop (this or an
// earlier barrier gave up).
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned& epoch, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    uint32_t it = 0;
    bool ok = true;
    while (ld_acquire(bar) < target) {
      if (++it == kSpinLimit) {
        atomicOr(err, ST_TIMEOUT);
        ok = false;
        break;
      }
    }
    if (ok && ld_acquire(reinterpret_cast<unsigned*>(err)) != 0) ok = false;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Named barrier of one 128-thread attention group.
__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, 128;" ::"r"(grp + 1) : "memory");
}

// Raw activation sources of a GEMV prologue (row, column) -> value.  Reads of
// data written by other blocks in this launch bypass L1.
struct SrcRows {
  const float* p;
  int stride;
  __device__ float operator()(int row, int c) const { return __ldcg(p + (size_t)row * stride + c); }
};
template <int FMT>
struct SrcEmbed {
  const void* E;
  const float* scale;
  int d;
  const StreamDev* st;
  const int32_t* slots;
  __device__ float operator()(int row, int c) const {
    return embed_at<FMT>(E, scale, d, st[slots[row]].last_tok, c);
  }
};

// Warm L2 with the rows this warp will read in a later GEMV phase.
template <int FMT>
__device__ __forceinline__ void prefetch_rows(const Mat& m, int gw, int GW, int lane) {
  const size_t row_bytes = (size_t)m.cols * WFmt<FMT>::ESZ;
  const size_t total = (size_t)m.rows * row_bytes;
  const char* base = static_cast<const char*>(m.w);
  for (int rp = gw; 2 * rp < m.rows; rp += GW) {
    const size_t first = (size_t)2 * rp * row_bytes;
    const size_t nbytes = (2 * rp + 1 < m.rows ? 2 : 1) * row_bytes;
    for (size_t off = (size_t)lane * 128; off < nbytes; off += 32 * 128)
      if (first + off < total) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + first + off));
  }
}

// One GEMV phase over the batch (B <= BT rows, one activation tile).
template <int FMT, int EPI, bool RMS, int BT, typename Src>
__device__ __noinline__ void phase_gemv(const Dims& D, const Mat& m, Src src, const float* gain, int B, float* xs,
                                        ProScratch& ps, GemvOut out, int gw, int GW) {
  const int tid = threadIdx.x, lane = tid & 31;
  prologue<RMS>(D, src, gain, m.cols, 0, B, xs, ps, tid, kStepThreads, [] { __syncthreads(); });
  const int nrp = (m.rows + 1) / 2;
  for (int rp = gw; rp < nrp; rp += GW) {
    uint4 h0[kHold], h1[kHold];
    load_rowpair<FMT, kHold>(m, rp, lane, h0, h1);
    gemv_rowpair<FMT, EPI, kHold, BT>(m, rp, xs, 0, B, h0, h1, lane, out);
  }
}

// One attention phase: this 128-thread group's units (row j, KV head g, chunk s).
template <int KBF16>
__device__ __noinline__ void phase_attn(const Dims& D, const Batch& b, int layer, int B, AttnSmem& sm,
                                        const AttnIO& aio, int gunit, int GU, int group, int gtid) {
  const int nsm = attn_splits_max_dev(D);
  const int n_units = B * D.hkv * nsm;
  for (int u = gunit; u < n_units; u += GU) {
    const int s = u % nsm, g = (u / nsm) % D.hkv, j = u / (nsm * D.hkv);
    StreamDev& st = b.st[b.slots[j]];
    const int a = st.n_coded, start = window_start(D, st);
    const int ns = (a - start + 1 + kAttnChunk - 1) / kAttnChunk;
    if (s >= ns) continue;                         // uniform across the group
    AttnPre<KBF16> pre;
    attn_preload<KBF16>(D, st, layer, g, s, start, a, gtid, sm, pre);
    attn_compute<KBF16>(D, st, layer, j, g, s, start, a, ns, gtid, sm, pre, aio, [group] { group_sync(group); });
  }
}

// Warm L2 with the cached keys / values of this group's units.
__device__ __forceinline__ void prefetch_attn(const Dims& D, const Batch& b, int layer, int B, int gunit, int GU,
                                              int gtid) {
  const int nsm = attn_splits_max_dev(D);
  const int n_units = B * D.hkv * nsm;
  for (int u = gunit; u < n_units; u += GU) {
    const int s = u % nsm, g = (u / nsm) % D.hkv, j = u / (nsm * D.hkv);
    const StreamDev& st = b.st[b.slots[j]];
    const int a = st.n_coded, start = window_start(D, st);
    const int ns = (a - start + 1 + kAttnChunk - 1) / kAttnChunk;
    if (s < ns) attn_prefetch(D, st, layer, g, s, start, a, gtid);
  }
}

template <int FMT, int KBF16, int BT>
__global__ void __launch_bounds__(kStepThreads, 1) k_step(Dims D, Batch b, StepArgs A) {
  extern __shared__ float4 smem4[];
  float* xs = reinterpret_cast<float*>(smem4);   // [kBT][max cols]
  __shared__ ProScratch ps;
  __shared__ AttnSmem asm_[kGroups];
  __shared__ int s_ok;
  __shared__ int s_B;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gw = blockIdx.x * kStepWarps + warp;          // global warp
  const int GW = gridDim.x * kStepWarps;
  const int group = warp >> 2, gtid = tid & 127;
  const int gunit = blockIdx.x * kGroups + group;
  const int GU = gridDim.x * kGroups;
  unsigned epoch = 0;

  // Launched without the PDL attribute and never signals early launch of its
  // dependents: a kernel that follows starts only after this grid completed.
  // rows of this step: all rows, or (encoder) the rows with tokens left;
  // rows are sorted longest first, so those are a prefix
  if (tid == 0) {
    int B = 0;
    if (A.encode) {
      for (int j = 0; j < b.Bmax; ++j) {
        const int nc = b.st[b.slots[j]].n_coded;
        const bool act = nc < A.lens[j];
        if (blockIdx.x == 0) A.obs[j] = act ? A.tok_flat[A.offs[j] + nc] : 0;
        B += act;
      }
      if (blockIdx.x == 0) *A.nB_out = B;
    } else {
      B = *b.nB;
    }
    s_B = B;
  }
  __syncthreads();
  const int B = s_B;
  if (B == 0) return;                              // uniform: every block sees the same B

  const int d = D.d;
  const GemvOut out_qkv{A.qkv, b.st, b.slots}, out_x{A.x, b.st, b.slots}, out_h{A.h, b.st, b.slots};
  const GemvOut out_z{nullptr, b.st, b.slots};
  const SrcRows src_x{A.x, d}, src_attn{A.attn_out, D.hq * kHeadDim}, src_h{A.h, D.F};
  const SrcEmbed<FMT> src_embed{A.embed, A.embed_scale, d, b.st, b.slots};
  const AttnIO aio{A.qkv, A.part, A.tickets, A.attn_out};
  const Mat head{A.embed, A.embed_scale, D.V, d};

  // embedding: block 0 writes the residual stream; every block feeds the
  // first QKV projection straight from the embedding rows
  if (blockIdx.x == 0)
    for (int e = tid; e < B * d; e += kStepThreads) A.x[e] = src_embed(e / d, e % d);
  for (int l = 0; l < D.n_layers; ++l) {
    const LayerW& L = A.layers[l];
    if (l == 0)
      phase_gemv<FMT, EPI_STORE, true, BT>(D, L.qkv, src_embed, L.g_attn, B, xs, ps, out_qkv, gw, GW);
    else
      phase_gemv<FMT, EPI_STORE, true, BT>(D, L.qkv, src_x, L.g_attn, B, xs, ps, out_qkv, gw, GW);
    prefetch_attn(D, b, l, B, gunit, GU, gtid);
    prefetch_rows<FMT>(L.o, gw, GW, lane);
    if (!grid_barrier(A.bar, A.err, epoch, &s_ok)) return;
    phase_attn<KBF16>(D, b, l, B, asm_[group], aio, gunit, GU, group, gtid);
    prefetch_rows<FMT>(L.gu, gw, GW, lane);
    if (!grid_barrier(A.bar, A.err, epoch, &s_ok)) return;
    phase_gemv<FMT, EPI_RESID, false, BT>(D, L.o, src_attn, nullptr, B, xs, ps, out_x, gw, GW);
    prefetch_rows<FMT>(L.down, gw, GW, lane);
    if (!grid_barrier(A.bar, A.err, epoch, &s_ok)) return;
    phase_gemv<FMT, EPI_SWIGLU, true, BT>(D, L.gu, src_x, L.g_ffn, B, xs, ps, out_h, gw, GW);
    if (l + 1 < D.n_layers) prefetch_rows<FMT>(A.layers[l + 1].qkv, gw, GW, lane);
    if (!grid_barrier(A.bar, A.err, epoch, &s_ok)) return;
    phase_gemv<FMT, EPI_RESID, false, BT>(D, L.down, src_h, nullptr, B, xs, ps, out_x, gw, GW);
    if (l + 1 == D.n_layers) prefetch_rows<FMT>(head, gw, GW, lane);
    if (!grid_barrier(A.bar, A.err, epoch, &s_ok)) return;
  }
  phase_gemv<FMT, EPI_LOGITS, true, BT>(D, head, src_x, A.g_final, B, xs, ps, out_z, gw, GW);
}

}  // namespace

size_t step_smem_bytes(const Dims& D) {
  const int cmax = D.d > D.F ? D.d : D.F;
  return (size_t)kBT * cmax * sizeof(float);
}

bool step_supported(const Dims& D, int Bmax) {
  return Bmax <= kBT && D.hq / D.hkv <= kMaxGroup && step_smem_bytes(D) <= 200 * 1024;
}

template <int BT>
static void (*step_kernel_bt(const Dims& D, int fmt))(Dims, Batch, StepArgs) {
  return fmt == NC_FP32 ? (D.kv_bf16 ? k_step<NC_FP32, 1, BT> : k_step<NC_FP32, 0, BT>)
         : fmt == NC_BF16 ? k_step<NC_BF16, 1, BT>
                          : k_step<NC_FP8E4M3, 1, BT>;
}

static void (*step_kernel(const Dims& D, int fmt, int Bmax))(Dims, Batch, StepArgs) {
  return Bmax <= 1 ? step_kernel_bt<1>(D, fmt) : step_kernel_bt<kBT>(D, fmt);
}

cudaError_t prepare_step_kernel(const Dims& D, int fmt) {
  cudaError_t e = cudaFuncSetAttribute(step_kernel(D, fmt, 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)step_smem_bytes(D));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_kernel(D, fmt, kBT), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_smem_bytes(D));
  return e;
}

cudaError_t launch_step(const Dims& D, const Batch& b, int fmt, const StepArgs& A, cudaStream_t s) {
  auto kern = step_kernel(D, fmt, b.Bmax);
  const size_t smem = step_smem_bytes(D);
  cudaError_t e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaMemsetAsync(A.bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sms);
  cfg.blockDim = dim3(kStepThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, D, b, A);
}

}  // namespace nc
