// tcgen05 tensor-core GEMM for the batched projections.
//
// Y[n][m] = sum_k W[m][k] X[n][k]: the weight matrix W [M, K] is the MMA's A
// operand (M = output channels, 128 per CTA), the batch of activation rows
// X [N, K] is the B operand (N = streams, BN per CTA).  Both are K-major and
// staged by TMA into 128-byte-swizzled shared memory through a ring of
// STAGES buffers; one thread issues tcgen05.mma (kind::f16 for BF16,
// kind::f8f6f4 for FP8 E4M3) into an FP32 accumulator in tensor memory; after
// the last K block the eight warps read the accumulator back with tcgen05.ld
// (two warps per lane quarter, one per half of the columns) and apply the
// fused epilogue.  Every output element accumulates its K
// blocks in the same order whatever BN, the grid or the batch, so results
// do not depend on how many streams share a step.
//
// Every wait on an mbarrier is bounded; a wait that gives up records an error
// in the context's status word and skips the remaining work.  Before the CTA
// frees its tensor memory and exits it waits, with the same bound, for what it
// already issued: the products (one commit after the last one issued) and the
// TMA loads no product consumed, so nothing lands in a CTA that has exited.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "internal.h"
#include "tc5.cuh"

namespace nc {

namespace {

using namespace tc5;

constexpr int kTcThreads = 256;              // 8 warps: all read the accumulator back
constexpr int kTileM = 128;
constexpr int kKBlockBytes = 128;            // one 128-byte swizzle row per operand row
// SiLU of the tensor-core path: a * (1 / (1 + e^-a)) with the fast exponential
// and a correctly rounded reciprocal (1 / inf = 0 for very negative a).  The
// decode step and the prefill forward run this same code.
__device__ __forceinline__ float silu_tc(float a) { return a * __frcp_rn(1.0f + __expf(-a)); }

template <int BN>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
}

template <int BN, int STAGES, int KP>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return 1024 /* alignment slack */ + (size_t)STAGES * KP * (kTileM + BN) * kKBlockBytes + 256;
}

// SwiGLU of two adjacent batch columns n, n + 1: rows 2j (gate) and 2j + 1
// (up) sit on adjacent lanes; the even lane computes h_j of column n, the odd
// lane h_j of column n + 1, each from one exchanged value; y0, y1 already
// carry the FP8 scales.
__device__ __forceinline__ void swiglu_pair(const TcGemm& g, int r, int n, int B, float y0, float y1) {
  const bool odd = r & 1;
  const float got = __shfl_xor_sync(0xffffffffu, odd ? y0 : y1, 1);
  const float gate = odd ? got : y0, up = odd ? y1 : got;
  const int col = n + (odd ? 1 : 0);
  if (col < B && r < g.M) {
    const float h = silu_tc(gate) * up;
    if (g.h16)
      static_cast<__nv_bfloat16*>(g.h16)[(size_t)col * (g.M / 2) + (r >> 1)] = __float2bfloat16_rn(h);
    else
      g.h_out[(size_t)col * (g.M / 2) + (r >> 1)] = h;
  }
}

// One output element (row r of the weights, batch row n) through the store,
// residual or logits epilogue; y already carries the FP8 scales.
template <int EPI>
__device__ __forceinline__ void epi_store(const TcGemm& g, int r, int n, int B, float y, float res) {
  if (n < B && r < g.M) {
    if (EPI == EPI_STORE) {
      g.y[(size_t)n * g.M + r] = y;
    } else if (EPI == EPI_RESID) {
      g.y[(size_t)n * g.M + r] = res + y;
    } else {
      if (g.zrows)
        g.zrows[(size_t)n * g.M + r] = y;
      else
        g.st[g.slots[n]].z[r] = y;
    }
  }
}

// The residual epilogue reads the first kPreCols columns' residuals of its
// row into registers while the products run; the rest, 16 columns at a
// time, one group ahead of the group it stores.
constexpr int kPreCols = 64;

// KP: K blocks per pipeline stage.  KP = 2 takes both operands' two K blocks
// in one 3D TMA box each (maps [K blocks][rows][128 bytes], K a multiple of
// the block), halving the copies; the products and their order are those of
// KP = 1.
template <int BN, int STAGES, int KIND_BF16, int EPI, int KP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, TcGemm g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr size_t kStageA = (size_t)KP * kTileM * kKBlockBytes, kStageB = (size_t)KP * BN * kKBlockBytes;
  uint8_t* sA = base;
  uint8_t* sB = base + STAGES * kStageA;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * kStageB);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  uint32_t* fail = tmem_slot + 1;
  int32_t* n_issued = reinterpret_cast<int32_t*>(fail + 1);     // stages whose TMA loads were issued
  int32_t* n_consumed = n_issued + 1;                          // stages the MMA issuer saw land

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM;
  const int n0 = blockIdx.y * BN;
  const int kblk = KIND_BF16 ? 64 : 128;             // elements per 128-byte K block
  const int nk = (g.K + kblk - 1) / kblk;            // the tail block reads zeros past K
  const int ns = (nk + KP - 1) / KP;                 // stages
  constexpr uint32_t kCols = tmem_cols<BN>();
  constexpr uint32_t kStageBytes = (uint32_t)(kStageA + kStageB);
  // stage ks's loads: K block ks of a 2D map, or K blocks KP ks .. of a 3D map
  auto load_a = [&](int ks, int s) {
    if (KP == 1) tma_load_2d(sA + s * kStageA, &tA, full + s, ks * kblk, m0);
    else tma_load_3d(sA + s * kStageA, &tA, full + s, 0, m0, KP * ks);
  };
  auto load_b = [&](int ks, int s) {
    if (KP == 1) tma_load_2d(sB + s * kStageB, &tB, full + s, ks * kblk, n0);
    else tma_load_3d(sB + s * kStageB, &tB, full + s, 0, n0, KP * ks);
  };

  // the row count was written by the step's prepare kernel, several launches
  // back, so it may be read before the wait on the previous kernel
  const int B = *g.nB;
  if (n0 >= B) return;                            // uniform across the CTA
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *fail = 0;
    *n_issued = 0;
    *n_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bool active = true;

  // weight tiles of the first stages do not depend on the previous kernel:
  // in flight before waiting on it; the operand tiles only after
  if (threadIdx.x == 0) {
    for (int ks = 0; ks < ns && ks < STAGES; ++ks) {
      mbar_expect_tx(full + ks, kStageBytes);
      load_a(ks, ks);
    }
  }
  pdl_wait();
  pdl_trigger();
  // the epilogue's first residuals (warp w: TMEM lanes 32 (w % 4) .., the
  // columns of half w / 4), in flight beside the products
  const int quarter = warp & 3, half = warp >> 2;
  const int r_ep = m0 + quarter * 32 + lane;         // weight row = TMEM lane
  const int c_ep = half * (BN / 2);
  constexpr int kPre = BN / 2 < kPreCols ? BN / 2 : kPreCols;
  float pre[kPre];
#pragma unroll
  for (int i = 0; i < kPre; ++i) {
    const int n = n0 + c_ep + i;
    pre[i] = (EPI == EPI_RESID && n < B && r_ep < g.M) ? __ldcg(g.y + (size_t)n * g.M + r_ep) : 0.f;
  }

  if (active && threadIdx.x == 0) {
    // TMA producer
    int ks = 0;
    for (; ks < ns; ++ks) {
      const int s = ks % STAGES;
      const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
      if (ks >= STAGES) {
        if (!mbar_wait(empty + s, ph ^ 1u)) {
          atomicOr(fail, 1u);
          break;
        }
        mbar_expect_tx(full + s, kStageBytes);
        load_a(ks, s);
      }
      load_b(ks, s);
    }
    // the first STAGES weight loads went out before the loop in any case
    *n_issued = max(ks, min(ns, STAGES));
  } else if (active && threadIdx.x == 32) {
    // MMA issuer: 4 instructions of 32 bytes of K per 128-byte block
    const uint32_t id = idesc(KIND_BF16, kTileM, BN);
    bool ok = true;
    for (int ks = 0; ks < ns && ok; ++ks) {
      const int s = ks % STAGES;
      const uint32_t ph = (uint32_t)(ks / STAGES) & 1u;
      if (!mbar_wait(full + s, ph)) {
        atomicOr(fail, 2u);
        ok = false;
        break;
      }
      *n_consumed = ks + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < KP; ++kk) {
        const int kb = KP * ks + kk;
        if (kb >= nk) break;                       // a 3D box's block past K: zeros, not multiplied
        const uint32_t a0 = smem_u32(sA + s * kStageA + (size_t)kk * kTileM * kKBlockBytes);
        const uint32_t b0 = smem_u32(sB + s * kStageB + (size_t)kk * BN * kKBlockBytes);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          mma_issue(KIND_BF16, tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), id, (kb | k) ? 1u : 0u);
      }
      mma_commit(empty + s);
    }
    mma_commit(done);
  }
  __syncwarp();
  // accumulator ready (or the pipeline gave up)
  bool ready = active;
  if (active && !mbar_wait(done, 0)) {
    atomicOr(fail, 4u);
    ready = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (*fail && threadIdx.x == 0) {
    // give-up path: nothing this CTA issued may land in its shared memory
    // after it exits.  Every MMA was committed to `done` (waited on above);
    // wait, with the same bound, for the TMA loads no MMA consumed.
    for (int kb = *n_consumed; kb < *n_issued; ++kb)
      if (!mbar_wait(full + kb % STAGES, (uint32_t)(kb / STAGES) & 1u)) break;
  }
  if (ready && *fail == 0) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its lane quarter) and the
    // columns of half w / 4 of the tile
    const int r = r_ep;
    const uint32_t tw = tmem + ((uint32_t)(quarter * 32) << 16);
    float ws = 1.f;
    if (!KIND_BF16 && r < g.M) ws = g.w_scale[r];
    // the columns whose residuals are already in registers
#pragma unroll
    for (int c0 = 0; c0 < kPre; c0 += 16) {
      float v[16];
      tmem_ld16(tw + (uint32_t)(c_ep + c0), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = n0 + c_ep + c0 + i;
        if (!KIND_BF16) v[i] *= ws * (n < B ? __ldg(g.x_scale + n) : 0.f);
        if (EPI != EPI_SWIGLU) epi_store<EPI>(g, r, n, B, v[i], pre[c0 + i]);
      }
      if (EPI == EPI_SWIGLU) {
#pragma unroll
        for (int i = 0; i < 16; i += 2) swiglu_pair(g, r, n0 + c_ep + c0 + i, B, v[i], v[i + 1]);
      }
    }
    // the remaining columns: the loads of group c + 16 (row scales,
    // residuals) are issued before group c is stored
    float xs[16], res[16];
    auto load_group = [&](int c) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = n0 + c + i;
        const bool in = c < c_ep + BN / 2 && n < B;
        xs[i] = (!KIND_BF16 && in) ? __ldg(g.x_scale + n) : 0.f;
        res[i] = (EPI == EPI_RESID && in && r < g.M) ? __ldcg(g.y + (size_t)n * g.M + r) : 0.f;
      }
    };
    if (kPre < BN / 2) load_group(c_ep + kPre);
#pragma unroll 1
    for (int c = c_ep + kPre; c < c_ep + BN / 2; c += 16) {
      float v[16], xc[16], rc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        xc[i] = xs[i];
        rc[i] = res[i];
      }
      load_group(c + 16);
      tmem_ld16(tw + (uint32_t)c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = n0 + c + i;
        if (!KIND_BF16) v[i] *= ws * xc[i];
        if (EPI != EPI_SWIGLU) epi_store<EPI>(g, r, n, B, v[i], rc[i]);
      }
      if (EPI == EPI_SWIGLU) {
#pragma unroll
        for (int i = 0; i < 16; i += 2) swiglu_pair(g, r, n0 + c + i, B, v[i], v[i + 1]);
      }
    }
  }
  if (threadIdx.x == 0 && *fail && g.status) atomicOr(g.status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// The bounded wait's give-up path, exercised without a fault: one thread
// waits (at most `polls` polls) on an mbarrier nothing arrives on, and
// records ST_TIMEOUT in *status when the wait gives up, as the pipelines do.
__global__ void k_wait_selftest(uint32_t polls, int32_t* status) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(&bar, 0, polls)) atomicOr(status, ST_TIMEOUT);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

template <int BN, int STAGES, int KB, int EPI, int KP>
cudaError_t prepare_tc_t() {
  return cudaFuncSetAttribute(k_gemm_tc<BN, STAGES, KB, EPI, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes<BN, STAGES, KP>());
}

template <int KB, int EPI>
cudaError_t prepare_tc_epi() {
  cudaError_t e = prepare_tc_t<32, 10, KB, EPI, 1>();
  if (e == cudaSuccess) e = prepare_tc_t<64, 8, KB, EPI, 1>();
  if (e == cudaSuccess) e = prepare_tc_t<128, 6, KB, EPI, 1>();
  if (e == cudaSuccess) e = prepare_tc_t<256, 4, KB, EPI, 1>();
  if (KB) {
    if (e == cudaSuccess) e = prepare_tc_t<32, 5, KB, EPI, 2>();
    if (e == cudaSuccess) e = prepare_tc_t<64, 4, KB, EPI, 2>();
    if (e == cudaSuccess) e = prepare_tc_t<128, 3, KB, EPI, 2>();
    if (e == cudaSuccess) e = prepare_tc_t<256, 2, KB, EPI, 2>();
  }
  return e;
}

template <int BN, int STAGES, int KB, int EPI, int KP>
cudaError_t launch_tc_t(const TcGemm& g, cudaStream_t s, bool pdl) {
  constexpr size_t smem = tc_smem_bytes<BN, STAGES, KP>();
  auto kern = k_gemm_tc<BN, STAGES, KB, EPI, KP>;
  dim3 grid((g.M + kTileM - 1) / kTileM, (g.Bmax + BN - 1) / BN);
  const CUtensorMap* a = reinterpret_cast<const CUtensorMap*>(g.tmap_a);
  const CUtensorMap* b = reinterpret_cast<const CUtensorMap*>(g.tmap_b);
  return launch_kernel(kern, grid, dim3(kTcThreads), smem, s, pdl, *a, *b, g);
}

template <int KB, int EPI>
cudaError_t launch_tc_epi(const TcGemm& g, cudaStream_t s, bool pdl) {
  if (KB && g.kp == 2 && g.K % 64 == 0) {
    switch (g.bn) {
      case 32: return launch_tc_t<32, 5, KB, EPI, 2>(g, s, pdl);
      case 64: return launch_tc_t<64, 4, KB, EPI, 2>(g, s, pdl);
      case 128: return launch_tc_t<128, 3, KB, EPI, 2>(g, s, pdl);
      case 256: return launch_tc_t<256, 2, KB, EPI, 2>(g, s, pdl);
    }
    return cudaErrorInvalidValue;
  }
  if (g.kp == 2) return cudaErrorInvalidValue;
  switch (g.bn) {
    case 32: return launch_tc_t<32, 10, KB, EPI, 1>(g, s, pdl);
    case 64: return launch_tc_t<64, 8, KB, EPI, 1>(g, s, pdl);
    case 128: return launch_tc_t<128, 6, KB, EPI, 1>(g, s, pdl);
    case 256: return launch_tc_t<256, 4, KB, EPI, 1>(g, s, pdl);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------- activation preparation
// RMSNorm of x into the GEMM operand (BF16, or E4M3 with one scale per row).
template <int KB>
__global__ void k_act_rmsnorm(Dims D, Batch b, const float* x, const float* gain, int cols, void* out,
                              float* out_scale) {
  __shared__ float red[32];
  __shared__ float sc;
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x;
  if (j >= *b.nB) return;
  const float* xr = x + (size_t)j * cols;
  float ss = 0.f;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) ss = fmaf(xr[c], xr[c], ss);
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    sc = 1.0f / sqrtf(t / (float)cols + D.eps);
  }
  __syncthreads();
  const float inv = sc;
  if (KB) {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + (size_t)j * cols;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) o[c] = __float2bfloat16_rn(xr[c] * inv * gain[c]);
  } else {
    // per-row E4M3 scale: amax / 448 (max is order-independent)
    float m = 0.f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) m = fmaxf(m, fabsf(xr[c] * inv * gain[c]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
      const float s = t > 0.f ? __fdiv_rn(t, 448.0f) : 1.0f;
      out_scale[j] = s;
      red[0] = s;
    }
    __syncthreads();
    const float s = red[0];
    __nv_fp8_storage_t* o = static_cast<__nv_fp8_storage_t*>(out) + (size_t)j * cols;
    for (int c = threadIdx.x; c < cols; c += blockDim.x)
      o[c] = __nv_cvt_float_to_fp8(__fdiv_rn(xr[c] * inv * gain[c], s), __NV_SATFINITE, __NV_E4M3);
  }
}

// Write a row held in shared memory as the GEMM operand: BF16, or E4M3 with
// the row's scale amax / 448.
template <int KB>
__device__ void write_operand(const float* buf, int cols, int j, void* out, float* out_scale, float* red) {
  if (KB) {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + (size_t)j * cols;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) o[c] = __float2bfloat16_rn(buf[c]);
    return;
  }
  float m = 0.f;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) m = fmaxf(m, fabsf(buf[c]));
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    const float sc = t > 0.f ? __fdiv_rn(t, 448.0f) : 1.0f;
    out_scale[j] = sc;
    red[32] = sc;
  }
  __syncthreads();
  const float sc = red[32];
  __nv_fp8_storage_t* o = static_cast<__nv_fp8_storage_t*>(out) + (size_t)j * cols;
  for (int c = threadIdx.x; c < cols; c += blockDim.x)
    o[c] = __nv_cvt_float_to_fp8(__fdiv_rn(buf[c], sc), __NV_SATFINITE, __NV_E4M3);
}

// An FP32 activation row (attention output, SwiGLU output) as the GEMM operand.
template <int KB>
__global__ void k_act_plain(Dims D, Batch b, const float* x, int cols, void* out, float* out_scale) {
  __shared__ float red[33];
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x;
  if (j >= *b.nB) return;
  write_operand<KB>(x + (size_t)j * cols, cols, j, out, out_scale, red);
}

}  // namespace

cudaError_t launch_wait_selftest(uint32_t polls, int32_t* status, cudaStream_t s) {
  k_wait_selftest<<<1, 1, 0, s>>>(polls, status);
  return cudaGetLastError();
}

cudaError_t launch_act_plain(const Dims& D, const Batch& b, const float* x, int cols, int kind_bf16, void* out,
                             float* out_scale, cudaStream_t s) {
  return launch_kernel(kind_bf16 ? k_act_plain<1> : k_act_plain<0>, dim3(b.Bmax), dim3(256), 0, s, D.pdl, D, b, x,
                       cols, out, out_scale);
}

bool tc_encode_tmap3(void* tmap, const void* base, int elem_bytes, int64_t K, int64_t rows, int box_rows) {
  // [K / kblk][rows][kblk]: element (j, r, i) at base + r K + j kblk + i
  EncodeTiled fn = encode_fn();
  const int64_t kblk = kKBlockBytes / elem_bytes;
  if (!fn || K % kblk) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kblk, (cuuint64_t)rows, (cuuint64_t)(K / kblk)};
  cuuint64_t strides[2] = {(cuuint64_t)(K * elem_bytes), (cuuint64_t)kKBlockBytes};
  cuuint32_t box[3] = {(cuuint32_t)kblk, (cuuint32_t)box_rows, 2};
  cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  return fn(reinterpret_cast<CUtensorMap*>(tmap), dt, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_tmap(void* tmap, const void* base, int elem_bytes, int64_t inner, int64_t outer, int box_outer) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(inner * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)(kKBlockBytes / elem_bytes), (cuuint32_t)box_outer};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  return fn(reinterpret_cast<CUtensorMap*>(tmap), dt, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t prepare_tc_kernels() {
  static bool done = false;                        // per-kernel attributes: once per process
  if (done) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int kb = 0; kb < 2 && e == cudaSuccess; ++kb) {
    if (kb) {
      e = prepare_tc_epi<1, EPI_STORE>();
      if (e == cudaSuccess) e = prepare_tc_epi<1, EPI_RESID>();
      if (e == cudaSuccess) e = prepare_tc_epi<1, EPI_SWIGLU>();
      if (e == cudaSuccess) e = prepare_tc_epi<1, EPI_LOGITS>();
    } else {
      e = prepare_tc_epi<0, EPI_STORE>();
      if (e == cudaSuccess) e = prepare_tc_epi<0, EPI_RESID>();
      if (e == cudaSuccess) e = prepare_tc_epi<0, EPI_SWIGLU>();
      if (e == cudaSuccess) e = prepare_tc_epi<0, EPI_LOGITS>();
    }
  }
  done = e == cudaSuccess;
  return e;
}

cudaError_t launch_gemm_tc(const TcGemm& g, int epi, cudaStream_t s, bool pdl) {
  if (g.kind_bf16) {
    switch (epi) {
      case EPI_STORE: return launch_tc_epi<1, EPI_STORE>(g, s, pdl);
      case EPI_RESID: return launch_tc_epi<1, EPI_RESID>(g, s, pdl);
      case EPI_SWIGLU: return launch_tc_epi<1, EPI_SWIGLU>(g, s, pdl);
      case EPI_LOGITS: return launch_tc_epi<1, EPI_LOGITS>(g, s, pdl);
    }
  } else {
    switch (epi) {
      case EPI_STORE: return launch_tc_epi<0, EPI_STORE>(g, s, pdl);
      case EPI_RESID: return launch_tc_epi<0, EPI_RESID>(g, s, pdl);
      case EPI_SWIGLU: return launch_tc_epi<0, EPI_SWIGLU>(g, s, pdl);
      case EPI_LOGITS: return launch_tc_epi<0, EPI_LOGITS>(g, s, pdl);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_act_rmsnorm(const Dims& D, const Batch& b, const float* x, const float* gain, int cols,
                               int kind_bf16, void* out, float* out_scale, cudaStream_t s) {
  return launch_kernel(kind_bf16 ? k_act_rmsnorm<1> : k_act_rmsnorm<0>, dim3(b.Bmax), dim3(256), 0, s, D.pdl, D, b,
                       x, gain, cols, out, out_scale);
}

}  // namespace nc
