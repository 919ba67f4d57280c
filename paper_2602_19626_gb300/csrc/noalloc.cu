// CDF quantisation for callers that must not allocate device memory.
//
// nc_probs_to_cdf keeps one status word per row in a buffer it allocates on
// every call.  Some callers cannot let a library allocate:
// - a serving process whose allocator has already reserved all free HBM;
// - a latency-critical loop where cudaMalloc / cudaFree would synchronise the device;
// - code that shares a device with a framework that owns every allocation.
// nc_probs_to_cdf_noalloc does the same work, but the status words live in the
// fixed array below.  The array is part of the library image, so every GPU
// that loads the library holds it until the process exits.
#include <cuda.h>

#include <mutex>

#include "internal.h"

namespace {

// Status words of at most NC_NOALLOC_MAX_ROWS rows; shared by every call.
static __device__ __align__(256) int32_t g_noalloc_status[NC_NOALLOC_MAX_ROWS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_status_ptr[kMaxDevices] = {};        // device address of the array, per device
unsigned long long g_ctx_id[kMaxDevices] = {};  // the context the address belongs to

// Unique id of the current context (0 when it cannot be read).  A device
// reset gives the device a new primary context with a new id, in which the
// library image, and so the array, may sit at another address.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qb != cudaDriverEntryPointSuccess)
      return 0;
    get_current = reinterpret_cast<GetCurrent>(a);
    get_id = reinterpret_cast<GetId>(b);
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the array on the current device.  Host code cannot use
// the symbol itself: on the host it names a stand-in, not device memory.
// Set-up, once per device (again after a reset of that device's context):
// the address is looked up with cudaGetSymbolAddress while the device is
// current and kept for later calls.
int status_words(int32_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NC_ECUDA;
  // before the runtime's first call on this device there is no current
  // context (id 0): the look-up below creates it, and the id is read again
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_status_ptr[dev] || id == 0 || id != g_ctx_id[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_status) != cudaSuccess || !p) return NC_ECUDA;
    g_status_ptr[dev] = static_cast<int32_t*>(p);
    g_ctx_id[dev] = id ? id : current_ctx_id();
  }
  *out = g_status_ptr[dev];
  return NC_OK;
}

}  // namespace

extern "C" int nc_probs_to_cdf_noalloc(const float* p, int n, int V, int log2_total, uint32_t floor_c,
                                       uint32_t* cdf, void* stream) {
  if (!p || !cdf || n < 1 || V < 2 || V > 65535 || log2_total < 1 || log2_total > 24 || floor_c < 1 ||
      (uint64_t)V * floor_c >= (1ull << log2_total))
    return NC_EINVAL;
  if (n > NC_NOALLOC_MAX_ROWS) return NC_EINVAL;   // more rows than the fixed status array holds
  int32_t* status = nullptr;
  int rc = status_words(&status);
  if (rc != NC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t hs[NC_NOALLOC_MAX_ROWS];
  // the words keep the previous call's values: clear the ones this call uses
  if (cudaMemsetAsync(status, 0, (size_t)n * sizeof(int32_t), s) != cudaSuccess ||
      nc::launch_probs_to_cdf(p, n, V, log2_total, floor_c, cdf, status, s) != cudaSuccess ||
      cudaMemcpyAsync(hs, status, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NC_ECUDA;
  for (int j = 0; j < n; ++j)
    if (hs[j]) return NC_ENUMERIC;
  return NC_OK;
}
