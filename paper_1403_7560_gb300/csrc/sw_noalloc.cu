// Cluster labeling of a caller's bond mask without any device allocation.
//
// Some callers cannot call cudaMalloc: a serving loop or a plugin that runs
// inside a host framework owning every device byte through its own pool, or
// code on a latency-critical path where cudaMalloc/cudaFree would
// synchronise the device and stall every other stream.  This entry point
// gives them the labeling step with its working memory (the union-find
// forest and an error flag) in a fixed array of this library's module,
// instead of a buffer allocated per handle.
#include <cstdio>
#include <string>

#include "../../include/sw.h"
#include "sw_internal.h"

namespace {

// Scratch shared by every call on a device: the forest (one word per site)
// plus 64 words whose first holds the device error flag.  Loaded with the
// library and held by every GPU that loads it until the process exits.
constexpr uint32_t kNoallocWords = SW_NOALLOC_MAX_SITES + 64u;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocWords];

int noalloc_fail(int code, const std::string& msg) {
  swgb::set_last_error(msg);
  return code;
}

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in; the address is looked up on
// every call, with the caller's device current, so that it stays valid
// after a cudaDeviceReset (which reloads the module at a new address).
int scratch_for_current_device(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return noalloc_fail(SW_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = static_cast<uint32_t*>(p);
  return SW_OK;
}

}  // namespace

extern "C" {

int sw_label_from_bonds_noalloc(int dim, int L, const uint32_t* dev_mask, int32_t* dev_labels,
                                void* stream) {
  swgb::set_last_error("");
  if (dim != 2 && dim != 3) return noalloc_fail(SW_ERR_BAD_ARG, "dim must be 2 or 3");
  if (L < 4) return noalloc_fail(SW_ERR_BAD_ARG, "L must be >= 4");
  if (!dev_mask || !dev_labels) return noalloc_fail(SW_ERR_BAD_ARG, "NULL buffer");
  double n = 1.0;
  for (int d = 0; d < dim; ++d) n *= L;
  if (n > (double)SW_NOALLOC_MAX_SITES)
    return noalloc_fail(SW_ERR_BAD_ARG, "lattice too large for the no-allocation scratch: L^dim must be <= " +
                                            std::to_string(SW_NOALLOC_MAX_SITES) + " sites");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the call reads its error flag back and synchronises the stream, which a
  // stream capture does not allow: refuse before any GPU work
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cs);
  if (ce != cudaSuccess)
    return noalloc_fail(SW_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
  if (cs != cudaStreamCaptureStatusNone)
    return noalloc_fail(SW_ERR_BAD_ARG, "label_from_bonds_noalloc cannot run inside a stream capture");
  uint32_t* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != SW_OK) return rc;

  swgb::Lattice lat{};
  lat.N = (uint32_t)n;
  lat.L = L;
  lat.dim = dim;
  lat.W = (L + 31) / 32;
  lat.R = lat.N / (uint32_t)L;
  swgb::tiles_for(dim, L, &lat.ntx, &lat.nty, &lat.ntz);
  lat.q = 2;
  lat.sbits = 0;
  lat.planes = const_cast<uint32_t*>(dev_mask);  // only read on the mask path
  lat.forest = scratch;
  lat.err = reinterpret_cast<int*>(scratch + SW_NOALLOC_MAX_SITES);
  lat.spins = nullptr;
  lat.model = swgb::kIsing;
  lat.hooked = nullptr;   // labeling only: the merge keeps no hooked lists
  lat.nhooked = nullptr;
  lat.cap = swgb::kLoopCap;

  int flag = 0;
  cudaError_t e = cudaMemsetAsync(lat.err, 0, sizeof(int), st);  // the flag must start at zero
  if (e == cudaSuccess) e = swgb::launch_label(lat, 0u, true, st);
  if (e == cudaSuccess) e = swgb::launch_merge(lat, st);
  if (e == cudaSuccess) e = swgb::launch_labels_out(lat, dev_labels, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, lat.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(SW_ERR_CUDA, std::string("label_from_bonds_noalloc: ") + cudaGetErrorString(e));
  if (flag != 0) return noalloc_fail(flag, "a device loop hit its iteration cap");
  return SW_OK;
}

}  // extern "C"
