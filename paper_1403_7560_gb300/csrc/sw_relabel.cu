// Labeling-method comparison on the same bond planes: this library's tile
// union-find + global merge, against the label-equivalence scheme the paper
// runs (Sec. 2: Hawick et al. with Kalentev et al.'s refinement), written
// here from that description.
//
// Label equivalence (one label array, no separate reference array):
//   init      label[i] = i
//   scanning  each site takes the smallest label among itself and the sites
//             it is bonded to, and lowers the entry of its current root to
//             it (atomicMin)
//   analysis  every site jumps to the root of its label chain
// The two kernels repeat until a scan changes nothing; the host reads the
// change flag after every iteration, as the paper's loop does.  Labels only
// decrease and each cluster's smallest index never changes, so the result
// is the canonical label (smallest site index of the cluster).
#include <string>

#include "../../include/sw.h"
#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

constexpr int kT = 256;

__global__ void __launch_bounds__(kT) k_le_init(uint32_t N, int32_t* label) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    label[i] = (int32_t)i;
}

__device__ __forceinline__ bool plane_bit(const Lattice& lat, int d, uint32_t row, int x) {
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  return (__ldg(&lat.planes[d * plane + row * (uint32_t)lat.W + (uint32_t)(x >> 5)]) >> (x & 31)) & 1u;
}

template <int D>
__global__ void __launch_bounds__(kT) k_le_scan(Lattice lat, int32_t* label, int* changed) {
  const int L = lat.L;
  // L a power of two: a site's coordinates by shifts and masks
  const bool pow2 = (L & (L - 1)) == 0;
  const int lsh = __ffs(L) - 1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    int x, y, z;
    uint32_t row;
    if (pow2) {
      x = (int)(i & (uint32_t)(L - 1));
      row = i >> lsh;
      y = (int)(row & (uint32_t)(L - 1));
      z = (D == 3) ? (int)(row >> lsh) : 0;
    } else {
      x = (int)(i % (uint32_t)L);
      row = i / (uint32_t)L;
      y = (int)(row % (uint32_t)L);
      z = (D == 3) ? (int)(row / (uint32_t)L) : 0;
    }
    const int32_t l = __ldcg(&label[i]);
    int32_t m = l;
    // +d neighbours (bond owned by i) and -d neighbours (bond owned by them)
    const int xp = (x + 1 == L) ? 0 : x + 1, xm = (x == 0) ? L - 1 : x - 1;
    const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
    const uint32_t base = i - (uint32_t)x;
    if (plane_bit(lat, 0, row, x)) m = min(m, __ldcg(&label[base + xp]));
    if (plane_bit(lat, 0, row, xm)) m = min(m, __ldcg(&label[base + xm]));
    const uint32_t rowyp = (uint32_t)yp + (uint32_t)L * (uint32_t)z;
    const uint32_t rowym = (uint32_t)ym + (uint32_t)L * (uint32_t)z;
    if (plane_bit(lat, 1, row, x)) m = min(m, __ldcg(&label[rowyp * L + x]));
    if (plane_bit(lat, 1, rowym, x)) m = min(m, __ldcg(&label[rowym * L + x]));
    if (D == 3) {
      const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
      const uint32_t rowzp = (uint32_t)y + (uint32_t)L * (uint32_t)zp;
      const uint32_t rowzm = (uint32_t)y + (uint32_t)L * (uint32_t)zm;
      if (plane_bit(lat, 2, row, x)) m = min(m, __ldcg(&label[rowzp * L + x]));
      if (plane_bit(lat, 2, rowzm, x)) m = min(m, __ldcg(&label[rowzm * L + x]));
    }
    if (m < l) {
      atomicMin(&label[l], m);
      *changed = 1;
    }
  }
}

__global__ void __launch_bounds__(kT) k_le_analysis(uint32_t N, int32_t* label, int* err, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int32_t r = __ldcg(&label[i]);
    uint32_t it = 0;
    for (; it < cap; ++it) {
      const int32_t p = __ldcg(&label[r]);
      if (p == r) break;
      r = p;
    }
    if (it == cap) atomicExch(err, kErrTimeout);
    label[i] = r;
  }
}

unsigned grid(uint32_t n) {
  unsigned g = (n + kT - 1) / kT;
  return g > 152u * 16u ? 152u * 16u : (g ? g : 1u);
}

}  // namespace
}  // namespace swgb

extern "C" int sw_relabel(sw_handle* h, int method, int32_t* host_labels, float* ms, int* iterations) {
  if (!h) {
    swgb::set_last_error("NULL handle");
    return SW_ERR_BAD_ARG;
  }
  if (method != SW_LABEL_TILE_UF && method != SW_LABEL_EQUIVALENCE) {
    swgb::set_last_error("method must be SW_LABEL_TILE_UF or SW_LABEL_EQUIVALENCE");
    return SW_ERR_BAD_ARG;
  }
  const swgb::Lattice& lat = h->lat;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  if (!h->d_labels) e = swgb::dev_alloc((void**)&h->d_labels, (size_t)lat.N * 4, st);
  int* d_flag = nullptr;
  int* h_flag = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&h_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int iters = 0;
  bool timed_out = false;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    if (method == SW_LABEL_TILE_UF) {
      // the sweep's own labeling, from the planes: tile union-find, merge,
      // canonical labels
      e = swgb::launch_label(lat, 0u, true, st);
      if (e == cudaSuccess) e = swgb::launch_merge(lat, st);
      if (e == cudaSuccess) e = swgb::launch_labels_out(lat, h->d_labels, st);
      iters = 1;
    } else {
      swgb::k_le_init<<<swgb::grid(lat.N), swgb::kT, 0, st>>>(lat.N, h->d_labels);
      // at most N + 1 scans change a label (each lowers one); the handle's
      // loop cap can lower the limit further
      uint32_t cap = lat.N < 1000000u ? lat.N + 2u : 1000000u;
      if (lat.cap < cap) cap = lat.cap;
      bool converged = false;
      for (iters = 0; (uint32_t)iters < cap && e == cudaSuccess;) {
        e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
        if (lat.dim == 2) swgb::k_le_scan<2><<<swgb::grid(lat.N), swgb::kT, 0, st>>>(lat, h->d_labels, d_flag);
        else swgb::k_le_scan<3><<<swgb::grid(lat.N), swgb::kT, 0, st>>>(lat, h->d_labels, d_flag);
        swgb::k_le_analysis<<<swgb::grid(lat.N), swgb::kT, 0, st>>>(lat.N, h->d_labels, lat.err, lat.cap);
        ++iters;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && *h_flag == 0) {
          converged = true;
          break;
        }
      }
      if (e == cudaSuccess && !converged) timed_out = true;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess && host_labels)
    e = cudaMemcpy(host_labels, h->d_labels, (size_t)lat.N * 4, cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_flag);
  cudaFreeHost(h_flag);
  if (e != cudaSuccess) {
    swgb::set_last_error(std::string("relabel: ") + cudaGetErrorString(e));
    return SW_ERR_CUDA;
  }
  if (ms) *ms = t;
  if (iterations) *iterations = iters;
  const int rc = sw_sync(h);
  if (rc == SW_OK && timed_out) {
    swgb::set_last_error("label equivalence: the iteration cap was reached before convergence");
    return SW_ERR_TIMEOUT;
  }
  return rc;
}
