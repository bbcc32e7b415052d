// Ragged batches: many Ising/Potts lattices of one dimension advanced
// together, one launch per phase over every tile of every member, the whole
// sweep captured once in a CUDA graph and replayed.
//
// A batch holds existing handles; each keeps its own buffers, sweep counter,
// seed and accumulators, and the Philox keying (seed, sweep, site, purpose)
// contains no batch position, so a lattice's trajectory is the same alone
// and in any batch.  Measurement follows the single-lattice scheme: the
// labeling kernel of sweep k measures the state after sweep k-1 and the
// compression kernel's first tile of each member writes that record; the
// last sweep of a call stays pending on the handle.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/sw.h"
#include "sw_internal.h"

using swgb::BatchMember;
using swgb::BatchView;

struct sw_batch {
  int dim = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<sw_handle*> members;
  bool dirty = true;                  // membership changed since the graph was built
  BatchMember* d_members = nullptr;   // device descriptors
  BatchMember* h_members = nullptr;   // pinned staging copy
  size_t cap_members = 0;
  uint32_t* d_tiles = nullptr;        // [2][cap_tiles]: member, tile
  size_t cap_tiles = 0;
  uint32_t* d_step = nullptr;
  uint32_t ntiles = 0;
  uint32_t ising_tiles = 0;           // the tile map lists the Ising members' tiles first
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev = nullptr;
};

namespace {

int bfail(int code, const std::string& msg) {
  swgb::set_last_error(msg);
  return code;
}

int bcuda(cudaError_t e, const char* what) {
  return bfail(SW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void drop_graph(sw_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

BatchView view(const sw_batch* b) {
  BatchView v;
  v.members = b->d_members;
  v.tile_lattice = b->d_tiles;
  v.tile_index = b->d_tiles + b->cap_tiles;
  v.step = b->d_step;
  return v;
}

// Rebuild the tile map and the captured sweep after a membership change.
int rebuild(sw_batch* b) {
  size_t ntiles = 0;
  for (sw_handle* h : b->members) ntiles += (size_t)h->lat.ntx * h->lat.nty * h->lat.ntz;
  if (ntiles > 0x7fffffffu) return bfail(SW_ERR_BAD_ARG, "batch has too many tiles");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch sync");
  if (b->members.size() > b->cap_members) {
    cudaFree(b->d_members);
    cudaFreeHost(b->h_members);
    b->d_members = nullptr;
    b->h_members = nullptr;
    const size_t cap = std::max<size_t>(16, b->members.size() * 2);
    if ((e = cudaMalloc(&b->d_members, cap * sizeof(BatchMember))) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_members, cap * sizeof(BatchMember))) != cudaSuccess)
      return bfail(SW_ERR_OOM, std::string("batch descriptors: ") + cudaGetErrorString(e));
    b->cap_members = cap;
  }
  if (ntiles > b->cap_tiles) {
    cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    const size_t cap = std::max<size_t>(1024, ntiles * 2);
    if ((e = cudaMalloc(&b->d_tiles, 2 * cap * sizeof(uint32_t))) != cudaSuccess)
      return bfail(SW_ERR_OOM, std::string("batch tile map: ") + cudaGetErrorString(e));
    b->cap_tiles = cap;
  }
  std::vector<uint32_t> lat(ntiles), idx(ntiles);
  size_t t = 0;
  for (int pass = 0; pass < 2; ++pass) {  // Ising members' tiles, then Potts
    for (size_t m = 0; m < b->members.size(); ++m) {
      const sw_handle* h = b->members[m];
      if ((h->model == SW_POTTS) != (pass == 1)) continue;
      const uint32_t n = (uint32_t)((size_t)h->lat.ntx * h->lat.nty * h->lat.ntz);
      for (uint32_t k = 0; k < n; ++k, ++t) {
        lat[t] = (uint32_t)m;
        idx[t] = k;
      }
    }
    if (pass == 0) b->ising_tiles = (uint32_t)t;
  }
  if (ntiles) {
    if ((e = cudaMemcpy(b->d_tiles, lat.data(), ntiles * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_tiles + b->cap_tiles, idx.data(), ntiles * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bcuda(e, "batch tile map");
  }
  b->ntiles = (uint32_t)ntiles;
  drop_graph(b);
  if (ntiles) {
    // capture one sweep: labels (+ measurement), merge, compression, apply, step
    cudaGraph_t g = nullptr;
    const BatchView v = view(b);
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = swgb::launch_label_batch(v, b->dim, b->ising_tiles, b->ntiles - b->ising_tiles, b->stream);
      if (le == cudaSuccess) le = swgb::launch_merge_batch(v, b->dim, b->ntiles, b->stream);
      if (le == cudaSuccess) le = swgb::launch_flip_batch(v, b->dim, b->ntiles, b->stream);
      e = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      drop_graph(b);
      return bcuda(e, "batch graph capture");
    }
  }
  b->dirty = false;
  return SW_OK;
}

}  // namespace

extern "C" {

sw_batch* sw_batch_create(int dim) {
  swgb::set_last_error("");
  if (dim != 2 && dim != 3) {
    bfail(SW_ERR_BAD_ARG, "dim must be 2 or 3");
    return nullptr;
  }
  sw_batch* b = new (std::nothrow) sw_batch();
  if (!b) {
    bfail(SW_ERR_OOM, "host allocation");
    return nullptr;
  }
  b->dim = dim;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) b->own_stream = true;
  if (e == cudaSuccess) e = cudaMalloc(&b->d_step, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    bcuda(e, "batch create");
    sw_batch_destroy(b);
    return nullptr;
  }
  return b;
}

void sw_batch_destroy(sw_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (sw_handle* h : b->members) h->batch = nullptr;
  drop_graph(b);
  cudaFree(b->d_members);
  cudaFreeHost(b->h_members);
  cudaFree(b->d_tiles);
  cudaFree(b->d_step);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int sw_batch_add(sw_batch* b, sw_handle* h) {
  if (!b || !h) return bfail(SW_ERR_BAD_ARG, "NULL argument");
  if (h->model != SW_ISING && h->model != SW_POTTS)
    return bfail(SW_ERR_BAD_ARG, "batches hold Ising and Potts lattices only");
  if (h->dim != b->dim) return bfail(SW_ERR_BAD_ARG, "lattice dimension differs from the batch's");
  if (h->batch) return bfail(SW_ERR_BAD_ARG, "lattice already belongs to a batch");
  // the batch stream does not wait for the lattice's own stream or uploads
  cudaError_t e = swgb::wait_io(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bcuda(e, "lattice sync");
  b->members.push_back(h);
  h->batch = b;
  b->dirty = true;
  return SW_OK;
}

int sw_batch_remove(sw_batch* b, sw_handle* h) {
  if (!b || !h) return bfail(SW_ERR_BAD_ARG, "NULL argument");
  auto it = std::find(b->members.begin(), b->members.end(), h);
  if (it == b->members.end()) return bfail(SW_ERR_BAD_ARG, "lattice is not in this batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch sync");
  b->members.erase(it);
  h->batch = nullptr;
  b->dirty = true;
  return SW_OK;
}

size_t sw_batch_size(sw_batch* b) { return b ? b->members.size() : 0; }

int sw_batch_set_stream(sw_batch* b, void* stream) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  if (!stream) return bfail(SW_ERR_BAD_ARG, "a batch needs a non-default stream (graph capture)");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch sync");
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->own_stream = false;
  b->stream = static_cast<cudaStream_t>(stream);
  b->dirty = true;
  return SW_OK;
}

int sw_batch_sweep(sw_batch* b, int n) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  if (n < 0) return bfail(SW_ERR_BAD_ARG, "n < 0");
  if (n == 0 || b->members.empty()) return SW_OK;
  for (sw_handle* h : b->members)
    if (h->sweep + (uint64_t)n >= 0xffffffffull) return bfail(SW_ERR_BAD_ARG, "sweep counter exhausted");
  if (b->dirty) {
    const int rc = rebuild(b);
    if (rc != SW_OK) return rc;
  }
  // every member's earlier work (and its pending record) precedes the batch
  cudaError_t e = cudaStreamSynchronize(b->stream);  // the staging copy below is reused
  for (sw_handle* h : b->members) {
    if (e == cudaSuccess) e = swgb::flush_pending(h);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev, 0);
  }
  if (e != cudaSuccess) return bcuda(e, "batch ordering");
  for (size_t m = 0; m < b->members.size(); ++m) {
    const sw_handle* h = b->members[m];
    b->h_members[m].lat = h->lat;
    b->h_members[m].meas = h->meas;
    b->h_members[m].sweep0 = (uint32_t)h->sweep;
  }
  if ((e = cudaMemcpyAsync(b->d_members, b->h_members, b->members.size() * sizeof(BatchMember),
                           cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(b->d_step, 0, sizeof(uint32_t), b->stream)) != cudaSuccess)
    return bcuda(e, "batch descriptors");
  for (int s = 0; s < n; ++s)
    if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return bcuda(e, "batch sweep");
  // later work on each member waits for the batch
  if ((e = cudaEventRecord(b->ev, b->stream)) != cudaSuccess) return bcuda(e, "batch event");
  for (sw_handle* h : b->members) {
    if ((e = cudaStreamWaitEvent(h->stream, b->ev, 0)) != cudaSuccess) return bcuda(e, "batch event");
    h->sweep += (uint64_t)n;
    h->pending = h->sweep;  // the last sweep's record, written on demand
  }
  return SW_OK;
}

size_t sw_device_bytes(int model, int dim, int L, int q) {
  if ((dim != 2 && dim != 3) || L < 4 || model < SW_ISING || model > SW_CLOCK) return 0;
  double n = 1.0;
  for (int d = 0; d < dim; ++d) n *= L;
  if (n > 4294967295.0) return 0;
  int ntx, nty, ntz;
  swgb::tiles_for(dim, L, &ntx, &nty, &ntz);
  const size_t N = (size_t)n;
  const size_t words = (size_t)dim * (N / (size_t)L) * (size_t)((L + 31) / 32);
  const size_t ntiles = (size_t)ntx * nty * ntz;
  const size_t spins = N * (model == SW_XY ? 4 : model == SW_CLOCK ? 2 : 1);
  const size_t clock = (model == SW_CLOCK) ? (size_t)4 * q * q * 4 + (size_t)2 * q * 8 + 3 * swgb::kSlots * 8 : 0;
  return spins + 4 * words + 4 * N + ntiles * (size_t)swgb::merge_list_capacity(dim) * 4 + ntiles * 4 +
         swgb::handle_block_bytes() + clock;
}

}  // extern "C"
