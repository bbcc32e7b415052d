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

static_assert(SW_BATCH_TILE_SHAPES == swgb::kTileShapes && SW_BATCH_SCHEDULES == swgb::kBatchSchedules,
              "configuration counts of the public header");

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
  int shape = 0;                      // tile shape (index into the shape table)
  int schedule = 0;                   // label layout (bit 0) and grid form (bit 1)
  // small members (whole sweeps in one CTA's shared memory): member indices,
  // the Ising ones then the Potts ones, run on a forked branch of the graph
  uint32_t* d_small = nullptr;
  size_t cap_small = 0;
  uint32_t n_small_ising = 0, n_small_potts = 0;
  std::vector<bool> is_small;         // per member
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
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

// A member's lattice view in the batch's tile shape (tile counts and the
// capacity of a tile's hooked list; the buffers hold the largest shape).
swgb::Lattice member_view(const sw_batch* b, const sw_handle* h) {
  swgb::Lattice lat = h->lat;
  swgb::tiles_for(b->dim, h->L, &lat.ntx, &lat.nty, &lat.ntz, b->shape);
  lat.hook_cap = swgb::merge_list_capacity(b->dim, b->shape);
  return lat;
}

size_t member_tiles(const sw_batch* b, const sw_handle* h) {
  const swgb::Lattice lat = member_view(b, h);
  return (size_t)lat.ntx * lat.nty * lat.ntz;
}

// Rebuild the tile map and the captured sweep after a change of membership
// or configuration.
int rebuild(sw_batch* b) {
  size_t ntiles = 0;
  std::vector<uint32_t> small_ising, small_potts;
  b->is_small.assign(b->members.size(), false);
  for (size_t m = 0; m < b->members.size(); ++m) {
    sw_handle* h = b->members[m];
    if (swgb::small_lattice(h->lat)) {
      b->is_small[m] = true;
      (h->model == SW_POTTS ? small_potts : small_ising).push_back((uint32_t)m);
    } else {
      ntiles += member_tiles(b, h);
    }
  }
  if (ntiles > 0x7fffffffu) return bfail(SW_ERR_BAD_ARG, "batch has too many tiles");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch sync");
  if (b->members.size() > b->cap_members) {
    swgb::dev_free(b->d_members, b->stream);
    cudaFreeHost(b->h_members);
    b->d_members = nullptr;
    b->h_members = nullptr;
    const size_t cap = std::max<size_t>(16, b->members.size() * 2);
    if ((e = swgb::dev_alloc((void**)&b->d_members, cap * sizeof(BatchMember), b->stream)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_members, cap * sizeof(BatchMember))) != cudaSuccess)
      return bfail(SW_ERR_OOM, std::string("batch descriptors: ") + cudaGetErrorString(e));
    b->cap_members = cap;
  }
  if (ntiles > b->cap_tiles) {
    swgb::dev_free(b->d_tiles, b->stream);
    b->d_tiles = nullptr;
    const size_t cap = std::max<size_t>(1024, ntiles * 2);
    if ((e = swgb::dev_alloc((void**)&b->d_tiles, 2 * cap * sizeof(uint32_t), b->stream)) != cudaSuccess)
      return bfail(SW_ERR_OOM, std::string("batch tile map: ") + cudaGetErrorString(e));
    b->cap_tiles = cap;
  }
  const size_t nsmall = small_ising.size() + small_potts.size();
  if (nsmall > b->cap_small) {
    swgb::dev_free(b->d_small, b->stream);
    b->d_small = nullptr;
    const size_t cap = std::max<size_t>(64, nsmall * 2);
    if ((e = swgb::dev_alloc((void**)&b->d_small, cap * sizeof(uint32_t), b->stream)) != cudaSuccess)
      return bfail(SW_ERR_OOM, std::string("batch small-member list: ") + cudaGetErrorString(e));
    b->cap_small = cap;
  }
  // the (re)allocations above are ordered on the batch stream; the copies
  // below run on the legacy stream
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bcuda(e, "batch sync");
  if (nsmall) {
    std::vector<uint32_t> all(small_ising);
    all.insert(all.end(), small_potts.begin(), small_potts.end());
    if ((e = cudaMemcpy(b->d_small, all.data(), nsmall * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bcuda(e, "batch small-member list");
    if (!b->side) {
      if ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return bcuda(e, "batch side stream");
    }
    if ((e = swgb::prepare_small_batch()) != cudaSuccess) return bcuda(e, "small-lattice kernels");
  }
  b->n_small_ising = (uint32_t)small_ising.size();
  b->n_small_potts = (uint32_t)small_potts.size();
  std::vector<uint32_t> lat(ntiles), idx(ntiles);
  size_t t = 0;
  for (int pass = 0; pass < 2; ++pass) {  // Ising members' tiles, then Potts
    for (size_t m = 0; m < b->members.size(); ++m) {
      const sw_handle* h = b->members[m];
      if (b->is_small[m] || (h->model == SW_POTTS) != (pass == 1)) continue;
      const uint32_t n = (uint32_t)member_tiles(b, h);
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
  if (ntiles || nsmall) {
    // capture one sweep: the small members on a forked branch; labels (+
    // measurement), merge, compression, apply of the tiled ones; the step
    cudaGraph_t g = nullptr;
    const BatchView v = view(b);
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaSuccess;
      if (nsmall) {
        le = cudaEventRecord(b->ev_fork, b->stream);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
        if (le == cudaSuccess)
          le = swgb::launch_small_batch(v, b->dim, b->d_small, b->n_small_ising, b->d_small + b->n_small_ising,
                                        b->n_small_potts, b->side);
        if (le == cudaSuccess) le = cudaEventRecord(b->ev_join, b->side);
      }
      if (le == cudaSuccess && ntiles) {
        le = swgb::launch_label_batch(v, b->dim, b->shape, b->schedule, b->ising_tiles, b->ntiles - b->ising_tiles,
                                      b->stream);
        if (le == cudaSuccess)
          le = swgb::launch_merge_batch(v, b->dim, b->shape, b->schedule, b->ntiles, b->stream);
        if (le == cudaSuccess)
          le = swgb::launch_flip_batch(v, b->dim, b->shape, b->schedule, b->ntiles, b->stream);
      }
      if (le == cudaSuccess && nsmall) le = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
      if (le == cudaSuccess) le = swgb::launch_advance(v, b->stream);
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
  b->shape = swgb::kSingleShape[dim - 2];
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) b->own_stream = true;
  if (e == cudaSuccess) e = swgb::dev_alloc((void**)&b->d_step, sizeof(uint32_t), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
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
  swgb::dev_free(b->d_members, b->stream);
  cudaFreeHost(b->h_members);
  swgb::dev_free(b->d_tiles, b->stream);
  swgb::dev_free(b->d_small, b->stream);
  swgb::dev_free(b->d_step, b->stream);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->side) cudaStreamDestroy(b->side);
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

int sw_batch_query(sw_batch* b) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  // the graph's side branch joins the batch stream, which therefore covers it
  const cudaError_t e = cudaStreamQuery(b->stream);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return bcuda(e, "batch stream query");
}

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

}  // extern "C"

namespace {

// Up to n sweeps of every member (graph replays): a member with a sweep
// target stops there.  With ms != nullptr the replays alone are timed with
// events on the batch stream (a host wait).
int batch_sweep(sw_batch* b, int n, float* ms) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  if (n < 0) return bfail(SW_ERR_BAD_ARG, "n < 0");
  if (n == 0 || b->members.empty()) return SW_OK;
  std::vector<uint32_t> count(b->members.size());
  uint32_t replays = 0;
  for (size_t m = 0; m < b->members.size(); ++m) {
    const sw_handle* h = b->members[m];
    uint64_t c = (uint64_t)n;
    if (h->target) c = h->target > h->sweep ? std::min<uint64_t>(c, h->target - h->sweep) : 0;
    if (h->sweep + c >= 0xffffffffull) return bfail(SW_ERR_BAD_ARG, "sweep counter exhausted");
    count[m] = (uint32_t)c;
    replays = std::max(replays, count[m]);
  }
  if (replays == 0) return SW_OK;
  if (b->dirty) {
    const int rc = rebuild(b);
    if (rc != SW_OK) return rc;
  }
  // every member's earlier work precedes the batch; a tiled member's pending
  // record (of its current state) is measured by the batch's first step
  cudaError_t e = cudaStreamSynchronize(b->stream);  // the staging copy below is reused
  for (size_t m = 0; m < b->members.size(); ++m) {
    sw_handle* h = b->members[m];
    const bool measure0 = !b->is_small[m] && count[m] > 0 && h->pending != 0 && h->pending == h->sweep;
    if (e == cudaSuccess && count[m] > 0 && !measure0) e = swgb::flush_pending(h);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev, 0);
    b->h_members[m].lat = member_view(b, h);
    b->h_members[m].meas = h->meas;
    b->h_members[m].sweep0 = (uint32_t)h->sweep;
    b->h_members[m].nsweeps = count[m];
    b->h_members[m].measure0 = measure0 ? 1u : 0u;  // pending is replaced once the replays are enqueued
  }
  if (e != cudaSuccess) return bcuda(e, "batch ordering");
  if ((e = cudaMemcpyAsync(b->d_members, b->h_members, b->members.size() * sizeof(BatchMember),
                           cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(b->d_step, 0, sizeof(uint32_t), b->stream)) != cudaSuccess)
    return bcuda(e, "batch descriptors");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (ms) {
    if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess ||
        (e = cudaEventRecord(t0, b->stream)) != cudaSuccess) {
      if (t0) cudaEventDestroy(t0);
      return bcuda(e, "batch timing");
    }
  }
  for (uint32_t s = 0; s < replays && e == cudaSuccess; ++s) e = cudaGraphLaunch(b->graph, b->stream);
  if (e == cudaSuccess && ms) e = cudaEventRecord(t1, b->stream);
  // later work on each member waits for the batch
  if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->stream);
  if (e == cudaSuccess) {
    for (size_t m = 0; m < b->members.size(); ++m) {
      sw_handle* h = b->members[m];
      if ((e = cudaStreamWaitEvent(h->stream, b->ev, 0)) != cudaSuccess) break;
      if (count[m] == 0) continue;
      h->sweep += count[m];
      // a tiled member's last record is written on demand; a small member
      // writes every record in its sweep
      if (!b->is_small[m]) h->pending = h->sweep;
    }
  }
  if (e == cudaSuccess && ms) e = cudaEventSynchronize(t1);
  if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, t0, t1);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  return e == cudaSuccess ? SW_OK : bcuda(e, "batch sweep");
}

}  // namespace

extern "C" {

int sw_batch_sweep(sw_batch* b, int n) { return batch_sweep(b, n, nullptr); }

int sw_batch_set_config(sw_batch* b, int shape, int schedule) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  if (shape < 0 || shape >= swgb::kTileShapes) return bfail(SW_ERR_BAD_ARG, "tile shape out of range");
  if (schedule < 0 || schedule >= swgb::kBatchSchedules) return bfail(SW_ERR_BAD_ARG, "schedule out of range");
  if (shape != b->shape || schedule != b->schedule) {
    cudaError_t e = cudaStreamSynchronize(b->stream);  // the replays in flight use the old tile map
    if (e != cudaSuccess) return bcuda(e, "batch sync");
    b->shape = shape;
    b->schedule = schedule;
    b->dirty = true;
  }
  return SW_OK;
}

int sw_batch_get_config(const sw_batch* b, int* shape, int* schedule, int* tile_y, int* tile_z) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  if (shape) *shape = b->shape;
  if (schedule) *schedule = b->schedule;
  if (tile_y) *tile_y = swgb::kShapeTY[b->dim - 2][b->shape];
  if (tile_z) *tile_z = swgb::kShapeTZ[b->dim - 2][b->shape];
  return SW_OK;
}

int sw_batch_autotune(sw_batch* b, int sweeps, float* ms_per_sweep) {
  if (!b) return bfail(SW_ERR_BAD_ARG, "NULL batch");
  if (sweeps < 1) return bfail(SW_ERR_BAD_ARG, "sweeps < 1");
  constexpr int kConfigs = swgb::kTileShapes * swgb::kBatchSchedules;
  if (ms_per_sweep)
    for (int c = 0; c < kConfigs; ++c) ms_per_sweep[c] = -1.0f;
  if (b->members.empty()) return SW_OK;
  bool ising = false, potts = false;
  for (const sw_handle* h : b->members) (h->model == SW_POTTS ? potts : ising) = true;
  // one label launch differs from two only when both kinds are present
  // (schedule bit 0); both grid forms (bit 1) and merge forms (bit 2) are
  // always tried
  const bool both = ising && potts;
  const uint64_t total = (uint64_t)swgb::kTileShapes * (both ? 8 : 4) * ((uint64_t)sweeps + 1);
  for (const sw_handle* h : b->members) {
    if (h->sweep + total >= 0xffffffffull) return bfail(SW_ERR_BAD_ARG, "sweep counter exhausted");
    // every configuration must time the same members
    if (h->target && h->target < h->sweep + total)
      return bfail(SW_ERR_BAD_ARG, "a member's sweep target falls within the tuning sweeps");
  }
  int best_shape = b->shape, best_schedule = b->schedule;
  float best = -1.0f;
  for (int sh = 0; sh < swgb::kTileShapes; ++sh) {
    for (int sc = 0; sc < swgb::kBatchSchedules; ++sc) {
      if ((sc & 1) && !both) continue;
      int rc = sw_batch_set_config(b, sh, sc);
      if (rc == SW_OK) rc = batch_sweep(b, 1, nullptr);  // graph capture and upload, untimed
      float ms = 0.0f;
      if (rc == SW_OK) rc = batch_sweep(b, sweeps, &ms);
      if (rc != SW_OK) return rc;
      ms /= (float)sweeps;
      if (ms_per_sweep) ms_per_sweep[sh * swgb::kBatchSchedules + sc] = ms;
      if (best < 0.0f || ms < best) {
        best = ms;
        best_shape = sh;
        best_schedule = sc;
      }
    }
  }
  return sw_batch_set_config(b, best_shape, best_schedule);
}

size_t sw_device_bytes(int model, int dim, int L, int q) {
  if ((dim != 2 && dim != 3) || L < 4 || model < SW_ISING || model > SW_CLOCK) return 0;
  double n = 1.0;
  for (int d = 0; d < dim; ++d) n *= L;
  if (n > 4294967295.0) return 0;
  const size_t N = (size_t)n;
  const size_t words = (size_t)dim * (N / (size_t)L) * (size_t)((L + 31) / 32);
  size_t ntiles = 0, hook_words = 0;
  swgb::tile_buffers(model, dim, L, &ntiles, &hook_words);
  const size_t spins = N * (model == SW_XY ? 4 : model == SW_CLOCK ? 2 : 1);
  const size_t clock =
      (model == SW_CLOCK) ? (size_t)4 * q * q * 4 + (size_t)2 * q * 8 + 3 * swgb::kSlots * 8 + (size_t)2 * q * 4 : 0;
  return spins + 4 * words + 4 * N + hook_words * 4 + ntiles * 4 + swgb::handle_block_bytes() + clock;
}

}  // extern "C"
