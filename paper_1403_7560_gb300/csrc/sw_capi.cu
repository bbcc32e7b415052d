// C ABI of the SW engine (include/sw.h): handle life cycle, argument
// validation, the sweep schedule on the handle's stream, and the debug /
// integration getters.  All SW arithmetic runs in sw_kernels.cu; the host
// computes only the per-run constants (bond threshold, 2/T) in sw_create.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/sw.h"
#include "sw_internal.h"

using swgb::Lattice;
using swgb::Measure;

namespace {
thread_local std::string g_last_error;
}  // namespace

void swgb::set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {
constexpr int kMaxPoolDevices = 64;
// freed memory the pool keeps for reuse before returning any to the driver
constexpr uint64_t kPoolKeepBytes = 16ull << 30;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaError_t device_pool(cudaMemPool_t* out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
    uint64_t keep = kPoolKeepBytes;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}
}  // namespace

int swgb::sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 1;
    n = v;
  }
  return n;
}

cudaError_t swgb::dev_alloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  const cudaError_t e = device_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void swgb::dev_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

namespace {

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kSeriesCap = 4096;

}  // namespace


namespace {

// Offsets of the small per-handle buffers inside one allocation: error
// flag, accumulators, cluster counts [2][kSlots], slot sums [kSlots][2],
// slot histograms [kSlots][256], XY partials, series ring.
struct BlockLayout {
  size_t err, done, acc, ncl, sums, hist, pd, series, total;
};

BlockLayout block_layout() {
  BlockLayout b;
  b.err = 0;
  b.done = 8;
  b.acc = 64;
  b.ncl = 128;
  b.sums = b.ncl + 2 * 8 * (size_t)swgb::kSlots;
  b.hist = b.sums + 16 * (size_t)swgb::kSlots;
  b.pd = b.hist + 8 * 256 * (size_t)swgb::kSlots;
  b.series = b.pd + 3 * 8 * (size_t)swgb::kMeasureBlocks;
  b.total = b.series + sizeof(swgb::Record) * (size_t)kSeriesCap;
  return b;
}

// Bond probability (Sec. 2, step (1), sign restored): Ising
// p = 1 - exp(-2/T); Potts (H = -sum(delta - 1)) p = 1 - exp(-1/T).  The
// kernel tests draw < t with t = floor(p 2^32), p = -expm1(-a) in double.
uint32_t bond_threshold(int model, double T) {
  const double a = (model == SW_ISING) ? 2.0 / T : 1.0 / T;
  double t = std::floor(-std::expm1(-a) * 4294967296.0);
  if (t > 4294967295.0) t = 4294967295.0;
  if (t < 0.0) t = 0.0;
  return (uint32_t)t;
}

// Clock model tables, per the definition in include/sw.h: fixed-point
// round(2^30 cos/sin((2 pi p)/q)), and thresholds
// floor(-expm1(-(2/T) x_a x_b) 2^32) with x_k = sin((pi k)/q), zero where
// x_a x_b <= 0.
constexpr double kPi = 3.141592653589793238463;

void clock_tables(int q, double T, std::vector<uint32_t>& tab, std::vector<long long>& fix,
                  std::vector<float>& proj) {
  const int q2 = 2 * q;
  std::vector<double> x(q2);
  for (int k = 0; k < q2; ++k) x[k] = std::sin((kPi * (double)k) / (double)q);
  // the projections in float: the bond kernel's estimate of a threshold
  proj.assign(q2, 0.0f);
  for (int k = 0; k < q2; ++k) proj[k] = (float)x[k];
  const double twoK = 2.0 / T;
  tab.assign((size_t)q2 * q2, 0u);
  for (int a = 0; a < q2; ++a)
    for (int b = 0; b < q2; ++b) {
      const double prod = x[a] * x[b];
      if (prod > 0.0) {
        double f = std::floor(-std::expm1(-(twoK * prod)) * 4294967296.0);
        if (f > 4294967295.0) f = 4294967295.0;
        tab[(size_t)a * q2 + b] = (uint32_t)f;
      }
    }
  fix.assign(q2, 0);
  for (int p = 0; p < q; ++p) {
    const double ang = (2.0 * kPi * (double)p) / (double)q;
    fix[p] = std::llround(std::ldexp(std::cos(ang), 30));
    fix[q + p] = std::llround(std::ldexp(std::sin(ang), 30));
  }
}

int draw_bits(int model, int q) {
  if (model != SW_POTTS) return 1;
  int b = 0;
  while ((1 << b) < q) ++b;
  return b;
}

void release(sw_handle* h) {
  if (!h) return;
  swgb::release_io(h);
  // every stream that used the buffers has been synchronised (sw_destroy,
  // release_io): the frees are ordered on the handle's stream and do not
  // wait for the rest of the device
  cudaStream_t st = h->stream;
  swgb::dev_free(h->lat.spins, st);
  swgb::dev_free(h->lat.planes, st);
  swgb::dev_free(h->lat.forest, st);
  swgb::dev_free(h->lat.hooked, st);
  swgb::dev_free(h->lat.nhooked, st);
  swgb::dev_free(h->d_labels, st);
  swgb::dev_free(h->d_block, st);
  swgb::dev_free(h->d_clock, st);
  if (h->own_stream && st) cudaStreamDestroy(st);
  delete h;
}

int check_device_error(sw_handle* h) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, h->lat.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  if (flag != 0) {
    cudaMemsetAsync(h->lat.err, 0, sizeof(int), h->stream);
    return fail(flag, "a device loop hit its iteration cap");
  }
  return SW_OK;
}

// Step (1) and the tile half of step (2): Ising/Potts bonds are drawn inside
// the labeling kernel, which also measures the incoming state when the
// previous sweep's record is pending; XY and clock bonds come from their own
// kernels, which measure the pending state the same way.  Sets *finalize to
// the pending sweep whose record the flip kernel of this sweep must write
// (0 if none).
cudaError_t launch_bonds_labels(sw_handle* h, uint32_t k, uint32_t* finalize) {
  *finalize = 0u;
  if (h->model == SW_XY || h->model == SW_CLOCK) {
    cudaError_t e;
    if (h->model == SW_XY) {
      const swgb::Measure* m = nullptr;
      if (h->pending) {
        *finalize = (uint32_t)h->pending;
        h->pending = 0;
        m = &h->meas;
      }
      int blocks = 0;
      e = swgb::launch_bonds_xy(h->lat, k, m, &blocks, h->stream);
      if (m) h->meas.xy_blocks = blocks;
    } else {
      const swgb::Measure* m = nullptr;
      if (h->pending) {
        *finalize = (uint32_t)h->pending;
        h->pending = 0;
        m = &h->meas;
      }
      e = swgb::launch_bonds_clock(h->lat, k, m, h->stream);
    }
    if (e != cudaSuccess) return e;
    return swgb::launch_label(h->lat, k, true, h->stream);
  }
  if (h->pending) {
    *finalize = (uint32_t)h->pending;
    h->pending = 0;
    return swgb::launch_label_measured(h->lat, k, h->meas, h->stream);
  }
  return swgb::launch_label(h->lat, k, false, h->stream);
}

}  // namespace

size_t swgb::handle_block_bytes() { return block_layout().total; }

// Write the record of a pending measured sweep with the stand-alone kernel.
cudaError_t swgb::flush_pending(sw_handle* h) {
  if (!h->pending) return cudaSuccess;
  const uint32_t k = (uint32_t)h->pending;
  h->pending = 0;
  return swgb::launch_measure(h->lat, h->model, k, h->meas, h->stream);
}

namespace {
using swgb::flush_pending;

// One sweep; the measurement stays pending (it is taken from the next
// sweep's bond kernel, or by flush_pending).
cudaError_t one_sweep(sw_handle* h, uint32_t k, bool measure, cudaEvent_t* ev) {
  cudaError_t e = cudaSuccess;
  uint32_t finalize = 0u;
  if (ev) e = cudaEventRecord(ev[0], h->stream);
  if (e == cudaSuccess) e = launch_bonds_labels(h, k, &finalize);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], h->stream);
  if (e == cudaSuccess) e = swgb::launch_merge(h->lat, h->stream);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], h->stream);
  // the flip writes the spins: a download of them goes first
  if (e == cudaSuccess) e = swgb::guard_state_write(h, h->lat.spins, h->stream);
  if (e == cudaSuccess) e = swgb::launch_flip(h->lat, h->model, k, h->meas, measure, finalize, h->stream);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], h->stream);
  if (e == cudaSuccess && measure) {
    h->pending = k;
  }
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4], h->stream);
  return e;
}

int run_sweeps(sw_handle* h, int n, bool measure) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  if (n < 0) return fail(SW_ERR_BAD_ARG, "n < 0");
  if (n > 0 && swgb::small_lattice(h->lat)) {
    // the whole lattice in one CTA's shared memory, many sweeps per launch
    if (h->sweep + (uint64_t)n >= 0xffffffffull) return fail(SW_ERR_BAD_ARG, "sweep counter exhausted");
    cudaError_t e = flush_pending(h);
    if (e == cudaSuccess) e = swgb::guard_state_write(h, h->lat.spins, h->stream);
    for (int done = 0; e == cudaSuccess && done < n;) {
      const int chunk = n - done < 256 ? n - done : 256;
      e = swgb::launch_sweeps_small(h->lat, h->meas, (uint32_t)h->sweep, chunk, measure, h->stream);
      if (e == cudaSuccess) {
        h->sweep += (uint64_t)chunk;
        done += chunk;
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    return SW_OK;
  }
  for (int s = 0; s < n; ++s) {
    if (h->sweep >= 0xffffffffull) return fail(SW_ERR_BAD_ARG, "sweep counter exhausted");
    const uint32_t k = (uint32_t)(++h->sweep);
    const cudaError_t e = one_sweep(h, k, measure, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
  }
  return SW_OK;
}

}  // namespace

extern "C" {

const char* sw_last_error(void) { return g_last_error.c_str(); }

size_t sw_series_capacity(void) { return kSeriesCap; }

sw_handle* sw_create(int model, int dim, int L, int q, double T, uint64_t seed) {
  g_last_error.clear();
  if (model < SW_ISING || model > SW_CLOCK) { fail(SW_ERR_BAD_ARG, "model must be 0 (Ising), 1 (Potts), 2 (XY) or 3 (clock)"); return nullptr; }
  if (dim != 2 && dim != 3) { fail(SW_ERR_BAD_ARG, "dim must be 2 or 3"); return nullptr; }
  if (L < 4) { fail(SW_ERR_BAD_ARG, "L must be >= 4"); return nullptr; }
  if (!(T > 0.0) || !std::isfinite(T)) { fail(SW_ERR_BAD_ARG, "T must be finite and > 0"); return nullptr; }
  if (model == SW_POTTS && (q < 2 || q > 256)) { fail(SW_ERR_BAD_ARG, "Potts q must be in 2..256"); return nullptr; }
  if (model == SW_CLOCK && (q < 2 || q > swgb::kMaxClockQ)) { fail(SW_ERR_BAD_ARG, "clock q must be in 2..1024"); return nullptr; }
  if (model != SW_POTTS && model != SW_CLOCK) q = 2;
  const int sb = draw_bits(model, q);
  const double Nd = std::pow((double)L, dim);
  if (Nd * std::ldexp(1.0, sb + 1) > 4294967296.0) {
    fail(SW_ERR_BAD_ARG, "lattice too large: N * 2^(drawbits+1) must fit in 32 bits");
    return nullptr;
  }
  const uint32_t N = (uint32_t)Nd;

  sw_handle* h = new (std::nothrow) sw_handle();
  if (!h) { fail(SW_ERR_OOM, "host allocation"); return nullptr; }
  h->model = model; h->dim = dim; h->L = L; h->q = q; h->T = T; h->seed = seed;
  h->spin_bytes = (size_t)N * (model == SW_XY ? sizeof(float) : model == SW_CLOCK ? sizeof(uint16_t) : 1);

  Lattice& lat = h->lat;
  lat.N = N; lat.L = L; lat.dim = dim; lat.W = (L + 31) / 32;
  lat.R = (uint32_t)(N / (uint32_t)L);
  swgb::tiles_for(dim, L, &lat.ntx, &lat.nty, &lat.ntz);
  lat.q = q; lat.sbits = sb;
  lat.dq = (model == SW_POTTS) ? q : 2;
  lat.t_bond = (model == SW_XY) ? 0u : bond_threshold(model, T);
  lat.twoK = (float)(2.0 / T);
  swgb::set_philox_key(lat, seed);
  lat.model = model;
  h->bond_words = (size_t)dim * lat.R * (size_t)lat.W;
  lat.hook_cap = swgb::merge_list_capacity(dim);
  lat.cap = swgb::kLoopCap;
  size_t tile_bufs = 0, hook_words = 0;  // sized for every tile shape a batch may use
  swgb::tile_buffers(model, dim, L, &tile_bufs, &hook_words);

  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { cuda_fail(e, "stream"); release(h); return nullptr; }
  h->own_stream = true;

  // small buffers, carved from one block (layout in block_layout)
  const BlockLayout bl = block_layout();
  const size_t off_err = bl.err, off_acc = bl.acc, off_ncl = bl.ncl, off_sums = bl.sums;
  const size_t off_hist = bl.hist, off_pd = bl.pd, off_series = bl.series;
  const size_t block_bytes = bl.total;

  cudaStream_t st = h->stream;
  if ((e = swgb::dev_alloc(&lat.spins, h->spin_bytes, st)) != cudaSuccess ||
      (e = swgb::dev_alloc((void**)&lat.planes, h->bond_words * 4, st)) != cudaSuccess ||
      (e = swgb::dev_alloc((void**)&lat.forest, (size_t)N * 4, st)) != cudaSuccess ||
      (e = swgb::dev_alloc((void**)&lat.hooked, hook_words * 4, st)) != cudaSuccess ||
      (e = swgb::dev_alloc((void**)&lat.nhooked, tile_bufs * 4, st)) != cudaSuccess ||
      (e = swgb::dev_alloc(&h->d_block, block_bytes, st)) != cudaSuccess) {
    fail(e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA,
         std::string("device allocation: ") + cudaGetErrorString(e));
    cudaGetLastError();
    release(h);
    return nullptr;
  }
  char* blk = static_cast<char*>(h->d_block);
  lat.err = reinterpret_cast<int*>(blk + off_err);
  h->meas.nclusters = reinterpret_cast<unsigned long long*>(blk + off_ncl);
  h->meas.sums = reinterpret_cast<unsigned long long*>(blk + off_sums);
  h->meas.hist = reinterpret_cast<unsigned long long*>(blk + off_hist);
  h->meas.acc = reinterpret_cast<double*>(blk + off_acc);
  h->meas.part_d = reinterpret_cast<double*>(blk + off_pd);
  h->meas.xy_blocks = 0;
  h->meas.done = reinterpret_cast<unsigned int*>(blk + bl.done);
  h->meas.series = blk + off_series;
  h->meas.series_cap = kSeriesCap;

  if (model == SW_CLOCK) {
    // clock tables (thresholds, fixed-point cos/sin) and slot sums in one allocation
    std::vector<uint32_t> tab;
    std::vector<long long> trig;
    std::vector<float> proj;
    clock_tables(q, T, tab, trig, proj);
    const size_t tab_bytes = tab.size() * 4, trig_bytes = trig.size() * 8;
    const size_t hist_bytes = (size_t)3 * swgb::kSlots * 8, proj_bytes = proj.size() * 4;
    if ((e = swgb::dev_alloc(&h->d_clock, tab_bytes + trig_bytes + hist_bytes + proj_bytes, st)) != cudaSuccess) {
      fail(SW_ERR_OOM, std::string("clock tables: ") + cudaGetErrorString(e));
      cudaGetLastError();
      release(h);
      return nullptr;
    }
    char* c = static_cast<char*>(h->d_clock);
    lat.ctab = reinterpret_cast<const uint32_t*>(c);
    h->meas.cfix = reinterpret_cast<const long long*>(c + tab_bytes);
    h->meas.csums = reinterpret_cast<unsigned long long*>(c + tab_bytes + trig_bytes);
    lat.cproj = reinterpret_cast<const float*>(c + tab_bytes + trig_bytes + hist_bytes);
    // copies on the allocating stream, from host vectors that live until
    // the synchronisation at the end of sw_create
    if ((e = cudaMemcpyAsync(c, tab.data(), tab_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c + tab_bytes, trig.data(), trig_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c + tab_bytes + trig_bytes, 0, hist_bytes, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c + tab_bytes + trig_bytes + hist_bytes, proj.data(), proj_bytes,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      cuda_fail(e, "clock tables");
      release(h);
      return nullptr;
    }
  }

  if ((e = cudaMemsetAsync(h->d_block, 0, block_bytes, h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(blk + off_series, 0xff, block_bytes - off_series, h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(lat.planes, 0, h->bond_words * 4, h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(lat.forest, 0, (size_t)N * 4, h->stream)) != cudaSuccess ||
      (e = swgb::launch_init(lat, model, h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    cuda_fail(e, "init");
    release(h);
    return nullptr;
  }
  return h;
}

void sw_destroy(sw_handle* h) {
  if (!h) return;
  if (h->batch) sw_batch_remove(h->batch, h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
}

int sw_sweep(sw_handle* h, int n) { return run_sweeps(h, n, true); }

int sw_sweep_timed(sw_handle* h, float* phase_ms, int nphase) {
  if (!h || !phase_ms) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (nphase < 4) return fail(SW_ERR_BAD_ARG, "nphase < 4");
  if (h->sweep >= 0xffffffffull) return fail(SW_ERR_BAD_ARG, "sweep counter exhausted");
  cudaEvent_t ev[5];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < 5 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) {
    for (int k = 0; k < made - 1; ++k) cudaEventDestroy(ev[k]);
    return cuda_fail(e, "event");
  }
  const uint32_t k = (uint32_t)(++h->sweep);
  e = one_sweep(h, k, true, ev);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
  for (int p = 0; p < 4 && e == cudaSuccess; ++p) e = cudaEventElapsedTime(&phase_ms[p], ev[p], ev[p + 1]);
  for (int p = 0; p < 5; ++p) cudaEventDestroy(ev[p]);
  if (e != cudaSuccess) return cuda_fail(e, "timed sweep");
  return check_device_error(h);
}

int sw_discard(sw_handle* h, int n) { return run_sweeps(h, n, false); }

int sw_sync(sw_handle* h) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  const cudaError_t e = swgb::wait_io(h);
  if (e != cudaSuccess) return cuda_fail(e, "asynchronous I/O");
  return check_device_error(h);
}

int sw_query(sw_handle* h) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  const cudaError_t e = cudaStreamQuery(h->stream);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return cuda_fail(e, "stream query");
}

int sw_set_loop_cap(sw_handle* h, long long cap) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  if (cap > (long long)swgb::kLoopCap) return fail(SW_ERR_BAD_ARG, "cap above the production cap 2^22");
  h->lat.cap = cap < 0 ? swgb::kLoopCap : (uint32_t)cap;
  return SW_OK;
}

int sw_measure(sw_handle* h, sw_moments* out) {
  if (!h || !out) return fail(SW_ERR_BAD_ARG, "NULL argument");
  double acc[6];
  cudaError_t e = flush_pending(h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, h->meas.acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->meas.acc, 0, sizeof(acc), h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "measure copy");
  const int rc = check_device_error(h);
  if (rc != SW_OK) return rc;
  std::memset(out, 0, sizeof(*out));
  out->n_sweeps = acc[0];
  out->sum_M2 = acc[1];
  out->sum_M4 = acc[2];
  out->sum_E = acc[3];
  out->sum_E2 = acc[4];
  out->sum_nclusters = acc[5];
  if (acc[0] > 0) {
    const double n = acc[0], N = (double)h->lat.N;
    const double m2 = acc[1] / n, m4 = acc[2] / n, e1 = acc[3] / n, e2 = acc[4] / n;
    out->U = m2 > 0 ? m4 / (m2 * m2) : 0.0;
    out->e_per_spin = e1 / N;
    out->c_per_spin = (e2 - e1 * e1) / (N * h->T * h->T);
    out->mean_cluster_size = acc[5] > 0 ? N / (acc[5] / n) : 0.0;
  }
  return SW_OK;
}

int sw_set_stream(sw_handle* h, void* stream) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  h->stream = static_cast<cudaStream_t>(stream);
  return SW_OK;
}

uint64_t sw_sweep_counter(sw_handle* h) { return h ? h->sweep : 0; }

int sw_set_sweep_counter(sw_handle* h, uint64_t k) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  if (k >= 0xffffffffull) return fail(SW_ERR_BAD_ARG, "sweep counter must be < 2^32 - 1");
  const cudaError_t e = flush_pending(h);
  if (e != cudaSuccess) return cuda_fail(e, "pending measurement");
  h->sweep = k;
  return SW_OK;
}

int sw_set_sweep_target(sw_handle* h, uint64_t target) {
  if (!h) return fail(SW_ERR_BAD_ARG, "NULL handle");
  if (target >= 0xffffffffull) return fail(SW_ERR_BAD_ARG, "sweep target must be < 2^32 - 1");
  h->target = target;
  return SW_OK;
}

size_t sw_num_sites(sw_handle* h) { return h ? h->lat.N : 0; }
size_t sw_spin_bytes(sw_handle* h) { return h ? h->spin_bytes : 0; }
size_t sw_bond_words(sw_handle* h) { return h ? h->bond_words : 0; }

int sw_get_spins(sw_handle* h, void* host, size_t bytes) {
  if (!h || !host) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (bytes != h->spin_bytes) return fail(SW_ERR_BAD_ARG, "bytes != sw_spin_bytes");
  cudaError_t e = cudaMemcpyAsync(host, h->lat.spins, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_spins");
  return check_device_error(h);
}

int sw_set_spins(sw_handle* h, const void* host, size_t bytes) {
  if (!h || !host) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (bytes != h->spin_bytes) return fail(SW_ERR_BAD_ARG, "bytes != sw_spin_bytes");
  cudaError_t e = flush_pending(h);
  if (e == cudaSuccess) e = swgb::guard_state_write(h, h->lat.spins, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->lat.spins, host, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_spins");
  return check_device_error(h);
}

int sw_get_spins_device(sw_handle* h, void* dev, size_t bytes) {
  if (!h || !dev) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (bytes != h->spin_bytes) return fail(SW_ERR_BAD_ARG, "bytes != sw_spin_bytes");
  cudaError_t e = cudaMemcpyAsync(dev, h->lat.spins, bytes, cudaMemcpyDeviceToDevice, h->stream);
  return e == cudaSuccess ? SW_OK : cuda_fail(e, "get_spins_device");
}

int sw_set_spins_device(sw_handle* h, const void* dev, size_t bytes) {
  if (!h || !dev) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (bytes != h->spin_bytes) return fail(SW_ERR_BAD_ARG, "bytes != sw_spin_bytes");
  cudaError_t e = flush_pending(h);
  if (e == cudaSuccess) e = swgb::guard_state_write(h, h->lat.spins, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->lat.spins, dev, bytes, cudaMemcpyDeviceToDevice, h->stream);
  return e == cudaSuccess ? SW_OK : cuda_fail(e, "set_spins_device");
}

int sw_get_labels(sw_handle* h, int32_t* host, size_t n) {
  if (!h || !host) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (n != h->lat.N) return fail(SW_ERR_BAD_ARG, "n != number of sites");
  cudaError_t e = cudaSuccess;
  if (!h->d_labels) e = swgb::dev_alloc((void**)&h->d_labels, (size_t)h->lat.N * 4, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "labels buffer");
  if ((e = swgb::launch_labels_out(h->lat, h->d_labels, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(host, h->d_labels, n * 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
    return cuda_fail(e, "get_labels");
  return check_device_error(h);
}

int sw_get_bonds(sw_handle* h, uint32_t* host, size_t words) {
  if (!h || !host) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (words != h->bond_words) return fail(SW_ERR_BAD_ARG, "words != sw_bond_words");
  cudaError_t e = cudaMemcpyAsync(host, h->lat.planes, words * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_bonds");
  return check_device_error(h);
}

int sw_label_from_bonds(sw_handle* h, const uint32_t* host_mask, int32_t* host_labels) {
  if (!h || !host_mask || !host_labels) return fail(SW_ERR_BAD_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(h->lat.planes, host_mask, h->bond_words * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = swgb::launch_label(h->lat, 0u, true, h->stream);
  if (e == cudaSuccess) e = swgb::launch_merge(h->lat, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "label_from_bonds");
  return sw_get_labels(h, host_labels, h->lat.N);
}

int sw_get_series(sw_handle* h, uint64_t first, size_t count, sw_record* host) {
  if (!h || (!host && count)) return fail(SW_ERR_BAD_ARG, "NULL argument");
  if (count > (size_t)kSeriesCap) return fail(SW_ERR_RANGE, "count exceeds the retained series");
  const cudaError_t fe = flush_pending(h);
  if (fe != cudaSuccess) return cuda_fail(fe, "pending measurement");
  const int rc = check_device_error(h);
  if (rc != SW_OK) return rc;
  static_assert(sizeof(swgb::Record) == sizeof(sw_record), "record layout");
  if (count == 0) return SW_OK;
  std::vector<sw_record> ring(kSeriesCap);
  cudaError_t e = cudaMemcpy(ring.data(), h->meas.series, sizeof(sw_record) * kSeriesCap,
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "get_series");
  for (size_t k = 0; k < count; ++k) {
    const uint64_t s = first + k;
    host[k] = ring[s % kSeriesCap];
    if (host[k].sweep != s) return fail(SW_ERR_RANGE, "sweep record not retained or not measured");
  }
  return SW_OK;
}

}  // extern "C"
