// Internal interface between the C-ABI layer (sw_capi.cu, sw_noalloc.cu) and
// the kernels (sw_label.cu, sw_flip.cu, sw_measure.cu).  Not installed; the
// public interface is include/sw.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

struct sw_handle;
struct sw_batch;

namespace swgb {

enum Model { kIsing = 0, kPotts = 1, kXY = 2, kClock = 3 };

// Device-side view of one lattice, passed by value to every kernel.
struct Lattice {
  void* spins;          // int8 (Ising), uint8 (Potts) or float (XY), N entries
  uint32_t* planes;     // bond bit-planes, dim * R * W words
  uint32_t* forest;     // per site: (parent << sbits) | cluster draw
  int* err;             // device error flag (0 = ok, else an sw_status)
  uint32_t N;           // L^dim
  int L, dim, W;        // W = words per lattice row
  uint32_t R;           // rows = L^(dim-1)
  int ntx, nty, ntz;    // tiles per axis
  int q, sbits;         // Potts states; bits of the cluster draw
  uint32_t t_bond;      // Ising/Potts: bond active iff draw < t_bond
  float twoK;           // XY: 2/T as float
  uint32_t key0, key1;  // Philox key = seed
  uint32_t rk[20];      // Philox round keys: (key0 + r*0x9E3779B9, key1 + r*0xBB67AE85), r = 0..9
  int model;            // Model
  int dq;               // modulus of the cluster draw: q (Potts) or 2
  const uint32_t* ctab; // clock: bond thresholds [2q][2q]
  const float* cproj;   // clock: projections x_k = sin(pi k / q) rounded to float [2q]
  uint32_t* hooked;     // per tile: roots hooked by the merge [ntiles * hook_cap]
  uint32_t* nhooked;    // per tile: number of hooked roots [ntiles]
  int hook_cap;         // capacity of a tile's hooked list
  uint32_t cap;         // iteration cap of the capped device loops (kLoopCap unless lowered
                        // by sw_set_loop_cap); a loop that reaches it sets *err and gives up
};

// Production iteration cap of the device loops whose length depends on the
// data (union retries, global union-find and compression walks, the label
// equivalence walks).  Every such loop ends far below it on valid input:
// parents only decrease, so a walk is bounded by the index range.
constexpr uint32_t kLoopCap = 1u << 22;

// Sets the Philox key (seed low, seed high) and its ten round keys.
inline void set_philox_key(Lattice& lat, uint64_t seed) {
  lat.key0 = (uint32_t)(seed & 0xffffffffu);
  lat.key1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    lat.rk[2 * r] = lat.key0 + (uint32_t)r * 0x9E3779B9u;
    lat.rk[2 * r + 1] = lat.key1 + (uint32_t)r * 0xBB67AE85u;
  }
}

// Buffers of the moment reduction (the per-sweep record and accumulators).
// Integer sums are spread over kSlots slots (by block index) so that no
// single word takes an atomic from every block; the record is finalised by
// one block of a later kernel in the same stream.
constexpr int kSlots = 64;
struct Measure {
  unsigned long long* nclusters;  // roots counted by the flip kernel, [2][kSlots] by sweep parity
  unsigned long long* sums;       // [kSlots][2]: integer M, E (two's complement)
  unsigned long long* hist;       // [kSlots][256]: Potts histogram
  double* part_d;                 // XY per-block partials [3 * kMeasureBlocks]
  unsigned long long* csums;      // clock: [kSlots][3] integer sums of C[p_i], S[p_i], C[p_i - p_j]
  const long long* cfix;          // clock: C[p] = round(2^30 cos(2 pi p / q)) [q], then S [q]
  int xy_blocks;                  // blocks that wrote part_d
  unsigned int* done;             // blocks of a stand-alone measurement that have added their sums
  double* acc;                    // n, sum M2, M4, E, E2, nclusters
  void* series;                   // sw_record ring
  int series_cap;
};

// One lattice of a batch: its device view, measurement buffers and the
// sweep counter before the current batch call.
struct BatchMember {
  Lattice lat;
  Measure meas;
  uint32_t sweep0;
  uint32_t nsweeps;   // sweeps of this member in the current batch call (steps >= nsweeps skip it)
  uint32_t measure0;  // 1: the first step also measures the incoming state (the record of sweep0)
};

// Device-side description of a batch: members, the tile -> (member, tile)
// map of one launch over every member's tiles, and the step counter of the
// current batch call (advanced on the device after every sweep, so that a
// captured sweep can be replayed).
struct BatchView {
  const BatchMember* members;
  const uint32_t* tile_lattice;
  const uint32_t* tile_index;
  uint32_t* step;
};

// Record layout written by the measurement kernel (mirrors sw_record).
struct Record {
  unsigned long long sweep;
  long long M, E, nclusters, S2;
  double mx, my, e_xy, M2, Ed;
};

constexpr int kMeasureBlocks = 1216;  // 152 SMs x 8 blocks of 256 threads
constexpr int kMaxClockQ = 1024;      // largest q of the clock model

// Tile shapes of the labeling and merge kernels: 32 sites along x (one
// bit-plane word) by TY (by TZ); one CTA of TY*TZ threads (a thread per row
// word) per tile.  Single lattices use shape kSingleShape of their
// dimension (2D 32 x 128, 3D 32 x 16 x 16, the faster ones on the GB300);
// a batch runs any of them (sw_batch_autotune times them).  A tile's shape
// changes no result: bond words, draws and canonical roots are keyed by row
// word and site index only.
constexpr int kTileShapes = 3;
constexpr int kShapeTY[2][kTileShapes] = {{256, 128, 64}, {16, 16, 8}};
constexpr int kShapeTZ[2][kTileShapes] = {{1, 1, 1}, {16, 8, 8}};
constexpr int kSingleShape[2] = {1, 0};

// Launches kernel k with programmatic stream serialisation: its launch is
// processed while the preceding kernel in the stream runs, and it waits for
// that kernel with griddepcontrol.wait (pdl_wait in sw_device.cuh) before
// touching global memory.  Every kernel launched this way must make that
// call.
template <class... K, class... A>
cudaError_t launch_pdl(void (*k)(K...), unsigned grid, unsigned block, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

// Tiles per axis of an L^dim lattice in tile shape `shape` (-1: the
// single-lattice shape of dim).
void tiles_for(int dim, int L, int* ntx, int* nty, int* ntz, int shape = -1);
// Bonds that leave one tile (its +x, +y, +z faces): the most roots one
// tile's merge can hook.
int merge_list_capacity(int dim, int shape = -1);
// Sizes of a lattice's per-tile buffers (the hooked-root counters and
// lists): for Ising/Potts lattices, which may join a batch, the largest
// over all tile shapes; for the others, the single-lattice shape's.
void tile_buffers(int model, int dim, int L, size_t* ntiles, size_t* hook_words);

// Message returned by sw_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// Stream-ordered device memory from a pool the library keeps per device
// (cudaMallocFromPoolAsync / cudaFreeAsync).  Creating or destroying a
// handle or a batch therefore never synchronises the device (cudaFree
// does), and freed blocks stay cached in the pool for the next handle.  An
// allocation is ordered on `st`: other streams may use it once `st` has
// been synchronised past it.  dev_free(nullptr, st) does nothing.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);

cudaError_t launch_init(const Lattice& lat, int model, cudaStream_t st);
// Bonds of the XY model (lane per site) into the bit-planes.
// XY bonds of `sweep`; with m != nullptr the kernel also measures the
// incoming state into m's XY partials, one per block (*blocks = grid).
cudaError_t launch_bonds_xy(const Lattice& lat, uint32_t sweep, const Measure* m, int* blocks,
                            cudaStream_t st);
// Bonds of the clock model (lane per site, table thresholds).
// Clock bonds of `sweep`; with m != nullptr the kernel also measures the
// incoming state into m's clock slot sums.
cudaError_t launch_bonds_clock(const Lattice& lat, uint32_t sweep, const Measure* m, cudaStream_t st);
// Tile labels (+ Ising/Potts bonds when from_mask is false; cluster draws
// when sweep != 0) into the forest.
cudaError_t launch_label(const Lattice& lat, uint32_t sweep, bool from_mask, cudaStream_t st);
// Same for Ising/Potts, also measuring the incoming spins (the state after
// sweep - 1) into the record of sweep - 1.
cudaError_t launch_label_measured(const Lattice& lat, uint32_t sweep, const Measure& m,
                                  cudaStream_t st);
cudaError_t launch_merge(const Lattice& lat, cudaStream_t st);
// Flip of `sweep`; counts roots into m.nclusters[sweep & 1] when `count`;
// when finalize != 0 its first block first writes the record of sweep
// `finalize` from the sums a previous kernel left in m.
cudaError_t launch_flip(const Lattice& lat, int model, uint32_t sweep, const Measure& m, bool count,
                        uint32_t finalize, cudaStream_t st);
// Stand-alone measurement of the current spins as the record of `sweep`
// (sums, then a one-block finalisation).
cudaError_t launch_measure(const Lattice& lat, int model, uint32_t sweep, const Measure& m,
                           cudaStream_t st);
// Stand-alone Ising/Potts measurement as the record of `sweep` (a thread per
// row word, sw_label.cu); the last block to finish writes the record.
cudaError_t launch_measure_rows(const Lattice& lat, uint32_t sweep, const Measure& m, cudaStream_t st);
cudaError_t launch_labels_out(const Lattice& lat, int32_t* out, cudaStream_t st);

// Batched phases: one launch per phase over every tile of every member
// (Ising/Potts, one dimension, tile shape `shape`), then the step counter
// advances.  The tile map lists the Ising members' tiles first (ising_tiles
// of them), then the Potts members' tiles.  A schedule has two bits:
//   bit 0 (label layout): 0 = the Ising tiles in one launch (two-state
//     layout), the Potts tiles in another; 1 = every tile in one launch
//     (Potts layout, the member's model picked per tile);
//   bit 1 (grid form): 0 = one CTA per tile-map entry; 1 = a persistent grid
//     of resident CTAs (the SM count times the CTAs one SM holds), each
//     striding over the tile map;
//   bit 2 (merge): 0 = one launch joins every face of every tile; 1 = one
//     launch per axis (the x faces of every tile, then y, then z).
constexpr int kBatchSchedules = 8;
cudaError_t launch_label_batch(const BatchView& bv, int dim, int shape, int schedule, uint32_t ising_tiles,
                               uint32_t potts_tiles, cudaStream_t st);
cudaError_t launch_merge_batch(const BatchView& bv, int dim, int shape, int schedule, uint32_t ntiles,
                               cudaStream_t st);
cudaError_t launch_flip_batch(const BatchView& bv, int dim, int shape, int schedule, uint32_t ntiles,
                              cudaStream_t st);

// Grid of a persistent launch of kernel k with `threads` threads per CTA
// over n tile-map entries: the device's SM count times the CTAs of k one SM
// holds (the occupancy calculator's figure for that kernel), at most n.
// Queried when the batch's graph is captured, not per sweep.
int sm_count();
template <class K>
unsigned batch_grid(K* k, int threads, uint32_t n) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const uint64_t g = (uint64_t)sm_count() * (uint64_t)per_sm;
  return (unsigned)(g < n ? g : (n ? n : 1u));
}
// Advances the batch step counter (after every member's sweep).
cudaError_t launch_advance(const BatchView& bv, cudaStream_t st);
// Small members of a batch (sw_small.cu): one CTA per member, whole sweeps
// in shared memory; lists of member indices, Ising and Potts.
// prepare_small_batch sets the kernels' shared-memory limit (once, before
// capture).
cudaError_t prepare_small_batch();
cudaError_t launch_small_batch(const BatchView& bv, int dim, const uint32_t* ising_list, uint32_t n_ising,
                               const uint32_t* potts_list, uint32_t n_potts, cudaStream_t st);

// Write the record of a pending measured sweep of h (stand-alone kernel).
cudaError_t flush_pending(struct ::sw_handle* h);
// Bytes of the small per-handle buffers (records, sums, accumulators).
size_t handle_block_bytes();
// Small Ising/Potts lattices (sw_small.cu): whole sweeps by one CTA with
// the lattice in shared memory, n sweeps per launch, records written as
// the tiled path writes them.
constexpr int kSmallSites = 8192;  // the shared-memory layout's capacity
size_t small_layout_bytes_max();
// Largest lattice (sites) that takes the one-CTA path: 2D Ising 4096, 2D
// Potts 8192, 3D 1024 (where it beats the tiled path).
uint32_t small_sites_limit(int model, int dim);
bool small_lattice(const Lattice& lat);
cudaError_t launch_sweeps_small(const Lattice& lat, const Measure& m, uint32_t sweep0, int n, bool measure,
                                cudaStream_t st);
// Waits for the handle's asynchronous uploads and downloads (no-op if none).
cudaError_t wait_io(sw_handle* h);
// Frees the asynchronous I/O streams, events and buffers.
void release_io(sw_handle* h);
// Called before any work enqueued on stream st writes the spin buffer buf:
// if a download of buf may still be in flight, st waits for it.
cudaError_t guard_state_write(sw_handle* h, const void* buf, cudaStream_t st);

}  // namespace swgb

// One lattice and everything the library allocated for it (include/sw.h:
// sw_handle).
struct sw_handle {
  int model = 0, dim = 0, L = 0, q = 2;
  double T = 0.0;
  uint64_t seed = 0;
  uint64_t sweep = 0;
  size_t spin_bytes = 0, bond_words = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  swgb::Lattice lat{};
  swgb::Measure meas{};
  uint64_t pending = 0;         // measured sweep whose record is not yet written
  uint64_t target = 0;          // batch sweeps stop at this counter value (0: no target)
  int32_t* d_labels = nullptr;  // debug readout buffer, allocated on first use
  void* d_block = nullptr;      // one allocation holding every small buffer
  void* d_clock = nullptr;      // clock model: thresholds, fixed-point cos/sin, slot sums
  struct sw_batch* batch = nullptr;  // batch the lattice belongs to, if any
  // asynchronous host I/O (sw_io.cu), created on first use: an upload and a
  // download stream, the upload target (swapped with lat.spins when the
  // upload is installed), with their events; the two spin buffers
  // (lat.spins and stage_in in either order) each have an event marking the
  // end of their last download and a flag saying that no write has waited
  // for it yet
  cudaStream_t io_in = nullptr, io_out = nullptr;
  void* stage_in = nullptr;
  void* io_buf[2] = {nullptr, nullptr};
  cudaEvent_t ev_in_done = nullptr, ev_in_free = nullptr, ev_state = nullptr, ev_rec = nullptr;
  cudaEvent_t ev_down[2] = {nullptr, nullptr};
  bool down_wait[2] = {false, false};
  bool in_free_set = false;
};
