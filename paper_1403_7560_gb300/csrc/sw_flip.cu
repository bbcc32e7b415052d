// The global half of step (2) and step (3) of the SW sweep (Komura & Okabe,
// Sec. 2).
//
// Forest word of a site: (parent << (sb+1)) | (local-root marker << sb) |
// cluster draw (sb bits).  After k_label every site points to its tile-local
// root (a site of the same tile, marker set on the root itself).  Only
// local roots take part in the global union-find, so the words of all other
// sites keep pointing at their tile's local root.
//
// k_merge: bonds that leave a tile join the local roots at their two ends
//   with atomicMin hooking of the larger root under the smaller; a warp
//   performs each distinct (root, root) pair once.
// k_merge also lists, per tile, the roots it hooked under another tree.
// k_compress: every listed root walks to its global root (the smallest site
//   index of the cluster), takes that root's draw and stores (root, draw) in
//   its own word.
// k_apply: every site reads its local root's word (or its own) and writes
//   its new state (set at random for Ising/Potts, reflection about the
//   mirror line for XY); global roots are counted.  A thread takes four
//   consecutive sites.
// k_labels_out: canonical labels (walk to the root) for readout.
#include <algorithm>

#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

template <class S>
struct MergeShape {
  // face bonds a tile owns: +x face, +y face (and +z face)
  static constexpr int kMax = S::ROWS + 32 * S::TZ + (S::D == 3 ? 32 * S::TY : 0);
  static constexpr int kPerThread = (kMax + S::THREADS - 1) / S::THREADS;
};

template <class S>
struct MergeSmem {
  uint2 list[MergeShape<S>::kMax];
  int n;
};

// faces: which of the tile's +x (1), +y (2), +z (4) faces to join; a merge
// split into one launch per axis starts the tile's hooked list with the x
// faces and appends to it in the later launches.
template <class S>
__device__ __forceinline__ void merge_tile(const Lattice& lat, uint32_t tile, MergeSmem<S>& sm,
                                           uint32_t faces = 7u) {
  constexpr int D = S::D, TY = S::TY, TZ = S::TZ, NT = S::THREADS;
  constexpr int NC = MergeShape<S>::kPerThread;
  uint2* s_list = sm.list;
  int& s_n = sm.n;
  const TileCoord tc = tile_coord<S>(lat, tile);
  const int L = lat.L;
  const int shift = lat.sbits + 1;
  const int nx = min(32, L - tc.x0), ny = min(TY, L - tc.y0), nz = (D == 3) ? min(TZ, L - tc.z0) : 1;
  const int cx = (lat.ntx > 1 && (faces & 1u)) ? ny * nz : 0;
  const int cy = (lat.nty > 1 && (faces & 2u)) ? nx * nz : 0;
  const int cz = (D == 3 && lat.ntz > 1 && (faces & 4u)) ? nx * ny : 0;
  const int total = cx + cy + cz;
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_n = 0;
  pdl_wait();

  // this thread's face bonds: bond bits first, then both forest words
  uint32_t ii[NC], jj[NC], a[NC], b[NC];
  bool on[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int c = threadIdx.x + k * NT;
    on[k] = false;
    ii[k] = jj[k] = 0u;
    if (c >= total) continue;
    int x, y, z, d;
    if (c < cx) {
      d = 0; x = tc.x0 + nx - 1; y = tc.y0 + c % ny; z = tc.z0 + c / ny;
    } else if (c < cx + cy) {
      const int e = c - cx;
      d = 1; x = tc.x0 + e % nx; y = tc.y0 + ny - 1; z = tc.z0 + e / nx;
    } else {
      const int e = c - cx - cy;
      d = 2; x = tc.x0 + e % nx; y = tc.y0 + e / nx; z = tc.z0 + nz - 1;
    }
    if (D == 2) z = 0;
    const uint32_t row = (uint32_t)y + (uint32_t)L * (uint32_t)z;
    const uint32_t bits = __ldg(&lat.planes[d * plane + row * lat.W + (x >> 5)]);
    on[k] = (bits >> (x & 31)) & 1u;
    const uint32_t i = (uint32_t)x + (uint32_t)L * row;
    ii[k] = i;
    if (d == 0) jj[k] = (x + 1 == L) ? i - (uint32_t)x : i + 1u;
    else if (d == 1) jj[k] = (y + 1 == L) ? i - (uint32_t)y * L : i + (uint32_t)L;
    else jj[k] = (z + 1 == L) ? i - (uint32_t)z * L * L : i + (uint32_t)L * L;
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    a[k] = on[k] ? __ldcg(&lat.forest[ii[k]]) >> shift : 0u;
    b[k] = on[k] ? __ldcg(&lat.forest[jj[k]]) >> shift : 0u;
  }
  __syncthreads();
  // distinct (root, root) pairs of each warp go to the tile's work list
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const bool want = on[k] && a[k] != b[k];
    const unsigned long long key = ((unsigned long long)a[k] << 32) | b[k];
    const unsigned grp = __match_any_sync(kFull, want ? key : ~0ull);
    if (want && lane == __ffs(grp) - 1) s_list[atomicAdd(&s_n, 1)] = make_uint2(a[k], b[k]);
  }
  __syncthreads();
  const int n = s_n;
  // every root this tile hooks goes to the tile's hooked list for k_compress
  // (no list on the labeling-only paths)
  uint32_t* hooked = lat.hooked ? lat.hooked + (size_t)tile * (size_t)lat.hook_cap : nullptr;
  __syncthreads();
  if (threadIdx.x == 0) s_n = (hooked && !(faces & 1u)) ? (int)__ldcg(&lat.nhooked[tile]) : 0;
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += NT) {
    const uint32_t h = gunion(lat.forest, s_list[e].x, s_list[e].y, lat.sbits, lat.err, lat.cap);
    if (hooked && h != 0xffffffffu) hooked[atomicAdd(&s_n, 1)] = h;
  }
  __syncthreads();
  if (hooked && threadIdx.x == 0) lat.nhooked[tile] = (uint32_t)s_n;
}

// Eight 256-thread CTAs per SM, proportionally more of smaller tiles.
constexpr int merge_blocks(int threads) { return 8 * 256 / threads > 32 ? 32 : 8 * 256 / threads; }

template <int D>
__global__ void __launch_bounds__(Tile<D>::THREADS, merge_blocks(Tile<D>::THREADS))
    k_merge(Lattice lat, uint32_t faces) {
  __shared__ MergeSmem<Tile<D>> sm;
  merge_tile<Tile<D>>(lat, blockIdx.x, sm, faces);
}

// Batch kernels: PERSISTENT false launches one CTA per tile-map entry
// (entry blockIdx.x); PERSISTENT true a grid of resident CTAs, each taking
// entries t = blockIdx.x, blockIdx.x + gridDim.x, ... below n.  Separate
// instantiations, so that the loop costs the one-entry kernels no registers.
template <class S, bool PERSISTENT>
__global__ void __launch_bounds__(S::THREADS, PERSISTENT ? (merge_blocks(S::THREADS) * 3) / 4 : merge_blocks(S::THREADS))
    k_merge_batch(BatchView bv, uint32_t n, uint32_t faces) {
  __shared__ MergeSmem<S> sm;
  pdl_wait();
  const uint32_t step = *bv.step;
  auto entry = [&](uint32_t t) {
    const BatchMember& m = bv.members[__ldg(&bv.tile_lattice[t])];
    if (step >= m.nsweeps) return;  // the member has had its sweeps this call
    const Lattice lat = m.lat;  // a private copy: global stores cannot alias it
    merge_tile<S>(lat, __ldg(&bv.tile_index[t]), sm, faces);
  };
  if constexpr (PERSISTENT) {
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) {
      __syncthreads();  // the previous entry's readers of sm are done
      entry(t);
    }
  } else {
    entry(blockIdx.x);
  }
}

constexpr int kFlipThreads = 256, kFlipWarps = kFlipThreads / 32;
constexpr unsigned kFlipBlocks = 152u * 8u;

// The roots one tile's merge hooked walk to their global root and store
// (root, marker, root draw) in their own word.  The walks read through L1
// (they meet on the same upper nodes): the merge is over (its stores are
// visible after the wait on it), so the only stores racing with a read are
// these final words, and an older word read in their place points to an
// ancestor of the same tree.
__device__ __forceinline__ void compress_tile(const Lattice& lat, uint32_t t) {
  const int sb = lat.sbits, shift = sb + 1;
  const uint32_t lr_bit = 1u << sb, dmask = lr_bit - 1u;
  const uint32_t n = __ldcg(&lat.nhooked[t]);
  const uint32_t* list = lat.hooked + (size_t)t * (size_t)lat.hook_cap;
  for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
    const uint32_t a = __ldcg(&list[e]);
    uint32_t cur = a, v = __ldcg(&lat.forest[a]);
    uint32_t it = 0;
    for (; it < lat.cap; ++it) {
      const uint32_t p = v >> shift;
      if (p == cur) break;
      cur = p;
      v = __ldca(&lat.forest[cur]);
    }
    if (it == lat.cap) atomicExch(lat.err, kErrTimeout);
    __stcg(&lat.forest[a], (cur << shift) | lr_bit | (v & dmask));
  }
}

// Every root the merge hooked under another tree (the tiles' hooked lists)
// walks to its global root and stores (root, marker, root draw) in its own
// word, so that every site is at most two loads away from its cluster's
// draw.  Block 0 first writes the record of the previous measured sweep,
// from the sums its successor's labeling kernel left behind.
__global__ void __launch_bounds__(kFlipThreads, 8) k_compress(Lattice lat, Measure mb, uint32_t finalize) {
  __shared__ long long s_red[kFlipWarps];
  __shared__ double s_rd[kFlipWarps];
  pdl_wait();
  if (finalize != 0u && blockIdx.x == 0) finalize_record<kFlipWarps>(lat, mb, finalize, s_red, s_rd);
  const uint32_t ntiles = (uint32_t)(lat.ntx * lat.nty * lat.ntz);
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) compress_tile(lat, t);
}

// Batch: one CTA per member tile; the CTA of each member's tile 0 first
// writes that member's previous record (every step after the first).
template <bool PERSISTENT>
__global__ void __launch_bounds__(kFlipThreads, PERSISTENT ? 4 : 6) k_compress_batch(BatchView bv, uint32_t n) {
  __shared__ long long s_red[kFlipWarps];
  __shared__ double s_rd[kFlipWarps];
  pdl_wait();
  const uint32_t step = *bv.step;
  auto entry = [&](uint32_t t) {
    const BatchMember& m = bv.members[__ldg(&bv.tile_lattice[t])];
    const uint32_t tile = __ldg(&bv.tile_index[t]);
    if (step >= m.nsweeps) return;
    const Lattice lat = m.lat;  // a private copy: global stores cannot alias it
    if (tile == 0u && (step > 0u || m.measure0))
      finalize_record<kFlipWarps>(lat, m.meas, m.sweep0 + step, s_red, s_rd);
    compress_tile(lat, tile);
  };
  if constexpr (PERSISTENT) {
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) entry(t);
  } else {
    entry(blockIdx.x);
  }
}

// Every site takes its cluster's draw from its own word (local roots, now
// compressed) or its local root's word and gets its new state: Ising and
// Potts take the draw (Ising: 1 = -1); XY and clock reflect a drawn cluster
// (XY about the sweep's mirror line, clock s -> mirror - s).  A thread takes
// four consecutive sites per step: one 16-byte load of their forest words,
// one load and one store of their four states (4, 8 or 16 bytes).  The
// local-root words are read through L1: each of a warp's four gathers (site
// j of every lane) spans the warp's 128 sites, so the four reach the same
// lines, and L1 serves the repeats (the forest is read-only in this kernel).
// All buffers come from the device pool, so these accesses are aligned; the
// last N mod 4 sites are taken one by one.
template <int MODEL>
__global__ void __launch_bounds__(kFlipThreads) k_apply(Lattice lat, uint32_t sweep, Measure mb,
                                                         bool count) {
  __shared__ float s_phi;
  __shared__ uint32_t s_mirror;
  __shared__ long long s_red[kFlipWarps];
  if (MODEL == kXY || MODEL == kClock) {
    if (threadIdx.x == 0) {
      if (MODEL == kXY) s_phi = xy_phi(lat, sweep);
      else s_mirror = clock_mirror(lat, sweep);
    }
    __syncthreads();
  }
  pdl_wait();
  const int sb = lat.sbits, shift = sb + 1;
  const uint32_t lr_bit = 1u << sb, dmask = lr_bit - 1u;
  const uint32_t nq = lat.N >> 2;
  const uint4* f4 = reinterpret_cast<const uint4*>(lat.forest);
  // the new state of a site (its state bits) from its old one and its draw
  auto update = [&](uint32_t old, uint32_t draw) -> uint32_t {
    if (MODEL == kIsing) return draw ? 0xffu : 0x01u;
    if (MODEL == kPotts) return draw;
    if (!draw) return old;
    if (MODEL == kClock) return (uint32_t)wrap_mod((int)s_mirror - clock_state(old, lat.q), lat.q);
    const float two_pi = 0x1.921fb6p+2f, pi = 0x1.921fb6p+1f;
    float t = __fsub_rn(__fadd_rn(__fmul_rn(2.0f, s_phi), pi), __uint_as_float(old));
    if (t >= two_pi) t = __fsub_rn(t, two_pi);
    if (t >= two_pi) t = __fsub_rn(t, two_pi);
    if (t < 0.0f) t = __fadd_rn(t, two_pi);
    return __float_as_uint(t);
  };
  long long roots = 0;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const uint4 w4 = __ldcg(&f4[q]);
    uint32_t v[4] = {w4.x, w4.y, w4.z, w4.w};
    // XY and clock: the old states are loaded beside the forest words
    // rather than after the roots' words (a shorter load chain)
    uint32_t old[4] = {0u, 0u, 0u, 0u};
    if (MODEL == kXY) {
      const uint4 o = __ldcg(&static_cast<const uint4*>(lat.spins)[q]);
      old[0] = o.x; old[1] = o.y; old[2] = o.z; old[3] = o.w;
    } else if (MODEL == kClock) {
      const uint2 o = __ldcg(&static_cast<const uint2*>(lat.spins)[q]);
      old[0] = o.x & 0xffffu; old[1] = o.x >> 16; old[2] = o.y & 0xffffu; old[3] = o.y >> 16;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!(v[j] & lr_bit)) v[j] = __ldg(&lat.forest[v[j] >> shift]);
      else if ((v[j] >> shift) == 4u * q + (uint32_t)j) ++roots;  // a cluster's root
    }
    uint32_t n[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) n[j] = update(old[j], v[j] & dmask);
    if (MODEL == kXY) {
      static_cast<uint4*>(lat.spins)[q] = make_uint4(n[0], n[1], n[2], n[3]);
    } else if (MODEL == kClock) {
      static_cast<uint2*>(lat.spins)[q] = make_uint2(n[0] | (n[1] << 16), n[2] | (n[3] << 16));
    } else {
      static_cast<uint32_t*>(lat.spins)[q] = n[0] | (n[1] << 8) | (n[2] << 16) | (n[3] << 24);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < (lat.N & 3u)) {
    const uint32_t i = 4u * nq + threadIdx.x;
    uint32_t v = __ldcg(&lat.forest[i]);
    uint32_t old = 0u;
    if (MODEL == kXY) old = __ldcg(&static_cast<const uint32_t*>(lat.spins)[i]);
    if (MODEL == kClock) old = __ldcg(&static_cast<const uint16_t*>(lat.spins)[i]);
    if (!(v & lr_bit)) v = __ldg(&lat.forest[v >> shift]);
    else if ((v >> shift) == i) ++roots;
    const uint32_t n = update(old, v & dmask);
    if (MODEL == kXY) static_cast<uint32_t*>(lat.spins)[i] = n;
    else if (MODEL == kClock) static_cast<uint16_t*>(lat.spins)[i] = (uint16_t)n;
    else static_cast<uint8_t*>(lat.spins)[i] = (uint8_t)n;
  }
  if (count) {
    const long long tot = block_combine<kFlipWarps>(warp_sum(roots), s_red);
    if (threadIdx.x == 0 && tot)
      atomicAdd(mb.nclusters + kSlots * (sweep & 1u) + (blockIdx.x % kSlots), (unsigned long long)tot);
  }
}

// Batch apply: one CTA per member tile, warps over the tile's rows, lanes
// over x; the member's model picks the state update.
template <class S>
__device__ __forceinline__ void apply_tile(const BatchMember& m, uint32_t tile, uint32_t step, long long* s_red);

template <class S, bool PERSISTENT>
__global__ void __launch_bounds__(kFlipThreads) k_apply_batch(BatchView bv, uint32_t n) {
  __shared__ long long s_red[kFlipThreads / 32];
  pdl_wait();
  const uint32_t step = *bv.step;
  if constexpr (PERSISTENT) {
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) {
      const BatchMember& m = bv.members[__ldg(&bv.tile_lattice[t])];
      if (step >= m.nsweeps) continue;
      apply_tile<S>(m, __ldg(&bv.tile_index[t]), step, s_red);
    }
  } else {
    const BatchMember& m = bv.members[__ldg(&bv.tile_lattice[blockIdx.x])];
    if (step >= m.nsweeps) return;
    apply_tile<S>(m, __ldg(&bv.tile_index[blockIdx.x]), step, s_red);
  }
}

// One member tile of the batch apply: warps over the tile's rows, lanes
// over x; the member's model picks the state update; the tile's roots are
// added to the member's cluster count.
template <class S>
__device__ __forceinline__ void apply_tile(const BatchMember& m, uint32_t tile, uint32_t step, long long* s_red) {
  constexpr int D = S::D, TY = S::TY, ROWS = S::ROWS, NW = kFlipThreads / 32, RPW = ROWS / NW;
  constexpr int B = 8;
  static_assert(RPW % B == 0, "whole batches of rows per warp");
  const Lattice lat = m.lat;  // a private copy: the spin stores cannot alias it
  const uint32_t sweep = m.sweep0 + step + 1u;
  const TileCoord tc = tile_coord<S>(lat, tile);
  const int L = lat.L, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sb = lat.sbits, shift = sb + 1;
  const uint32_t lr_bit = 1u << sb, dmask = lr_bit - 1u;
  const int x = tc.x0 + lane;
  long long roots = 0;
#pragma unroll 1
  for (int k0 = 0; k0 < RPW; k0 += B) {
    uint32_t idx[B], v[B];
    bool ok[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int rr = warp + NW * (k0 + k);
      const int y = tc.y0 + rr % TY, z = tc.z0 + rr / TY;
      ok[k] = x < L && y < L && (D == 2 || z < L);
      idx[k] = ok[k] ? (uint32_t)x + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z) : 0u;
      v[k] = ok[k] ? __ldcg(&lat.forest[idx[k]]) : lr_bit;
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (!(v[k] & lr_bit)) v[k] = __ldcg(&lat.forest[v[k] >> shift]);
      else if (ok[k] && (v[k] >> shift) == idx[k]) ++roots;
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (!ok[k]) continue;
      const uint32_t draw = v[k] & dmask;
      if (lat.model == kIsing) static_cast<int8_t*>(lat.spins)[idx[k]] = draw ? (int8_t)-1 : (int8_t)1;
      else static_cast<uint8_t*>(lat.spins)[idx[k]] = (uint8_t)draw;
    }
  }
  const long long tot = block_combine<NW>(warp_sum(roots), s_red);
  if (threadIdx.x == 0 && tot)
    atomicAdd(m.meas.nclusters + kSlots * (sweep & 1u) + (tile % kSlots), (unsigned long long)tot);
}

__global__ void k_advance(uint32_t* step) {
  pdl_wait();
  *step += 1u;
}

__global__ void __launch_bounds__(256) k_labels_out(Lattice lat, int32_t* out) {
  const int shift = lat.sbits + 1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    uint32_t r = lat.forest[i] >> shift;
    uint32_t it = 0;
    for (; it < lat.cap; ++it) {
      const uint32_t r2 = lat.forest[r] >> shift;
      if (r2 == r) break;
      r = r2;
    }
    if (it == lat.cap) atomicExch(lat.err, kErrTimeout);
    out[i] = (int32_t)r;
  }
}

}  // namespace

namespace {
template <int D>
int merge_capacity_dim(int shape) {
  if (shape == 1) return MergeShape<ShapeOf<D, 1>>::kMax;
  if (shape == 2) return MergeShape<ShapeOf<D, 2>>::kMax;
  return MergeShape<ShapeOf<D, 0>>::kMax;
}
}  // namespace

int merge_list_capacity(int dim, int shape) {
  if (shape < 0) shape = kSingleShape[dim - 2];
  return dim == 2 ? merge_capacity_dim<2>(shape) : merge_capacity_dim<3>(shape);
}

void tile_buffers(int model, int dim, int L, size_t* ntiles, size_t* hook_words) {
  const bool batchable = model == kIsing || model == kPotts;
  *ntiles = *hook_words = 0;
  // the single-lattice shape (-1) always; every batch shape for the models a
  // batch can hold
  for (int s = -1; s < (batchable ? kTileShapes : 0); ++s) {
    int ntx, nty, ntz;
    tiles_for(dim, L, &ntx, &nty, &ntz, s);
    const size_t n = (size_t)ntx * nty * ntz;
    *ntiles = std::max(*ntiles, n);
    *hook_words = std::max(*hook_words, n * (size_t)merge_list_capacity(dim, s));
  }
}

cudaError_t launch_merge(const Lattice& lat, cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  if (lat.dim == 2) return launch_pdl(k_merge<2>, g, (unsigned)Tile<2>::THREADS, st, lat, 7u);
  return launch_pdl(k_merge<3>, g, (unsigned)Tile<3>::THREADS, st, lat, 7u);
}

cudaError_t launch_flip(const Lattice& lat, int model, uint32_t sweep, const Measure& m, bool count,
                        uint32_t finalize, cudaStream_t st) {
  // a thread per four sites; at most kFlipBlocks CTAs striding over them
  unsigned g = (unsigned)((lat.N + 4u * kFlipThreads - 1) / (4u * kFlipThreads));
  if (g > kFlipBlocks) g = kFlipBlocks;
  if (g == 0) g = 1;
  const unsigned ntiles = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  const cudaError_t e = launch_pdl(k_compress, ntiles, kFlipThreads, st, lat, m, finalize);
  if (e != cudaSuccess) return e;
  if (model == kIsing) return launch_pdl(k_apply<kIsing>, g, kFlipThreads, st, lat, sweep, m, count);
  if (model == kPotts) return launch_pdl(k_apply<kPotts>, g, kFlipThreads, st, lat, sweep, m, count);
  if (model == kClock) return launch_pdl(k_apply<kClock>, g, kFlipThreads, st, lat, sweep, m, count);
  return launch_pdl(k_apply<kXY>, g, kFlipThreads, st, lat, sweep, m, count);
}

namespace {

// One merge launch over every tile's faces, or (split) one launch per axis:
// the x faces of every tile, then the y faces, then the z faces.
template <int D, int SH>
cudaError_t merge_batch_shape(const BatchView& bv, uint32_t ntiles, bool persistent, bool split, cudaStream_t st) {
  using S = ShapeOf<D, SH>;
  const unsigned g = persistent ? batch_grid(k_merge_batch<S, true>, S::THREADS, ntiles) : ntiles;
  auto one = [&](uint32_t faces) {
    return persistent ? launch_pdl(k_merge_batch<S, true>, g, (unsigned)S::THREADS, st, bv, ntiles, faces)
                      : launch_pdl(k_merge_batch<S, false>, g, (unsigned)S::THREADS, st, bv, ntiles, faces);
  };
  if (!split) return one(7u);
  cudaError_t e = cudaSuccess;
  for (int d = 0; d < D && e == cudaSuccess; ++d) e = one(1u << d);
  return e;
}

template <int D, int SH>
cudaError_t flip_batch_shape(const BatchView& bv, uint32_t ntiles, bool persistent, cudaStream_t st) {
  using S = ShapeOf<D, SH>;
  cudaError_t e;
  if (!persistent) {
    e = launch_pdl(k_compress_batch<false>, ntiles, kFlipThreads, st, bv, ntiles);
    if (e == cudaSuccess) e = launch_pdl(k_apply_batch<S, false>, ntiles, kFlipThreads, st, bv, ntiles);
    return e;
  }
  const unsigned gc = batch_grid(k_compress_batch<true>, kFlipThreads, ntiles);
  const unsigned ga = batch_grid(k_apply_batch<S, true>, kFlipThreads, ntiles);
  e = launch_pdl(k_compress_batch<true>, gc, kFlipThreads, st, bv, ntiles);
  if (e == cudaSuccess) e = launch_pdl(k_apply_batch<S, true>, ga, kFlipThreads, st, bv, ntiles);
  return e;
}

template <int D>
cudaError_t merge_batch_dim(const BatchView& bv, int shape, uint32_t ntiles, bool persistent, bool split,
                            cudaStream_t st) {
  if (shape == 1) return merge_batch_shape<D, 1>(bv, ntiles, persistent, split, st);
  if (shape == 2) return merge_batch_shape<D, 2>(bv, ntiles, persistent, split, st);
  return merge_batch_shape<D, 0>(bv, ntiles, persistent, split, st);
}

template <int D>
cudaError_t flip_batch_dim(const BatchView& bv, int shape, uint32_t ntiles, bool persistent, cudaStream_t st) {
  if (shape == 1) return flip_batch_shape<D, 1>(bv, ntiles, persistent, st);
  if (shape == 2) return flip_batch_shape<D, 2>(bv, ntiles, persistent, st);
  return flip_batch_shape<D, 0>(bv, ntiles, persistent, st);
}

}  // namespace

cudaError_t launch_merge_batch(const BatchView& bv, int dim, int shape, int schedule, uint32_t ntiles,
                               cudaStream_t st) {
  static_assert(kTileShapes == 3, "one instantiation per shape");
  const bool persistent = (schedule & 2) != 0, split = (schedule & 4) != 0;
  return dim == 2 ? merge_batch_dim<2>(bv, shape, ntiles, persistent, split, st)
                  : merge_batch_dim<3>(bv, shape, ntiles, persistent, split, st);
}

cudaError_t launch_flip_batch(const BatchView& bv, int dim, int shape, int schedule, uint32_t ntiles,
                              cudaStream_t st) {
  const bool persistent = (schedule & 2) != 0;
  return dim == 2 ? flip_batch_dim<2>(bv, shape, ntiles, persistent, st)
                  : flip_batch_dim<3>(bv, shape, ntiles, persistent, st);
}

cudaError_t launch_advance(const BatchView& bv, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(bv.step);
  return cudaGetLastError();
}

cudaError_t launch_labels_out(const Lattice& lat, int32_t* out, cudaStream_t st) {
  unsigned g = (lat.N + 255u) / 256u;
  if (g > 4096u) g = 4096u;
  k_labels_out<<<g, 256, 0, st>>>(lat, out);
  return cudaGetLastError();
}

}  // namespace swgb
