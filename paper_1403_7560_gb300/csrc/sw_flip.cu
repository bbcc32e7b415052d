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
// k_flip: per tile, every local root walks to its global root (the smallest
//   site index of the cluster), takes that root's draw and stores
//   (root, draw) in its own word; after a CTA barrier every site reads its
//   local root's word and writes its new state (set at random for
//   Ising/Potts, reflection about the mirror line for XY).
// k_labels_out: canonical labels (walk to the root) for readout.
#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

template <int D>
__global__ void __launch_bounds__(kTileThreads) k_merge(Lattice lat) {
  constexpr int TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  const TileCoord tc = tile_coord<D>(lat);
  const int L = lat.L;
  const int shift = lat.sbits + 1;
  const int nx = min(32, L - tc.x0), ny = min(TY, L - tc.y0), nz = (D == 3) ? min(TZ, L - tc.z0) : 1;
  const int cx = (lat.ntx > 1) ? ny * nz : 0;
  const int cy = (lat.nty > 1) ? nx * nz : 0;
  const int cz = (D == 3 && lat.ntz > 1) ? nx * ny : 0;
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  const int lane = threadIdx.x & 31;
  for (int c = threadIdx.x; c < cx + cy + cz; c += blockDim.x) {
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
    if (!((bits >> (x & 31)) & 1u)) continue;
    const uint32_t i = (uint32_t)x + (uint32_t)L * row;
    uint32_t j;
    if (d == 0) j = (x + 1 == L) ? i - (uint32_t)x : i + 1u;
    else if (d == 1) j = (y + 1 == L) ? i - (uint32_t)y * L : i + (uint32_t)L;
    else j = (z + 1 == L) ? i - (uint32_t)z * L * L : i + (uint32_t)L * L;
    const uint32_t a = __ldcg(&lat.forest[i]) >> shift;
    const uint32_t b = __ldcg(&lat.forest[j]) >> shift;
    if (a == b) continue;
    const unsigned long long key = ((unsigned long long)a << 32) | b;
    const unsigned grp = __match_any_sync(__activemask(), key);
    if (lane == __ffs(grp) - 1) gunion(lat.forest, a, b, lat.sbits, lat.err);
  }
}

template <int MODEL, int D>
__global__ void __launch_bounds__(kTileThreads) k_flip(Lattice lat, uint32_t sweep,
                                                        unsigned long long* nclusters) {
  constexpr int TY = Tile<D>::TY, ROWS = Tile<D>::ROWS, NW = kTileThreads / 32, RPW = ROWS / NW;
  __shared__ float s_phi;
  __shared__ long long s_red[NW];
  if (MODEL == kXY) {
    if (threadIdx.x == 0) s_phi = xy_phi(lat, sweep);
    __syncthreads();
  }
  const TileCoord tc = tile_coord<D>(lat);
  const int L = lat.L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sb = lat.sbits, shift = sb + 1;
  const uint32_t lr_bit = 1u << sb, dmask = lr_bit - 1u;
  const int x = tc.x0 + lane;
  long long roots = 0;

  // local roots: walk to the global root, store (root, marker, root draw)
#pragma unroll 1
  for (int k = 0; k < RPW; ++k) {
    const int rr = warp + NW * k;
    const int y = tc.y0 + rr % TY, z = tc.z0 + rr / TY;
    if (x >= L || y >= L || (D == 3 && z >= L)) continue;
    const uint32_t i = (uint32_t)x + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z);
    const uint32_t f = __ldcg(&lat.forest[i]);
    if (!(f & lr_bit)) continue;
    uint32_t cur = i, v = f;
    int it = 0;
    for (; it < (1 << 22); ++it) {
      const uint32_t p = v >> shift;
      if (p == cur) break;
      cur = p;
      v = __ldcg(&lat.forest[cur]);
    }
    if (it == (1 << 22)) atomicExch(lat.err, kErrTimeout);
    if (cur == i) ++roots;
    else __stcg(&lat.forest[i], (cur << shift) | lr_bit | (v & dmask));
  }
  __syncthreads();

  // every site: the draw of its cluster from its local root's word
#pragma unroll 1
  for (int k = 0; k < RPW; ++k) {
    const int rr = warp + NW * k;
    const int y = tc.y0 + rr % TY, z = tc.z0 + rr / TY;
    if (x >= L || y >= L || (D == 3 && z >= L)) continue;
    const uint32_t i = (uint32_t)x + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z);
    uint32_t v = __ldcg(&lat.forest[i]);
    if (!(v & lr_bit)) v = __ldcg(&lat.forest[v >> shift]);
    const uint32_t draw = v & dmask;
    if (MODEL == kIsing) {
      static_cast<int8_t*>(lat.spins)[i] = draw ? (int8_t)-1 : (int8_t)1;
    } else if (MODEL == kPotts) {
      static_cast<uint8_t*>(lat.spins)[i] = (uint8_t)draw;
    } else if (draw) {
      float* th = static_cast<float*>(lat.spins);
      const float phi = s_phi;
      const float two_pi = 0x1.921fb6p+2f, pi = 0x1.921fb6p+1f;
      float t = __fsub_rn(__fadd_rn(__fmul_rn(2.0f, phi), pi), th[i]);
      if (t >= two_pi) t = __fsub_rn(t, two_pi);
      if (t >= two_pi) t = __fsub_rn(t, two_pi);
      if (t < 0.0f) t = __fadd_rn(t, two_pi);
      th[i] = t;
    }
  }
  if (nclusters) {
    const long long tot = block_combine<NW>(warp_sum(roots), s_red);
    if (threadIdx.x == 0 && tot) atomicAdd(nclusters, (unsigned long long)tot);
  }
}

__global__ void __launch_bounds__(256) k_labels_out(Lattice lat, int32_t* out) {
  const int shift = lat.sbits + 1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    uint32_t r = lat.forest[i] >> shift;
    int it = 0;
    for (; it < (1 << 22); ++it) {
      const uint32_t r2 = lat.forest[r] >> shift;
      if (r2 == r) break;
      r = r2;
    }
    if (it == (1 << 22)) atomicExch(lat.err, kErrTimeout);
    out[i] = (int32_t)r;
  }
}

}  // namespace

cudaError_t launch_merge(const Lattice& lat, cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  if (lat.dim == 2) k_merge<2><<<g, kTileThreads, 0, st>>>(lat);
  else k_merge<3><<<g, kTileThreads, 0, st>>>(lat);
  return cudaGetLastError();
}

cudaError_t launch_flip(const Lattice& lat, int model, uint32_t sweep,
                        unsigned long long* nclusters, cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  if (lat.dim == 2) {
    if (model == kIsing) k_flip<kIsing, 2><<<g, kTileThreads, 0, st>>>(lat, sweep, nclusters);
    else if (model == kPotts) k_flip<kPotts, 2><<<g, kTileThreads, 0, st>>>(lat, sweep, nclusters);
    else k_flip<kXY, 2><<<g, kTileThreads, 0, st>>>(lat, sweep, nclusters);
  } else {
    if (model == kIsing) k_flip<kIsing, 3><<<g, kTileThreads, 0, st>>>(lat, sweep, nclusters);
    else if (model == kPotts) k_flip<kPotts, 3><<<g, kTileThreads, 0, st>>>(lat, sweep, nclusters);
    else k_flip<kXY, 3><<<g, kTileThreads, 0, st>>>(lat, sweep, nclusters);
  }
  return cudaGetLastError();
}

cudaError_t launch_labels_out(const Lattice& lat, int32_t* out, cudaStream_t st) {
  unsigned g = (lat.N + 255u) / 256u;
  if (g > 4096u) g = 4096u;
  k_labels_out<<<g, 256, 0, st>>>(lat, out);
  return cudaGetLastError();
}

}  // namespace swgb
