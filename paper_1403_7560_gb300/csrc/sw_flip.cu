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
struct MergeShape {
  // face bonds a tile owns: +x face, +y face (and +z face)
  static constexpr int kMax = Tile<D>::ROWS + 32 * Tile<D>::TZ + (D == 3 ? 32 * Tile<D>::TY : 0);
  static constexpr int kPerThread = (kMax + kTileThreads - 1) / kTileThreads;
};

template <int D>
__global__ void __launch_bounds__(kTileThreads) k_merge(Lattice lat) {
  constexpr int TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NC = MergeShape<D>::kPerThread;
  __shared__ uint2 s_list[MergeShape<D>::kMax];
  __shared__ int s_n;
  const TileCoord tc = tile_coord<D>(lat);
  const int L = lat.L;
  const int shift = lat.sbits + 1;
  const int nx = min(32, L - tc.x0), ny = min(TY, L - tc.y0), nz = (D == 3) ? min(TZ, L - tc.z0) : 1;
  const int cx = (lat.ntx > 1) ? ny * nz : 0;
  const int cy = (lat.nty > 1) ? nx * nz : 0;
  const int cz = (D == 3 && lat.ntz > 1) ? nx * ny : 0;
  const int total = cx + cy + cz;
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_n = 0;

  // this thread's face bonds: bond bits first, then both forest words
  uint32_t ii[NC], jj[NC], a[NC], b[NC];
  bool on[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int c = threadIdx.x + k * kTileThreads;
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
  for (int e = threadIdx.x; e < n; e += kTileThreads) gunion(lat.forest, s_list[e].x, s_list[e].y, lat.sbits, lat.err);
}

constexpr int kFlipThreads = 256;
constexpr int kFlipBatch = 8;  // rows whose loads and root walks advance together

template <int MODEL, int D>
__global__ void __launch_bounds__(kFlipThreads) k_flip(Lattice lat, uint32_t sweep, Measure mb,
                                                        bool count, uint32_t finalize) {
  constexpr int TY = Tile<D>::TY, ROWS = Tile<D>::ROWS, NW = kFlipThreads / 32, RPW = ROWS / NW;
  constexpr int B = kFlipBatch;
  static_assert(RPW % B == 0, "rows per warp must be a multiple of the batch");
  __shared__ float s_phi;
  __shared__ long long s_red[NW];
  __shared__ double s_rd[NW];
  // the record of the previous measured sweep, from the sums its successor's
  // labeling kernel left behind
  if (finalize != 0u && blockIdx.x == 0) finalize_record<NW>(lat, mb, finalize, s_red, s_rd);
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

  // local roots walk to their global root and store (root, marker, draw);
  // the loads and walks of B rows advance together
#pragma unroll 1
  for (int k0 = 0; k0 < RPW; k0 += B) {
    uint32_t idx[B], cur[B], v[B];
    bool pend[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int rr = warp + NW * (k0 + k);
      const int y = tc.y0 + rr % TY, z = tc.z0 + rr / TY;
      const bool ok = x < L && y < L && (D == 2 || z < L);
      idx[k] = ok ? (uint32_t)x + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z) : 0u;
      v[k] = ok ? __ldcg(&lat.forest[idx[k]]) : 0u;
      const bool lr = ok && (v[k] & lr_bit);
      pend[k] = lr && (v[k] >> shift) != idx[k];
      if (lr && !pend[k]) ++roots;
      cur[k] = v[k] >> shift;
    }
    for (int it = 0; it < (1 << 22); ++it) {
      bool any = false;
#pragma unroll
      for (int k = 0; k < B; ++k)
        if (pend[k]) v[k] = __ldcg(&lat.forest[cur[k]]);
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (!pend[k]) continue;
        const uint32_t p = v[k] >> shift;
        if (p == cur[k]) {
          pend[k] = false;
          __stcg(&lat.forest[idx[k]], (cur[k] << shift) | lr_bit | (v[k] & dmask));
        } else {
          cur[k] = p;
          any = true;
        }
      }
      if (!any) break;
      if (it == (1 << 22) - 1) atomicExch(lat.err, kErrTimeout);
    }
  }
  __syncthreads();

  // every site: its cluster's draw from its local root's word
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
      v[k] = ok[k] ? __ldcg(&lat.forest[idx[k]]) : 0u;
    }
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (ok[k] && !(v[k] & lr_bit)) v[k] = __ldcg(&lat.forest[v[k] >> shift]);
#pragma unroll
    for (int k = 0; k < B; ++k) {
      if (!ok[k]) continue;
      const uint32_t draw = v[k] & dmask;
      const uint32_t i = idx[k];
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
  }
  if (count) {
    const long long tot = block_combine<NW>(warp_sum(roots), s_red);
    if (threadIdx.x == 0 && tot) atomicAdd(mb.nclusters + (sweep & 1u), (unsigned long long)tot);
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

cudaError_t launch_flip(const Lattice& lat, int model, uint32_t sweep, const Measure& m, bool count,
                        uint32_t finalize, cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  if (lat.dim == 2) {
    if (model == kIsing) k_flip<kIsing, 2><<<g, kFlipThreads, 0, st>>>(lat, sweep, m, count, finalize);
    else if (model == kPotts) k_flip<kPotts, 2><<<g, kFlipThreads, 0, st>>>(lat, sweep, m, count, finalize);
    else k_flip<kXY, 2><<<g, kFlipThreads, 0, st>>>(lat, sweep, m, count, finalize);
  } else {
    if (model == kIsing) k_flip<kIsing, 3><<<g, kFlipThreads, 0, st>>>(lat, sweep, m, count, finalize);
    else if (model == kPotts) k_flip<kPotts, 3><<<g, kFlipThreads, 0, st>>>(lat, sweep, m, count, finalize);
    else k_flip<kXY, 3><<<g, kFlipThreads, 0, st>>>(lat, sweep, m, count, finalize);
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
