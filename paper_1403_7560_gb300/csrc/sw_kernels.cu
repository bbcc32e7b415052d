// Kernels of one Swendsen-Wang sweep (Komura & Okabe, Sec. 2) for sm_103a.
//
//   k_bond_label  step (1) + the tile-local half of step (2): one CTA per
//                 32 x TY (x TZ) tile draws the site's Philox words, decides
//                 its +d bonds, writes the bond bit-planes (one __ballot_sync
//                 word per row and direction), joins x-runs with ballot bit
//                 arithmetic and the remaining in-tile bonds with a
//                 shared-memory union-find, and writes each site's forest
//                 word (tile-local root as a global index, plus the site's own
//                 cluster draw in the low bits).
//   k_merge       the global half of step (2): bonds that leave a tile are
//                 joined in the global forest with atomicMin hooking of the
//                 larger root under the smaller (path halving in find), so
//                 every root ends as the smallest site index of its cluster.
//   k_flip        step (3): each site walks to its root, takes the root's
//                 draw and writes its new state; roots are counted.
//   k_measure     measurement (Sec. 2: M, E; Potts M^2 equation): block and
//                 warp reductions, per-block partials, and the last block
//                 finalises the sweep record and the FP64 accumulators.
//
// Every device loop is bounded by construction (parents only decrease) and
// additionally capped; hitting a cap sets the error flag instead of hanging.
#include "sw_internal.h"

namespace swgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kErrTimeout = -4;

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds; per round two 32x32
// multiplications whose high words are xor-ed with the other counter words
// and the round key, key bumped by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t word(const uint4& w, int d) {
  return d == 0 ? w.x : d == 1 ? w.y : d == 2 ? w.z : w.w;
}

// XY mirror direction of a sweep: phi = (w0 >> 8) * fl(2 pi)/2^24 in float.
__device__ __forceinline__ float xy_phi(const Lattice& lat, uint32_t sweep) {
  const uint4 w = philox(0u, sweep, 3u, 0u, lat.key0, lat.key1);
  return __fmul_rn((float)(w.x >> 8), 0x1.921fb6p-22f);
}

// Cluster draw of a site from word `dim` of its bond draw.
template <int MODEL>
__device__ __forceinline__ uint32_t cluster_draw(uint32_t w, int q) {
  if (MODEL == kPotts) return (uint32_t)(((unsigned long long)w * (unsigned)q) >> 32);
  return w >> 31;
}

template <int D>
struct TileDims;
template <>
struct TileDims<2> {
  static constexpr int TY = kTileY2, TZ = 1;
};
template <>
struct TileDims<3> {
  static constexpr int TY = kTileY3, TZ = kTileZ3;
};

// ---------------------------------------------------------------- init
template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_init(Lattice lat) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    const uint32_t w = philox(i, 0u, 0u, 0u, lat.key0, lat.key1).x;
    if (MODEL == kIsing) {
      static_cast<int8_t*>(lat.spins)[i] = (w >> 31) ? (int8_t)-1 : (int8_t)1;
    } else if (MODEL == kPotts) {
      static_cast<uint8_t*>(lat.spins)[i] = (uint8_t)(((unsigned long long)w * (unsigned)lat.q) >> 32);
    } else {
      static_cast<float*>(lat.spins)[i] = __fmul_rn((float)(w >> 8), 0x1.921fb6p-22f);
    }
  }
}

// ---------------------------------------------------------------- shared UF
__device__ __forceinline__ uint32_t sfind(volatile uint32_t* par, uint32_t x) {
  for (int it = 0; it < 4096; ++it) {
    const uint32_t p = par[x];
    if (p == x) return x;
    const uint32_t gp = par[p];
    if (gp == p) return p;
    par[x] = gp;  // path halving on a non-root
    x = gp;
  }
  return x;
}

__device__ __forceinline__ void sunion(uint32_t* par, uint32_t a, uint32_t b, int* err) {
  volatile uint32_t* vp = par;
  for (int it = 0; it < 4096; ++it) {
    a = sfind(vp, a);
    b = sfind(vp, b);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicMin(&par[a], b);
    if (old == a) return;
    a = old;
  }
  atomicExch(err, kErrTimeout);
}

// ---------------------------------------------------------------- global UF
__device__ __forceinline__ uint32_t gfind(uint32_t* f, uint32_t x, int sb) {
  for (int it = 0; it < (1 << 22); ++it) {
    const uint32_t p = __ldcg(&f[x]) >> sb;
    if (p == x) return x;
    const uint32_t gp = __ldcg(&f[p]) >> sb;
    if (gp == p) return p;
    __stcg(&f[x], gp << sb);  // path halving on a non-root
    x = gp;
  }
  return x;
}

__device__ __forceinline__ void gunion(uint32_t* f, uint32_t a, uint32_t b, int sb, int* err) {
  for (int it = 0; it < (1 << 20); ++it) {
    a = gfind(f, a, sb);
    b = gfind(f, b, sb);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicMin(&f[a], b << sb);
    if ((old >> sb) == a) return;
    a = old >> sb;
  }
  atomicExch(err, kErrTimeout);
}

// ---------------------------------------------------------------- bonds + tile labels
template <int MODEL, int D, bool FROM_MASK>
__global__ void __launch_bounds__(kThreads) k_bond_label(Lattice lat, uint32_t sweep) {
  constexpr int TY = TileDims<D>::TY, TZ = TileDims<D>::TZ;
  constexpr int ROWS = TY * TZ, RPW = ROWS / kWarps, TS = 32 * ROWS;
  __shared__ uint32_t par[TS];
  __shared__ float s_phi;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int b = blockIdx.x;
  const int tx = b % lat.ntx;
  b /= lat.ntx;
  const int ty = b % lat.nty;
  const int tz = b / lat.nty;
  const int L = lat.L;
  const int x0 = tx * 32, y0 = ty * TY, z0 = tz * TZ;
  const int x = x0 + lane;
  const uint32_t plane = lat.R * (uint32_t)lat.W;

  if (MODEL == kXY && !FROM_MASK) {
    if (threadIdx.x == 0) s_phi = xy_phi(lat, sweep);
    __syncthreads();
  }

  // bits 0..2: bond (i,d) active; bit 3: valid site; bits 8..15: draw
  uint32_t info[RPW];
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const int r = warp + kWarps * j;
    const int ry = r % TY, rz = r / TY;
    const int y = y0 + ry, z = z0 + rz;
    const bool rowv = (y < L) && (D == 2 || z < L);
    const bool v = rowv && (x < L);
    const uint32_t row = (uint32_t)y + (uint32_t)L * (uint32_t)z;
    const uint32_t i = (uint32_t)x + (uint32_t)L * row;
    uint32_t a = 0, draw = 0;
    if (v) {
      if (FROM_MASK) {
#pragma unroll
        for (int d = 0; d < D; ++d)
          a |= ((__ldg(&lat.planes[d * plane + row * lat.W + tx]) >> lane) & 1u) << d;
      } else {
        const uint4 w = philox(i, sweep, 1u, 0u, lat.key0, lat.key1);
        uint32_t jn[3];
        jn[0] = (x + 1 == L) ? i - (uint32_t)x : i + 1u;
        jn[1] = (y + 1 == L) ? i - (uint32_t)y * L : i + (uint32_t)L;
        jn[2] = (D == 3) ? ((z + 1 == L) ? i - (uint32_t)z * L * L : i + (uint32_t)L * L) : 0u;
        if (MODEL == kIsing || MODEL == kPotts) {
          const uint8_t* s = static_cast<const uint8_t*>(lat.spins);
          const uint8_t si = s[i];
#pragma unroll
          for (int d = 0; d < D; ++d)
            a |= (uint32_t)((s[jn[d]] == si) && (word(w, d) < lat.t_bond)) << d;
        } else {
          const float* th = static_cast<const float*>(lat.spins);
          const float phi = s_phi;
          const float xi = cosf(__fsub_rn(th[i], phi));
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float xj = cosf(__fsub_rn(th[jn[d]], phi));
            const float prod = __fmul_rn(xi, xj);
            bool act = false;
            if (prod > 0.0f) {
              const float p = -expm1f(-__fmul_rn(lat.twoK, prod));
              const float u = __fmul_rn((float)(word(w, d) >> 8), 0x1p-24f);
              act = u < p;
            }
            a |= (uint32_t)act << d;
          }
        }
        draw = cluster_draw<MODEL>(word(w, D), lat.q);
      }
    }
    if (!FROM_MASK) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const uint32_t bal = __ballot_sync(kFull, (a >> d) & 1u);
        if (rowv && lane == d) lat.planes[d * plane + row * lat.W + tx] = bal;
      }
    }
    // x-runs: lanes m..l are joined when bonds m..l-1 are all active
    const uint32_t bx = __ballot_sync(kFull, (a & 1u) && lane < 31 && x + 1 < L);
    const uint32_t below = ~bx & ((1u << lane) - 1u);
    const int m = below ? 32 - __clz(below) : 0;
    par[lane + 32 * r] = (uint32_t)(m + 32 * r);
    info[j] = a | (v ? 8u : 0u) | (draw << 8);
  }
  __syncthreads();

  // remaining in-tile bonds: x wrap (tile spans the whole row), +y, +z
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const uint32_t inf = info[j];
    if (!(inf & 8u)) continue;
    const int r = warp + kWarps * j;
    const int ry = r % TY, rz = r / TY;
    const uint32_t t = (uint32_t)(lane + 32 * r);
    if ((inf & 1u) && x + 1 == L && x0 == 0) sunion(par, t, t - (uint32_t)lane, lat.err);
    if (inf & 2u) {
      const int y = y0 + ry;
      const int y1 = (y + 1 == L) ? 0 : y + 1;
      if (y1 - y0 >= 0 && y1 - y0 < TY) sunion(par, t, (uint32_t)((int)t + 32 * (y1 - y)), lat.err);
    }
    if (D == 3 && (inf & 4u)) {
      const int z = z0 + rz;
      const int z1 = (z + 1 == L) ? 0 : z + 1;
      if (z1 - z0 >= 0 && z1 - z0 < TZ) sunion(par, t, (uint32_t)((int)t + 32 * TY * (z1 - z)), lat.err);
    }
  }
  __syncthreads();

  // forest word: tile-local root as a global site index, plus the draw
#pragma unroll
  for (int j = 0; j < RPW; ++j) {
    const uint32_t inf = info[j];
    if (!(inf & 8u)) continue;
    const int r = warp + kWarps * j;
    const int ry = r % TY, rz = r / TY;
    const uint32_t lr = sfind(par, (uint32_t)(lane + 32 * r));
    const uint32_t lrow = lr >> 5;
    const uint32_t gx = (uint32_t)x0 + (lr & 31u);
    const uint32_t gy = (uint32_t)y0 + lrow % TY;
    const uint32_t gz = (uint32_t)z0 + lrow / TY;
    const uint32_t g = gx + (uint32_t)L * (gy + (uint32_t)L * gz);
    const uint32_t i = (uint32_t)x + (uint32_t)L * ((uint32_t)(y0 + ry) + (uint32_t)L * (uint32_t)(z0 + rz));
    lat.forest[i] = (g << lat.sbits) | (inf >> 8);
  }
}

// ---------------------------------------------------------------- tile-boundary merge
template <int D>
__global__ void __launch_bounds__(kThreads) k_merge(Lattice lat) {
  constexpr int TY = TileDims<D>::TY, TZ = TileDims<D>::TZ;
  int b = blockIdx.x;
  const int tx = b % lat.ntx;
  b /= lat.ntx;
  const int ty = b % lat.nty;
  const int tz = b / lat.nty;
  const int L = lat.L;
  const int x0 = tx * 32, y0 = ty * TY, z0 = tz * TZ;
  const int nx = min(32, L - x0), ny = min(TY, L - y0), nz = (D == 3) ? min(TZ, L - z0) : 1;
  const int cx = (lat.ntx > 1) ? ny * nz : 0;
  const int cy = (lat.nty > 1) ? nx * nz : 0;
  const int cz = (D == 3 && lat.ntz > 1) ? nx * ny : 0;
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  for (int c = threadIdx.x; c < cx + cy + cz; c += blockDim.x) {
    int x, y, z, d;
    if (c < cx) {
      d = 0; x = x0 + nx - 1; y = y0 + c % ny; z = z0 + c / ny;
    } else if (c < cx + cy) {
      const int e = c - cx;
      d = 1; x = x0 + e % nx; y = y0 + ny - 1; z = z0 + e / nx;
    } else {
      const int e = c - cx - cy;
      d = 2; x = x0 + e % nx; y = y0 + e / nx; z = z0 + nz - 1;
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
    gunion(lat.forest, i, j, lat.sbits, lat.err);
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Block total (fixed order) from each warp's total; valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_combine(T warp_total, T* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = warp_total;
  __syncthreads();
  T r = T(0);
  if (threadIdx.x < 32) {
    r = (lane < kWarps) ? scratch[lane] : T(0);
    r = warp_sum(r);
  }
  return r;
}

// Block sum (fixed order) of one value per thread; valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  return block_combine(warp_sum(v), scratch);
}

// ---------------------------------------------------------------- flip
template <int MODEL, int D>
__global__ void __launch_bounds__(kThreads) k_flip(Lattice lat, uint32_t sweep,
                                                   unsigned long long* nclusters) {
  __shared__ float s_phi;
  __shared__ long long s_red[kWarps];
  if (MODEL == kXY) {
    if (threadIdx.x == 0) s_phi = xy_phi(lat, sweep);
    __syncthreads();
  }
  const int sb = lat.sbits;
  const uint32_t dmask = (1u << sb) - 1u;
  long long roots = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    uint32_t v = lat.forest[i];
    uint32_t r = v >> sb;
    if (r == i) {
      ++roots;
    } else {
      int it = 0;
      for (; it < (1 << 22); ++it) {
        const uint32_t v2 = lat.forest[r];
        const uint32_t r2 = v2 >> sb;
        if (r2 == r) {
          v = v2;
          break;
        }
        r = r2;
      }
      if (it == (1 << 22)) atomicExch(lat.err, kErrTimeout);
    }
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
    const long long tot = block_sum(roots, s_red);
    if (threadIdx.x == 0 && tot) atomicAdd(nclusters, (unsigned long long)tot);
  }
}

// ---------------------------------------------------------------- measurement
template <int MODEL, int D>
__global__ void __launch_bounds__(kThreads) k_measure(Lattice lat, uint32_t sweep, Measure mb) {
  __shared__ unsigned int s_hist[256];
  __shared__ long long s_ri[kWarps];
  __shared__ double s_rd[kWarps];
  __shared__ bool s_last;
  const int L = lat.L;
  if (MODEL == kPotts) {
    for (int k = threadIdx.x; k < lat.q; k += blockDim.x) s_hist[k] = 0;
    __syncthreads();
  }
  long long m = 0, e = 0;
  float fx = 0.f, fy = 0.f, fe = 0.f;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    const uint32_t x = i % L, y = (i / L) % L, z = (D == 3) ? i / ((uint32_t)L * L) : 0u;
    uint32_t jn[3];
    jn[0] = (x + 1 == (uint32_t)L) ? i - x : i + 1u;
    jn[1] = (y + 1 == (uint32_t)L) ? i - y * L : i + (uint32_t)L;
    jn[2] = (D == 3) ? ((z + 1 == (uint32_t)L) ? i - z * L * L : i + (uint32_t)L * L) : 0u;
    if (MODEL == kIsing) {
      const int8_t* s = static_cast<const int8_t*>(lat.spins);
      const int si = s[i];
      int nb = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) nb += s[jn[d]];
      m += si;
      e -= si * nb;
    } else if (MODEL == kPotts) {
      const uint8_t* s = static_cast<const uint8_t*>(lat.spins);
      const uint8_t si = s[i];
      atomicAdd(&s_hist[si], 1u);
#pragma unroll
      for (int d = 0; d < D; ++d) e += (s[jn[d]] != si) ? 1 : 0;
    } else {
      const float* th = static_cast<const float*>(lat.spins);
      const float ti = th[i];
      float sn, cs;
      sincosf(ti, &sn, &cs);
      fx = __fadd_rn(fx, cs);
      fy = __fadd_rn(fy, sn);
#pragma unroll
      for (int d = 0; d < D; ++d) fe = __fsub_rn(fe, cosf(__fsub_rn(ti, th[jn[d]])));
    }
  }
  if (MODEL == kPotts) {
    __syncthreads();
    for (int k = threadIdx.x; k < lat.q; k += blockDim.x)
      if (s_hist[k]) atomicAdd(&mb.hist[k], (unsigned long long)s_hist[k]);
  }
  if (MODEL == kXY) {
    // float within a warp, double across warps and blocks
    const double sx = block_combine((double)warp_sum(fx), s_rd);
    const double sy = block_combine((double)warp_sum(fy), s_rd);
    const double se = block_combine((double)warp_sum(fe), s_rd);
    if (threadIdx.x == 0) {
      mb.part_d[3 * blockIdx.x + 0] = sx;
      mb.part_d[3 * blockIdx.x + 1] = sy;
      mb.part_d[3 * blockIdx.x + 2] = se;
    }
  } else {
    const long long sm = block_sum(m, s_ri);
    const long long se = block_sum(e, s_ri);
    if (threadIdx.x == 0) {
      mb.part_i[2 * blockIdx.x + 0] = sm;
      mb.part_i[2 * blockIdx.x + 1] = se;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(mb.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // last block: fixed-order reduction of the partials, record, accumulators
  long long M = 0, E = 0, S2 = 0;
  double mx = 0.0, my = 0.0, exy = 0.0;
  if (MODEL == kXY) {
    double a = 0.0, c = 0.0, g = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      a = __dadd_rn(a, __ldcg(&mb.part_d[3 * k + 0]));
      c = __dadd_rn(c, __ldcg(&mb.part_d[3 * k + 1]));
      g = __dadd_rn(g, __ldcg(&mb.part_d[3 * k + 2]));
    }
    mx = block_sum(a, s_rd);
    my = block_sum(c, s_rd);
    exy = block_sum(g, s_rd);
  } else {
    long long a = 0, c = 0, g = 0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
      a += __ldcg(&mb.part_i[2 * k + 0]);
      c += __ldcg(&mb.part_i[2 * k + 1]);
    }
    if (MODEL == kPotts) {
      for (int k = threadIdx.x; k < lat.q; k += blockDim.x) {
        const long long n = (long long)__ldcg(&mb.hist[k]);
        g += n * n;
        mb.hist[k] = 0ull;
      }
    }
    M = block_sum(a, s_ri);
    E = block_sum(c, s_ri);
    S2 = block_sum(g, s_ri);
  }
  if (threadIdx.x != 0) return;
  const long long ncl = (long long)__ldcg(mb.nclusters);
  *mb.nclusters = 0ull;
  *mb.ticket = 0u;
  double M2, Ed;
  if (MODEL == kIsing) {
    M2 = __dmul_rn((double)M, (double)M);
    Ed = (double)E;
  } else if (MODEL == kPotts) {
    const long long N = (long long)lat.N;
    M2 = __ddiv_rn((double)((long long)lat.q * S2 - N * N), (double)(lat.q - 1));
    Ed = (double)E;
  } else {
    M2 = __dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my));
    Ed = exy;
  }
  Record* rec = static_cast<Record*>(mb.series) + (sweep % (uint32_t)mb.series_cap);
  rec->sweep = sweep;
  rec->M = M;
  rec->E = E;
  rec->nclusters = ncl;
  rec->S2 = S2;
  rec->mx = mx;
  rec->my = my;
  rec->e_xy = exy;
  rec->M2 = M2;
  rec->Ed = Ed;
  double* acc = mb.acc;
  acc[0] = __dadd_rn(acc[0], 1.0);
  acc[1] = __dadd_rn(acc[1], M2);
  acc[2] = __dadd_rn(acc[2], __dmul_rn(M2, M2));
  acc[3] = __dadd_rn(acc[3], Ed);
  acc[4] = __dadd_rn(acc[4], __dmul_rn(Ed, Ed));
  acc[5] = __dadd_rn(acc[5], (double)ncl);
}

// ---------------------------------------------------------------- labels readout
__global__ void __launch_bounds__(kThreads) k_labels_out(Lattice lat, int32_t* out) {
  const int sb = lat.sbits;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    uint32_t r = lat.forest[i] >> sb;
    int it = 0;
    for (; it < (1 << 22); ++it) {
      const uint32_t r2 = lat.forest[r] >> sb;
      if (r2 == r) break;
      r = r2;
    }
    if (it == (1 << 22)) atomicExch(lat.err, kErrTimeout);
    out[i] = (int32_t)r;
  }
}

unsigned grid_for(uint32_t n, unsigned cap) {
  const unsigned g = (unsigned)((n + kThreads - 1) / kThreads);
  return g < cap ? (g ? g : 1u) : cap;
}

}  // namespace

void tiles_for(int dim, int L, int* ntx, int* nty, int* ntz) {
  *ntx = (L + 31) / 32;
  if (dim == 2) {
    *nty = (L + kTileY2 - 1) / kTileY2;
    *ntz = 1;
  } else {
    *nty = (L + kTileY3 - 1) / kTileY3;
    *ntz = (L + kTileZ3 - 1) / kTileZ3;
  }
}

cudaError_t launch_init(const Lattice& lat, int model, cudaStream_t st) {
  const unsigned g = grid_for(lat.N, 4096);
  if (model == kIsing) k_init<kIsing><<<g, kThreads, 0, st>>>(lat);
  else if (model == kPotts) k_init<kPotts><<<g, kThreads, 0, st>>>(lat);
  else k_init<kXY><<<g, kThreads, 0, st>>>(lat);
  return cudaGetLastError();
}

template <int MODEL, int D>
static void bond_label_md(const Lattice& lat, uint32_t sweep, bool from_mask, unsigned g,
                          cudaStream_t st) {
  if (from_mask) k_bond_label<MODEL, D, true><<<g, kThreads, 0, st>>>(lat, sweep);
  else k_bond_label<MODEL, D, false><<<g, kThreads, 0, st>>>(lat, sweep);
}

cudaError_t launch_bond_label(const Lattice& lat, int model, uint32_t sweep, bool from_mask,
                              cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  if (from_mask) model = kIsing;  // the mask path reads no spins
  if (lat.dim == 2) {
    if (model == kIsing) bond_label_md<kIsing, 2>(lat, sweep, from_mask, g, st);
    else if (model == kPotts) bond_label_md<kPotts, 2>(lat, sweep, from_mask, g, st);
    else bond_label_md<kXY, 2>(lat, sweep, from_mask, g, st);
  } else {
    if (model == kIsing) bond_label_md<kIsing, 3>(lat, sweep, from_mask, g, st);
    else if (model == kPotts) bond_label_md<kPotts, 3>(lat, sweep, from_mask, g, st);
    else bond_label_md<kXY, 3>(lat, sweep, from_mask, g, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_merge(const Lattice& lat, cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  if (lat.dim == 2) k_merge<2><<<g, kThreads, 0, st>>>(lat);
  else k_merge<3><<<g, kThreads, 0, st>>>(lat);
  return cudaGetLastError();
}

cudaError_t launch_flip(const Lattice& lat, int model, uint32_t sweep,
                        unsigned long long* nclusters, cudaStream_t st) {
  const unsigned g = grid_for(lat.N, kFlipBlocks);
  if (lat.dim == 2) {
    if (model == kIsing) k_flip<kIsing, 2><<<g, kThreads, 0, st>>>(lat, sweep, nclusters);
    else if (model == kPotts) k_flip<kPotts, 2><<<g, kThreads, 0, st>>>(lat, sweep, nclusters);
    else k_flip<kXY, 2><<<g, kThreads, 0, st>>>(lat, sweep, nclusters);
  } else {
    if (model == kIsing) k_flip<kIsing, 3><<<g, kThreads, 0, st>>>(lat, sweep, nclusters);
    else if (model == kPotts) k_flip<kPotts, 3><<<g, kThreads, 0, st>>>(lat, sweep, nclusters);
    else k_flip<kXY, 3><<<g, kThreads, 0, st>>>(lat, sweep, nclusters);
  }
  return cudaGetLastError();
}

cudaError_t launch_measure(const Lattice& lat, int model, uint32_t sweep, const Measure& m,
                           cudaStream_t st) {
  const unsigned g = grid_for(lat.N, kMeasureBlocks);
  if (lat.dim == 2) {
    if (model == kIsing) k_measure<kIsing, 2><<<g, kThreads, 0, st>>>(lat, sweep, m);
    else if (model == kPotts) k_measure<kPotts, 2><<<g, kThreads, 0, st>>>(lat, sweep, m);
    else k_measure<kXY, 2><<<g, kThreads, 0, st>>>(lat, sweep, m);
  } else {
    if (model == kIsing) k_measure<kIsing, 3><<<g, kThreads, 0, st>>>(lat, sweep, m);
    else if (model == kPotts) k_measure<kPotts, 3><<<g, kThreads, 0, st>>>(lat, sweep, m);
    else k_measure<kXY, 3><<<g, kThreads, 0, st>>>(lat, sweep, m);
  }
  return cudaGetLastError();
}

cudaError_t launch_labels_out(const Lattice& lat, int32_t* out, cudaStream_t st) {
  k_labels_out<<<grid_for(lat.N, 4096), kThreads, 0, st>>>(lat, out);
  return cudaGetLastError();
}

}  // namespace swgb
