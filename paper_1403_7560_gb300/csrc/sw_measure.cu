// Initial state and the measurement of a sweep (Komura & Okabe, Sec. 2:
// magnetization M, the energy of the Hamiltonian, the Potts M^2 equation;
// Sec. 3: the moments entering U = <M^4>/<M^2>^2).
//
// k_measure: one warp per 32-site row word (grid-stride), lane per site;
//   integer M / E / Potts histogram (warp-aggregated shared atomics) or
//   float XY sums; per-block partials; the last block to finish reduces the
//   partials in a fixed order, writes the sweep record and adds M2, M2^2, E,
//   E^2 and the cluster count to the FP64 accumulators (explicit
//   round-to-nearest operations, no contraction).
#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

template <int MODEL>
__global__ void __launch_bounds__(256) k_init(Lattice lat) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    const uint32_t w = philox(i, 0u, kInit, 0u, lat.key0, lat.key1).x;
    if (MODEL == kIsing) {
      static_cast<int8_t*>(lat.spins)[i] = (w >> 31) ? (int8_t)-1 : (int8_t)1;
    } else if (MODEL == kPotts) {
      static_cast<uint8_t*>(lat.spins)[i] = (uint8_t)draw_value(w, (uint32_t)lat.q);
    } else {
      static_cast<float*>(lat.spins)[i] = __fmul_rn((float)(w >> 8), 0x1.921fb6p-22f);
    }
  }
}

constexpr int kMThreads = 256, kMWarps = kMThreads / 32;

template <int MODEL, int D>
__global__ void __launch_bounds__(kMThreads) k_measure(Lattice lat, uint32_t sweep, Measure mb) {
  __shared__ unsigned int s_hist[256];
  __shared__ long long s_ri[kMWarps];
  __shared__ double s_rd[kMWarps];
  __shared__ bool s_last;
  const int L = lat.L, lane = threadIdx.x & 31;
  if (MODEL == kPotts) {
    for (int k = threadIdx.x; k < lat.q; k += blockDim.x) s_hist[k] = 0u;
    __syncthreads();
  }
  long long m = 0, e = 0;
  float fx = 0.f, fy = 0.f, fe = 0.f;
  const uint32_t nwords = lat.R * (uint32_t)lat.W;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = gw; g < nwords; g += nw) {
    const uint32_t row = g / (uint32_t)lat.W, xw = g % (uint32_t)lat.W;
    const uint32_t y = row % (uint32_t)L, z = row / (uint32_t)L;
    const int x = (int)(32 * xw) + lane;
    const bool valid = x < L;
    const uint32_t i = (uint32_t)min(x, L - 1) + (uint32_t)L * row;
    uint32_t jn[3];
    jn[0] = (x + 1 >= L) ? i - (uint32_t)min(x, L - 1) : i + 1u;
    jn[1] = (y + 1 == (uint32_t)L) ? i - y * L : i + (uint32_t)L;
    jn[2] = (D == 3) ? ((z + 1 == (uint32_t)L) ? i - z * L * L : i + (uint32_t)L * L) : 0u;
    if (MODEL == kIsing) {
      const int8_t* s = static_cast<const int8_t*>(lat.spins);
      if (valid) {
        const int si = s[i];
        int nb = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) nb += s[jn[d]];
        m += si;
        e -= si * nb;
      }
    } else if (MODEL == kPotts) {
      const uint8_t* s = static_cast<const uint8_t*>(lat.spins);
      const uint32_t si = valid ? s[i] : 0xffffffffu;
      if (valid) {
#pragma unroll
        for (int d = 0; d < D; ++d) e += (s[jn[d]] != si) ? 1 : 0;
      }
      const unsigned grp = __match_any_sync(kFull, si);
      if (valid && lane == __ffs(grp) - 1) atomicAdd(&s_hist[si], (unsigned)__popc(grp));
    } else if (valid) {
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
    const double sx = block_combine<kMWarps>((double)warp_sum(fx), s_rd);
    const double sy = block_combine<kMWarps>((double)warp_sum(fy), s_rd);
    const double se = block_combine<kMWarps>((double)warp_sum(fe), s_rd);
    if (threadIdx.x == 0) {
      mb.part_d[3 * blockIdx.x + 0] = sx;
      mb.part_d[3 * blockIdx.x + 1] = sy;
      mb.part_d[3 * blockIdx.x + 2] = se;
    }
  } else {
    const long long sm = block_combine<kMWarps>(warp_sum(m), s_ri);
    const long long se = block_combine<kMWarps>(warp_sum(e), s_ri);
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
    mx = block_combine<kMWarps>(warp_sum(a), s_rd);
    my = block_combine<kMWarps>(warp_sum(c), s_rd);
    exy = block_combine<kMWarps>(warp_sum(g), s_rd);
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
    M = block_combine<kMWarps>(warp_sum(a), s_ri);
    E = block_combine<kMWarps>(warp_sum(c), s_ri);
    S2 = block_combine<kMWarps>(warp_sum(g), s_ri);
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

unsigned grid_for(uint32_t n_warps_work, unsigned cap) {
  const unsigned g = (n_warps_work + kMWarps - 1) / kMWarps;
  return g < cap ? (g ? g : 1u) : cap;
}

}  // namespace

cudaError_t launch_init(const Lattice& lat, int model, cudaStream_t st) {
  unsigned g = (lat.N + 255u) / 256u;
  if (g > 4096u) g = 4096u;
  if (model == kIsing) k_init<kIsing><<<g, 256, 0, st>>>(lat);
  else if (model == kPotts) k_init<kPotts><<<g, 256, 0, st>>>(lat);
  else k_init<kXY><<<g, 256, 0, st>>>(lat);
  return cudaGetLastError();
}

cudaError_t launch_measure(const Lattice& lat, int model, uint32_t sweep, const Measure& m,
                           cudaStream_t st) {
  const unsigned g = grid_for(lat.R * (uint32_t)lat.W, kMeasureBlocks);
  if (lat.dim == 2) {
    if (model == kIsing) k_measure<kIsing, 2><<<g, kMThreads, 0, st>>>(lat, sweep, m);
    else if (model == kPotts) k_measure<kPotts, 2><<<g, kMThreads, 0, st>>>(lat, sweep, m);
    else k_measure<kXY, 2><<<g, kMThreads, 0, st>>>(lat, sweep, m);
  } else {
    if (model == kIsing) k_measure<kIsing, 3><<<g, kMThreads, 0, st>>>(lat, sweep, m);
    else if (model == kPotts) k_measure<kPotts, 3><<<g, kMThreads, 0, st>>>(lat, sweep, m);
    else k_measure<kXY, 3><<<g, kMThreads, 0, st>>>(lat, sweep, m);
  }
  return cudaGetLastError();
}

}  // namespace swgb
