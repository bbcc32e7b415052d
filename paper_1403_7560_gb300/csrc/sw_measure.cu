// Initial state and the measurement of a sweep (Komura & Okabe, Sec. 2:
// magnetization M, the energy of the Hamiltonian, the Potts M^2 equation;
// Sec. 3: the moments entering U = <M^4>/<M^2>^2).
//
// k_measure: one warp per lattice row (grid-stride), lane per site; the
//   clock model's fixed-point cos / sin sums added to the measurement
//   slots, or float XY per-block partials (Ising/Potts states are measured
//   by a thread per row word, k_measure_rows in sw_label.cu).
// k_finalize (after k_measure): one block sums slots / partials in a fixed
//   order, writes the sweep record and adds M2, M2^2, E, E^2 and the cluster count to the FP64
//   accumulators (explicit round-to-nearest operations, no contraction).
#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

template <int MODEL>
__global__ void __launch_bounds__(256) k_init(const __grid_constant__ Lattice lat) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lat.N; i += gridDim.x * blockDim.x) {
    const uint32_t w = philox(i, 0u, kInit, 0u, lat.rk).x;
    if (MODEL == kIsing) {
      static_cast<int8_t*>(lat.spins)[i] = (w >> 31) ? (int8_t)-1 : (int8_t)1;
    } else if (MODEL == kPotts) {
      static_cast<uint8_t*>(lat.spins)[i] = (uint8_t)draw_value(w, (uint32_t)lat.q);
    } else if (MODEL == kClock) {
      static_cast<uint16_t*>(lat.spins)[i] = (uint16_t)draw_value(w, (uint32_t)lat.q);
    } else {
      static_cast<float*>(lat.spins)[i] = __fmul_rn((float)(w >> 8), 0x1.921fb6p-22f);
    }
  }
}

constexpr int kMThreads = 256, kMWarps = kMThreads / 32;

// XY and clock states (Ising/Potts: k_measure_rows in sw_label.cu).
template <int MODEL, int D>
__global__ void __launch_bounds__(kMThreads) k_measure(Lattice lat, uint32_t sweep, Measure mb) {
  static_assert(MODEL == kXY || MODEL == kClock, "row-word kernel for Ising/Potts");
  __shared__ long long s_ri[kMWarps];
  __shared__ double s_rd[kMWarps];
  const int L = lat.L, lane = threadIdx.x & 31;
  long long m = 0, e = 0, cb = 0;
  float fx = 0.f, fy = 0.f, fe = 0.f;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  // one warp per lattice row (y, z); the row's words are walked in order
  for (uint32_t row = gw; row < lat.R; row += nw) {
    const uint32_t y = row % (uint32_t)L, z = row / (uint32_t)L;
    const uint32_t rowL = row * (uint32_t)L;
    const uint32_t dy = (y + 1 == (uint32_t)L) ? 0u - y * L : (uint32_t)L;
    const uint32_t dz = (D == 3) ? ((z + 1 == (uint32_t)L) ? 0u - z * L * L : (uint32_t)L * L) : 0u;
#pragma unroll 4
    for (int x = lane; x < L; x += 32) {
      const uint32_t i = rowL + (uint32_t)x;
      uint32_t jn[3];
      jn[0] = (x + 1 == L) ? rowL : i + 1u;
      jn[1] = i + dy;
      jn[2] = i + dz;
      if (MODEL == kClock) {
        // fixed-point sums: C[p_i], S[p_i] and C[(p_i - p_j) mod q]
        const uint16_t* sp = static_cast<const uint16_t*>(lat.spins);
        const int q = lat.q;
        const int pi = clock_state(sp[i], q);
        m += __ldg(&mb.cfix[pi]);
        e += __ldg(&mb.cfix[q + pi]);
#pragma unroll
        for (int d = 0; d < D; ++d) cb += __ldg(&mb.cfix[wrap_mod(pi - clock_state(sp[jn[d]], q), q)]);
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
  }
  if (MODEL == kClock) {
    add_clock_sums<kMWarps>(mb, blockIdx.x, m, e, cb, s_ri);
    return;
  }
  // XY: float within a warp, double across warps; per-block partials are
  // reduced in a fixed order by the finalising block
  const double sx = block_combine<kMWarps>((double)warp_sum(fx), s_rd);
  const double sy = block_combine<kMWarps>((double)warp_sum(fy), s_rd);
  const double se = block_combine<kMWarps>((double)warp_sum(fe), s_rd);
  if (threadIdx.x == 0) {
    mb.part_d[3 * blockIdx.x + 0] = sx;
    mb.part_d[3 * blockIdx.x + 1] = sy;
    mb.part_d[3 * blockIdx.x + 2] = se;
  }
}

__global__ void __launch_bounds__(kMThreads) k_finalize(Lattice lat, uint32_t sweep, Measure mb) {
  __shared__ long long s_ri[kMWarps];
  __shared__ double s_rd[kMWarps];
  finalize_record<kMWarps>(lat, mb, sweep, s_ri, s_rd);
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
  else if (model == kClock) k_init<kClock><<<g, 256, 0, st>>>(lat);
  else k_init<kXY><<<g, 256, 0, st>>>(lat);
  return cudaGetLastError();
}

cudaError_t launch_measure(const Lattice& lat, int model, uint32_t sweep, const Measure& m,
                           cudaStream_t st) {
  const unsigned g = grid_for(lat.R, kMeasureBlocks);
  if (model == kIsing || model == kPotts) return launch_measure_rows(lat, sweep, m, st);  // finalises itself
  if (lat.dim == 2) {
    if (model == kClock) k_measure<kClock, 2><<<g, kMThreads, 0, st>>>(lat, sweep, m);
    else k_measure<kXY, 2><<<g, kMThreads, 0, st>>>(lat, sweep, m);
  } else {
    if (model == kClock) k_measure<kClock, 3><<<g, kMThreads, 0, st>>>(lat, sweep, m);
    else k_measure<kXY, 3><<<g, kMThreads, 0, st>>>(lat, sweep, m);
  }
  Measure mf = m;
  mf.xy_blocks = (int)g;
  k_finalize<<<1, kMThreads, 0, st>>>(lat, sweep, mf);
  return cudaGetLastError();
}

}  // namespace swgb
