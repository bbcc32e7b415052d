// Small Ising/Potts lattices (N <= small_sites_limit: 2D 8192, 3D 4096):
// whole sweeps by one CTA with the lattice in shared memory, n sweeps per
// launch.
//
// The tiled path pays four kernel launches and a global merge per sweep,
// which for a lattice of a few thousand sites is nearly all of the time.
// Here one CTA of 1024 threads keeps the spins, the bond planes and a
// union-find forest over every site in shared memory and loops over the
// sweeps: step (1) bonds with the same bit-sliced Philox words as the tiled
// path (equality masks by warp ballots, a thread per row word and
// direction for the Bernoulli words), step (2) the union-find of the tiled
// path over the whole periodic lattice (every site's parent is its x-run
// start, then threads per row word, one per range of its bits, join the
// runs bonded to the +y / +z rows, one of them also the run bonded to the
// next row word; the smallest index becomes the root, so labels are
// canonical), step (3) every site takes its root's draw (the same draw
// definitions), and the new state is measured into the same per-sweep
// record and FP64 accumulators.  After the last sweep the spins, that
// sweep's bond planes and a forest of (root, marker, draw) words are
// written back, so every readout call sees the same state as after tiled
// sweeps.  The whole lattice is on one SM, so every phase's slowest thread
// holds the others at the next barrier: the unions are split for that.
#include <string>

#include "../../include/sw.h"
#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

constexpr int kSmallThreads = 1024, kSmallWarps = kSmallThreads / 32;

struct SmallLayout {
  size_t par, planes, draws, starts, spins, pdraw, total;
};

__host__ __device__ SmallLayout small_layout(const Lattice& lat, bool potts) {
  const size_t rw = (size_t)lat.R * (size_t)lat.W;
  SmallLayout s;
  s.par = 0;
  s.planes = s.par + 4 * (size_t)lat.N;
  s.draws = s.planes + 4 * (size_t)lat.dim * rw;
  s.starts = s.draws + 4 * rw;
  s.spins = s.starts + 4 * rw;
  s.pdraw = s.spins + (size_t)lat.N;
  s.total = s.pdraw + (potts ? (size_t)lat.N : 0);
  s.total = (s.total + 15) & ~(size_t)15;
  return s;
}

// Shared memory of a small sweep besides the dynamic lattice block.
struct SmallScratch {
  long long s_ri[4 * kSmallWarps];  // per-warp partials of the record's four sums
  unsigned int s_hist[256];
  double s_acc[6];  // the FP64 accumulators, written back at the end
};

// Division by an invariant divisor d (Granlund & Montgomery, "Division by
// invariant integers using multiplication", 1994): with m = floor((2^32 -
// 1) / d) + 1, floor(n / d) = umulhi(n, m) whenever n * d < 2^32 (the
// product overshoots n / d by less than n / 2^32 < 1 / d, which cannot
// carry the quotient past the next integer); d = 1 takes n itself.  The
// small lattices' indices (n <= 3 N, d <= N, N <= 8192) are far inside.
struct InvDiv {
  uint32_t d, m;
  __device__ explicit InvDiv(uint32_t dv) : d(dv), m(dv > 1u ? 0xffffffffu / dv + 1u : 0u) {}
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return d > 1u ? __umulhi(n, m) : n; }
  __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};

// n sweeps after sweep0 of one small lattice by the whole CTA.
template <int D, bool POTTS>
__device__ __forceinline__ void sweep_small(const Lattice& lat, const Measure& mb, uint32_t sweep0, int n,
                                            bool measure, const SmallLayout& lay, unsigned char* smem,
                                            SmallScratch& sc) {
  long long* s_ri = sc.s_ri;
  unsigned int* s_hist = sc.s_hist;
  double* s_acc = sc.s_acc;
  uint32_t* par = reinterpret_cast<uint32_t*>(smem + lay.par);
  uint32_t* pl = reinterpret_cast<uint32_t*>(smem + lay.planes);
  uint32_t* dw = reinterpret_cast<uint32_t*>(smem + lay.draws);
  uint32_t* ss = reinterpret_cast<uint32_t*>(smem + lay.starts);  // x-run starts of each row word
  uint8_t* sp = smem + lay.spins;
  uint8_t* pd = smem + lay.pdraw;
  const uint32_t N = lat.N, L = (uint32_t)lat.L, W = (uint32_t)lat.W, RW = lat.R * W;
  const InvDiv byL(L), byW(W), byRW(RW);
  // the unions of a row word are split by bit range over 2^segsh threads:
  // the largest power of two up to 16 whose threads for all row words stay
  // within about one CTA (a thread then walks at most 32 >> segsh unions
  // of a row word, instead of all of them)
  uint32_t segsh = 0;
  while (segsh < 4u && (RW << (segsh + 1u)) <= kSmallThreads + kSmallThreads / 8u) ++segsh;
  const uint32_t segb = 32u >> segsh, segbits = segb == 32u ? kFull : (1u << segb) - 1u;
  const uint32_t tid = threadIdx.x;
  const int q = lat.q, sb = lat.sbits, shift = sb + 1;
  const bool two_state = lat.dq == 2;
  const uint32_t lr_bit = 1u << sb;
  const uint8_t* gs = static_cast<const uint8_t*>(lat.spins);
  for (uint32_t i = tid; i < N; i += kSmallThreads) sp[i] = gs[i];
  if (tid < 6) s_acc[tid] = mb.acc[tid];
  const uint32_t lane = tid & 31u, warp = tid >> 5;

  for (int s = 0; s < n; ++s) {
    const uint32_t sweep = sweep0 + (uint32_t)s + 1u;
    const bool last = s + 1 == n;
    __syncthreads();
    // step (1a): equality masks, a warp per row word (lane per site, ballots)
    for (uint32_t g = warp; g < RW; g += kSmallWarps) {
      const uint32_t row = byW.div(g), x = 32u * (g - row * W) + lane;
      const uint32_t z = byL.div(row), y = row - z * L;
      bool q0 = false, q1 = false, q2 = false;
      if (x < L) {
        const uint8_t si = sp[row * L + x];
        q0 = sp[row * L + (x + 1u == L ? 0u : x + 1u)] == si;
        q1 = sp[((y + 1u == L ? 0u : y + 1u) + L * z) * L + x] == si;
        if (D == 3) q2 = sp[(y + L * (z + 1u == L ? 0u : z + 1u)) * L + x] == si;
      }
      const uint32_t b0 = __ballot_sync(kFull, q0), b1 = __ballot_sync(kFull, q1), b2 = __ballot_sync(kFull, q2);
      if (lane < (uint32_t)D) pl[lane * RW + g] = lane == 0 ? b0 : lane == 1 ? b1 : b2;
    }
    __syncthreads();
    // step (1b): Bernoulli words, a thread per (row word, direction); the
    // two-state draw words
    for (uint32_t c = tid; c < (uint32_t)D * RW; c += kSmallThreads) {
      const uint32_t d = byRW.div(c), g = c - d * RW;
      const uint32_t e = pl[c];
      pl[c] = e ? (e & bernoulli_word(g, sweep, (int)d, lat.t_bond, e, lat.rk)) : 0u;
    }
    if (two_state)
      for (uint32_t g = tid; g < RW; g += kSmallThreads) dw[g] = philox(g, sweep, kDraw, 1u, lat.rk).x;
    if (POTTS && !two_state) {
      // Potts draw of every site: word (i & 3) of Philox(i >> 2, sweep, DRAW, 0)
      for (uint32_t c = tid; 4u * c < N; c += kSmallThreads) {
        const uint4 w = philox(c, sweep, kDraw, 0u, lat.rk);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4u * c + (uint32_t)k < N) pd[4u * c + (uint32_t)k] = (uint8_t)draw_value(word_of(w, k), (uint32_t)lat.dq);
      }
    }
    __syncthreads();
    // step (2a): every site's parent is the start of its x-run inside its
    // row word (a warp per row word, lane per site)
    for (uint32_t g = warp; g < RW; g += kSmallWarps) {
      const uint32_t row = byW.div(g), x0 = 32u * (g - row * W);
      const int nvalid = (int)min(32u, L - x0);
      const uint32_t vmask = nvalid >= 32 ? kFull : ((1u << nvalid) - 1u);
      const uint32_t S = ~((pl[g] & (vmask >> 1)) << 1) & vmask;
      if (lane == 0) ss[g] = S;
      if ((int)lane < nvalid) par[row * L + x0 + lane] = row * L + x0 + run_start(S, (int)lane);
    }
    __syncthreads();
    // step (2b): threads per row word (one per bit range) join the runs
    // bonded to the +y row and to the +z row; runs already joined through
    // the previous bit are skipped; the last range's thread also joins the
    // run bonded to the next row word along x (or around)
    for (uint32_t c = tid; c < (RW << segsh); c += kSmallThreads) {
      const uint32_t g = c >> segsh, seg = c & ((1u << segsh) - 1u);
      const uint32_t segmask = segbits << (segb * seg);
      const uint32_t row = byW.div(g), xw = g - row * W, x0 = 32u * xw;
      const uint32_t z = byL.div(row), y = row - z * L;
      const int nvalid = (int)min(32u, L - x0);
      const uint32_t vmask = nvalid >= 32 ? kFull : ((1u << nvalid) - 1u);
      const uint32_t A0 = pl[g], X = A0 & (vmask >> 1), S = ss[g], base = row * L + x0;
      if (seg == (1u << segsh) - 1u && ((A0 >> (nvalid - 1)) & 1u)) {
        const uint32_t i = base + (uint32_t)(nvalid - 1);
        sunion(par, base + run_start(S, nvalid - 1), x0 + (uint32_t)nvalid == L ? row * L : i + 1u, lat.err,
               lat.cap);
      }
#pragma unroll
      for (int d = 1; d < D; ++d) {
        const uint32_t rown = (d == 1) ? (y + 1u == L ? 0u : y + 1u) + L * z
                                       : y + L * (z + 1u == L ? 0u : z + 1u);
        const uint32_t gn = rown * W + xw, Yd = pl[d * RW + g];
        if (!Yd) continue;
        const uint32_t Xn = pl[gn] & (vmask >> 1), Sn = ss[gn], basen = rown * L + x0;
        uint32_t U = Yd & ~((Yd & X & Xn) << 1) & segmask;
        while (U) {
          const int b = __ffs(U) - 1;
          U &= U - 1u;
          sunion(par, base + run_start(S, b), basen + run_start(Sn, b), lat.err, lat.cap);
        }
      }
    }
    __syncthreads();
    // step (3): every site takes its root's draw; roots counted
    long long roots = 0;
    for (uint32_t g = warp; g < RW; g += kSmallWarps) {
      const uint32_t row = byW.div(g), x = 32u * (g - row * W) + lane;
      if (x >= L) continue;
      const uint32_t i = row * L + x;
      const uint32_t r = sfind(par, i);
      if (r == i) ++roots;
      const uint32_t rr = byL.div(r), xr = r - rr * L, gr = rr * W + (xr >> 5);
      const uint32_t v = two_state ? (dw[gr] >> (xr & 31u)) & 1u : pd[r];
      sp[i] = POTTS ? (uint8_t)v : (uint8_t)(v ? (int8_t)-1 : (int8_t)1);
      if (last) {
        const uint32_t own = two_state ? (dw[g] >> lane) & 1u : pd[i];
        lat.forest[i] = (r << shift) | (r == i ? lr_bit : 0u) | own;
      }
    }
    if (!measure) continue;
    // the new state's record: M, E (Potts: E and the histogram), roots
    if (POTTS) {
      __syncthreads();
      for (int k = tid; k < 256; k += kSmallThreads) s_hist[k] = 0u;
    }
    __syncthreads();
    long long m = 0, en = 0;
    for (uint32_t g = warp; g < RW; g += kSmallWarps) {
      const uint32_t row = byW.div(g), x = 32u * (g - row * W) + lane;
      if (x >= L) continue;
      const uint32_t z = byL.div(row), y = row - z * L, i = row * L + x;
      uint32_t j[3];
      j[0] = x + 1u == L ? i - x : i + 1u;
      j[1] = y + 1u == L ? i - y * L : i + L;
      j[2] = (D == 3) ? (z + 1u == L ? i - z * L * L : i + L * L) : i;
      if (POTTS) {
        const uint32_t si = sp[i];
        atomicAdd(&s_hist[si], 1u);
#pragma unroll
        for (int d = 0; d < D; ++d) en += sp[j[d]] != si;
      } else {
        const int si = (int8_t)sp[i];
        m += si;
#pragma unroll
        for (int d = 0; d < D; ++d) en -= si * (int)(int8_t)sp[j[d]];
      }
    }
    long long s2 = 0;
    if (POTTS) {
      __syncthreads();
      if (tid < (uint32_t)q) s2 = (long long)s_hist[tid] * (long long)s_hist[tid];
    }
    // the four sums in one block reduction (two barriers instead of eight:
    // the whole lattice is on one SM, so every barrier is on the critical path)
    const long long part[4] = {warp_sum(m), warp_sum(en), warp_sum(s2), warp_sum(roots)};
    __syncthreads();
    if (lane == 0)
      for (int k = 0; k < 4; ++k) s_ri[k * kSmallWarps + warp] = part[k];
    __syncthreads();
    if (warp == 0) {
      long long tot[4];
      for (int k = 0; k < 4; ++k) tot[k] = warp_sum(s_ri[k * kSmallWarps + lane]);
      if (lane == 0) write_record(lat, mb, sweep, tot[0], tot[1], tot[2], 0.0, 0.0, 0.0, tot[3], s_acc);
    }
  }
  __syncthreads();
  uint8_t* out = static_cast<uint8_t*>(lat.spins);
  for (uint32_t i = tid; i < N; i += kSmallThreads) out[i] = sp[i];
  for (uint32_t w = tid; w < (uint32_t)D * RW; w += kSmallThreads) lat.planes[w] = pl[w];
  if (tid < 6) mb.acc[tid] = s_acc[tid];
}

template <int D, bool POTTS>
__global__ void __launch_bounds__(kSmallThreads, 1)
    k_sweep_small(const __grid_constant__ Lattice lat, const __grid_constant__ Measure mb, uint32_t sweep0,
                  int n, int measure, SmallLayout lay) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SmallScratch sc;
  sweep_small<D, POTTS>(lat, mb, sweep0, n, measure != 0, lay, smem, sc);
}

// Small members of a batch, one CTA per member (list[blockIdx.x]), one
// measured sweep per launch: sweep number from the batch step counter; a
// member stops after its own number of sweeps.
template <int D, bool POTTS>
__global__ void __launch_bounds__(kSmallThreads, 1) k_sweep_small_batch(BatchView bv, const uint32_t* list) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SmallScratch sc;
  __shared__ Lattice s_lat;  // read on every Philox round
  static_assert(sizeof(Lattice) % 4 == 0 && sizeof(Lattice) / 4 <= kSmallThreads, "lattice copy");
  const BatchMember& m = bv.members[__ldg(&list[blockIdx.x])];
  if (*bv.step >= m.nsweeps) return;  // the member has had its sweeps this call
  if (threadIdx.x < sizeof(Lattice) / 4)
    reinterpret_cast<uint32_t*>(&s_lat)[threadIdx.x] = reinterpret_cast<const uint32_t*>(&m.lat)[threadIdx.x];
  __syncthreads();
  const SmallLayout lay = small_layout(s_lat, POTTS);
  sweep_small<D, POTTS>(s_lat, m.meas, m.sweep0 + *bv.step, 1, true, lay, smem, sc);
}

template <int D, bool POTTS>
cudaError_t launch_small_t(const Lattice& lat, const Measure& m, uint32_t sweep0, int n, bool measure,
                           cudaStream_t st) {
  const SmallLayout lay = small_layout(lat, POTTS);
  static thread_local int configured_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device != dev) {
    e = cudaFuncSetAttribute(k_sweep_small<D, POTTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)small_layout_bytes_max());
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  k_sweep_small<D, POTTS><<<1, kSmallThreads, lay.total, st>>>(lat, m, sweep0, n, measure ? 1 : 0, lay);
  return cudaGetLastError();
}

}  // namespace

size_t small_layout_bytes_max() {
  // N <= kSmallSites, bond planes of at most N / 8 words per direction
  // beyond N / 32 (rows padded to words), and Potts draws
  return (size_t)kSmallSites * 4 + 3 * 4 * (size_t)kSmallSites / 4 + 4 * (size_t)kSmallSites / 4 +
         2 * (size_t)kSmallSites + 16;
}

uint32_t small_sites_limit(int model, int dim) {
  // measured on the GB300 against the tiled path (with its overlapped
  // launches), us per sweep at T_c over back-to-back sweeps: 2D Ising L = 80:
  // 18.8 here, 28.6 tiled; L = 90: 26.8 here, 30.1 tiled; 3D Ising L = 12:
  // 20.4 here, 23.1 tiled; L = 16: 24.3 here, 27.7 tiled; L = 20: 36.4 here,
  // 33.2 tiled; 3D Potts q = 3 L = 16: 26.5 here, 31.7 tiled; L = 20: 40.3
  // here, 37.4 tiled.  2D: the layout's whole capacity.
  (void)model;
  return dim == 2 ? (uint32_t)kSmallSites : 4096u;
}

bool small_lattice(const Lattice& lat) {
  if (lat.model != kIsing && lat.model != kPotts) return false;
  if (lat.N > small_sites_limit(lat.model, lat.dim)) return false;
  return small_layout(lat, lat.model == kPotts).total <= small_layout_bytes_max();
}

cudaError_t prepare_small_batch() {
  const int bytes = (int)small_layout_bytes_max();
  cudaError_t e = cudaFuncSetAttribute(k_sweep_small_batch<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweep_small_batch<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweep_small_batch<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweep_small_batch<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_small_batch(const BatchView& bv, int dim, const uint32_t* ising_list, uint32_t n_ising,
                               const uint32_t* potts_list, uint32_t n_potts, cudaStream_t st) {
  const size_t bytes = small_layout_bytes_max();
  if (n_ising) {
    if (dim == 2) k_sweep_small_batch<2, false><<<n_ising, kSmallThreads, bytes, st>>>(bv, ising_list);
    else k_sweep_small_batch<3, false><<<n_ising, kSmallThreads, bytes, st>>>(bv, ising_list);
  }
  if (n_potts) {
    if (dim == 2) k_sweep_small_batch<2, true><<<n_potts, kSmallThreads, bytes, st>>>(bv, potts_list);
    else k_sweep_small_batch<3, true><<<n_potts, kSmallThreads, bytes, st>>>(bv, potts_list);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweeps_small(const Lattice& lat, const Measure& m, uint32_t sweep0, int n, bool measure,
                                cudaStream_t st) {
  const bool potts = lat.model == kPotts;
  if (lat.dim == 2) return potts ? launch_small_t<2, true>(lat, m, sweep0, n, measure, st)
                                 : launch_small_t<2, false>(lat, m, sweep0, n, measure, st);
  return potts ? launch_small_t<3, true>(lat, m, sweep0, n, measure, st)
               : launch_small_t<3, false>(lat, m, sweep0, n, measure, st);
}

}  // namespace swgb
