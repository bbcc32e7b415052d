// Steps (1) and (2) of the SW sweep (Komura & Okabe, Sec. 2): active bond
// generation and the tile-local half of the cluster labeling.
//
// k_label: one CTA per 32 x TY (x TZ) tile, one thread per 32-site row word.
//   phase 1 (thread per row word): Ising/Potts bonds from the int8/uint8
//     spins -- equality of the row with its +x/+y/+z neighbour rows from
//     byte-lane compares, AND a bit-sliced Bernoulli word per direction
//     (u < t decided for 32 sites at once from whole Philox words) -- and
//     the row's cluster draws (one Philox word per row word for two-state
//     draws, one per four sites for Potts); or the bonds read from the
//     bit-planes.
//   Before it, every site is its own parent in the shared-memory forest; an
//   x-run is represented by its start, the only site of it ever looked up.
//   phase 2 (thread per row word): one shared-memory union per pair of runs
//     joined by +y / +z bonds inside the tile (runs already joined through
//     the previous bit are skipped).
//   phase 3 (lane per site): find the tile-local root of the site's run
//     start and write the forest word (root as a global index, local-root
//     marker, cluster draw).
//   With MEASURE the row threads also measure the incoming spins (the state
//   after the previous sweep) from the same bytes and equality masks.
// k_bonds_xy: XY bonds: project on the sweep's mirror axis (once per site,
//   through a shared-memory block with halo) and test the embedded-Ising
//   probability; ballot into the bit-planes; optionally measure the
//   incoming state from the same projections.
#include "sw_device.cuh"

namespace swgb {
namespace {

using namespace dev;

constexpr int kSmallQ = 16;  // Potts histograms up to this q are counted per thread

// The 32 spin bytes of a row word and of its +x, +y, +z neighbour words.
struct RowBytes {
  uint32_t a[8], ax[8], ay[8], az[8];
};

template <int D>
__device__ __forceinline__ void load_rows(const uint8_t* s, int L, int x0, uint32_t row,
                                          uint32_t row_y, uint32_t row_z, RowBytes& rb) {
  const uint32_t base = row * (uint32_t)L + (uint32_t)x0;
  if ((L & 31) == 0) {
    // 32-byte aligned rows: two 16-byte loads per row word
    const uint4* p = reinterpret_cast<const uint4*>(s + base);
    const uint4* py = reinterpret_cast<const uint4*>(s + row_y * (uint32_t)L + (uint32_t)x0);
    uint4 v0 = __ldg(p), v1 = __ldg(p + 1);
    rb.a[0] = v0.x; rb.a[1] = v0.y; rb.a[2] = v0.z; rb.a[3] = v0.w;
    rb.a[4] = v1.x; rb.a[5] = v1.y; rb.a[6] = v1.z; rb.a[7] = v1.w;
    v0 = __ldg(py); v1 = __ldg(py + 1);
    rb.ay[0] = v0.x; rb.ay[1] = v0.y; rb.ay[2] = v0.z; rb.ay[3] = v0.w;
    rb.ay[4] = v1.x; rb.ay[5] = v1.y; rb.ay[6] = v1.z; rb.ay[7] = v1.w;
    if (D == 3) {
      const uint4* pz = reinterpret_cast<const uint4*>(s + row_z * (uint32_t)L + (uint32_t)x0);
      v0 = __ldg(pz); v1 = __ldg(pz + 1);
      rb.az[0] = v0.x; rb.az[1] = v0.y; rb.az[2] = v0.z; rb.az[3] = v0.w;
      rb.az[4] = v1.x; rb.az[5] = v1.y; rb.az[6] = v1.z; rb.az[7] = v1.w;
    }
    // +x neighbours: the row shifted by one byte; the last one wraps to x = 0
    const uint32_t nx = (x0 + 32 < L) ? s[base + 32] : s[row * (uint32_t)L];
#pragma unroll
    for (int k = 0; k < 7; ++k) rb.ax[k] = __byte_perm(rb.a[k], rb.a[k + 1], 0x4321);
    rb.ax[7] = __byte_perm(rb.a[7], nx, 0x4321);
  } else {
    // general L: byte loads of the valid sites, zero elsewhere
#pragma unroll
    for (int k = 0; k < 8; ++k) rb.a[k] = rb.ax[k] = rb.ay[k] = rb.az[k] = 0u;
    const uint32_t rowL = row * (uint32_t)L, rowyL = row_y * (uint32_t)L, rowzL = row_z * (uint32_t)L;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const int x = x0 + b;
      if (x < L) {
        const int x1 = (x + 1 == L) ? 0 : x + 1;
        const int sh = 8 * (b & 3);
        rb.a[b >> 2] |= (uint32_t)s[rowL + x] << sh;
        rb.ax[b >> 2] |= (uint32_t)s[rowL + x1] << sh;
        rb.ay[b >> 2] |= (uint32_t)s[rowyL + x] << sh;
        if (D == 3) rb.az[b >> 2] |= (uint32_t)s[rowzL + x] << sh;
      }
    }
  }
}

// Measurement of one 32-site row word from its bytes and the equality masks
// e0..e2 with its +x/+y/+z neighbours.  MM 1 (Ising): M = #(+1) - #(-1) and
// E = -(#parallel - #antiparallel) over the +d bonds.  MM 2 (Potts): E = the
// number of unequal +d bonds, and the histogram n[k] of the states (per-warp
// bins for q <= kSmallQ, shared bins above).
template <int D, int MM>
__device__ __forceinline__ void measure_row(const RowBytes& rb, uint32_t e0, uint32_t e1, uint32_t e2,
                                            uint32_t vmask, int nvalid, int q, int& m_acc, int& e_acc,
                                            unsigned int* warp_hist, unsigned int* s_hist) {
  const int par_bonds = __popc(e0) + __popc(e1) + (D == 3 ? __popc(e2) : 0);
  if (MM == 1) {
    uint32_t ones[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ones[k] = 0x01010101u;
    m_acc += 2 * __popc(eq_bits(rb.a, ones) & vmask) - nvalid;
    e_acc -= 2 * par_bonds - D * nvalid;
  } else if (MM == 2) {
    e_acc += D * nvalid - par_bonds;
    if (q <= kSmallQ) {
      for (int k = 0; k < q; ++k) {
        uint32_t kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) kk[j] = 0x01010101u * (uint32_t)k;
        const unsigned c = (unsigned)__popc(eq_bits(rb.a, kk) & vmask);
        if (c) atomicAdd(&warp_hist[k], c);
      }
    } else {
#pragma unroll
      for (int b = 0; b < 32; ++b)
        if (b < nvalid) atomicAdd(&s_hist[(rb.a[b >> 2] >> (8 * (b & 3))) & 0xffu], 1u);
    }
  }
}

// MM (measurement mode) 1 = Ising, 2 = Potts: also measure the incoming
// spins (the state after sweep - 1): M and E from the row words' equality
// masks and the Potts histogram, added to the measurement slots (the flip
// kernel of this sweep writes the record of sweep - 1).  MM 0 and 3: no
// measurement, two-state (0: Ising, and XY / clock from their bond planes)
// or Potts (3) cluster draws.
// Shared memory of one tile's labeling in measurement mode MM (the Potts
// draw words and histograms only where Potts lattices can run).
template <class S, int MM>
struct LabelSmem {
  static constexpr int ROWS = S::ROWS, NW = S::THREADS / 32;
  static constexpr bool kPottsDraws = MM >= 2;  // MM 0 and 1: two-state draws only
  static constexpr int kDrawWords = (kPottsDraws ? 8 : 1) * (ROWS + 1);
  static constexpr int kHist = MM == 2 ? 256 : 1, kWHist = MM == 2 ? NW * kSmallQ : 1;
  alignas(16) uint32_t par[ROWS * 32];
  uint32_t srow[ROWS];  // global index of each row word's first site
  // cluster draws of the tile: two-state draws, row r's 32 bits in word r;
  // Potts, row r's bytes 4j..4j+3 in word j*(ROWS+1)+r (row-thread stores
  // and lane reads both bank-conflict free)
  uint32_t sdraw[kDrawWords];
  uint32_t sX[ROWS], sS[ROWS];
  // Potts histogram: per-warp bins for q <= kSmallQ, shared bins above
  unsigned int s_hist[kHist];
  unsigned int s_whist[kWHist];
  long long s_red[NW];
};

template <class Sh, bool FROM_MASK, int MM, class Smem>
__device__ __forceinline__ void label_tile(const Lattice& lat, uint32_t tile, uint32_t sweep,
                                           const Measure& mb, Smem& sm) {
  constexpr bool MEASURE = MM == 1 || MM == 2;
  constexpr int D = Sh::D, TY = Sh::TY, TZ = Sh::TZ, ROWS = Sh::ROWS, NT = Sh::THREADS;
  constexpr int NW = NT / 32, RPW = ROWS / NW;
  static_assert(ROWS == NT && NT % 32 == 0, "one thread per row word, whole warps");
  static_assert(!(MEASURE && FROM_MASK), "measurement needs the spins");
  uint32_t* par = sm.par;
  uint32_t* sdraw = sm.sdraw;
  uint32_t* sX = sm.sX;
  uint32_t* sS = sm.sS;
  unsigned int* s_hist = sm.s_hist;
  unsigned int* s_whist = sm.s_whist;
  long long* s_red = sm.s_red;
  int m_acc = 0, e_acc = 0;
  if (MM == 2) {
    for (int k = threadIdx.x; k < 256; k += NT) s_hist[k] = 0u;
    for (int k = threadIdx.x; k < NW * kSmallQ; k += NT) s_whist[k] = 0u;
    __syncthreads();
  }

  const TileCoord tc = tile_coord<Sh>(lat, tile);
  const int L = lat.L;
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  const int nvalid = min(32, L - tc.x0);
  const uint32_t vmask = (nvalid >= 32) ? kFull : ((1u << nvalid) - 1u);
  const bool draws = (sweep != 0u);
  const bool two_state = lat.dq == 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // every run start is its own parent until the unions (other sites are
  // never looked up: a site's root is the root of its run start)
  {
    uint4* p4 = reinterpret_cast<uint4*>(par);
#pragma unroll
    for (int k = 0; k < ROWS * 32 / 4 / NT; ++k) {
      const uint32_t t = 4u * (uint32_t)(threadIdx.x + k * NT);
      p4[threadIdx.x + k * NT] = make_uint4(t, t + 1u, t + 2u, t + 3u);
    }
  }

  // global memory only after the preceding kernel of the sweep is done
  pdl_wait();

  // ---- phase 1: bonds, runs and draws of this thread's row word
  const int r = threadIdx.x;
  const int ry = r % TY, rz = r / TY;
  const int y = tc.y0 + ry, z = tc.z0 + rz;
  const bool rowv = (y < L) && (D == 2 || z < L);
  const int y1 = (y + 1 == L) ? 0 : y + 1;
  const int z1 = (D == 3) ? ((z + 1 == L) ? 0 : z + 1) : 0;
  uint32_t X = 0u, Y = 0u, Z = 0u, S = 0u, XW = 0u;
  if (rowv) {
    const uint32_t row = (uint32_t)y + (uint32_t)L * (uint32_t)z;
    sm.srow[r] = row * (uint32_t)L + (uint32_t)tc.x0;
    const uint32_t g = row * (uint32_t)lat.W + (uint32_t)tc.tx;
    uint32_t A0, A1, A2 = 0u;
    if (FROM_MASK) {
      A0 = __ldg(&lat.planes[g]) & vmask;
      A1 = __ldg(&lat.planes[plane + g]) & vmask;
      if (D == 3) A2 = __ldg(&lat.planes[2 * plane + g]) & vmask;
    } else {
      RowBytes rb;
      const uint32_t row_y = (uint32_t)y1 + (uint32_t)L * (uint32_t)z;
      const uint32_t row_z = (uint32_t)y + (uint32_t)L * (uint32_t)z1;
      load_rows<D>(static_cast<const uint8_t*>(lat.spins), L, tc.x0, row, row_y, row_z, rb);
      // equality masks (and the measurement) first, so the row bytes are
      // dead before the Bernoulli words are drawn
      const uint32_t e0 = eq_bits(rb.a, rb.ax) & vmask;
      const uint32_t e1 = eq_bits(rb.a, rb.ay) & vmask;
      const uint32_t e2 = (D == 3) ? (eq_bits(rb.a, rb.az) & vmask) : 0u;
      if (MEASURE) measure_row<D, MM>(rb, e0, e1, e2, vmask, nvalid, lat.q, m_acc, e_acc, s_whist + warp * kSmallQ, s_hist);
      A0 = e0 ? (e0 & bernoulli_word(g, sweep, 0, lat.t_bond, e0, lat.rk)) : 0u;
      A1 = e1 ? (e1 & bernoulli_word(g, sweep, 1, lat.t_bond, e1, lat.rk)) : 0u;
      if (D == 3) A2 = e2 ? (e2 & bernoulli_word(g, sweep, 2, lat.t_bond, e2, lat.rk)) : 0u;
      lat.planes[g] = A0;
      lat.planes[plane + g] = A1;
      if (D == 3) lat.planes[2 * plane + g] = A2;
    }
    X = A0 & (vmask >> 1);          // x-bonds whose +x site is in the same word
    S = ~(X << 1) & vmask;          // x-run starts
    XW = (tc.x0 == 0 && L <= 32) ? ((A0 >> (L - 1)) & 1u) : 0u;  // wrap inside the word
    Y = (y1 - tc.y0 >= 0 && y1 - tc.y0 < TY) ? A1 : 0u;
    Z = (D == 3 && z1 - tc.z0 >= 0 && z1 - tc.z0 < TZ) ? A2 : 0u;
    if (draws && two_state) {
      // two-state cluster draws: bit (x & 31) of word 0 of Philox(g, sweep, DRAW, 1)
      sdraw[r] = philox(g, sweep, kDraw, 1u, lat.rk).x;
    } else if (draws && Smem::kPottsDraws) {
      // Potts cluster draw of every site: word (i & 3) of Philox(i >> 2, sweep, DRAW, 0)
      const uint32_t i0 = row * (uint32_t)L + (uint32_t)tc.x0;
      const uint32_t dq = (uint32_t)lat.dq;
      if ((L & 3) == 0) {
        // L a multiple of 4 (the same branch for the whole lattice): the row
        // word starts a Philox group, and group j holds the draws of its
        // sites 4j..4j+3 (those past the end of the row go unused)
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
          const uint4 w = philox((i0 >> 2) + (uint32_t)j, sweep, kDraw, 0u, lat.rk);
          sdraw[j * (ROWS + 1) + r] = draw_value(w.x, dq) | (draw_value(w.y, dq) << 8) |
                                      (draw_value(w.z, dq) << 16) | (draw_value(w.w, dq) << 24);
        }
      } else {
        uint32_t cached = 0xffffffffu;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
          uint32_t packed = 0u;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int b = 4 * j + t;
            if (b < nvalid) {
              const uint32_t i = i0 + (uint32_t)b;
              if ((i >> 2) != cached) {
                cached = i >> 2;
                w = philox(cached, sweep, kDraw, 0u, lat.rk);
              }
              packed |= draw_value(word_of(w, (int)(i & 3u)), dq) << (8 * t);
            }
          }
          sdraw[j * (ROWS + 1) + r] = packed;
        }
      }
    }
  }
  sX[r] = X;
  sS[r] = S;
  __syncthreads();

  // ---- phase 2: unions of runs joined by in-tile +y / +z bonds
  const uint32_t cap = lat.cap;
  if (rowv) {
    if (Y) {
      const int rn = r + (y1 - y);
      const uint32_t Xn = sX[rn], Sn = sS[rn];
      uint32_t U = Y & ~((Y & X & Xn) << 1);
      while (U) {
        const int b = __ffs(U) - 1;
        U &= U - 1u;
        sunion(par, (uint32_t)(32 * r) + run_start(S, b), (uint32_t)(32 * rn) + run_start(Sn, b), lat.err, cap);
      }
    }
    if (D == 3 && Z) {
      const int rn = r + TY * (z1 - z);
      const uint32_t Xn = sX[rn], Sn = sS[rn];
      uint32_t U = Z & ~((Z & X & Xn) << 1);
      while (U) {
        const int b = __ffs(U) - 1;
        U &= U - 1u;
        sunion(par, (uint32_t)(32 * r) + run_start(S, b), (uint32_t)(32 * rn) + run_start(Sn, b), lat.err, cap);
      }
    }
    if (XW) sunion(par, (uint32_t)(32 * r) + run_start(S, L - 1), (uint32_t)(32 * r), lat.err, cap);
  }
  __syncthreads();

  // ---- phase 3: forest word of every site
  const uint32_t lr_bit = 1u << lat.sbits;
  const int shift = lat.sbits + 1;
#pragma unroll 2
  for (int k = 0; k < RPW; ++k) {
    const int rr = warp + NW * k;
    const uint32_t st = sS[rr];
    if (st == 0u || lane >= nvalid) continue;
    const uint32_t t = (uint32_t)(32 * rr + lane);
    const uint32_t lr = sfind(par, (uint32_t)(32 * rr) + run_start(st, lane));
    const uint32_t gidx = sm.srow[lr >> 5] + (lr & 31u);
    const uint32_t i = sm.srow[rr] + (uint32_t)lane;
    const uint32_t draw = !draws ? 0u
                          : (two_state || !Smem::kPottsDraws)
                              ? (sdraw[rr] >> lane) & 1u
                              : (sdraw[(lane >> 2) * (ROWS + 1) + rr] >> (8 * (lane & 3))) & 0xffu;
    lat.forest[i] = (gidx << shift) | (lr == t ? lr_bit : 0u) | draw;
  }
  if (MEASURE) {
    if (MM == 2) {
      __syncthreads();
      for (int k = threadIdx.x; k < kSmallQ; k += NT)
        for (int w = 0; w < NW; ++w) s_hist[k] += s_whist[w * kSmallQ + k];
      __syncthreads();
      add_histogram(lat, mb, tile, s_hist);
    }
    add_integer_sums<NW>(mb, tile, (long long)m_acc, (long long)e_acc, s_red);
  }
}

// Five 256-thread CTAs per SM, proportionally more of smaller tiles.
template <int D, bool FROM_MASK, int MM>
__global__ void __launch_bounds__(Tile<D>::THREADS, 5 * 256 / Tile<D>::THREADS)
    k_label(const __grid_constant__ Lattice lat, uint32_t sweep, const __grid_constant__ Measure mb) {
  __shared__ LabelSmem<Tile<D>, MM> sm;
  label_tile<Tile<D>, FROM_MASK, MM>(lat, blockIdx.x, sweep, mb, sm);
}

// Ising/Potts lattices of a batch, one tile of shape S per CTA; sweep
// numbers come from the batch step counter, and every step after the first
// (the first too when the member's last record is pending) also measures
// the incoming state of its lattice (the record of the previous sweep).  A
// member stops after its own number of sweeps.  The tile map lists the
// Ising members' tiles first.
// LAYOUT 1: Ising tiles only, two-state layout; LAYOUT 2: Potts tiles only;
// LAYOUT 3: any tile, Potts layout, the member's model picked per tile.
// Resident CTAs per SM: five 256-thread CTAs (two-state layout) or four
// (Potts layout), and proportionally more of smaller tiles.
constexpr int label_blocks(int threads, int layout) {
  return (layout == 1 ? 5 : 4) * 256 / threads > 32 ? 32 : (layout == 1 ? 5 : 4) * 256 / threads;
}

// One tile-map entry of a batch label launch: the member's lattice view is
// copied to shared memory (the Philox round keys are read on every round).
template <class S, int LAYOUT, class Smem>
__device__ __forceinline__ void label_batch_entry(const BatchView& bv, uint32_t e, uint32_t step, Smem& sm,
                                                  Lattice& s_lat) {
  static_assert(sizeof(Lattice) % 4 == 0, "lattice copy");
  const uint32_t b = __ldg(&bv.tile_lattice[e]);
  const uint32_t tile = __ldg(&bv.tile_index[e]);
  const BatchMember& m = bv.members[b];
  for (uint32_t k = threadIdx.x; k < sizeof(Lattice) / 4; k += S::THREADS)
    reinterpret_cast<uint32_t*>(&s_lat)[k] = reinterpret_cast<const uint32_t*>(&m.lat)[k];
  __syncthreads();
  if (step >= m.nsweeps) return;  // the member has had its sweeps this call
  const uint32_t sweep = m.sweep0 + step + 1u;
  const bool potts = LAYOUT == 2 || (LAYOUT == 3 && s_lat.model == kPotts);
  if (step == 0u && !m.measure0) label_tile<S, false, 0>(s_lat, tile, sweep, m.meas, sm);
  else if (LAYOUT != 1 && potts) label_tile<S, false, 2>(s_lat, tile, sweep, m.meas, sm);
  else if (LAYOUT != 2) label_tile<S, false, 1>(s_lat, tile, sweep, m.meas, sm);
}

// PERSISTENT false: CTA k labels tile-map entry first + k (the grid covers
// the map).  PERSISTENT true: a grid of resident CTAs, each taking entries
// first + t for t = blockIdx.x, blockIdx.x + gridDim.x, ... below first + n.
// Separate instantiations, so that the loop costs the one-entry kernel no
// registers; the persistent one allows a quarter fewer CTAs per SM (its
// grid is sized by the occupancy it gets), so that its loop does not spill.
constexpr int persistent_blocks(int blocks) { return blocks * 3 / 4 > 1 ? blocks * 3 / 4 : 1; }

template <class S, int LAYOUT, bool PERSISTENT>
__global__ void __launch_bounds__(S::THREADS, PERSISTENT ? persistent_blocks(label_blocks(S::THREADS, LAYOUT))
                                                         : label_blocks(S::THREADS, LAYOUT))
    k_label_batch(BatchView bv, uint32_t first, uint32_t n) {
  __shared__ LabelSmem<S, LAYOUT == 1 ? 1 : 2> sm;
  __shared__ Lattice s_lat;
  pdl_wait();
  const uint32_t step = *bv.step;
  if constexpr (PERSISTENT) {
    for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) {
      __syncthreads();  // the previous entry's readers of s_lat and sm are done
      label_batch_entry<S, LAYOUT>(bv, first + t, step, sm, s_lat);
    }
  } else {
    label_batch_entry<S, LAYOUT>(bv, first + blockIdx.x, step, sm, s_lat);
  }
}

// Stand-alone measurement of an Ising (MM 1) or Potts (MM 2) state as the
// record of `sweep`: a thread per 32-site row word (grid-stride), the
// labeling kernel's row loads and equality masks, sums added to the
// measurement slots by block; the last block to finish (a counter) writes
// the record and the FP64 accumulators from the complete slots.
template <int D, int MM>
__global__ void __launch_bounds__(256) k_measure_rows(const __grid_constant__ Lattice lat,
                                                      const __grid_constant__ Measure mb, uint32_t sweep) {
  constexpr int NW = 256 / 32;
  __shared__ unsigned int s_hist[MM == 2 ? 256 : 1];
  __shared__ unsigned int s_whist[MM == 2 ? NW * kSmallQ : 1];
  __shared__ long long s_red[NW];
  __shared__ double s_rd[NW];
  __shared__ bool s_last;
  const int warp = threadIdx.x >> 5;
  if (MM == 2) {
    for (int k = threadIdx.x; k < 256; k += 256) s_hist[k] = 0u;
    for (int k = threadIdx.x; k < NW * kSmallQ; k += 256) s_whist[k] = 0u;
    __syncthreads();
  }
  const int L = lat.L;
  const uint32_t words = lat.R * (uint32_t)lat.W;
  int m_acc = 0, e_acc = 0;
  // L a power of two (then so is W): indices by shifts and masks
  const bool pow2 = (L & (L - 1)) == 0;
  const int lsh = __ffs(L) - 1, wsh = __ffs(lat.W) - 1;
  for (uint32_t g = blockIdx.x * 256u + threadIdx.x; g < words; g += gridDim.x * 256u) {
    uint32_t row, tx, y, z;
    if (pow2) {
      row = g >> wsh;
      tx = g & (uint32_t)(lat.W - 1);
      y = row & (uint32_t)(L - 1);
      z = row >> lsh;
    } else {
      row = g / (uint32_t)lat.W;
      tx = g % (uint32_t)lat.W;
      y = row % (uint32_t)L;
      z = row / (uint32_t)L;
    }
    const int x0 = 32 * (int)tx;
    const int nvalid = min(32, L - x0);
    const uint32_t vmask = (nvalid >= 32) ? kFull : ((1u << nvalid) - 1u);
    const uint32_t y1 = (y + 1u == (uint32_t)L) ? 0u : y + 1u;
    const uint32_t z1 = (D == 3) ? ((z + 1u == (uint32_t)L) ? 0u : z + 1u) : 0u;
    RowBytes rb;
    load_rows<D>(static_cast<const uint8_t*>(lat.spins), L, x0, row, y1 + (uint32_t)L * z, y + (uint32_t)L * z1, rb);
    const uint32_t e0 = eq_bits(rb.a, rb.ax) & vmask;
    const uint32_t e1 = eq_bits(rb.a, rb.ay) & vmask;
    const uint32_t e2 = (D == 3) ? (eq_bits(rb.a, rb.az) & vmask) : 0u;
    measure_row<D, MM>(rb, e0, e1, e2, vmask, nvalid, lat.q, m_acc, e_acc, s_whist + warp * kSmallQ, s_hist);
  }
  if (MM == 2) {
    __syncthreads();
    for (int k = threadIdx.x; k < kSmallQ; k += 256)
      for (int w = 0; w < NW; ++w) s_hist[k] += s_whist[w * kSmallQ + k];
    __syncthreads();
    add_histogram(lat, mb, blockIdx.x, s_hist);
  }
  add_integer_sums<NW>(mb, blockIdx.x, (long long)m_acc, (long long)e_acc, s_red);
  // this block's slot additions are visible before it counts itself done
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(mb.done, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  finalize_record<NW>(lat, mb, sweep, s_red, s_rd);
  if (threadIdx.x == 0) *mb.done = 0u;
}

// ---------------------------------------------------------------- XY bonds
// One CTA per 32 x BY (x BZ) block of sites, grid-strided over the blocks.
// The projections (x, y) = (cos, sin)(theta - phi) on the sweep's mirror
// axis are computed once per site of the block and its +x/+y/+z halo into
// shared memory; bond (i,d) is active iff x_i x_j > 0 and the uniform of
// word d of Philox(i, sweep, BOND, 0) is below 1 - exp(-2K x_i x_j); warps
// ballot their rows into the bit-planes.  With MEASURE the same values
// measure the incoming state (the state after sweep - 1): sum x, sum y and
// the bond energies x_i x_j + y_i y_j (cos(theta_i - theta_j), invariant
// under the rotation by phi) in float per thread, then double per block;
// the block's (sum cos theta, sum sin theta, E) partial, rotated back by
// phi, goes to slot blockIdx of the XY partials.
template <int D>
struct XYBlock;
template <>
struct XYBlock<2> {
  static constexpr int BY = 128, BZ = 1;
};
template <>
struct XYBlock<3> {
  static constexpr int BY = 16, BZ = 8;
};

template <int D, bool MEASURE>
__global__ void __launch_bounds__(256) k_bonds_xy(const __grid_constant__ Lattice lat, uint32_t sweep,
                                                   const __grid_constant__ Measure mb) {
  constexpr int BY = XYBlock<D>::BY, BZ = XYBlock<D>::BZ;
  constexpr int HX = 33, HY = BY + 1, HZ = (D == 3) ? BZ + 1 : 1, NBOX = HX * HY * HZ;
  constexpr int NW = 256 / 32;
  __shared__ float2 sv[NBOX];
  __shared__ float s_phi;
  __shared__ double s_rd[NW];
  if (threadIdx.x == 0) s_phi = xy_phi(lat, sweep);
  pdl_wait();
  __syncthreads();
  const float phi = s_phi;
  const int L = lat.L, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t plane = lat.R * (uint32_t)lat.W;
  const float* th = static_cast<const float*>(lat.spins);
  const uint32_t nbx = (uint32_t)lat.W, nby = (uint32_t)((L + BY - 1) / BY);
  const uint32_t nbz = (D == 3) ? (uint32_t)((L + BZ - 1) / BZ) : 1u;
  const uint32_t nblocks = nbx * nby * nbz;
  float fx = 0.f, fy = 0.f, fe = 0.f;
  for (uint32_t t = blockIdx.x; t < nblocks; t += gridDim.x) {
    const int x0 = 32 * (int)(t % nbx), y0 = BY * (int)((t / nbx) % nby), z0 = BZ * (int)(t / (nbx * nby));
    const int nx = min(32, L - x0), ny = min(BY, L - y0), nz = (D == 3) ? min(BZ, L - z0) : 1;
    __syncthreads();  // the previous block's values are no longer read
    // a warp per halo row (yy, zz), lanes along x; then the +x halo column
    // (entry 32 of every row) a thread per row
    for (int hr = warp; hr < HY * HZ; hr += NW) {
      const int yy = hr % HY, zz = hr / HY;
      if (yy > ny || zz > nz || lane > nx) continue;  // beyond the valid sites and their halo
      int gy = y0 + yy, gz = (D == 3) ? z0 + zz : 0;
      if (gy >= L) gy -= L;
      if (gz >= L) gz -= L;
      int gx = x0 + lane;
      if (gx >= L) gx -= L;
      float sn, cs;
      sincosf(__fsub_rn(__ldg(&th[(uint32_t)gx + (uint32_t)L * ((uint32_t)gy + (uint32_t)L * (uint32_t)gz)]),
                        phi), &sn, &cs);
      sv[hr * HX + lane] = make_float2(cs, sn);
    }
    if (nx == 32) {
      for (int hr = threadIdx.x; hr < HY * HZ; hr += 256) {
        const int yy = hr % HY, zz = hr / HY;
        if (yy > ny || zz > nz) continue;
        int gy = y0 + yy, gz = (D == 3) ? z0 + zz : 0;
        if (gy >= L) gy -= L;
        if (gz >= L) gz -= L;
        int gx = x0 + 32;
        if (gx >= L) gx -= L;
        float sn, cs;
        sincosf(__fsub_rn(__ldg(&th[(uint32_t)gx + (uint32_t)L * ((uint32_t)gy + (uint32_t)L * (uint32_t)gz)]),
                          phi), &sn, &cs);
        sv[hr * HX + 32] = make_float2(cs, sn);
      }
    }
    __syncthreads();
    for (int rr = warp; rr < BY * BZ; rr += NW) {
      const int yy = rr % BY, zz = rr / BY;
      const bool rowv = yy < ny && zz < nz;
      uint32_t a = 0u;
      if (rowv && lane < nx) {
        const uint32_t y = (uint32_t)(y0 + yy), z = (uint32_t)(z0 + zz);
        const uint32_t i = (uint32_t)(x0 + lane) + (uint32_t)L * (y + (uint32_t)L * z);
        const uint4 w = philox(i, sweep, kBond, 0u, lat.rk);
        const int c = lane + HX * (yy + HY * zz);
        const float2 si = sv[c];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float2 sj = sv[c + (d == 0 ? 1 : d == 1 ? HX : HX * HY)];
          const float prod = __fmul_rn(si.x, sj.x);
          bool act = false;
          if (prod > 0.0f) {
            // u < p with p = -expm1f(-2K prod): a fast estimate of p decides
            // unless u lies within a margin far above the estimate's error
            // (|a| <= 2K keeps __expf within a few ulp), where expm1f decides
            const float a2 = __fmul_rn(lat.twoK, prod);
            const float u = __fmul_rn((float)(word_of(w, d) >> 8), 0x1p-24f);
            const float pf = __fsub_rn(1.0f, __expf(-a2));
            if (fabsf(__fsub_rn(u, pf)) > 0x1p-16f) act = u < pf;
            else act = u < -expm1f(-a2);
          }
          a |= (uint32_t)act << d;
          if (MEASURE) fe = __fadd_rn(fe, __fadd_rn(prod, __fmul_rn(si.y, sj.y)));
        }
        if (MEASURE) {
          fx = __fadd_rn(fx, si.x);
          fy = __fadd_rn(fy, si.y);
        }
      }
      const uint32_t row = (uint32_t)(y0 + yy) + (uint32_t)L * (uint32_t)(z0 + zz);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const uint32_t bal = __ballot_sync(kFull, (a >> d) & 1u);
        if (rowv && lane == d) lat.planes[d * plane + row * (uint32_t)lat.W + (uint32_t)(x0 >> 5)] = bal;
      }
    }
  }
  if (MEASURE) {
    const double sx = block_combine<NW>((double)warp_sum(fx), s_rd);
    const double sy = block_combine<NW>((double)warp_sum(fy), s_rd);
    const double se = block_combine<NW>((double)warp_sum(fe), s_rd);
    if (threadIdx.x == 0) {
      const double c = cos((double)phi), sn = sin((double)phi);
      mb.part_d[3 * blockIdx.x + 0] = __dsub_rn(__dmul_rn(c, sx), __dmul_rn(sn, sy));
      mb.part_d[3 * blockIdx.x + 1] = __dadd_rn(__dmul_rn(sn, sx), __dmul_rn(c, sy));
      mb.part_d[3 * blockIdx.x + 2] = -se;
    }
  }
}

// ---------------------------------------------------------------- clock bonds
// q-state clock: x_i = sin(pi k_i / q), k_i = (2 p_i - s) mod 2q for the
// sweep's mirror index s; bond (i,d) active iff u(i,d) < t[k_i][k_j] (the
// table is 0 where x_i x_j <= 0); u(i,d) = word d of Philox(i, sweep, BOND, 0).
// The comparison is decided from a float estimate of t (the projections in
// shared memory, __expf) unless the draw lies within a margin far above the
// estimate's error, where the exact table entry decides: the result is the
// table's, without a table gather per bond.
// With MEASURE the same loads measure the incoming state: integer sums of
// the fixed-point tables C[p_i], S[p_i] and C[(p_i - p_j) mod q], added to
// the clock slots per block.
template <int D, bool MEASURE>
__global__ void __launch_bounds__(256) k_bonds_clock(const __grid_constant__ Lattice lat, uint32_t sweep,
                                                      const __grid_constant__ Measure mb) {
  __shared__ uint32_t s_mirror;
  __shared__ long long s_red[256 / 32];
  __shared__ float s_x[2 * kMaxClockQ];
  // the fixed-point cos / sin tables of the measurement (gathered per site)
  __shared__ long long s_fix[MEASURE ? 2 * kMaxClockQ : 1];
  if (threadIdx.x == 0) s_mirror = clock_mirror(lat, sweep);
  pdl_wait();
  const int L = lat.L, lane = threadIdx.x & 31;
  const int q = lat.q, q2 = 2 * q;
  for (int k = threadIdx.x; k < q2; k += 256) {
    s_x[k] = __ldg(&lat.cproj[k]);
    if (MEASURE) s_fix[k] = __ldg(&mb.cfix[k]);
  }
  __syncthreads();
  // Error of the float threshold estimate below against the exact table
  // entry t/2^32 (x rounded to float, products and 2K in float, __expf,
  // the draw rounded to float): below 2K * 2.5e-7 + 4e-7; the margin is
  // about four times that, and draws inside it read the exact entry.
  const float margin = __fadd_rn(0x1p-16f, __fmul_rn(lat.twoK, 0x1p-20f));
  const int mirror = (int)s_mirror;
  const uint32_t nwords = lat.R * (uint32_t)lat.W;
  const uint32_t plane = nwords;
  const uint16_t* sp = static_cast<const uint16_t*>(lat.spins);
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  long long cx = 0, sy = 0, eb = 0;
  // L a power of two (then so is W): a row word's indices by shifts and
  // masks instead of four divisions (the same branch for the whole lattice)
  const bool pow2 = (L & (L - 1)) == 0;
  const int lsh = __ffs(L) - 1, wsh = __ffs(lat.W) - 1;
  for (uint32_t g = gw; g < nwords; g += nw) {
    uint32_t row, xw, y, z;
    if (pow2) {
      row = g >> wsh;
      xw = g & (uint32_t)(lat.W - 1);
      y = row & (uint32_t)(L - 1);
      z = row >> lsh;
    } else {
      row = g / (uint32_t)lat.W;
      xw = g % (uint32_t)lat.W;
      y = row % (uint32_t)L;
      z = row / (uint32_t)L;
    }
    const int x = (int)(32 * xw) + lane;
    uint32_t a = 0u;
    if (x < L) {
      const uint32_t i = (uint32_t)x + (uint32_t)L * row;
      const uint4 w = philox(i, sweep, kBond, 0u, lat.rk);
      uint32_t jn[3];
      jn[0] = (x + 1 == L) ? i - (uint32_t)x : i + 1u;
      jn[1] = (y + 1 == (uint32_t)L) ? i - y * L : i + (uint32_t)L;
      jn[2] = (D == 3) ? ((z + 1 == (uint32_t)L) ? i - z * L * L : i + (uint32_t)L * L) : 0u;
      const int pi = clock_state(sp[i], q);
      const int ki = wrap_mod(2 * pi - mirror, q2);
      if (MEASURE) {
        cx += s_fix[pi];
        sy += s_fix[q + pi];
      }
      const float xi = s_x[ki];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int pj = clock_state(sp[jn[d]], q);
        const int kj = wrap_mod(2 * pj - mirror, q2);
        // the table entry is 0 where x_i x_j <= 0 (the sign of a float
        // product is the exact one; |x| >= sin(pi/q) off k = 0, q)
        const float prod = __fmul_rn(xi, s_x[kj]);
        bool act = false;
        if (prod > 0.0f) {
          const uint32_t wd = word_of(w, d);
          const float pf = __fsub_rn(1.0f, __expf(-__fmul_rn(lat.twoK, prod)));
          const float diff = __fsub_rn(__fmul_rn(__uint2float_rn(wd), 0x1p-32f), pf);
          act = (fabsf(diff) > margin) ? diff < 0.0f
                                       : wd < __ldg(&lat.ctab[(size_t)ki * (size_t)q2 + (size_t)kj]);
        }
        a |= (uint32_t)act << d;
        if (MEASURE) eb += s_fix[wrap_mod(pi - pj, q)];
      }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const uint32_t bal = __ballot_sync(kFull, (a >> d) & 1u);
      if (lane == d) lat.planes[d * plane + g] = bal;
    }
  }
  if (MEASURE) add_clock_sums<256 / 32>(mb, blockIdx.x, cx, sy, eb, s_red);
}

}  // namespace

cudaError_t launch_bonds_clock(const Lattice& lat, uint32_t sweep, const Measure* m, cudaStream_t st) {
  const uint32_t words = lat.R * (uint32_t)lat.W;
  unsigned g = (words + 7u) / 8u;
  if (g > 4096u) g = 4096u;
  cudaError_t e = cudaSuccess;
  const Measure none{};
  if (lat.dim == 2) {
    if (m) e = launch_pdl(k_bonds_clock<2, true>, g, 256, st, lat, sweep, *m);
    else e = launch_pdl(k_bonds_clock<2, false>, g, 256, st, lat, sweep, none);
  } else {
    if (m) e = launch_pdl(k_bonds_clock<3, true>, g, 256, st, lat, sweep, *m);
    else e = launch_pdl(k_bonds_clock<3, false>, g, 256, st, lat, sweep, none);
  }
  return e;
}

void tiles_for(int dim, int L, int* ntx, int* nty, int* ntz, int shape) {
  if (shape < 0) shape = kSingleShape[dim - 2];
  const int ty = kShapeTY[dim - 2][shape], tz = kShapeTZ[dim - 2][shape];
  *ntx = (L + 31) / 32;
  *nty = (L + ty - 1) / ty;
  *ntz = (dim == 2) ? 1 : (L + tz - 1) / tz;
}

namespace {
template <int D>
cudaError_t launch_label_dim(const Lattice& lat, uint32_t sweep, bool from_mask, bool potts_draws,
                             cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz), t = (unsigned)Tile<D>::THREADS;
  const Measure none{};
  if (from_mask) {
    if (potts_draws) return launch_pdl(k_label<D, true, 3>, g, t, st, lat, sweep, none);
    return launch_pdl(k_label<D, true, 0>, g, t, st, lat, sweep, none);
  }
  if (potts_draws) return launch_pdl(k_label<D, false, 3>, g, t, st, lat, sweep, none);
  return launch_pdl(k_label<D, false, 0>, g, t, st, lat, sweep, none);
}
}  // namespace

cudaError_t launch_label(const Lattice& lat, uint32_t sweep, bool from_mask, cudaStream_t st) {
  // the Potts layout (a draw byte per site in shared memory) only where
  // Potts draws are made; two-state draws or none take the smaller layout
  const bool potts_draws = sweep != 0u && lat.dq != 2;
  if (lat.dim == 2) return launch_label_dim<2>(lat, sweep, from_mask, potts_draws, st);
  return launch_label_dim<3>(lat, sweep, from_mask, potts_draws, st);
}

namespace {

// Schedule bit 0: Ising and Potts tiles in one launch (Potts layout) or
// two; bit 1: persistent grids (batch_grid).
template <class S, int LAYOUT>
cudaError_t label_batch_launch(const BatchView& bv, uint32_t first, uint32_t n, bool persistent,
                               cudaStream_t st) {
  if (!persistent) return launch_pdl(k_label_batch<S, LAYOUT, false>, n, (unsigned)S::THREADS, st, bv, first, n);
  const unsigned g = batch_grid(k_label_batch<S, LAYOUT, true>, S::THREADS, n);
  return launch_pdl(k_label_batch<S, LAYOUT, true>, g, (unsigned)S::THREADS, st, bv, first, n);
}

template <int D, int SH>
cudaError_t label_batch_shape(const BatchView& bv, int schedule, uint32_t ising_tiles, uint32_t potts_tiles,
                              cudaStream_t st) {
  using S = ShapeOf<D, SH>;
  const bool persistent = (schedule & 2) != 0;
  if ((schedule & 1) && ising_tiles && potts_tiles)
    return label_batch_launch<S, 3>(bv, 0u, ising_tiles + potts_tiles, persistent, st);
  cudaError_t e = cudaSuccess;
  if (ising_tiles) e = label_batch_launch<S, 1>(bv, 0u, ising_tiles, persistent, st);
  if (e == cudaSuccess && potts_tiles) e = label_batch_launch<S, 2>(bv, ising_tiles, potts_tiles, persistent, st);
  return e;
}

template <int D>
cudaError_t label_batch_dim(const BatchView& bv, int shape, int schedule, uint32_t ising_tiles,
                            uint32_t potts_tiles, cudaStream_t st) {
  if (shape == 1) return label_batch_shape<D, 1>(bv, schedule, ising_tiles, potts_tiles, st);
  if (shape == 2) return label_batch_shape<D, 2>(bv, schedule, ising_tiles, potts_tiles, st);
  return label_batch_shape<D, 0>(bv, schedule, ising_tiles, potts_tiles, st);
}

}  // namespace

cudaError_t launch_label_batch(const BatchView& bv, int dim, int shape, int schedule, uint32_t ising_tiles,
                               uint32_t potts_tiles, cudaStream_t st) {
  static_assert(kTileShapes == 3, "one instantiation per shape");
  if (dim == 2) return label_batch_dim<2>(bv, shape, schedule, ising_tiles, potts_tiles, st);
  return label_batch_dim<3>(bv, shape, schedule, ising_tiles, potts_tiles, st);
}

cudaError_t launch_measure_rows(const Lattice& lat, uint32_t sweep, const Measure& m, cudaStream_t st) {
  const uint32_t words = lat.R * (uint32_t)lat.W;
  unsigned g = (words + 255u) / 256u;
  if (g > (unsigned)kMeasureBlocks) g = (unsigned)kMeasureBlocks;
  if (g == 0) g = 1;
  const bool potts = lat.model == kPotts;
  if (lat.dim == 2) {
    if (potts) k_measure_rows<2, 2><<<g, 256, 0, st>>>(lat, m, sweep);
    else k_measure_rows<2, 1><<<g, 256, 0, st>>>(lat, m, sweep);
  } else {
    if (potts) k_measure_rows<3, 2><<<g, 256, 0, st>>>(lat, m, sweep);
    else k_measure_rows<3, 1><<<g, 256, 0, st>>>(lat, m, sweep);
  }
  return cudaGetLastError();
}

cudaError_t launch_label_measured(const Lattice& lat, uint32_t sweep, const Measure& m,
                                  cudaStream_t st) {
  const unsigned g = (unsigned)(lat.ntx * lat.nty * lat.ntz);
  cudaError_t e = cudaSuccess;
  const bool potts = lat.model == kPotts;
  if (lat.dim == 2) {
    if (potts) e = launch_pdl(k_label<2, false, 2>, g, (unsigned)Tile<2>::THREADS, st, lat, sweep, m);
    else e = launch_pdl(k_label<2, false, 1>, g, (unsigned)Tile<2>::THREADS, st, lat, sweep, m);
  } else {
    if (potts) e = launch_pdl(k_label<3, false, 2>, g, (unsigned)Tile<3>::THREADS, st, lat, sweep, m);
    else e = launch_pdl(k_label<3, false, 1>, g, (unsigned)Tile<3>::THREADS, st, lat, sweep, m);
  }
  return e;
}

cudaError_t launch_bonds_xy(const Lattice& lat, uint32_t sweep, const Measure* m, int* blocks,
                            cudaStream_t st) {
  const uint32_t ny = (uint32_t)((lat.L + XYBlock<3>::BY - 1) / XYBlock<3>::BY);
  const uint32_t nb = (lat.dim == 2)
                          ? (uint32_t)lat.W * (uint32_t)((lat.L + XYBlock<2>::BY - 1) / XYBlock<2>::BY)
                          : (uint32_t)lat.W * ny * (uint32_t)((lat.L + XYBlock<3>::BZ - 1) / XYBlock<3>::BZ);
  // one wave: the CTAs the GPU holds at once (the box of projections and the
  // registers allow five per SM), each striding over the blocks; at most
  // kMeasureBlocks (the slots of the XY partials)
  unsigned g = 0;
  auto launch = [&](auto kernel, const Measure& mm) {
    g = batch_grid(kernel, 256, nb);
    if (g > (unsigned)kMeasureBlocks) g = (unsigned)kMeasureBlocks;
    return launch_pdl(kernel, g, 256, st, lat, sweep, mm);
  };
  cudaError_t e = cudaSuccess;
  const Measure none{};
  if (lat.dim == 2) {
    if (m) e = launch(k_bonds_xy<2, true>, *m);
    else e = launch(k_bonds_xy<2, false>, none);
  } else {
    if (m) e = launch(k_bonds_xy<3, true>, *m);
    else e = launch(k_bonds_xy<3, false>, none);
  }
  if (blocks) *blocks = (int)g;
  return e;
}

}  // namespace swgb
