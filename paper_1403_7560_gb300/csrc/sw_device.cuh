// Device helpers shared by the SW kernels: Philox4x32-10, the bit-sliced
// Bernoulli word, byte-lane comparisons, tile geometry, union-find in shared
// and global memory, and warp/block reductions.
#pragma once

#include "sw_internal.h"

namespace swgb {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch.  The kernels of a sweep are launched with
// programmatic stream serialisation (launch_pdl): the launch of a kernel is
// processed while its predecessor runs, and pdl_wait() blocks until the
// predecessor has completed and its writes are visible (it returns at once
// for a kernel launched without the attribute).  Every such kernel calls
// pdl_wait() before its first global memory access.  No kernel triggers its
// successor early (griddepcontrol.launch_dependents): successors resident
// ahead of time, waiting, made the sweep slower on the GB300.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
constexpr int kErrTimeout = -4;

// Philox purposes (third counter word).
constexpr uint32_t kInit = 0u, kBond = 1u, kDraw = 2u, kAxis = 3u;

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds; per round two 32x32
// multiplications whose high words are xor-ed with the other counter words
// and the round key.  The round keys (the key bumped by the Weyl increments
// r times) are precomputed per lattice and read from the kernel parameters.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ rk[2 * r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, int j) {
  return j == 0 ? w.x : j == 1 ? w.y : j == 2 ? w.z : w.w;
}

// XY mirror direction of a sweep: phi = (w0 >> 8) * fl(2 pi)/2^24 in float.
__device__ __forceinline__ float xy_phi(const Lattice& lat, uint32_t sweep) {
  const uint4 w = philox(0u, sweep, kAxis, 0u, lat.rk);
  return __fmul_rn((float)(w.x >> 8), 0x1.921fb6p-22f);
}

// Clock model mirror index of a sweep: s = floor(w 2q / 2^32), the
// reflection p -> (s - p) mod q.
__device__ __forceinline__ uint32_t clock_mirror(const Lattice& lat, uint32_t sweep) {
  const uint4 w = philox(0u, sweep, kAxis, 0u, lat.rk);
  return (uint32_t)(((unsigned long long)w.x * (unsigned)(2 * lat.q)) >> 32);
}

// One step of the bit-sliced comparison u < t, most significant bit first:
// r holds bit `hb` of the 32 lanes' uniforms.
__device__ __forceinline__ void cmp_step(uint32_t& lt, uint32_t& eq, uint32_t r, uint32_t t, int hb) {
  if ((t >> hb) & 1u) {
    lt |= eq & ~r;
    eq &= r;
  } else {
    eq &= ~r;
  }
}

// Bernoulli word of row word g, direction d: bit b is set iff the 32-bit
// uniform u(b) < t, where bit 31-k of u(b) is bit b of the k-th word of the
// sequence, word k = word (k & 3) of Philox(g, sweep, BOND, 8d + k/4).  The
// comparison covers only the lanes in `live` (the others are masked off by
// the caller) and stops once all of them are decided; undecided lanes
// after 32 bits have u == t and stay 0.
__device__ __forceinline__ uint32_t bernoulli_word(uint32_t g, uint32_t sweep, int d, uint32_t t,
                                                   uint32_t live, const uint32_t* rk) {
  uint32_t lt = 0u, eq = live;
#pragma unroll 1
  for (int c = 0; c < 8; ++c) {
    const uint4 w = philox(g, sweep, kBond, (uint32_t)(8 * d + c), rk);
    const int hb = 31 - 4 * c;
    cmp_step(lt, eq, w.x, t, hb);
    cmp_step(lt, eq, w.y, t, hb - 1);
    cmp_step(lt, eq, w.z, t, hb - 2);
    cmp_step(lt, eq, w.w, t, hb - 3);
    if (eq == 0u) break;
  }
  return lt;
}

// Cluster draw value of a site from its 32-bit draw word w: floor(w q / 2^32)
// (Ising and XY use q = 2: 1 = flip to -1 / reflect).
__device__ __forceinline__ uint32_t draw_value(uint32_t w, uint32_t q) {
  return (uint32_t)(((unsigned long long)w * q) >> 32);
}

// 32 equality bits of two 32-byte rows held as 8 little-endian words.  A
// byte of x = a ^ b is zero iff bit 7 of ((x & 0x7f) + 0x7f) | x is clear
// (no carry crosses a byte); the four flags are gathered into a nibble by
// one multiplication (bits 7, 15, 23, 31 land on bits 28..31).
__device__ __forceinline__ uint32_t eq_bits(const uint32_t* a, const uint32_t* b) {
  uint32_t m = 0u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t x = a[k] ^ b[k];
    const uint32_t nz = (((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;
    const uint32_t z = nz ^ 0x80808080u;          // bit 7 of each byte: byte equal
    m |= ((z * 0x00204081u) >> 28) << (4 * k);
  }
  return m;
}

// v mod m for v in (-m, 2m), without a division.
__device__ __forceinline__ int wrap_mod(int v, int m) {
  return v < 0 ? v + m : (v >= m ? v - m : v);
}

// A clock state as an index into the model's tables: states set by the
// caller outside [0, q) are reduced mod q instead of indexing past a table
// (the branch is never taken for valid states).
__device__ __forceinline__ int clock_state(uint32_t p, int q) {
  return p < (uint32_t)q ? (int)p : (int)(p % (uint32_t)q);
}

// Highest set bit of `starts` at or below bit b (the start of b's x-run).
__device__ __forceinline__ uint32_t run_start(uint32_t starts, int b) {
  return 31u - __clz(starts & (kFull >> (31 - b)));
}

// ---------------------------------------------------------------- tiles
// A tile is 32 (one bit-plane word) x TY x TZ sites; one CTA of
// THREADS = TY*TZ threads (a thread per row word) labels it.  Shape S of
// dimension D is the S-th entry of the shape table; Tile<D> is the
// single-lattice tile.
template <int D_, int TY_, int TZ_>
struct TileShape {
  static constexpr int D = D_, TY = TY_, TZ = TZ_, ROWS = TY_ * TZ_, THREADS = TY_ * TZ_;
};
template <int D, int S>
using ShapeOf = TileShape<D, kShapeTY[D - 2][S], kShapeTZ[D - 2][S]>;
template <int D>
using Tile = ShapeOf<D, kSingleShape[D - 2]>;

struct TileCoord {
  int tx, x0, y0, z0;
};

template <class S>
__device__ __forceinline__ TileCoord tile_coord(const Lattice& lat, uint32_t tile) {
  int b = (int)tile;
  TileCoord c;
  c.tx = b % lat.ntx;
  b /= lat.ntx;
  c.x0 = c.tx * 32;
  c.y0 = (b % lat.nty) * S::TY;
  c.z0 = (b / lat.nty) * S::TZ;
  return c;
}

// ---------------------------------------------------------------- union-find
// Shared-memory forest of one tile: parents only decrease, so every loop is
// bounded by the tile size; the caps only guard against corrupted input.
__device__ __forceinline__ uint32_t sfind(volatile uint32_t* par, uint32_t x) {
  for (int it = 0; it < 65536; ++it) {
    const uint32_t p = par[x];
    if (p == x) return x;
    const uint32_t gp = par[p];
    if (gp == p) return p;
    par[x] = gp;  // path halving on a non-root
    x = gp;
  }
  return x;
}

__device__ __forceinline__ void sunion(uint32_t* par, uint32_t a, uint32_t b, int* err, uint32_t cap) {
  volatile uint32_t* vp = par;
  for (uint32_t it = 0; it < cap; ++it) {
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

// Global forest over tile-local roots: word = (parent << shift) | marker |
// draw, shift = sb + 1, marker = 1 << sb set on every local root (the only
// nodes these functions touch).  Links always point to a smaller index, so
// the root of every tree is its smallest site index.
// The roots of a and b, the two walks advanced in lockstep so that their
// loads are in flight together; each step on a non-root halves its path
// (the word of the node walked from is pointed at its grandparent).
// The walks read through L1 (ld.global.ca): the walks of one CTA meet on
// the same upper nodes.  L1 is not coherent with the other SMs' stores, so
// a word read may be older than L2's, but every word ever stored points to
// a smaller index of the same tree: an old word sends a walk along a longer
// path to an ancestor, or ends it at a node that has since been hooked, and
// gunion's atomicMin (in L2) then returns the node's real parent and the
// union continues from there.  Path halving with an old grandparent still
// stores an ancestor.  Only the atomic decides that a root is hooked.
// Earlier kernels' stores are not an issue: every caller reads the forest
// after griddepcontrol.wait (or a kernel boundary), which makes them
// visible to the grid's loads.
__device__ __forceinline__ void gfind2(uint32_t* f, uint32_t& a, uint32_t& b, int shift, uint32_t marker) {
  bool da = false, db = false;
  for (int it = 0; it < (1 << 22); ++it) {
    const uint32_t pa = da ? a : __ldca(&f[a]) >> shift;
    const uint32_t pb = db ? b : __ldca(&f[b]) >> shift;
    da = da || pa == a;
    db = db || pb == b;
    if (da && db) return;
    const uint32_t ga = da ? a : __ldca(&f[pa]) >> shift;
    const uint32_t gb = db ? b : __ldca(&f[pb]) >> shift;
    if (!da) {
      if (ga == pa) {
        a = pa;
        da = true;
      } else {
        __stcg(&f[a], (ga << shift) | marker);
        a = ga;
      }
    }
    if (!db) {
      if (gb == pb) {
        b = pb;
        db = true;
      } else {
        __stcg(&f[b], (gb << shift) | marker);
        b = gb;
      }
    }
    if (da && db) return;
  }
}

// Joins the trees of a and b; returns the root that was hooked under the
// other tree (each root is hooked at most once), or 0xffffffff if the two
// were already one tree.
__device__ __forceinline__ uint32_t gunion(uint32_t* f, uint32_t a, uint32_t b, int sb, int* err,
                                           uint32_t cap) {
  const int shift = sb + 1;
  const uint32_t marker = 1u << sb;
  for (uint32_t it = 0; it < cap; ++it) {
    gfind2(f, a, b, shift, marker);
    if (a == b) return 0xffffffffu;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicMin(&f[a], (b << shift) | marker);
    if ((old >> shift) == a) return a;
    a = old >> shift;
  }
  atomicExch(err, kErrTimeout);
  return 0xffffffffu;
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
template <int NW, typename T>
__device__ __forceinline__ T block_combine(T warp_total, T* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = warp_total;
  __syncthreads();
  T r = T(0);
  if (threadIdx.x < 32) {
    r = (lane < NW) ? scratch[lane] : T(0);
    r = warp_sum(r);
  }
  return r;
}

// ---------------------------------------------------------------- records
// Add a block's integer M, E (any thread's share) into slot slot_of % kSlots;
// called by all threads of the block.
template <int NW>
__device__ __forceinline__ void add_integer_sums(const Measure& mb, uint32_t slot_of, long long m,
                                                 long long e, long long* s_red) {
  const long long M = block_combine<NW>(warp_sum(m), s_red);
  const long long E = block_combine<NW>(warp_sum(e), s_red);
  if (threadIdx.x == 0) {
    unsigned long long* slot = mb.sums + 2 * (slot_of % kSlots);
    if (M) atomicAdd(&slot[0], (unsigned long long)M);
    if (E) atomicAdd(&slot[1], (unsigned long long)E);
  }
}

// Add a block's clock sums (fixed-point cos, sin of the states and cos of
// the bond differences) into its slot.
template <int NW>
__device__ __forceinline__ void add_clock_sums(const Measure& mb, uint32_t slot_of, long long cx,
                                               long long sy, long long eb, long long* s_red) {
  const long long X = block_combine<NW>(warp_sum(cx), s_red);
  const long long Y = block_combine<NW>(warp_sum(sy), s_red);
  const long long B = block_combine<NW>(warp_sum(eb), s_red);
  if (threadIdx.x == 0) {
    unsigned long long* slot = mb.csums + 3 * (slot_of % kSlots);
    if (X) atomicAdd(&slot[0], (unsigned long long)X);
    if (Y) atomicAdd(&slot[1], (unsigned long long)Y);
    if (B) atomicAdd(&slot[2], (unsigned long long)B);
  }
}

// Add a block's Potts histogram (shared bins) into its slot.
__device__ __forceinline__ void add_histogram(const Lattice& lat, const Measure& mb, uint32_t slot_of,
                                              const unsigned int* s_hist) {
  unsigned long long* slot = mb.hist + 256 * (slot_of % kSlots);
  for (int k = threadIdx.x; k < lat.q; k += blockDim.x)
    if (s_hist[k]) atomicAdd(&slot[k], (unsigned long long)s_hist[k]);
}

template <int NW>
__device__ __forceinline__ void commit_record(const Lattice& lat, const Measure& mb, uint32_t sweep,
                                              long long M, long long E, long long S2, double mx,
                                              double my, double exy, long long* s_ri);

// Record of `sweep` and the FP64 accumulators, from the slot sums (Ising /
// Potts) or the XY per-block partials, summed in a fixed order; the slots
// and the sweep's cluster count are reset.  Called by all threads of ONE
// block of a kernel that runs after every kernel that added to the sums.
// Every double operation rounds to nearest, no contraction.
template <int NW>
__device__ __forceinline__ void finalize_record(const Lattice& lat, const Measure& mb, uint32_t sweep,
                                                long long* s_ri, double* s_rd) {
  long long M = 0, E = 0, S2 = 0;
  double mx = 0.0, my = 0.0, exy = 0.0;
  if (lat.model == kXY) {
    double a = 0.0, c = 0.0, g = 0.0;
    for (int k = threadIdx.x; k < mb.xy_blocks; k += blockDim.x) {
      a = __dadd_rn(a, __ldcg(&mb.part_d[3 * k + 0]));
      c = __dadd_rn(c, __ldcg(&mb.part_d[3 * k + 1]));
      g = __dadd_rn(g, __ldcg(&mb.part_d[3 * k + 2]));
    }
    mx = block_combine<NW>(warp_sum(a), s_rd);
    my = block_combine<NW>(warp_sum(c), s_rd);
    exy = block_combine<NW>(warp_sum(g), s_rd);
  } else if (lat.model == kClock) {
    // exact integer sums, converted to double once
    long long a = 0, c = 0, g = 0;
    for (int k = threadIdx.x; k < kSlots; k += blockDim.x) {
      a += (long long)__ldcg(&mb.csums[3 * k + 0]);
      c += (long long)__ldcg(&mb.csums[3 * k + 1]);
      g += (long long)__ldcg(&mb.csums[3 * k + 2]);
      mb.csums[3 * k + 0] = 0ull;
      mb.csums[3 * k + 1] = 0ull;
      mb.csums[3 * k + 2] = 0ull;
    }
    const long long X = block_combine<NW>(warp_sum(a), s_ri);
    const long long Y = block_combine<NW>(warp_sum(c), s_ri);
    const long long B = block_combine<NW>(warp_sum(g), s_ri);
    mx = __dmul_rn((double)X, 0x1p-30);
    my = __dmul_rn((double)Y, 0x1p-30);
    exy = -__dmul_rn((double)B, 0x1p-30);
  } else {
    long long a = 0, c = 0, g = 0;
    for (int k = threadIdx.x; k < kSlots; k += blockDim.x) {
      a += (long long)__ldcg(&mb.sums[2 * k + 0]);
      c += (long long)__ldcg(&mb.sums[2 * k + 1]);
      mb.sums[2 * k + 0] = 0ull;
      mb.sums[2 * k + 1] = 0ull;
    }
    if (lat.model == kPotts) {
      // n[k] = sum over slots, all (slot, k) pairs spread over the block
      __shared__ unsigned long long s_n[256];
      for (int k = threadIdx.x; k < 256; k += blockDim.x) s_n[k] = 0ull;
      __syncthreads();
      for (int t = threadIdx.x; t < kSlots * lat.q; t += blockDim.x) {
        const int sl = t / lat.q, k = t % lat.q;
        const unsigned long long v = __ldcg(&mb.hist[256 * sl + k]);
        if (v) {
          atomicAdd(&s_n[k], v);
          mb.hist[256 * sl + k] = 0ull;
        }
      }
      __syncthreads();
      for (int k = threadIdx.x; k < lat.q; k += blockDim.x) g += (long long)(s_n[k] * s_n[k]);
    }
    M = block_combine<NW>(warp_sum(a), s_ri);
    E = block_combine<NW>(warp_sum(c), s_ri);
    S2 = block_combine<NW>(warp_sum(g), s_ri);
  }
  commit_record<NW>(lat, mb, sweep, M, E, S2, mx, my, exy, s_ri);
}

// The record of `sweep` from its sums and cluster count, and the update of
// the FP64 accumulators acc[6] (global, or a shared copy).  Called by one
// thread.
__device__ __forceinline__ void write_record(const Lattice& lat, const Measure& mb, uint32_t sweep,
                                             long long M, long long E, long long S2, double mx, double my,
                                             double exy, long long ncl, double* acc) {
  double M2, Ed;
  if (lat.model == kIsing) {
    M2 = __dmul_rn((double)M, (double)M);
    Ed = (double)E;
  } else if (lat.model == kPotts) {
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
  acc[0] = __dadd_rn(acc[0], 1.0);
  acc[1] = __dadd_rn(acc[1], M2);
  acc[2] = __dadd_rn(acc[2], __dmul_rn(M2, M2));
  acc[3] = __dadd_rn(acc[3], Ed);
  acc[4] = __dadd_rn(acc[4], __dmul_rn(Ed, Ed));
  acc[5] = __dadd_rn(acc[5], (double)ncl);
}

// Record of `sweep` from its gathered sums plus the sweep's cluster count
// (slots reset), and the FP64 accumulators.  Called by all threads of one
// block; thread 0 writes.
template <int NW>
__device__ __forceinline__ void commit_record(const Lattice& lat, const Measure& mb, uint32_t sweep,
                                              long long M, long long E, long long S2, double mx,
                                              double my, double exy, long long* s_ri) {
  long long nc = 0;
  unsigned long long* ncl_slots = mb.nclusters + kSlots * (sweep & 1u);
  for (int k = threadIdx.x; k < kSlots; k += blockDim.x) {
    nc += (long long)__ldcg(&ncl_slots[k]);
    ncl_slots[k] = 0ull;
  }
  const long long ncl = block_combine<NW>(warp_sum(nc), s_ri);
  if (threadIdx.x != 0) return;
  write_record(lat, mb, sweep, M, E, S2, mx, my, exy, ncl, mb.acc);
}

}  // namespace dev
}  // namespace swgb
