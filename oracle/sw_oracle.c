/*
 * Swendsen-Wang oracle: a plain, single-threaded CPU implementation of one
 * SW sweep for the 2D/3D Ising, q-state Potts and classical XY models
 * (Komura & Okabe, "CUDA programs for GPU computing of Swendsen-Wang
 * multi-cluster spin flip algorithm", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and this file
 * shares no code, header, table or constant with that path.
 *
 * Every step follows the paper's three SW steps in the paper's order
 * (Sec. 2: (1) active bond generation, (2) cluster labeling, (3) spin flip)
 * followed by the measurement of M and E (Sec. 2, Eqs. for M and the Potts
 * M^2).  Where the paper leaves a choice open the reading taken is stated at
 * the function.  Floating point is IEEE double except where a float decides
 * an integer (the XY bond test), which is taken in float as the kernels do.
 *
 * Lattice conventions: N = L^D sites, site i = x + L*(y + L*z), x fastest,
 * periodic boundaries (Sec. 1, below the Ising Hamiltonian).  Bond (i,d)
 * joins i and its +d neighbour.  J = 1.
 *
 * Bond bit-planes: plane d holds one bit per site for bond (i,d); each
 * lattice row (fixed y,z) is padded to W = ceil(L/32) 32-bit words; word
 * index = d*(R*W) + row*W + (x>>5), bit x&31, with R = L^(D-1) rows and
 * row = y + L*z.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), key = (seed low, seed high),
 * 32-bit counter words (c0, c1 = sweep, c2 = purpose, c3).  The paper uses
 * an LCG and says any other generator may be used (Sec. 2, technical
 * remarks).
 *   purpose 0 (INIT):  counter (i, 0, 0, 0), word 0 -> initial state of i.
 *   purpose 1 (BOND):  Ising/Potts: the 32-bit uniform u(i,d) of bond (i,d)
 *                      is spread over a sequence of 32 words shared by the
 *                      32 sites of i's row word g = row*W + (x>>5): bit 31-k
 *                      of u(i,d) is bit (x & 31) of the k-th word, the k-th
 *                      word being word (k & 3) of counter (g, k, 1, 8d + k/4).
 *                      XY: counter (i, k, 1, 0), word d -> u(i,d).
 *   purpose 2 (DRAW):  the cluster draw w(i), used when i is a cluster
 *                      root.  Potts with q > 2: counter (i >> 2, k, 2, 0),
 *                      word (i & 3).  Two-state draws (Ising, Potts q = 2,
 *                      XY, clock): one bit, bit (x & 31) of word 0 of
 *                      counter (g, k, 2, 1) for i's row word g; w(i) is
 *                      that bit times 2^31.
 *   purpose 3 (AXIS):  counter (0, k, 3, 0), word 0 -> XY mirror angle, or
 *                      the clock model's mirror index.
 *   Clock bonds:       counter (i, k, 1, 0), word d -> u(i,d) (32 bits).
 * (k is the sweep number, starting at 1; the initial state uses 0.)
 *
 * q-state clock model (the paper's discretised XY, theta_p = 2 pi p / q,
 * q = 512 in Sec. 3): spins p in [0, q) as uint16.  Per sweep a mirror
 * index s = floor(w q2 / 2^32), q2 = 2q, picks the reflection p -> (s - p)
 * mod q (the mirror line at angle pi s / q); the Ising projection of site i
 * is x_i = sin(pi k_i / q) with k_i = (2 p_i - s) mod 2q.  Bond (i,d) is
 * active iff x_i x_j > 0 and u(i,d) < t[k_i][k_j], t = floor((1 - exp(-2K
 * x_a x_b)) 2^32) from a table evaluated in double.  Moments are exact
 * integer sums of fixed-point tables C[k] = round(2^30 cos(2 pi k / q)),
 * S[k] = round(2^30 sin(2 pi k / q)): mx = 2^-30 sum_i C[p_i], my likewise
 * with S, and E = -2^-30 sum_<ij> C[(p_i - p_j) mod q]; each integer sum is
 * converted to double once, so the result does not depend on the order of
 * the sites.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ISING 0
#define OR_POTTS 1
#define OR_XY 2
#define OR_CLOCK 3

#define PURPOSE_INIT 0u
#define PURPOSE_BOND 1u
#define PURPOSE_DRAW 2u
#define PURPOSE_AXIS 3u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the definition in Salmon et al. (SC'11),
 * Sec. 3: ten rounds of two 32x32->64 multiplications whose high halves are
 * xor-ed with the other counter words and the round key; the key is bumped
 * by the Weyl constants between rounds. */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw4(uint64_t seed, uint32_t c0, uint32_t sweep, uint32_t purpose, uint32_t c3,
                  uint32_t w[4]) {
  uint32_t ctr[4] = {c0, sweep, purpose, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------------------------ */
/* Geometry helpers. */
static int64_t n_sites(int dim, int L) {
  int64_t n = 1;
  for (int d = 0; d < dim; ++d) n *= L;
  return n;
}

static int64_t row_words(int L) { return (L + 31) / 32; }

int64_t oracle_plane_words(int dim, int L) {
  return (int64_t)dim * n_sites(dim - 1, L) * row_words(L);
}

/* +d neighbour of site i with periodic wrap. */
static int64_t neighbour(int dim, int L, int64_t i, int d) {
  int64_t x = i % L;
  int64_t y = (i / L) % L;
  int64_t z = (dim == 3) ? i / ((int64_t)L * L) : 0;
  if (d == 0) x = (x + 1) % L;
  if (d == 1) y = (y + 1) % L;
  if (d == 2) z = (z + 1) % L;
  return x + (int64_t)L * (y + (int64_t)L * z);
}

static int64_t plane_word_index(int dim, int L, int64_t i, int d) {
  int64_t x = i % L;
  int64_t row = i / L;
  int64_t R = n_sites(dim - 1, L);
  return (int64_t)d * R * row_words(L) + row * row_words(L) + (x >> 5);
}

static int plane_bit(const uint32_t* planes, int dim, int L, int64_t i, int d) {
  return (int)((planes[plane_word_index(dim, L, i, d)] >> ((i % L) & 31)) & 1u);
}

/* ------------------------------------------------------------------------ */
/* Bond probability (Sec. 2, step (1)).  The printed formula
 * p = 1 - e^{2J/T} has lost its minus sign; the Ising SW probability is
 * p = 1 - exp(-2J/T).  For the Potts Hamiltonian H = -J sum(delta - 1)
 * (Sec. 1) the same construction gives p = 1 - exp(-J/T).  The bond test
 * is taken on integers: active iff the 32-bit draw u < t with
 * t = floor(p * 2^32), p evaluated in double as -expm1(-a). */
uint32_t oracle_bond_threshold(int model, double T) {
  double a = (model == OR_ISING) ? 2.0 / T : 1.0 / T;
  double p = -expm1(-a);
  double t = floor(p * 4294967296.0);
  if (t > 4294967295.0) t = 4294967295.0;
  if (t < 0.0) t = 0.0;
  return (uint32_t)t;
}

/* XY mirror angle for sweep k (Sec. 2, remark on ispr: one random direction
 * shared by all sites): phi = (w0 >> 8) * (2 pi / 2^24), taken in float. */
float oracle_xy_phi(uint64_t seed, uint32_t sweep) {
  uint32_t w[4];
  draw4(seed, 0u, sweep, PURPOSE_AXIS, 0u, w);
  const float step = (float)(6.283185307179586476925 / 16777216.0);
  return (float)(w[0] >> 8) * step;
}

/* ------------------------------------------------------------------------ */
/* Clock model tables.  Angle of state p: (2 pi p) / q in double; the
 * fixed-point cos/sin tables of the moments; the projection table x(k) = sin((pi k) / q) for k in [0, 2q); the threshold
 * table t[a][b] = floor(-expm1(-(2/T) x(a) x(b)) 2^32) where x(a) x(b) > 0,
 * else 0. */
static const double OR_PI = 3.141592653589793238463;

/* Fixed-point clock tables: C[p] = round(2^30 cos(2 pi p / q)), S[p] =
 * round(2^30 sin(2 pi p / q)) (nearest, halves away from zero). */
void oracle_clock_fixed(int q, int64_t* C, int64_t* S) {
  for (int p = 0; p < q; ++p) {
    const double a = (2.0 * OR_PI * (double)p) / (double)q;
    C[p] = llround(ldexp(cos(a), 30));
    S[p] = llround(ldexp(sin(a), 30));
  }
}

void oracle_clock_thresholds(int q, double T, uint32_t* t) {
  const int q2 = 2 * q;
  double* x = (double*)malloc(sizeof(double) * (size_t)q2);
  for (int k = 0; k < q2; ++k) x[k] = sin((OR_PI * (double)k) / (double)q);
  const double twoK = 2.0 / T;
  for (int a = 0; a < q2; ++a)
    for (int b = 0; b < q2; ++b) {
      const double prod = x[a] * x[b];
      uint32_t v = 0u;
      if (prod > 0.0) {
        double f = floor(-expm1(-(twoK * prod)) * 4294967296.0);
        if (f > 4294967295.0) f = 4294967295.0;
        v = (uint32_t)f;
      }
      t[(size_t)a * (size_t)q2 + (size_t)b] = v;
    }
  free(x);
}

/* The threshold table of the last (q, T) asked for, kept between sweeps. */
static const uint32_t* clock_table(int q, double T) {
  static uint32_t* tab = NULL;
  static int tab_q = 0;
  static double tab_T = 0.0;
  if (!tab || tab_q != q || tab_T != T) {
    free(tab);
    tab = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(2 * q) * (size_t)(2 * q));
    oracle_clock_thresholds(q, T, tab);
    tab_q = q;
    tab_T = T;
  }
  return tab;
}

uint32_t oracle_clock_mirror(uint64_t seed, uint32_t sweep, int q) {
  uint32_t w[4];
  draw4(seed, 0u, sweep, PURPOSE_AXIS, 0u, w);
  return (uint32_t)(((uint64_t)w[0] * (uint64_t)(2 * q)) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Initial configuration (paper: device_function_spinset; the distribution is
 * not stated, a uniformly random start is taken). */
int oracle_init(int model, int dim, int L, int q, uint64_t seed, void* spins) {
  int64_t N = n_sites(dim, L);
  const float step = (float)(6.283185307179586476925 / 16777216.0);
  for (int64_t i = 0; i < N; ++i) {
    uint32_t w[4];
    draw4(seed, (uint32_t)i, 0u, PURPOSE_INIT, 0u, w);
    if (model == OR_ISING) {
      ((int8_t*)spins)[i] = (w[0] >> 31) ? (int8_t)-1 : (int8_t)1;
    } else if (model == OR_POTTS) {
      ((uint8_t*)spins)[i] = (uint8_t)(((uint64_t)w[0] * (uint64_t)q) >> 32);
    } else if (model == OR_CLOCK) {
      ((uint16_t*)spins)[i] = (uint16_t)(((uint64_t)w[0] * (uint64_t)q) >> 32);
    } else {
      ((float*)spins)[i] = (float)(w[0] >> 8) * step;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The 32 words of the bond sequence of row word g and direction d: word k
 * is word (k & 3) of counter (g, sweep, 1, 8d + k/4). */
static void bond_sequence(uint64_t seed, uint32_t sweep, uint32_t g, int d, uint32_t R[32]) {
  for (int c = 0; c < 8; ++c) {
    uint32_t w[4];
    draw4(seed, g, sweep, PURPOSE_BOND, (uint32_t)(8 * d + c), w);
    for (int j = 0; j < 4; ++j) R[4 * c + j] = w[j];
  }
}

/* u(i,d) of the site at bit b of the row word: bit 31-k of u is bit b of
 * the k-th word of the sequence. */
static uint32_t bond_uniform(const uint32_t R[32], int b) {
  uint32_t u = 0;
  for (int k = 0; k < 32; ++k) u |= ((R[k] >> b) & 1u) << (31 - k);
  return u;
}

/* Step (1): active bond generation (Sec. 2).
 * Ising/Potts: bond (i,j) active iff s_i == s_j and u(i,d) < t.
 * XY (embedded Ising clusters, Wolff 1989; Sec. 1 and Sec. 2 remarks on the
 * clock model): project on r = (cos phi, sin phi): x_i = cos(theta_i - phi);
 * bond active iff x_i x_j > 0 and u < 1 - exp(-2K x_i x_j), with
 * u = (w_d >> 8) 2^-24.  Taken in float (the decision is an integer). */
void oracle_bonds(int model, int dim, int L, int q, double T, uint64_t seed,
                  uint32_t sweep, const void* spins, uint32_t* planes) {
  (void)q;
  int64_t N = n_sites(dim, L);
  memset(planes, 0, sizeof(uint32_t) * (size_t)oracle_plane_words(dim, L));
  uint32_t t = (model == OR_XY) ? 0u : oracle_bond_threshold(model, T);
  float phi = (model == OR_XY) ? oracle_xy_phi(seed, sweep) : 0.0f;
  float twoK = (float)(2.0 / T);
  uint32_t R[3][32];           /* bond sequences of the current row word */
  int64_t cached_g = -1;
  const uint32_t* ctab = NULL;
  uint32_t mirror = 0;
  const int q2 = 2 * q;
  if (model == OR_CLOCK) {
    ctab = clock_table(q, T);
    mirror = oracle_clock_mirror(seed, sweep, q);
  }
  for (int64_t i = 0; i < N; ++i) {
    int64_t x = i % L;
    int64_t g = (i / L) * row_words(L) + (x >> 5);
    uint32_t w[4];
    if (model == OR_XY || model == OR_CLOCK) {
      draw4(seed, (uint32_t)i, sweep, PURPOSE_BOND, 0u, w);
    } else if (g != cached_g) {
      for (int d = 0; d < dim; ++d) bond_sequence(seed, sweep, (uint32_t)g, d, R[d]);
      cached_g = g;
    }
    for (int d = 0; d < dim; ++d) {
      int64_t j = neighbour(dim, L, i, d);
      int active = 0;
      if (model == OR_ISING) {
        active = (((const int8_t*)spins)[i] == ((const int8_t*)spins)[j]) &&
                 (bond_uniform(R[d], (int)(x & 31)) < t);
      } else if (model == OR_POTTS) {
        active = (((const uint8_t*)spins)[i] == ((const uint8_t*)spins)[j]) &&
                 (bond_uniform(R[d], (int)(x & 31)) < t);
      } else if (model == OR_CLOCK) {
        const int pi_ = ((const uint16_t*)spins)[i];
        const int pj_ = ((const uint16_t*)spins)[j];
        const int ka = ((2 * pi_ - (int)mirror) % q2 + q2) % q2;
        const int kb = ((2 * pj_ - (int)mirror) % q2 + q2) % q2;
        active = w[d] < ctab[(size_t)ka * (size_t)q2 + (size_t)kb];
      } else {
        float ti = ((const float*)spins)[i];
        float tj = ((const float*)spins)[j];
        float xi = cosf(ti - phi);
        float xj = cosf(tj - phi);
        float prod = xi * xj;
        if (prod > 0.0f) {
          float p = -expm1f(-(twoK * prod));
          float u = (float)(w[d] >> 8) * 0x1p-24f;
          active = u < p;
        }
      }
      if (active) planes[plane_word_index(dim, L, i, d)] |= 1u << (x & 31);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Step (2): cluster labeling (Sec. 2).  Sequential union-find, the class the
 * paper cites as the CPU standard (Hoshen-Kopelman); the larger root is
 * always linked under the smaller one, so every root is the smallest site
 * index of its tree and label[i] = find(i) is the minimum site index of i's
 * cluster. */
static int64_t uf_find(int64_t* parent, int64_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]]; /* path halving */
    x = parent[x];
  }
  return x;
}

static void uf_unite(int64_t* parent, int64_t a, int64_t b) {
  a = uf_find(parent, a);
  b = uf_find(parent, b);
  if (a == b) return;
  if (a < b) parent[b] = a;
  else parent[a] = b;
}

int oracle_labels(int dim, int L, const uint32_t* planes, int32_t* labels) {
  int64_t N = n_sites(dim, L);
  int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  if (!parent) return -1;
  for (int64_t i = 0; i < N; ++i) parent[i] = i;
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < dim; ++d)
      if (plane_bit(planes, dim, L, i, d)) uf_unite(parent, i, neighbour(dim, L, i, d));
  for (int64_t i = 0; i < N; ++i) labels[i] = (int32_t)uf_find(parent, i);
  free(parent);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step (3): spin flip (Sec. 2; paper: spin_select then spin_flip).  Each
 * cluster takes one new state from its root's cluster draw w (purpose 2):
 *   Ising: +1 if w < 2^31 else -1   (set at random, Sec. 2 step (3))
 *   Potts: floor(w q / 2^32)        (uniform of q states)
 *   XY:    reflect about the line perpendicular to r iff w >= 2^31:
 *          theta' = 2 phi + pi - theta, wrapped to [0, 2 pi)  (Wolff's
 *          embedded-cluster flip).
 *   Clock: reflect iff w >= 2^31: p' = (s - p) mod q.
 * Returns the number of clusters (roots). */
int64_t oracle_flip(int model, int dim, int L, int q, uint64_t seed, uint32_t sweep,
                    const int32_t* labels, void* spins) {
  int64_t N = n_sites(dim, L);
  int64_t nclusters = 0;
  uint32_t* root_draw = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  if (!root_draw) return -1;
  const int two_state = !(model == OR_POTTS && q > 2);
  for (int64_t r = 0; r < N; ++r) {
    if (labels[r] != r) continue;
    uint32_t w[4];
    if (two_state) {
      const int64_t x = r % L;
      const int64_t g = (r / L) * row_words(L) + (x >> 5);
      draw4(seed, (uint32_t)g, sweep, PURPOSE_DRAW, 1u, w);
      root_draw[r] = ((w[0] >> (x & 31)) & 1u) << 31;
    } else {
      draw4(seed, (uint32_t)(r >> 2), sweep, PURPOSE_DRAW, 0u, w);
      root_draw[r] = w[r & 3];
    }
    ++nclusters;
  }
  double phi = (model == OR_XY) ? (double)oracle_xy_phi(seed, sweep) : 0.0;
  const uint32_t clock_mirror = (model == OR_CLOCK) ? oracle_clock_mirror(seed, sweep, q) : 0u;
  const double two_pi = 6.283185307179586476925;
  const double pi = 3.141592653589793238463;
  for (int64_t i = 0; i < N; ++i) {
    uint32_t w = root_draw[labels[i]];
    if (model == OR_ISING) {
      ((int8_t*)spins)[i] = (w >> 31) ? (int8_t)-1 : (int8_t)1;
    } else if (model == OR_POTTS) {
      ((uint8_t*)spins)[i] = (uint8_t)(((uint64_t)w * (uint64_t)q) >> 32);
    } else if (model == OR_CLOCK) {
      if (w >> 31) {
        const int p_ = ((uint16_t*)spins)[i];
        ((uint16_t*)spins)[i] = (uint16_t)((((int)clock_mirror - p_) % q + q) % q);
      }
    } else if (w >> 31) {
      double th = 2.0 * phi + pi - (double)((float*)spins)[i];
      while (th >= two_pi) th -= two_pi;
      while (th < 0.0) th += two_pi;
      ((float*)spins)[i] = (float)th;
    }
  }
  free(root_draw);
  return nclusters;
}

/* ------------------------------------------------------------------------ */
/* Measurement (Sec. 2: M = sum s_i and the energy; Potts M^2 equation).
 *   Ising: M = sum s_i, E = -sum_<ij> s_i s_j, M2 = M^2
 *   Potts: n[k] histogram, S2 = sum n[k]^2, M2 = (q S2 - N^2)/(q-1),
 *          E = sum_<ij> (1 - delta(s_i,s_j))   (the paper's H with J = 1)
 *   XY:    mx = sum cos, my = sum sin, M2 = mx^2 + my^2,
 *          E = -sum_<ij> cos(theta_i - theta_j)
 * The quartic moment is M4 = (M2)^2 for every model (for Potts the paper
 * gives M^2 only; squaring it reduces to the Ising M^4 at q = 2). */
typedef struct {
  int64_t M;
  int64_t E;
  int64_t nclusters;
  int64_t S2;
  double mx;
  double my;
  double e_xy;
  double M2;
  double Ed;
} oracle_record;

void oracle_moments(int model, int dim, int L, int q, const void* spins,
                    oracle_record* rec) {
  int64_t N = n_sites(dim, L);
  memset(rec, 0, sizeof(*rec));
  if (model == OR_ISING) {
    const int8_t* s = (const int8_t*)spins;
    int64_t M = 0, E = 0;
    for (int64_t i = 0; i < N; ++i) {
      M += s[i];
      for (int d = 0; d < dim; ++d) E -= (int64_t)s[i] * s[neighbour(dim, L, i, d)];
    }
    rec->M = M;
    rec->E = E;
    rec->M2 = (double)M * (double)M;
    rec->Ed = (double)E;
  } else if (model == OR_POTTS) {
    const uint8_t* s = (const uint8_t*)spins;
    int64_t* n = (int64_t*)calloc((size_t)q, sizeof(int64_t));
    int64_t E = 0;
    for (int64_t i = 0; i < N; ++i) {
      n[s[i]] += 1;
      for (int d = 0; d < dim; ++d) E += (s[i] != s[neighbour(dim, L, i, d)]) ? 1 : 0;
    }
    int64_t S2 = 0;
    for (int k = 0; k < q; ++k) S2 += n[k] * n[k];
    free(n);
    rec->S2 = S2;
    rec->E = E;
    rec->M2 = (double)((int64_t)q * S2 - N * N) / (double)(q - 1);
    rec->Ed = (double)E;
  } else if (model == OR_CLOCK) {
    const uint16_t* s = (const uint16_t*)spins;
    int64_t* C = (int64_t*)malloc(sizeof(int64_t) * (size_t)q);
    int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (size_t)q);
    oracle_clock_fixed(q, C, S);
    int64_t mxi = 0, myi = 0, eb = 0;
    for (int64_t i = 0; i < N; ++i) {
      mxi += C[s[i]];
      myi += S[s[i]];
      for (int d = 0; d < dim; ++d) eb += C[((int)s[i] - (int)s[neighbour(dim, L, i, d)] + q) % q];
    }
    free(C); free(S);
    const double mx = (double)mxi * 0x1p-30, my = (double)myi * 0x1p-30;
    const double e = -((double)eb * 0x1p-30);
    rec->mx = mx;
    rec->my = my;
    rec->e_xy = e;
    rec->M2 = mx * mx + my * my;
    rec->Ed = e;
  } else {
    const float* th = (const float*)spins;
    double mx = 0.0, my = 0.0, e = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      mx += cos((double)th[i]);
      my += sin((double)th[i]);
      for (int d = 0; d < dim; ++d)
        e -= cos((double)th[i] - (double)th[neighbour(dim, L, i, d)]);
    }
    rec->mx = mx;
    rec->my = my;
    rec->e_xy = e;
    rec->M2 = mx * mx + my * my;
    rec->Ed = e;
  }
}

/* ------------------------------------------------------------------------ */
/* A whole run: the sample program's main loop (Sec. 2: mcs1 discarded
 * sweeps, mcs2 measured sweeps), accumulating sum M^2, M^4, E, E^2 and the
 * cluster count over measured sweeps in double, in sweep order. */
typedef struct {
  double n_sweeps;
  double sum_M2;
  double sum_M4;
  double sum_E;
  double sum_E2;
  double sum_nclusters;
} oracle_acc;

typedef struct {
  int model, dim, L, q;
  double T;
  uint64_t seed;
  int64_t N;
  uint32_t sweep;
  void* spins;
  uint32_t* planes;
  int32_t* labels;
  oracle_record last;
  oracle_acc acc;
} oracle_sw;

static size_t spin_bytes(int model) {
  return model == OR_XY ? sizeof(float) : model == OR_CLOCK ? sizeof(uint16_t) : 1;
}

oracle_sw* oracle_create(int model, int dim, int L, int q, double T, uint64_t seed) {
  if (model < 0 || model > 3 || dim < 2 || dim > 3 || L < 2 || !(T > 0.0)) return NULL;
  if (model == OR_POTTS && (q < 2 || q > 256)) return NULL;
  if (model == OR_CLOCK && (q < 2 || q > 1024)) return NULL;
  oracle_sw* o = (oracle_sw*)calloc(1, sizeof(oracle_sw));
  if (!o) return NULL;
  o->model = model; o->dim = dim; o->L = L; o->q = (model == OR_POTTS || model == OR_CLOCK) ? q : 2;
  o->T = T; o->seed = seed; o->N = n_sites(dim, L); o->sweep = 0;
  o->spins = calloc((size_t)o->N, spin_bytes(model));
  o->planes = (uint32_t*)calloc((size_t)oracle_plane_words(dim, L), sizeof(uint32_t));
  o->labels = (int32_t*)calloc((size_t)o->N, sizeof(int32_t));
  if (!o->spins || !o->planes || !o->labels) {
    free(o->spins); free(o->planes); free(o->labels); free(o);
    return NULL;
  }
  oracle_init(model, dim, L, o->q, seed, o->spins);
  return o;
}

void oracle_destroy(oracle_sw* o) {
  if (!o) return;
  free(o->spins); free(o->planes); free(o->labels); free(o);
}

static void accumulate(oracle_acc* a, const oracle_record* r) {
  double m2 = r->M2;
  double e = r->Ed;
  a->n_sweeps += 1.0;
  a->sum_M2 += m2;
  a->sum_M4 += m2 * m2;
  a->sum_E += e;
  a->sum_E2 += e * e;
  a->sum_nclusters += (double)r->nclusters;
}

/* One sweep with an optionally injected bond mask (NULL: draw the bonds). */
int oracle_sweep_with_planes(oracle_sw* o, const uint32_t* planes_in, int measure) {
  o->sweep += 1;
  if (planes_in)
    memcpy(o->planes, planes_in, sizeof(uint32_t) * (size_t)oracle_plane_words(o->dim, o->L));
  else
    oracle_bonds(o->model, o->dim, o->L, o->q, o->T, o->seed, o->sweep, o->spins, o->planes);
  if (oracle_labels(o->dim, o->L, o->planes, o->labels) != 0) return -1;
  int64_t ncl = oracle_flip(o->model, o->dim, o->L, o->q, o->seed, o->sweep, o->labels, o->spins);
  if (ncl < 0) return -1;
  if (measure) {
    oracle_moments(o->model, o->dim, o->L, o->q, o->spins, &o->last);
    o->last.nclusters = ncl;
    accumulate(&o->acc, &o->last);
  }
  return 0;
}

int oracle_sweep(oracle_sw* o, int n, int measure) {
  for (int k = 0; k < n; ++k)
    if (oracle_sweep_with_planes(o, NULL, measure) != 0) return -1;
  return 0;
}

void* oracle_spins(oracle_sw* o) { return o->spins; }
uint32_t* oracle_planes(oracle_sw* o) { return o->planes; }
int32_t* oracle_label_array(oracle_sw* o) { return o->labels; }
uint32_t oracle_sweep_counter(oracle_sw* o) { return o->sweep; }
void oracle_set_sweep_counter(oracle_sw* o, uint32_t k) { o->sweep = k; }
void oracle_last_record(oracle_sw* o, oracle_record* out) { *out = o->last; }
void oracle_take_acc(oracle_sw* o, oracle_acc* out) {
  *out = o->acc;
  memset(&o->acc, 0, sizeof(o->acc));
}
