/*
 * sw.h - C ABI of the GB300 Swendsen-Wang engine.
 *
 * One SW sweep (Komura & Okabe, Sec. 2) = (1) active bond generation,
 * (2) cluster labeling, (3) cluster flip, followed by the measurement of the
 * magnetization and energy (Sec. 2, equations for M and the Potts M^2; the
 * moment ratio U of Sec. 3).  Models: Ising (Eq. for H_Ising), q-state Potts
 * (Eq. for H_Potts) and classical XY (Eq. for H_XY) on the 2D square and 3D
 * simple cubic lattices with periodic boundaries (Sec. 1).  Every step runs
 * in CUDA kernels for sm_103a on one GPU; the host only launches them.
 *
 * Conventions shared by every call:
 *   - N = L^dim sites; site i = x + L*(y + L*z), x fastest; J = 1.
 *   - Spins (host or device buffers passed to the get/set calls):
 *       SW_ISING  int8_t  +1 / -1
 *       SW_POTTS  uint8_t 0 .. q-1
 *       SW_XY     float   angle theta in [0, 2 pi)
 *       SW_CLOCK  uint16  clock state p in [0, q), angle 2 pi p / q (a state
 *                         set outside [0, q) is read mod q)
 *   - Bond bit-planes: plane d (0 <= d < dim) holds bond (i, i + e_d); each
 *     row (fixed y, z) is padded to W = ceil(L/32) uint32 words; the bit of
 *     site i is word d*R*W + row*W + (x >> 5), bit (x & 31), with
 *     R = L^(dim-1) rows and row = y + L*z.
 *   - Labels: int32, label[i] = smallest site index in i's cluster.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *     key = (seed low 32 bits, seed high 32 bits) and counter
 *     (c0, sweep, purpose, c3); sweep k (1-based) of the run uses k, the
 *     initial state uses 0.  Purposes:
 *       0 initial state: counter (i, 0, 0, 0), word 0;
 *       1 bonds: Ising/Potts bond (i,d) is active iff the spins are equal
 *         and a 32-bit uniform u(i,d) < floor(p 2^32); bit 31-k of u(i,d)
 *         is bit (x & 31) of word k of the sequence of i's row word
 *         g = row*W + (x >> 5), word k = word (k & 3) of counter
 *         (g, k_sweep, 1, 8d + k/4).  XY: counter (i, sweep, 1, 0), word d;
 *       2 cluster draws, used when site i is the root of its cluster:
 *         Potts with q > 2: w = word (i & 3) of counter (i >> 2, sweep, 2, 0);
 *         two-state draws (Ising, Potts q = 2, XY, clock): one bit, bit
 *         (x & 31) of word 0 of counter (g, sweep, 2, 1) for i's row word
 *         g = row*W + (x >> 5), read as w = bit * 2^31;
 *       3 XY mirror angle: counter (0, sweep, 3, 0), word 0.
 *   - q-state clock model (the paper's discretised XY, Sec. 1 and Sec. 3,
 *     q = 512 there): per sweep a mirror index s = floor(w 2q / 2^32) from
 *     counter (0, sweep, 3, 0) word 0 picks the reflection p -> (s - p) mod q.
 *     The Ising projection of site i is x_i = sin(pi k_i / q), k_i =
 *     (2 p_i - s) mod 2q.  Bond (i,d) is active iff w_d < t[k_i][k_j], w_d =
 *     word d of counter (i, sweep, 1, 0) and t[a][b] = floor(-expm1(-(2/T)
 *     x_a x_b) 2^32) where x_a x_b > 0, else 0 (double, computed once per
 *     lattice).  Clusters reflect when their root's draw w >= 2^31.  Moments
 *     are exact integer sums of the fixed-point tables C[k] = round(2^30
 *     cos(2 pi k / q)) and S[k] = round(2^30 sin(2 pi k / q)): mx = 2^-30
 *     sum_i C[p_i], my = 2^-30 sum_i S[p_i], E = -2^-30 sum_<ij>
 *     C[(p_i - p_j) mod q], each integer sum converted to double once, so
 *     trajectories and moments are reproducible bit for bit.
 *   - Ownership: the handle owns every device buffer it allocates; host
 *     buffers passed in stay owned by the caller and are only read or
 *     written during the call (the call synchronises the handle's stream).
 *   - Errors: functions returning int return SW_OK (0) or a negative
 *     sw_status; sw_create returns NULL.  sw_last_error() gives a message
 *     for the last failure on the calling thread.  No C++ exception crosses
 *     this interface.
 *   - Streams: all GPU work of a handle is ordered on one CUDA stream (its
 *     own non-blocking stream unless sw_set_stream gave another).  sw_sweep
 *     and sw_discard only enqueue; the calls that return data synchronise.
 */
#ifndef SW_GB300_H
#define SW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum sw_model { SW_ISING = 0, SW_POTTS = 1, SW_XY = 2, SW_CLOCK = 3 };

enum sw_status {
  SW_OK = 0,
  SW_ERR_BAD_ARG = -1,  /* invalid argument, size or NULL handle          */
  SW_ERR_OOM = -2,      /* device or host allocation failed                */
  SW_ERR_CUDA = -3,     /* a CUDA call or kernel launch failed             */
  SW_ERR_TIMEOUT = -4,  /* a device-side loop hit its iteration cap        */
  SW_ERR_RANGE = -5     /* requested sweep records are no longer retained  */
};

typedef struct sw_handle sw_handle;

/* Sums over the measured sweeps since the previous sw_measure (Sec. 2,
 * outputs of the sample program; Sec. 3, moment ratio U).
 *   M2 per sweep: Ising M^2 with M = sum s_i; Potts (q sum_k n_k^2 - N^2)/(q-1)
 *   (Sec. 2, Potts equation); XY and clock (sum cos)^2 + (sum sin)^2.
 *   M4 = (M2)^2.  E per sweep: Ising -sum s_i s_j; Potts sum (1 - delta);
 *   XY and clock -sum cos(theta_i - theta_j).
 *   U = <M4>/<M2>^2;  e_per_spin = <E>/N;  c_per_spin = (<E^2>-<E>^2)/(N T^2);
 *   mean_cluster_size = N / <number of clusters>. */
typedef struct sw_moments {
  double n_sweeps;
  double sum_M2;
  double sum_M4;
  double sum_E;
  double sum_E2;
  double sum_nclusters;
  double U;
  double e_per_spin;
  double c_per_spin;
  double mean_cluster_size;
} sw_moments;

/* One measured sweep's record (the per-sweep series).  Ising: M, E; Potts:
 * E, S2 = sum_k n_k^2; XY: mx, my, e_xy.  M2 and Ed are the per-sweep M2 and
 * E used by the accumulators. */
typedef struct sw_record {
  uint64_t sweep;
  int64_t M;
  int64_t E;
  int64_t nclusters;
  int64_t S2;
  double mx;
  double my;
  double e_xy;
  double M2;
  double Ed;
} sw_record;

/* Create a lattice (paper: device_function_spinset + the parameters nx,
 * mcs1/mcs2 of Sec. 2).  model: sw_model; dim: 2 or 3; L >= 4; q: Potts
 * states 2..256 or clock states 2..1024 (ignored otherwise); T > 0 in units
 * of J; seed: Philox key.
 * The initial state is random from the seed (sweep counter 0).  Returns NULL
 * on a bad argument, an oversized lattice (N * 2^(b+1) must fit in 32 bits,
 * b = bits of the cluster draw: 1 for Ising/XY, ceil(log2 q) for Potts) or
 * a CUDA failure.  Uses the current CUDA device. */
sw_handle* sw_create(int model, int dim, int L, int q, double T, uint64_t seed);

/* Free every device buffer and the owned stream.  NULL is allowed. */
void sw_destroy(sw_handle* h);

/* Message for the last failing call on this thread ("" if none). */
const char* sw_last_error(void);

/* Enqueue n measured SW sweeps (Sec. 2 steps (1)-(3) + measurement): per
 * sweep the records and the accumulators of sw_measure are updated on the
 * device.  n >= 0.  Asynchronous: returns after the launches. */
int sw_sweep(sw_handle* h, int n);

/* Enqueue n SW sweeps without measurement (the paper's discarded mcs1
 * sweeps; also the "update only" timing of Tables 1 and 2). */
int sw_discard(sw_handle* h, int n);

/* Synchronise, copy the accumulators of the sweeps measured since the last
 * call into *out, then reset them.  Returns SW_ERR_TIMEOUT if any device
 * loop of the queued sweeps hit its cap. */
int sw_measure(sw_handle* h, sw_moments* out);

/* Synchronise the handle's stream and report any device error flag. */
int sw_sync(sw_handle* h);

/* Non-blocking completion test of the work enqueued so far on the handle's
 * stream: 1 if all of it has completed, 0 if some is still running, a
 * negative sw_status on error (SW_ERR_BAD_ARG for NULL, SW_ERR_CUDA).  It
 * neither waits nor reads the device error flag (sw_sync does both).  A
 * serving loop polls it to advance each lattice as soon as its previous
 * chunk of sweeps is done.  sw_batch_query (below) does the same for a
 * batch's stream. */
int sw_query(sw_handle* h);

/* Failure-detection hook (no counterpart in the paper).  Every device loop
 * whose trip count depends on the data -- the union retries of the tile
 * labeling (shared memory) and of the global merge, the compression and
 * canonical-label walks, the label-equivalence walks and iterations of
 * sw_relabel -- is capped.  On valid input each ends far below the cap
 * (parents only decrease), so the cap only turns a corrupted forest into an
 * error instead of a hang: a loop that reaches it writes SW_ERR_TIMEOUT to
 * the handle's device error flag and gives up, the kernel returns, and the
 * next synchronising call (sw_sync, sw_measure, the getters,
 * sw_label_from_bonds, sw_relabel) returns SW_ERR_TIMEOUT and clears the
 * flag.  The results of the affected call are then undefined; the handle
 * itself stays usable.
 *   cap >= 0   every capped loop of this handle's own launches gives up
 *              after cap steps (0: at once; used by the tests to exercise
 *              the error path without a fault)
 *   cap < 0    restores the production cap (2^22 steps)
 * Takes effect for launches enqueued after the call; a batch member runs
 * with the cap its handle had when the batch last captured its sweep (a
 * member joining or leaving, or a configuration change, recaptures it).
 * Returns SW_ERR_BAD_ARG for a NULL handle or cap > 2^22. */
int sw_set_loop_cap(sw_handle* h, long long cap);

/* Use `stream` (a cudaStream_t, e.g. torch.cuda.Stream.cuda_stream; NULL =
 * the legacy default stream) for all further work of the handle.  The
 * caller keeps ownership of the stream and must keep it alive while the
 * handle uses it. */
int sw_set_stream(sw_handle* h, void* stream);

/* Number of sweeps done so far (the sweep field of the Philox counter of
 * the last sweep), and its setter for checkpoint/resume. */
uint64_t sw_sweep_counter(sw_handle* h);
int sw_set_sweep_counter(sw_handle* h, uint64_t k);

/* Sizes of the buffers below: sites, bytes of the spin array, bond words. */
size_t sw_num_sites(sw_handle* h);
size_t sw_spin_bytes(sw_handle* h);
size_t sw_bond_words(sw_handle* h);

/* Copy the spin state to / from a caller-owned HOST buffer of exactly
 * sw_spin_bytes bytes.  Synchronous. */
int sw_get_spins(sw_handle* h, void* host, size_t bytes);
int sw_set_spins(sw_handle* h, const void* host, size_t bytes);

/* Same with a caller-owned DEVICE buffer; enqueued on the handle's stream
 * (asynchronous with respect to the host). */
int sw_get_spins_device(sw_handle* h, void* dev, size_t bytes);
int sw_set_spins_device(sw_handle* h, const void* dev, size_t bytes);

/* Canonical labels (min site index per cluster, Sec. 2 step (2)) of the
 * clusters of the last sweep, into a host int32 buffer of n = N entries
 * (all zero before the first sweep). */
int sw_get_labels(sw_handle* h, int32_t* host, size_t n);

/* Bond bit-planes of the last sweep into a host buffer of sw_bond_words
 * words. */
int sw_get_bonds(sw_handle* h, uint32_t* host, size_t words);

/* Label the clusters of an injected bond mask (host bit-planes, layout
 * above) with the same kernels the sweep uses, writing N canonical labels
 * to host_labels.  Overwrites the handle's bond and label buffers (the
 * spins are untouched).  For parity tests of the labeling step. */
int sw_label_from_bonds(sw_handle* h, const uint32_t* host_mask, int32_t* host_labels);

/* Label the handle's current bond planes (those of the last sweep, or of
 * the last sw_label_from_bonds) with one of two methods and time it:
 *   SW_LABEL_TILE_UF      the sweep's own labeling: union-find inside
 *                         32-wide tiles in shared memory, then a merge of
 *                         the tile-local roots across tile faces;
 *   SW_LABEL_EQUIVALENCE  the labeler the paper runs (Sec. 2, label
 *                         equivalence of Hawick et al. in the refinement of
 *                         Kalentev et al.): a scanning kernel lowers the
 *                         entry of each site's root to the smallest bonded
 *                         label, an analysis kernel jumps every label to its
 *                         root, and the host reads a change flag after each
 *                         iteration until a scan changes nothing.
 * Both write the same canonical labels (min site index per cluster) to the
 * handle's label buffer; host_labels (N int32, may be NULL) receives a copy.
 * *ms (may be NULL) gets the device time between events recorded on the
 * handle's stream around the labeling only (for EQUIVALENCE it includes the
 * per-iteration flag reads); *iterations (may be NULL) the number of
 * scan + analysis passes (1 for TILE_UF).  Synchronous.  The spins, the
 * sweep counter and the measurement state are untouched; the tile forest is
 * rebuilt by TILE_UF and left alone by EQUIVALENCE.  Errors: SW_ERR_BAD_ARG
 * (NULL handle, unknown method), SW_ERR_CUDA (launch or allocation failure;
 * message in sw_last_error). */
enum sw_label_method { SW_LABEL_TILE_UF = 0, SW_LABEL_EQUIVALENCE = 1 };
int sw_relabel(sw_handle* h, int method, int32_t* host_labels, float* ms, int* iterations);

/* One measured sweep, like sw_sweep(h, 1), with CUDA events recorded on
 * the handle's stream between its kernels.  Synchronises, then writes the
 * device time of each phase in milliseconds to phase_ms[0..3]:
 * [0] bonds + tile labels (Ising/Potts: including the measurement of the
 * incoming state, the previous sweep's record), [1] tile-boundary merge,
 * [2] flip, [3] stand-alone measurement (XY only; 0 otherwise).  nphase must
 * be >= 4.  For profiling. */
int sw_sweep_timed(sw_handle* h, float* phase_ms, int nphase);

/* Records of measured sweeps first .. first+count-1 into a host array.  The
 * handle retains the records of the last sw_series_capacity() measured
 * sweeps; SW_ERR_RANGE if a requested one is gone or was not measured. */
int sw_get_series(sw_handle* h, uint64_t first, size_t count, sw_record* host);
size_t sw_series_capacity(void);

/* ------------------------------------------------------------------------
 * Ragged batches (serving): many Ising/Potts lattices of one dimension,
 * each a normal handle with its own L, q, T, seed, buffers and accumulators,
 * advanced together with one launch per phase over all their tiles; one
 * sweep is captured in a CUDA graph and replayed.  Each lattice's trajectory
 * is the same alone and in a batch (the random numbers are keyed by seed,
 * sweep, site and purpose only).  The paper runs one lattice at a time; this
 * is the throughput path for many small lattices.
 *
 * sw_batch_create(dim)     new empty batch for dim = 2 or 3 (NULL on error);
 *                          it owns a non-blocking stream.
 * sw_batch_add(b, h)       h joins b (Ising/Potts of the batch's dim, in no
 *                          other batch); the handle stays owned by the caller.
 * sw_batch_remove(b, h)    h leaves b (synchronises the batch stream).
 * sw_batch_sweep(b, n)     n measured sweeps of every member (enqueued);
 *                          afterwards each member's counter has advanced by n
 *                          and its records and accumulators are read with the
 *                          usual per-handle calls, which wait for the batch.
 *                          A member with a sweep target (below) advances by
 *                          min(n, target - counter) only, 0 once there.
 * sw_set_sweep_target(h, t)  batch sweeps of h stop when its counter
 *                          reaches t (t = 0: no target; t >= 2^32 - 1 is
 *                          SW_ERR_BAD_ARG).  Single-lattice calls ignore it.
 *                          A serving loop gives each job its sweep count and
 *                          advances the whole batch by a fixed chunk.
 * sw_batch_query(b)        1 if the batch's enqueued sweeps have completed,
 *                          0 if not (non-blocking; see sw_query).
 * sw_batch_set_stream      run on a caller's non-default stream instead.
 * sw_batch_size            number of members.
 * sw_batch_destroy(b)      frees the batch (not its members).  sw_destroy of a
 *                          member removes it from its batch first.
 * sw_device_bytes          device bytes sw_create would allocate for a lattice
 *                          (0 for invalid arguments): the budget a serving
 *                          loop admits jobs against.
 *
 * Launch configuration.  A batch's tiles are 32 x tile_y (x tile_z) sites,
 * one CTA (a thread per 32-site row word) per tile, in one of
 * SW_BATCH_TILE_SHAPES shapes: 2D 32x256, 32x128, 32x64; 3D 32x16x16,
 * 32x16x8, 32x8x8 (single lattices use 32x128 in 2D, shape 1, and
 * 32x16x16 in 3D, shape 0, which a new batch starts with).  The schedule
 * (0 .. SW_BATCH_SCHEDULES - 1) has two bits.  Bit 0 is the label layout: 0
 * runs the Ising tiles in one launch with the two-state layout and the Potts
 * tiles in another, 1 runs all tiles in one launch with the Potts layout.
 * Bit 1 is the grid form of every phase (labels, merge, compression, apply):
 * 0 launches one CTA per tile, 1 launches a persistent grid -- the SM count
 * times the CTAs one SM holds -- whose CTAs stride over the tile map.  Bit 2
 * is the merge schedule: 0 joins every face of every tile in one launch, 1
 * in one launch per axis (the x faces of all tiles, then y, then z).  No
 * configuration changes any result: bonds, draws and canonical labels are
 * keyed by row word and site index, not by tile, CTA or union order.
 * sw_batch_set_config(b, shape, schedule)   selects one (SW_ERR_BAD_ARG out
 *                          of range); the next sweep recaptures the graph.
 * sw_batch_get_config(b, &shape, &schedule, &tile_y, &tile_z)   the current
 *                          one (any pointer may be NULL; tile_z = 1 in 2D).
 * sw_batch_autotune(b, sweeps, ms)   times every configuration on the
 *                          batch itself and keeps the fastest: per
 *                          configuration one untimed sweep (graph capture and
 *                          upload), then `sweeps` sweeps timed with CUDA
 *                          events (a host wait).  These are real measured
 *                          sweeps of every member, as sw_batch_sweep's: with
 *                          C = 3 shapes x 2 grid forms x 2 merge schedules
 *                          x (2 label layouts if the batch holds both Ising
 *                          and Potts lattices, else 1), every counter
 *                          advances by C * (sweeps + 1).  ms (NULL or
 *                          SW_BATCH_TILE_SHAPES * SW_BATCH_SCHEDULES floats,
 *                          index shape * 8 + schedule) receives the
 *                          time per sweep of each configuration, -1 where not
 *                          tried.  An empty batch returns SW_OK untouched;
 *                          sweeps < 1, or a member whose sweep target lies
 *                          within the C * (sweeps + 1) sweeps, is
 *                          SW_ERR_BAD_ARG. */
#define SW_BATCH_TILE_SHAPES 3
#define SW_BATCH_SCHEDULES 8
typedef struct sw_batch sw_batch;
sw_batch* sw_batch_create(int dim);
void sw_batch_destroy(sw_batch* b);
int sw_batch_add(sw_batch* b, sw_handle* h);
int sw_batch_remove(sw_batch* b, sw_handle* h);
int sw_batch_sweep(sw_batch* b, int n);
int sw_batch_query(sw_batch* b);
int sw_batch_set_stream(sw_batch* b, void* stream);
size_t sw_batch_size(sw_batch* b);
size_t sw_device_bytes(int model, int dim, int L, int q);
int sw_set_sweep_target(sw_handle* h, uint64_t target);
int sw_batch_set_config(sw_batch* b, int shape, int schedule);
int sw_batch_get_config(const sw_batch* b, int* shape, int* schedule, int* tile_y, int* tile_z);
int sw_batch_autotune(sw_batch* b, int sweeps, float* ms_per_sweep);

/* ------------------------------------------------------------------------
 * Asynchronous host I/O.  The paper has no counterpart (it times sweeps on a
 * resident lattice); a loop that streams states in and results out uses
 * these calls so that the transfers overlap the sweeps.  Host buffers must
 * be page-locked (cudaHostAlloc / pinned) and stay valid, and for uploads
 * unchanged, until sw_wait_io or sw_sync returns.  The handle creates two
 * copy streams and one device buffer of sw_spin_bytes on first use (not
 * counted by sw_device_bytes).  Not available for a lattice in a batch
 * (SW_ERR_BAD_ARG).
 *
 * sw_set_spins_async(h, host, bytes)  enqueues the upload of a new state;
 *     sweeps enqueued afterwards start from it.  The measurement pending on
 *     the replaced state is taken first, as in sw_set_spins.
 * sw_get_spins_async(h, host, bytes)  enqueues the download of the state
 *     after the sweeps enqueued so far: the state buffer is copied to the
 *     host on the download stream; later sweeps run meanwhile (they only
 *     read it until their flip), and the next write of that buffer (a
 *     flip, an upload into it, sw_set_spins) waits for the copy.
 * sw_get_record_async(h, sweep, host) enqueues the download of the record of
 *     a measured sweep (1 <= sweep <= sw_sweep_counter and among the last
 *     sw_series_capacity sweeps, else SW_ERR_RANGE) into one sw_record; the
 *     record's sweep field identifies it (a sweep that was not measured
 *     leaves another sweep's record in its slot).
 * sw_wait_io(h)  waits for every enqueued transfer and sweep of the handle.
 * Errors: SW_ERR_BAD_ARG (NULL, wrong size, batch member), SW_ERR_RANGE,
 * SW_ERR_CUDA (message in sw_last_error). */
int sw_set_spins_async(sw_handle* h, const void* host, size_t bytes);
int sw_get_spins_async(sw_handle* h, void* host, size_t bytes);
int sw_get_record_async(sw_handle* h, uint64_t sweep, sw_record* host);
int sw_wait_io(sw_handle* h);

/* ------------------------------------------------------------------------
 * Labeling without device allocation.  The paper has no counterpart: this
 * serves callers that may not allocate device memory themselves, such as a
 * plugin inside a host framework that owns every device byte through its
 * own pool, or a latency-critical loop where cudaMalloc / cudaFree would
 * synchronise the device and stall other streams.
 *
 * Computes exactly what sw_label_from_bonds computes (canonical min-index
 * labels of the clusters of a bond mask in the bit-plane layout above, with
 * the same kernels), but takes DEVICE buffers from the caller and allocates
 * nothing: no cudaMalloc, cudaFree or allocating library call.  Its working
 * memory (the union-find forest and an error flag) is one static device
 * array of SW_NOALLOC_MAX_SITES + 64 words (8 MiB + 256 B) in this library,
 * which every GPU that loads the library holds until the process exits.
 *
 *   dim, L       2 or 3, L >= 4, and L^dim <= SW_NOALLOC_MAX_SITES; larger
 *                lattices are rejected with SW_ERR_BAD_ARG before any GPU work
 *   dev_mask     device pointer, bond bit-planes (read only)
 *   dev_labels   device pointer, L^dim int32 labels (written)
 *   stream       cudaStream_t to run on (NULL = legacy default stream)
 *
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress), so the call stays valid across cudaDeviceReset.
 * The call cannot be captured into a CUDA graph: it reads its error flag
 * back and synchronises `stream`, so on a capturing stream it returns
 * SW_ERR_BAD_ARG before any GPU work.  Every call on a device shares the same array and leaves
 * its contents behind; the call clears the error flag itself, and the forest
 * needs no clearing.  Calls whose GPU work overlaps (on different streams or
 * from different threads) race on the array and must be serialised by the
 * caller.  The call synchronises `stream` before returning and reports a
 * device loop that hit its cap as SW_ERR_TIMEOUT; sw_last_error() gives the
 * message of a failure. */
#define SW_NOALLOC_MAX_SITES (1u << 21)
int sw_label_from_bonds_noalloc(int dim, int L, const uint32_t* dev_mask, int32_t* dev_labels,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SW_GB300_H */
