/*
 * fciqmc.h -- C ABI of libfciqmc: one FCIQMC time step over a sparse walker
 * vector for Bose-Hubbard Hamiltonians, run as hand-written CUDA kernels on
 * one GPU (sm_103a).  The method is the one of the Rimu.jl paper
 * (arXiv 2601.19505), Secs. 3.1-3.2, 4.2, 6.1-6.3 and 7.1.
 *
 * Calls follow the paper's statement of a calculation (Sec. 2.1): create a
 * Hamiltonian from its parameters, seed a walker vector, set the time step,
 * shift and target walker number, step n times, and read the shift, norm,
 * projected energy and occupied-configuration count.
 *
 * Conventions for every call:
 *  - Return 0 (FQ_OK) on success, a negative FQ_ERR_* code otherwise;
 *    fq_strerror() names it.  Nothing is changed when a call fails, except
 *    where a call says otherwise.
 *  - Handles (fq_ham, fq_run, fq_batch) are opaque, owned by the library and
 *    released by the matching *_destroy call.  A fq_ham must outlive every
 *    run created from it; runs must outlive every batch that holds them.
 *  - Input arrays are owned by the caller and copied before the call returns.
 *    Outputs are written into caller buffers whose capacity is passed in.
 *  - All pointers in this header are HOST pointers.  Device memory is owned
 *    by the library; it comes from the caller's allocator when one is given
 *    (e.g. PyTorch's caching allocator), else from cudaMallocAsync.
 *  - There is no CPU fallback: without a usable CUDA device, fq_run_create
 *    returns FQ_ERR_CUDA.
 *  - Stepping is asynchronous on the run's CUDA stream.  Errors that arise on
 *    the device (a full buffer, a dead population) are reported by the next
 *    call that synchronises (fq_run_sync, _stats, _history, _export); the
 *    run is then left at its last completed step ("rolled back").
 *  - Not thread-safe per handle: one host thread at a time per run or batch.
 */
#ifndef FCIQMC_H
#define FCIQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fq_ham fq_ham;
typedef struct fq_run fq_run;
typedef struct fq_batch fq_batch;

/* A Fock address (Sec. 6.1): the occupation bit string of N + M - 1 bits, n_m
 * one-bits for mode m and one zero-bit between consecutive modes, mode 1 in
 * the least significant bit of lo; bits 64..127 in hi (0 when N+M-1 <= 64).
 * Example: BoseFS(0,2,3,4,0,1) is lo = 0b100111101110110 = 20342, hi = 0. */
typedef struct { uint64_t lo, hi; } fq_key;

/* Hamiltonians (Eq. bose-hubbard-hamiltonian and its momentum-space form,
 * Sec. 6.3).  REAL_1D: periodic ring of Lx >= 3 sites (Ly = 1).  REAL_2D:
 * periodic Lx x Ly lattice, Lx, Ly >= 3, site x + Lx*y.  MOM_1D: Lx momentum
 * modes (Ly = 1, 2 <= Lx <= 64), mode j carries k = 2 pi (j - floor(Lx/2))/Lx. */
enum { FQ_BH_REAL_1D = 1, FQ_BH_REAL_2D = 2, FQ_BH_MOM_1D = 3 };

/* Walker representation.  INT: integer walkers (int64 amplitudes, the
 * original integer-coefficient formulation).  REAL64: FP64 amplitudes with
 * matrix and vector compression (Sec. 3.2).  REAL32: amplitudes, spawns and
 * the per-entry arithmetic (spawn values, diagonal update, annihilation sums)
 * in FP32; the one-norm is an exact sum rounded once to FP64, and the shift
 * and projected-energy sums are FP64.  DETERMINISTIC: no
 * compression at all, the power iteration of Eq. fciqmc (FP64). */
enum { FQ_MODE_INT = 0, FQ_MODE_REAL64 = 1, FQ_MODE_REAL32 = 2, FQ_MODE_DETERMINISTIC = 3 };

/* Annihilation strategy (Sec. 6.3: summing spawns to one address).  Both
 * arms scatter spawns into hash-segmented buckets.  HASH: one warp sums a
 * bucket's spawns per address in an open-addressing table in shared memory,
 * then the segment's entries take their sums.  SORT: one warp sorts a
 * bucket's contributions (the entries' diagonal terms, then the spawns) by a
 * 16-bit hash of the address with a stable LSD radix sort of two 8-bit
 * digits and sums each address's run (a segmented reduction).  Results are
 * the same up to the order of FP sums.  AUTO: fq_run_autotune /
 * fq_batch_autotune time both arms and keep the faster; HASH until then. */
enum { FQ_ANN_AUTO = 0, FQ_ANN_SORT = 1, FQ_ANN_HASH = 2 };

/* Where vector compression Pi acts (Sec. 7.1).  LATE (default, Eq.
 * late-comp): on each address's summed value after annihilation.  EARLY (Eq.
 * early-comp): on every spawn and every diagonal term on its own, before any
 * sum; a spawn below the threshold that compression drops is never written,
 * and the summed values are stored as they are (some may lie below the
 * threshold).  Real-valued walkers only: INT and DETERMINISTIC runs ignore
 * it.  The draw of a spawn's compression is the draw that picked it (attempt
 * a of its source), that of entry k of an exact column the draw of stream k,
 * and that of a diagonal term stream 0xFFFFFFFD of its address. */
enum { FQ_COMPRESS_LATE = 0, FQ_COMPRESS_EARLY = 1 };

enum {
    FQ_OK = 0,
    FQ_ERR_INVALID = -1,  /* bad argument or handle state                        */
    FQ_ERR_NOMEM = -2,    /* device allocation failed                            */
    FQ_ERR_CAPACITY = -3, /* spawn, vector or table capacity exceeded; rolled back */
    FQ_ERR_TIMEOUT = -4,  /* a bounded device-side wait expired; rolled back      */
    FQ_ERR_EMPTY = -5,    /* the population died (norm 0); rolled back            */
    FQ_ERR_CUDA = -6      /* a CUDA runtime error, or no usable device           */
};

/* Run parameters.  dt: time step (Eq. discretised).  target: target one-norm
 * N_t (Eq. shift-update).  zeta, xi: shift damping and forcing (Eq.
 * shift-update).  threshold: vector-compression threshold theta (Eq.
 * vec-compression with 1 -> theta).  t_rel: semistochastic threshold; a column
 * is spawned exactly when |c_i| t_rel >= m_i (Sec. 7.1).  mode: FQ_MODE_*.
 * annihilation: FQ_ANN_*.  seed, run_id: key of the counter-based random
 * draws.  compression: FQ_COMPRESS_*.  capacity_vec, capacity_spawn: maximum
 * occupied entries of the vector and spawn entries per step (0 = derived from
 * target and threshold). */
typedef struct {
    double dt, target, zeta, xi, threshold, t_rel;
    int32_t mode, annihilation;
    uint64_t seed;
    uint32_t run_id;
    int32_t compression;
    size_t capacity_vec, capacity_spawn;
} fq_params;

/* One row of the time series (Sec. 4): the step number, occupied
 * configurations (len), exact and stochastic columns spawned, spawn entries
 * written, and after the step the shift S, the one-norm ||c||_1 and the
 * projected-energy numerator y^T H c (hproj) and denominator y^T c (vproj). */
typedef struct {
    int64_t step, len, exact_steps, inexact_steps, n_spawns;
    double shift, norm, hproj, vproj;
} fq_stats;

/* Device-memory allocator used by a run instead of cudaMallocAsync.  alloc
 * returns a device pointer of at least `bytes` (NULL on failure) usable on
 * `stream`; free releases it.  Both are called from the host thread that
 * calls into the library. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
} fq_allocator;

const char *fq_version(void);
const char *fq_strerror(int code);

/* Defaults recovered from the paper's printed time series (Secs. 2.1, 4):
 * dt = 0.01, zeta = 0.08, xi = zeta^2/4, threshold = 1, t_rel = 1,
 * target = 1000, mode REAL64, seed 1, run_id 0, capacities derived. */
int fq_params_default(fq_params *p);
/* Set the shift damping zeta together with its critically damped forcing
 * xi = zeta^2/4 (Eq. shift-update; the value the paper's printed time series
 * are reproduced with, and the critical damping of x'' + zeta x' + xi x = 0).
 * FQ_ERR_INVALID unless zeta >= 0 is finite.  Set xi afterwards to depart
 * from it. */
int fq_params_set_zeta(fq_params *p, double zeta);

/* Create a Bose-Hubbard Hamiltonian with N bosons, hopping t, interaction u.
 * N >= 1, N + M - 1 <= 128.  FQ_ERR_INVALID for any other shape. */
int fq_ham_create(fq_ham **out, int kind, int Lx, int Ly, int N, double t, double u);
void fq_ham_destroy(fq_ham *h);
/* Number of modes M, address bits N + M - 1, and 64-bit words per address. */
int fq_ham_info(const fq_ham *h, int *M, int *nbits, int *key_words);
/* Fock-space dimension C(N + M - 1, N) (Sec. 2), as a double. */
int fq_ham_dimension(const fq_ham *h, double *dim);
/* Starting address: near-uniform filling in real space (floor(N/M) per
 * site, the first N mod M sites one more), all bosons in k = 0 in momentum
 * space. */
int fq_ham_starting_address(const fq_ham *h, fq_key *out);
/* Address <-> occupation numbers occ[0..M-1] (Sec. 6.1).  encode fails if
 * sum(occ) != N; decode fails if the key is not a valid address. */
int fq_encode(const fq_ham *h, const uint8_t *occ, fq_key *out);
int fq_decode(const fq_ham *h, fq_key key, uint8_t *occ);
/* The column of H at `key` (Sec. 6.2, operator_column), evaluated by the
 * device code the step uses: diagonal element and the m off-diagonal
 * entries in enumeration order (dest[k], val[k], k < min(m, cap)).  Runs on
 * the legacy default stream and synchronises. */
int fq_ham_column(const fq_ham *h, fq_key key, double *diag, fq_key *dest, double *val,
                  size_t cap, size_t *m);

/* fq_ham_column without any allocation (the paper has no counterpart: this
 * is a library-level variant).  The column is evaluated into one fixed
 * device array of 729,600 bytes that exists from the moment the library is
 * loaded, so the call works when device memory is exhausted (cudaMalloc
 * would fail) and never waits for the whole device (as cudaFree does).
 * Same arguments and results as fq_ham_column, with these limits:
 *  - columns longer than FQ_COLUMN_NOALLOC_MAX entries are rejected with
 *    FQ_ERR_CAPACITY, *m still set to the column's length; nothing else is
 *    written;
 *  - the array is shared per device: calls that overlap in time (several
 *    host threads) race on it, so callers must serialise them;
 *  - the work runs on a stream the library creates once per device with
 *    cudaStreamNonBlocking: it does not wait for the legacy default stream
 *    or for the caller's streams (queued steps keep running), and the call
 *    returns once its own copies have completed;
 *  - the first call on a device looks up the array's address (which may
 *    load the module) and creates that stream: make it outside any CUDA
 *    stream capture. */
#define FQ_COLUMN_NOALLOC_MAX 16384
int fq_ham_column_noalloc(const fq_ham *h, fq_key key, double *diag, fq_key *dest, double *val,
                          size_t cap, size_t *m);

/* Create a run: device buffers sized from the parameters, all on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  `alloc` may be NULL. */
int fq_run_create(fq_run **out, const fq_ham *h, const fq_params *p, void *stream,
                  const fq_allocator *alloc);
void fq_run_destroy(fq_run *r);
/* Replace the walker vector by n distinct (key, amplitude) pairs; zero
 * amplitudes are dropped.  INT runs need integral amplitudes; REAL32 runs
 * round them to FP32.  Also sets the shift S and the step counter, clears
 * the history, and takes the norm N^(0) = sum |c|.  FQ_ERR_INVALID on a
 * duplicate or invalid key, FQ_ERR_CAPACITY if a segment overflows. */
int fq_run_seed(fq_run *r, const fq_key *keys, const double *amps, size_t n, double shift,
                int64_t step);
/* The paper's default start (Secs. 2.1, 4.2): `weight` (N_w = 10) on the
 * starting address, shift = its diagonal element, step 0, and projected-
 * energy reference y = N_w e_start. */
int fq_run_seed_default(fq_run *r, double weight);
/* Reference vector y of the projected energy (Eq. ProjectedEnergy): n <= 64
 * distinct addresses with coefficients y.  hproj = y^T H c, vproj = y^T c. */
int fq_run_set_reference(fq_run *r, const fq_key *keys, const double *y, size_t n);
/* Change dt, the current shift, or the target norm before the next step. */
int fq_run_set_dt(fq_run *r, double dt);
int fq_run_set_shift(fq_run *r, double shift);
int fq_run_set_target(fq_run *r, double target);
/* Enqueue n steps c^(n+1) = Pi[1 + dt (S^(n) - H~)] c^(n) with the shift
 * update after each (Eq. stochasticTransitionOperator, Eq. shift-update).
 * Asynchronous; captured once into a CUDA graph and replayed. */
int fq_run_step(fq_run *r, int64_t n);
/* Wait for queued work; report a device-side error (the run is rolled back
 * to its last completed step and can continue). */
int fq_run_sync(fq_run *r);
/* The device-side cause of the last error a synchronising call reported:
 * bit 0 a spawn bucket, bit 1 a vector segment, bit 2 an on-chip or scratch
 * annihilation table was full, bit 3 the population died, bit 5 an
 * amplitude left the exact-norm range (|c| / threshold >= 2^63).  0 if none. */
int fq_run_error_bits(const fq_run *r, unsigned *bits);
/* Synchronise and return the row of the last completed step (step 0 after
 * seeding: len, shift and norm set, the rest 0). */
int fq_run_stats(fq_run *r, fq_stats *out);
/* Synchronise and move out the rows recorded since the last call (oldest
 * first, at most cap; *n = rows written).  The ring holds 65536 rows; older
 * rows are dropped. */
int fq_run_history(fq_run *r, fq_stats *out, size_t cap, size_t *n);
/* Synchronise and copy the walker vector, sorted by address, into caller
 * buffers (*n = occupied entries; min(*n, cap) written). */
int fq_run_export(fq_run *r, fq_key *keys, double *amps, size_t cap, size_t *n);
/* Dict-style read (Sec. 6.3): amps[i] = the amplitude of keys[i] in the
 * current vector, 0 when the address is not stored.  Synchronises. */
int fq_run_lookup(fq_run *r, const fq_key *keys, size_t n, double *amps);
/* A sample of the current vector: every entry of whole segments taken in an
 * order shuffled by `seed`, until at least `want` entries (*n = entries
 * sampled; min(*n, cap) written).  Synchronises. */
int fq_run_sample(fq_run *r, uint64_t seed, size_t want, fq_key *keys, double *amps, size_t cap,
                  size_t *n);
/* Kernel-level check: run only the spawning stage of the next step on the
 * current vector and copy out the spawn entries (destination, value; order
 * unspecified, *n = count).  The run's state does not change. */
int fq_run_spawns(fq_run *r, fq_key *dest, double *val, size_t cap, size_t *n);
/* Grow the vector and spawn capacities to at least these totals (never
 * shrinks), keeping the vector.  The usual answer to FQ_ERR_CAPACITY: the
 * run was rolled back, so grow and step again.  The vector's new buffers
 * are allocated while the old ones still hold it; the spawn buffers hold
 * nothing between steps and are released before their successors are
 * allocated.  FQ_ERR_NOMEM when the device memory cannot hold the new
 * sizes: the run keeps what it had (the spawn buffers are allocated again
 * at their old size; should even that fail, every later step and check of
 * the run returns FQ_ERR_NOMEM).  Synchronises. */
int fq_run_reserve(fq_run *r, size_t capacity_vec, size_t capacity_spawn);
/* Current total capacities (entries of the vector, spawns per step). */
int fq_run_capacity(const fq_run *r, size_t *capacity_vec, size_t *capacity_spawn);
/* Annihilation tables (tests and tuning; not in the paper).  A bucket's
 * spawns are summed in an on-chip table of `slots` entries per merge warp
 * when they fill at most 0.7 of it, else in that warp's table of
 * `scratch_slots` entries in device memory, which by default holds any
 * bucket within the run's capacities; a bucket beyond 0.9 of the scratch
 * table fails the step with FQ_ERR_CAPACITY (error bit 2) and the run is
 * rolled back.  Each size is a power of two >= 64 (slots: 8 warps' tables
 * within 200 KB of shared memory; scratch_slots <= 2^26); 0 restores the
 * default.  Synchronises; the next step rebuilds the launch. */
int fq_run_set_tables(fq_run *r, unsigned slots, unsigned scratch_slots);
/* Spawn-buffer layout (tests and tuning; not in the paper).  The first
 * `primary` slots of every spawn bucket lie in one dense region of the spawn
 * buffers, the bucket's other slots in a second region after it; a spawn is
 * stored in the first free slot of its bucket either way, so the results do
 * not depend on the split.  Spawns land in random buckets, and a small dense
 * region keeps their stores on few memory pages.  By default `primary` is
 * the steady-state bucket fill (spawns per step ~ 1.1 N_t / threshold) plus
 * three standard deviations, rounded up to a multiple of 32.  `primary` must
 * be a multiple of 32 and at most the bucket capacity (0: every slot in the
 * second region); else FQ_ERR_INVALID.  A later fq_run_reserve keeps it.
 * Synchronises. */
int fq_run_set_spawn_split(fq_run *r, unsigned primary);
/* Buckets the merge summed in the on-chip table and in the scratch table
 * since the run was seeded (a rolled-back step's buckets included).
 * Synchronises. */
int fq_run_merge_paths(fq_run *r, uint64_t *onchip, uint64_t *scratch);
/* Time the launch shapes on the current vector and keep the fastest.  Each
 * candidate runs `steps` real steps, so the run advances. */
int fq_run_autotune(fq_run *r, int steps);
/* The launch shape the run steps with (after fq_run_autotune, the tuned
 * one): shape[0..6] = spawn warps per block, spawn blocks, merge warps per
 * block, merge blocks, per merge warp the on-chip table slots (HASH) or
 * sort-workspace elements (SORT) and the device-memory table slots or
 * workspace elements for larger buckets, and the annihilation arm
 * (FQ_ANN_HASH or FQ_ANN_SORT).  Needs a seeded run. */
int fq_run_shape(fq_run *r, int *shape);
/* The last fq_run_autotune's best mean merge-kernel time (ms) of each
 * annihilation arm on the run's vector (0 for an arm it did not time). */
int fq_run_arm_times(fq_run *r, float *hash_ms, float *sort_ms);
/* Measurement: run n steps launched one kernel at a time (not from the graph)
 * with CUDA events around each kernel on the run's stream; ms[0], ms[1],
 * ms[2] = mean milliseconds per step of the spawning, merge and shift
 * kernels.  The run advances n steps (n <= 4096); synchronises. */
int fq_run_profile(fq_run *r, int n, float *ms);

/* A batch: B runs (same Hamiltonian kind, address width, mode and
 * annihilation strategy; any sizes and other parameters) stepped together by
 * one launch per kernel per step. */
int fq_batch_create(fq_batch **out, fq_run *const *runs, int B);
void fq_batch_destroy(fq_batch *b);
int fq_batch_step(fq_batch *b, int64_t n);
int fq_batch_sync(fq_batch *b);
int fq_batch_autotune(fq_batch *b, int steps);

/* Replica overlaps (Sec. 4.3, Eq. RayleighQuotientReplica): with R = 2..8
 * replicas in one batch (one Hamiltonian, equal sizes; statistically
 * independent through their run_id), record after every step, for every pair
 * A < B in the order (0,1), (0,2), ..., (1,2), ..., the vector-vector product
 * c_A^T c_B and the vector-operator-vector products c_A^T G2(d_k) c_B of the
 * density-density correlator G2(d) = (1/M) sum_i n_i (n_{i+d} - delta_{d0})
 * (Eq. g2; 1D real space only, 0 <= d_k < M, n_g2 <= 16; n_g2 = 0 records the
 * dot products alone).  The variational energy of Sec. 4.3 is then the ratio
 * of the means of (S_A + S_B)/2 c_A^T c_B and c_A^T c_B (shifts from each
 * run's history).  Each pair's sums over segments are added in a fixed
 * order, so repeated runs give identical rows.  Replaces any earlier
 * setting; FQ_ERR_INVALID for runs of different shapes or sizes. */
int fq_batch_set_overlaps(fq_batch *b, const int *g2_d, int n_g2);
/* Excited states (Sec. 2.2): runs 0..K-1 of the batch (2 <= K <= 8; one
 * Hamiltonian and equal sizes; real-valued or deterministic walkers) become
 * step-synchronised spectral states.  After every step's annihilation, run k
 * is orthogonalised to runs 0..k-1 (Gram-Schmidt): c_k <- c_k - sum_j
 * alpha_j c_j with alpha_j = (c_j^T c_k) / (c_j^T c_j), all alpha_j from the
 * same c_k; each value that changed is then compressed by Pi (Eq.
 * vec-compression, its draw from stream 0xFFFFFFFC of the address), and run
 * k's norm, shift update and projected energy follow the orthogonalised
 * vector.  The shift of run k estimates the k-th energy (shift_estimator).
 * Seed the runs differently (a later state must not start parallel to an
 * earlier one).  K = 0 turns it off; FQ_ERR_INVALID for integer walkers or
 * runs of different shapes or sizes. */
int fq_batch_set_spectral(fq_batch *b, int K);
/* Move out the overlap rows recorded since the last call, oldest first, at
 * most cap of them (*n = rows written).  A row is `width` doubles: the step,
 * then per pair c_A^T c_B followed by its n_g2 G2 products; width =
 * 1 + P (1 + n_g2) with P = R (R - 1) / 2.  The ring keeps at least the last
 * 1024 rows; steps that failed (rolled back) leave no row.  Synchronises. */
int fq_batch_overlaps(fq_batch *b, double *rows, size_t cap, size_t *n, int *width);

#ifdef __cplusplus
}
#endif

#endif /* FCIQMC_H */
