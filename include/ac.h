/*
 * ac.h -- C ABI of libac, an exact GB300 (sm_103a) simulator of
 * Poisson-asynchronous cellular arrays: Glauber's continuous-time Ising model
 * on a periodic 2D lattice, after Lubachevsky, "Efficient Parallel Simulations
 * of Asynchronous Cellular Arrays".
 *
 * Model (Sec. 1 "Poisson asynchrony"; Sec. 2, Eqs. (1)-(2)).  Each cell of a
 * rows x cols torus has an independent rate-1 Poisson clock.  At an arrival
 * the cell's spin s = +-1 flips with the heat-bath probability
 * p = 1 / (1 + exp(beta * dE)), dE = 2 s (J S + h), S the sum of the four
 * neighbour spins just before the arrival.  Energy E = -J sum s s' - h sum s
 * (appendix).  Arrivals are committed in global (tick, row-major index) order,
 * which every kernel reproduces exactly (the uniqueness argument of Sec. 3).
 *
 * Exact arithmetic conventions (shared by every entry point):
 *   time       int64 ticks, 2^32 ticks per unit time; a run to T commits every
 *              arrival with tick < t_end = T * 2^32.
 *   randomness Philox4x32-10 with key (seed & 0xffffffff, seed >> 32): arrival
 *              n of cell c (n = 0, 1, ...) uses block Philox({c, n+1, 0, 0});
 *              word y is its acceptance uniform, word x gives the gap to arrival
 *              n+1; block {c, 0, 0, 0} gives the first arrival, block
 *              {c, 0, 1, 0} the random initial spin (odd x: up).  One counter
 *              stream per cell (Sec. 5, and the invariance remark after
 *              Fig. 3.6).
 *   gap        integer stand-in for -ln r of Eq. (5): for a 32-bit word x,
 *              u = (2x+1)/2^33, gap = floor((33 - log2(2x+1)) ln2 * 2^32) + 1
 *              with log2 by 32 steps of truncated repeated squaring (Q1.31) and
 *              ln 2 = 0xB17217F7D1CF79AB / 2^64.
 *   threshold  thr[j + 5*(s > 0)] = min(floor(p * 2^32), 2^32 - 1) in IEEE
 *              binary64 on the host, j = number of up neighbours (0..4); the
 *              spin flips iff y < thr (the appendix's prob[] table).
 *   state      per cell: spin int8 (+1 / -1), next-arrival tick int64 (>= 1),
 *              committed-arrival count uint32; arrays row-major, rows*cols long.
 *
 * Ownership: the library owns all device memory of a simulation; every host
 * buffer passed in is owned by the caller and only read or written during the
 * call.  Calls on one handle are not thread-safe; distinct handles are
 * independent.  Every call returns a status; on failure ac_last_error() holds a
 * thread-local message.  Run calls are synchronous (they return when the device
 * work on the handle's stream has completed).
 */
#ifndef AC_H
#define AC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ac_sim ac_sim;

typedef enum {
  AC_OK = 0,
  AC_ERR_ARG = 1,     /* invalid argument; nothing was changed */
  AC_ERR_OOM = 2,     /* device or host allocation failed */
  AC_ERR_CUDA = 3,    /* a CUDA call failed; the handle's state is undefined */
  AC_ERR_STALL = 4,   /* the blocked kernel's watchdog saw no progress; state undefined */
  AC_ERR_STATE = 5    /* call not valid in the handle's current state */
} ac_status;

typedef enum { AC_INIT_RANDOM = 0, AC_INIT_UP = 1, AC_INIT_DOWN = 2 } ac_init;

typedef enum {
  AC_KERNEL_ROUND = 0,    /* (a) synchronous rounds, Fig. 3.2 */
  AC_KERNEL_BLOCKED = 1,  /* (b) blocked persistent kernel, Fig. 3.4: resident tiles, live edge words */
  AC_KERNEL_EPOCH = 2     /* (b) blocked persistent kernel, Fig. 3.4 at tile granularity: temporal-
                             blocked tiles ordered by per-tile epoch words in HBM */
} ac_kernel;

/* rows, cols >= 2 and rows * cols < 2^32. */
typedef struct {
  int32_t rows, cols;
  int32_t init; /* ac_init */
} ac_lattice;

/*
 * Create a simulation at time 0 (Sec. 2, initial state; first arrivals as
 * above).  beta >= 0, J and h finite.  Allocates key/count arrays (12 bytes per
 * cell) plus edge words for the tiling, and initialises them on the device.
 * Defaults: blocked kernel, tile side 64.  *out receives the handle.
 * Errors: AC_ERR_ARG (bad sizes or parameters), AC_ERR_OOM, AC_ERR_CUDA.
 */
ac_status ac_create(ac_lattice lat, double beta, double J, double h, uint64_t seed, ac_sim** out);

/*
 * Create the Ising array on the q-th degree neighbourhood of Sec. 3 (q = 2 or 3):
 * every cell within Manhattan distance q is a neighbour, M = 2q(q+1) of them.  The
 * heat-bath rule of ac_create uses S = the sum of their spins, i.e. the table
 * p = 1/(1 + exp(beta dE)), dE = 2 s (J S + h), thr = min(floor(p 2^32), 2^32 - 1),
 * index j + (M+1)(s > 0) for j up neighbours; a cell may commit once its
 * (tick, index) key is below all M neighbours' keys.  Initial state and arrivals
 * as for ac_create.  Needs rows, cols >= 4q.  Runs on the round kernel only
 * (temporal blocking, the region losing q rings per round; rounds per launch
 * capped at 16 / q and min(rows, cols) / (4q), default 6); not in batches; no
 * per-cell rates.  Observables of ac_stats keep the nearest-neighbour bonds.
 * Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.
 */
ac_status ac_create_q(ac_lattice lat, double beta, double J, double h, int32_t q, uint64_t seed, ac_sim** out);

/*
 * Create an asynchronous Life-like automaton instead of the Ising array: the
 * deterministic update of Sec. 3 (Conway's Game of Life is the paper's example)
 * under the same Poisson asynchrony, arrivals and random streams.  At an arrival
 * a cell with k live cells among its 8 Moore neighbours (states just before the
 * arrival) becomes alive iff bit k of `survive` (if alive) or of `birth` (if
 * dead) is set; Conway's rule is birth = AC_LIFE_CONWAY_BIRTH, survive =
 * AC_LIFE_CONWAY_SURVIVE.  A cell may commit once its (tick, index) key is below
 * those of all 8 Moore neighbours.  Initial state (lat.init): AC_INIT_RANDOM =
 * alive iff the word x of Philox block {c, 0, 1, 0} is < density (a 32-bit
 * fraction), AC_INIT_UP = all alive, AC_INIT_DOWN = all dead.  The state reads
 * and loads as for the Ising array with s = +1 alive, -1 dead; ticks and counts
 * are those of the Ising array with the same seed.  Needs rows, cols >= 4 and
 * 9-bit masks.  Runs on the round kernel only (temporal blocking with rounds per
 * launch capped at min(rows, cols) / 4, default 6); not in batches.
 * Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.
 */
#define AC_LIFE_CONWAY_BIRTH (1u << 3)
#define AC_LIFE_CONWAY_SURVIVE ((1u << 2) | (1u << 3))
ac_status ac_create_life(ac_lattice lat, uint32_t density, uint32_t birth, uint32_t survive, uint64_t seed,
                         ac_sim** out);

/* Use `cuda_stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later device work of this handle.  NULL selects the legacy default stream. */
ac_status ac_set_stream(ac_sim* sim, void* cuda_stream);

/*
 * Choose the kernel and its tuning for later run calls.
 *   kernel  AC_KERNEL_ROUND, AC_KERNEL_BLOCKED or AC_KERNEL_EPOCH
 *   Lb      tile side: 32, 64 or 128 (threads per CTA = 4 * Lb)
 *   rounds  round kernel: synchronous rounds per launch.  1 = one global round of
 *           Fig. 3.2 per launch, with per-round enabled counts (ac_round_history).
 *           2..16 = temporal blocking: each CTA loads its tile with a halo of depth
 *           `rounds` into a shared-memory region and runs `rounds` exact
 *           synchronous rounds per launch.  The region is 96 x 96 for rounds <= 12
 *           (384 threads per CTA, two CTAs per SM) and 128 x 128 for 13..16 (512
 *           threads, one CTA per SM); Lb = 128 selects the 128-wide region for any
 *           rounds, other Lb values are unused.  The tile side is the region side
 *           - 2*rounds.  Needs rows,
 *           cols >= 4*rounds; otherwise Lb-tiles with frozen halos run `rounds`
 *           rounds per launch.  When the lattice's counts are too uneven for the
 *           kernel's 16-bit count window, the call runs one round per launch.
 *           Blocked kernel: halo refresh period in rounds (>= 1).
 *   polls   blocked kernel: halo polls before a blocked tile is left (>= 0)
 * AC_KERNEL_EPOCH takes `rounds` and Lb as the round kernel does (synchronous rounds
 * per tile visit, the halo depth; Lb = 128 for the 128-wide region) and ignores polls.  It is one persistent launch per
 * run call: each CTA claims (epoch, tile) work items in order; a tile's visit loads
 * its region (tile plus halo) by bulk asynchronous copies, runs `rounds` rounds, writes
 * the tile back and publishes the tile's epoch with a release store; a visit of epoch
 * e starts once the tile and its 8 neighbour tiles have published epoch e (acquire
 * loads, bounded polls, the AC_OPT_WATCHDOG_NS watchdog).  The aggregated algorithm
 * of Fig. 3.4 with a tile per subarray and a tile's epoch as the local time its
 * neighbours wait on.  Needs the 4-neighbour Ising array, even cols, even `rounds`
 * (2..16) and rows, cols >= 4*rounds, and no snapshot frames; otherwise the handle
 * runs on the round kernel with the same `rounds`.
 * The trajectory does not depend on any of these (Sec. 3, invariance of the
 * aggregated algorithm under re-partitioning); only the speed does.
 * Errors: AC_ERR_ARG, AC_ERR_OOM (edge-word reallocation), AC_ERR_CUDA.
 */
ac_status ac_configure(ac_sim* sim, int32_t kernel, int32_t Lb, int32_t rounds, int32_t polls);

/*
 * Advance the trajectory: commit every arrival with tick < t_end (Fig. 3.1 loop
 * condition); afterwards every cell's tick is its first uncommitted arrival,
 * >= t_end.  t_end must be >= the previous t_end of this handle and < 2^61.
 * ac_run_until(T) uses t_end = floor(T * 2^32) (exact for integral T).
 * Errors: AC_ERR_ARG (t_end decreasing or out of range), AC_ERR_STALL,
 * AC_ERR_CUDA.
 */
ac_status ac_run_until(ac_sim* sim, double T);
ac_status ac_run_until_ticks(ac_sim* sim, int64_t t_end);

/*
 * Copy the state to caller-owned HOST arrays of rows*cols elements (row-major):
 * s (+1/-1), t (next-arrival ticks), n (committed arrivals per cell).  Any
 * pointer may be NULL to skip that array.  Errors: AC_ERR_ARG, AC_ERR_CUDA.
 */
ac_status ac_read_state(const ac_sim* sim, int8_t* s, int64_t* t, uint32_t* n);

/* Same as ac_read_state into caller-owned DEVICE arrays (e.g. torch CUDA tensors). */
ac_status ac_read_state_device(const ac_sim* sim, int8_t* s_dev, int64_t* t_dev, uint32_t* n_dev);

/*
 * Replace the state from caller-owned HOST arrays (the inverse of
 * ac_read_state) and declare it the state at time t_done: every s must be +-1
 * and every t in [max(t_done, 1), 2^61).  Together with ac_read_state this is
 * checkpoint/resume: the random streams are positioned by the counts n.
 * Errors: AC_ERR_ARG (invalid state), AC_ERR_CUDA.
 */
ac_status ac_load_state(ac_sim* sim, const int8_t* s, const int64_t* t, const uint32_t* n,
                        int64_t t_done);

/*
 * Asynchronous state transfers (checkpoint/resume and end-to-end runs that overlap
 * copies with compute).  Both enqueue their work on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) after all earlier work of the handle, and return
 * without waiting.  Host buffers should be pinned (cudaHostAlloc, or torch
 * pin_memory) for the copies to run asynchronously; they must stay valid until the
 * work on `stream` has completed.
 *
 * ac_load_state_async: as ac_load_state -- copy into the handle's staging buffers,
 *   validate on the device (every s +-1, every t in [max(t_done, 1), 2^61)), and only
 *   then replace the state -- but the outcome is known on the device only.  The
 *   handle's next call that uses its state (run, read, load, stats, class counts,
 *   reset, rates, frames, batch) first waits on the host for the load; if validation
 *   failed, that call returns AC_ERR_ARG naming the first bad cell and the state and
 *   time are left as they were.  The staging buffers are the second state buffer of
 *   the handle, so a transfer never overlaps the handle's own runs, only other
 *   handles' work.
 * ac_read_state_async: as ac_read_state into host arrays (any pointer may be NULL);
 *   the arrays hold the state once `stream` reaches this point.  The handle's next
 *   device work waits for the read on the device.
 * Errors: AC_ERR_ARG, AC_ERR_OOM (staging or events), AC_ERR_CUDA.
 */
ac_status ac_load_state_async(ac_sim* sim, const int8_t* s, const int64_t* t, const uint32_t* n, int64_t t_done,
                              void* stream);
ac_status ac_read_state_async(const ac_sim* sim, int8_t* s, int64_t* t, uint32_t* n, void* stream);

typedef struct {
  uint64_t events;          /* arrivals committed by run calls since create/load */
  uint64_t rounds;          /* tile rounds (commit phases) executed */
  uint64_t launches;        /* hot-path kernel launches */
  uint64_t scanned;         /* enable tests performed */
  uint64_t enabled;         /* enable tests that passed */
  uint64_t visits;          /* blocked kernel: tile visits */
  uint64_t polls;           /* blocked kernel: halo polls of blocked tiles */
  uint64_t global_rounds;   /* round kernel with rounds=1: synchronous rounds run */
  double device_ms;         /* device time of the run calls (CUDA events) */
  double enabled_frac_mean; /* Sec. 4 efficiency: mean over synchronous rounds of
                               enabled/N (round kernel, rounds=1); else enabled/scanned */
  int64_t sum_s;            /* current sum of spins */
  int64_t sum_bonds;        /* current sum over right and down bonds of s s' */
  uint64_t checksum;        /* sum_c mix(mix(mix(c) ^ t) ^ (2n + [s>0])) mod 2^64,
                               mix = SplitMix64 finaliser */
  uint64_t total_counts;    /* sum of per-cell counts */
  int64_t t_done;           /* t_end of the last completed run call */
  int32_t kernel, Lb, threads, rounds_per_launch;
  int32_t grid;             /* CTAs of the last launch */
  int32_t ctas_per_sm;      /* blocked kernel: resident CTAs per SM */
  uint64_t early_commits;   /* one-round kernel with AC_OPT_EARLY_REJECT: arrivals committed
                               early as certain rejections */
} ac_stats_t;

/* Statistics and observables of the handle (runs a reduction on the device). */
ac_status ac_stats(const ac_sim* sim, ac_stats_t* out);

/* Per-round enabled counts of the synchronous rounds run so far with the round
 * kernel at rounds=1 (Sec. 4 efficiency = counts / N).  Writes up to `cap`
 * entries and the number available to *n_rounds. */
ac_status ac_round_history(const ac_sim* sim, uint64_t* counts, int32_t cap, int32_t* n_rounds);

/*
 * BKL classes (Sec. 3, "The BKL algorithm"): the flip probability of a cell
 * depends only on its spin s and its number j of up neighbours, so the cells fall
 * into 10 classes; counts[j + 5 (s > 0)] receives the number of cells in each
 * (the index of the threshold table, so sum_k counts[k] * thr[k] / 2^32 is the
 * expected number of flips per unit time).  The 4-neighbour Ising array only.
 * Errors: AC_ERR_ARG, AC_ERR_CUDA.
 */
ac_status ac_class_counts(const ac_sim* sim, uint64_t counts[10]);

/*
 * Return the handle to time 0 with a new seed and initial condition, reusing its
 * device memory (the same initial state as ac_create; counters and statistics of
 * the trajectory restart).  No allocation.  Errors: AC_ERR_ARG, AC_ERR_CUDA.
 */
ac_status ac_reset(ac_sim* sim, uint64_t seed, int32_t init);

/*
 * Per-cell rates: the general asynchrony law (A) of Sec. 2, next arrival
 * t - ln(r) / p_c.  m[c] (a host array of rows * cols entries, each >= 1) gives
 * cell c the rate p_c = 2^20 / m[c]: each of its gaps, the first included, is
 * max(1, floor(e * m[c] / 2^20)) for the rate-1 gap e of ac_run_until (so
 * m[c] = 2^20 is rate 1 exactly).  NULL restores rate 1 everywhere.  Only at
 * time 0 (before the first run, or after ac_reset); the handle is re-initialised
 * with its seed and initial condition so that the first arrivals use the rates.
 * ac_reset keeps the rates.  Works with every kernel and in batches; the Ising
 * array only.  Errors: AC_ERR_ARG (a zero multiplier, a Life handle),
 * AC_ERR_STATE (after a run), AC_ERR_OOM, AC_ERR_CUDA.
 */
#define AC_RATE_ONE (1u << 20)
ac_status ac_set_rates(ac_sim* sim, const uint32_t* m);

/*
 * Snapshot frames at regular times K * dt (Sec. 3, "Generating the output",
 * Fig. 3.7).  Frame K is the array of all spins (int8 +-1, row-major) after every
 * arrival with tick <= K * dt_ticks has been committed and none later -- the
 * figure stores a subarray's image before it processes its first event later
 * than K dt.  (With ac_run_until's convention, frame K is the state after
 * ac_run_until_ticks(K * dt_ticks + 1).)  Frames are written by the kernels'
 * commits while the run proceeds; the library keeps B frame slots (the figure's
 * output buffer of B frames, B * rows * cols bytes of device memory) and never
 * lets a cell get further ahead than the B frames after the oldest one not yet
 * handed out (the figure's lag bound, between (B-1) dt and B dt).  Works with
 * every kernel and tuning; the trajectory and the final state do not change.
 *
 * ac_frames_configure: frames K0, K0+1, ... every dt_ticks ticks, B slots in
 *   [1, AC_MAX_FRAMES]; B = 0 turns frames off and frees the slots.  Needs
 *   dt_ticks >= 1, (B + 1) * dt_ticks <= 2^60, K0 * dt_ticks <= 2^60 and frame K0
 *   not before the state (K0 * dt_ticks + 1 >= the last t_end).  Replaces an
 *   earlier configuration.  ac_reset and ac_load_state turn frames off.
 *   Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.
 * ac_run_until_frames: as ac_run_until_ticks, and calls fn(user, K, frame, n)
 *   on the calling thread, in increasing K, once for every frame K with
 *   K * dt_ticks < t_end that was not handed out before.  `frame` points to
 *   n = rows * cols spins: device memory when on_host == 0 (the stream is
 *   synchronised before the call; the slot is reused after fn returns, so work
 *   that reads it must finish inside fn), else a library-owned pinned host buffer
 *   valid until fn returns.  fn may be NULL (frames are dropped).  While frames
 *   are configured, ac_run_until and ac_run_until_ticks behave as this call with
 *   fn = NULL, and ac_batch_run_until refuses the handle (AC_ERR_ARG).
 * ac_frames_status: next frame to be handed out, B and dt_ticks (B = 0: off).
 */
/*
 * Time-only round model (Sec. 4, the model behind the one-cell-per-PE efficiency
 * figure).  Cells carry only local times on an n-cell circle (dims = 1), an n x n
 * torus (2) or an n x n x n periodic array (3), row-major index
 * ((z n) + y) n + x.  Cell c starts at t = gap(B(c, 0).x); in each synchronous
 * round a cell advances iff t < t_end and (t, index) is below the keys of all
 * its neighbours (reading R1) -- the 2 dims nearest cells for q = 1, or, for
 * q > 1, every cell within Manhattan distance q (the q-th degree neighbourhood
 * of Sec. 3; needs n >= 2q+1, q <= 8) -- drawing its k-th increment from
 * B(c, k).x, where B(c, k) is Philox4x32-10 of {c, k, 0, 0} under the key
 * (seed lo, seed hi).  Increment laws:
 *   AC_LAW_EXP     exponential: the integer logarithm gap of ac_run_until
 *   AC_LAW_UNIFORM uniform on (0, 1]: x + 1 ticks
 *   AC_LAW_ROOT8   r^(1/8), r = (2x+1)/2^33: s1 = isqrt((2x+1) 2^31),
 *                  s2 = isqrt(s1 2^32), gap = isqrt(s2 2^32)
 * Runs until a round advances no cell or max_rounds rounds have run.  Writes the
 * number of advancing cells of each round to enabled[0 .. *rounds_out) (a host
 * array of max_rounds entries), and, when not NULL, the final times and advance
 * counts to host arrays t_out, n_out of n^dims entries and the device time of
 * the rounds to *device_ms.  Allocates and frees its own device memory.  Needs
 * n >= 2, n^dims < 2^32, t_end >= 0, max_rounds >= 1.
 * Errors: AC_ERR_ARG, AC_ERR_OOM, AC_ERR_CUDA.
 */
enum { AC_LAW_EXP = 0, AC_LAW_UNIFORM = 1, AC_LAW_ROOT8 = 2 };
ac_status ac_time_model(int32_t dims, int64_t n, int32_t q, int32_t law, uint64_t seed, int64_t t_end, int32_t max_rounds,
                        uint64_t* enabled, int32_t* rounds_out, int64_t* t_out, uint32_t* n_out,
                        double* device_ms);

#define AC_MAX_FRAMES 64
typedef void (*ac_frame_fn)(void* user, int64_t K, const int8_t* frame, size_t n);
ac_status ac_frames_configure(ac_sim* sim, int64_t dt_ticks, int64_t K0, int32_t B);
ac_status ac_run_until_frames(ac_sim* sim, int64_t t_end, ac_frame_fn fn, void* user, int32_t on_host);
ac_status ac_frames_status(const ac_sim* sim, int64_t* next_K, int32_t* B, int64_t* dt_ticks);

/* Tuning and verification options (ac_set_option):
 *   AC_OPT_WATCHDOG_NS   blocked and epoch kernels: no-progress limit in ns before
 *                        the run returns AC_ERR_STALL (default 5e9, >= 1e6)
 *   AC_OPT_MAX_ROUNDS    blocked kernel: cap on tile rounds per visit (0 = none)
 *   AC_OPT_DROP_PUBLISH  verification hook: 1 suppresses the publication of
 *                        boundary commits (blocked kernel) and of tile epochs (epoch
 *                        kernel), so that a lattice of several tiles cannot finish
 *                        and the watchdog must end the run with AC_ERR_STALL (no
 *                        fault, no unbounded wait); 0 restores it.
 *   AC_OPT_EARLY_REJECT  1: the round kernel with rounds = 1 (one synchronous round of
 *                        Fig. 3.2 per launch) also commits, out of (tick, index) order,
 *                        every pending arrival that is a rejection whatever the spins of
 *                        the neighbours that precede it turn out to be -- the observation
 *                        behind the BKL algorithm of Sec. 3 that at low temperature most
 *                        arrivals change nothing.  Such an arrival keeps the cell's spin,
 *                        so no neighbour's decision depends on its order; the trajectory is
 *                        unchanged.  The neighbours that do not precede the cell keep their
 *                        spins until after its arrival, so the number j of up neighbours at
 *                        the arrival lies in [their up count, that + the number that
 *                        precede it]; the arrival is a certain rejection iff
 *                        u >= thr[j + 5 (s > 0)] for every such j.  A per-cell byte (rows *
 *                        cols bytes of device memory, allocated on first use) caches the j
 *                        at which the pending arrival would flip; it is refilled at the
 *                        start of each run call and kept by the commits (one extra
 *                        Philox block per arrival).  The Ising array only; other kernels
 *                        ignore the option.  0 (default) turns it off. */
enum { AC_OPT_WATCHDOG_NS = 1, AC_OPT_MAX_ROUNDS = 2, AC_OPT_DROP_PUBLISH = 3, AC_OPT_EARLY_REJECT = 4 };
ac_status ac_set_option(ac_sim* sim, int32_t option, int64_t value);

/* Free all memory of the handle (NULL is ignored). */
void ac_destroy(ac_sim* sim);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* ac_last_error(void);

/* The threshold table the library uses for (beta, J, h) (the appendix's prob[],
 * quantised as above), written to thr[10]. */
ac_status ac_thresholds(double beta, double J, double h, uint32_t thr[10]);

/*
 * Batching.  ac_batch_create makes n independent simulations (arrays of n
 * lattices and parameters; seeds distinguish lattices, the counter carries no
 * lattice id) into out[0..n-1], each usable with every call above.
 * ac_batch_run_until advances sims[0..n-1] to t_end[i] each.  When every handle
 * is configured for the epoch kernel with the same rounds and fits it, ONE
 * persistent epoch-kernel launch covers the tiles of all handles (each tile waits
 * only on its own lattice's neighbour tiles; a further launch follows only if the
 * launch's epoch budget ran out first).  Otherwise, when every handle is configured
 * for the round or epoch kernel with the same rounds per launch (>= 2) and fits
 * temporal blocking, one work list holds the tiles of all handles and each
 * temporal-blocked launch advances all of them; launches are issued in chunks of
 * 8, replayed from a CUDA graph captured on the second call with the same list
 * of handles, and the host reads the device counters after each chunk to see
 * whether any arrival before t_end is left.  Otherwise the handles run in ONE
 * cooperative blocked-kernel launch over all their tiles (tile side Lb of
 * sims[0]), replayed from a CUDA graph captured on the first call for that list
 * of handles.  All handles must share the stream of sims[0] and a tile side;
 * only the 4-neighbour Ising array, without snapshot frames.  Results are
 * bit-identical to running each handle alone.  Errors as for
 * ac_run_until_ticks.
 */
ac_status ac_batch_create(int32_t n, const ac_lattice* lats, const double* beta, const double* J,
                          const double* h, const uint64_t* seed, ac_sim** out);
ac_status ac_batch_run_until(int32_t n, ac_sim* const* sims, const int64_t* t_end);

/*
 * Run without allocating.  The paper has no counterpart to this entry point.  It
 * serves callers that cannot let the library call cudaMalloc: applications whose
 * own memory pool has reserved the device's memory up front (a cudaMalloc from
 * the library would fail or fragment that pool), hosts that grant a plugin a
 * fixed device budget and account for every byte of it, and loops that must not
 * call cudaMalloc or cudaFree at all because those calls can synchronise the
 * whole device.
 *
 * Advances the lattice stored in the caller's DEVICE buffers to t_end with the
 * blocked persistent kernel (tile side 64), bit-identical to ac_run_until_ticks
 * on a handle with the same state and parameters.
 *   key_dev  rows*cols uint64, row-major: tick << 1 | (spin > 0); read and written
 *   cnt_dev  rows*cols uint32: committed arrivals per cell; read and written
 *   stream   cudaStream_t for the work (NULL: legacy default stream)
 * All other buffers the kernel needs (lattice descriptor, counters, tile flags,
 * edge words) live in one file-scope device array of AC_STATIC_SCRATCH_BYTES,
 * which every GPU that loads the library holds until the process exits.  The
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it for the process; make that first call before any
 * stream capture.  The cached address does not survive cudaDeviceReset or the
 * destruction of the device's primary context: after either, do not call this
 * entry point again in the same process.  Every call shares the array and clears
 * what must start at zero, so calls whose GPU work overlaps (other streams, other
 * threads) race and must not be issued.  The call is synchronous: it waits for
 * its GPU work on `stream` and reads the device counters back before returning.
 * Errors: AC_ERR_ARG (bad arguments, or a lattice needing more scratch than the
 * maximum: about 2000 tiles of 64 x 64, e.g. 2816 x 2816), AC_ERR_STALL,
 * AC_ERR_CUDA.
 */
#define AC_STATIC_SCRATCH_BYTES (4u << 20)
ac_status ac_run_blocked_static(int32_t rows, int32_t cols, double beta, double J, double h,
                                uint64_t seed, uint64_t* key_dev, uint32_t* cnt_dev, int64_t t_end,
                                void* stream);

/*
 * Row slabs of one lattice (Sec. 3, the aggregated algorithm over a partition of the array;
 * the trajectory does not depend on the partition, the remark after Fig. 3.6).  A handle that
 * holds the whole lattice can be restricted to rows [row0, row0 + nrows) of the torus and then
 * advanced one temporal-blocked launch at a time over that slab's tiles only: `rounds` exact
 * synchronous rounds of Fig. 3.2 per step, reading the `rounds` rows above and below the slab
 * from its own current state.  Between steps the caller copies each slab's first and last
 * `rounds` rows into the neighbouring slabs' handles (ac_slab_export / ac_slab_import: device
 * buffers of count * cols * 12 bytes, the keys tick << 1 | (s > 0) then the uint32 counts), so
 * that every slab's halo is the neighbours' state after the same number of steps; the steps
 * are then the global synchronous rounds, and the union of the slabs' own rows is the exact
 * trajectory.  The rows outside the slab are not kept current by the steps themselves.
 *   ac_slab_configure  needs the round or epoch kernel with rounds >= 2 (rows, cols >=
 *                      4 * rounds), the 4-neighbour Ising array, no frames, and
 *                      rounds <= nrows <= rows - 2 * rounds; nrows = 0 lifts the restriction.
 *   ac_slab_step       one step toward t_end; *live = 1 if a cell of the slab still has an
 *                      arrival before t_end.  Run every slab until no slab is live.  Does not
 *                      change the handle's t_done.  AC_ERR_STATE if the counts of a region left
 *                      the kernel's 16-bit window (the state is then unchanged).
 *   ac_slab_export     rows [row, row + count) of the current state into dst (synchronous)
 *   ac_slab_import     rows [row, row + count) of the current state from src (synchronous)
 * Errors: AC_ERR_ARG, AC_ERR_STATE, AC_ERR_OOM, AC_ERR_CUDA.
 */
ac_status ac_slab_configure(ac_sim* sim, int32_t row0, int32_t nrows);
ac_status ac_slab_step(ac_sim* sim, int64_t t_end, int32_t* live);
ac_status ac_slab_export(const ac_sim* sim, int32_t row, int32_t count, void* dst_dev);
ac_status ac_slab_import(ac_sim* sim, int32_t row, int32_t count, const void* src_dev);

/* Device-primitive probes (DEVICE pointers, n elements), for verification:
 * out[i] = gap of x[i];  out4[4i..4i+3] = Philox({c[i], k[i], w2, 0}) under seed. */
ac_status ac_dev_exp_ticks(const uint32_t* x_dev, uint64_t* out_dev, int64_t n);
ac_status ac_dev_philox(uint64_t seed, const uint32_t* c_dev, const uint32_t* k_dev, uint32_t w2,
                        uint32_t* out4_dev, int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* AC_H */
