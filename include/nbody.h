/*
 * nbody.h -- C ABI of libnbody, a GB300 (sm_103a) direct-sum Hermite N-body
 * force engine.
 *
 * The calls follow the paper's statement of one integration step (Groen,
 * Portegies Zwart, McMillan & Makino, "Distributed N-body Simulation on the
 * Grid Using Dedicated Hardware", Sec. 4.1 steps 1-7 and, for the split
 * between predicting all particles and computing forces on an active block,
 * Sec. 4.4 steps 2-7):
 *   set j-particles -> next block time + active block -> predict all N to t
 *   -> forces (acceleration, jerk, potential) on the active block from all N
 *   -> correct the block and choose new power-of-two time steps.
 *
 * Conventions (every entry point):
 *  - Returns NB_OK (0) or a negative NB_E* code; no exception or signal ever
 *    crosses the ABI.  The first error is also kept in the context ("sticky")
 *    and returned by nb_last_error until nb_clear_error.
 *  - The caller owns every pointer it passes.  The library copies inputs in
 *    and writes into caller-owned outputs; it keeps no caller pointer after
 *    the call returns.
 *  - ptr_kind says where caller buffers live: NB_PTR_HOST (pageable or pinned
 *    host memory; the call synchronises the context's stream before
 *    returning) or NB_PTR_DEVICE (device memory of the context's device; the
 *    work is enqueued on the context's stream and the call returns without
 *    synchronising).
 *  - Vectors are row-major [count][3] FP64 at the ABI; the library stores
 *    them structure-of-arrays internally.
 *  - Units: N-body units, G = 1.
 *  - One context per host thread at a time (contexts are not thread-safe);
 *    any number of contexts may coexist.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define NB_OK         0
#define NB_EINVAL    -1   /* bad argument (null pointer, range, ordering)   */
#define NB_ENOMEM    -2   /* device or host allocation failed               */
#define NB_ECUDA     -3   /* a CUDA runtime call failed                     */
#define NB_ENUMERIC  -4   /* NaN or Inf seen in a result                    */
#define NB_EDTMIN    -5   /* a step criterion fell below dt_min (clamped)   */
#define NB_ETIMEOUT  -6   /* a bounded device wait gave up                  */
#define NB_ESTATE    -7   /* call out of order (e.g. forces before predict) */

/* ---- force-path precision ---------------------------------------------- */
#define NB_FP64   0  /* IEEE FP64 pairwise arithmetic; 1/s from an FP32 seed
                        refined in FP64 (any s^2 > 0; s^2 = 0 only for the
                        self pair, which is excluded by index)                 */
#define NB_MIXED  1  /* FP32 pairwise arithmetic on double-single position
                        differences; the FP32 sum over each j-tile is folded
                        into a double-single (FP32 hi + lo, TwoSum)
                        accumulator; results converted to FP64.  Pair
                        distances must lie in the FP32 normal range
                        (s^2 >= 2^-126), which any eps >= 2^-63 ensures       */

/* ---- where caller buffers live ---------------------------------------- */
#define NB_PTR_HOST    0
#define NB_PTR_DEVICE  1

typedef struct nb_ctx nb_ctx;   /* opaque, owned by the library */

/*
 * nb_create -- make a context for up to n_max particles on CUDA device
 * `device`, working on `cuda_stream` (a cudaStream_t; NULL = a stream the
 * library creates and owns; pass cudaStreamLegacy to work on the legacy
 * default stream).  precision: NB_FP64 or NB_MIXED (changeable
 * with nb_set_precision).  Allocates all device memory the context needs up
 * front (about 0.3 KB per particle).  Parameters start at the paper's values
 * (Sec. 2): eps = 2^-8, dt in [2^-22, 2^-3], eta = 0.01.
 * Errors: NB_EINVAL (out == NULL, n_max < 1, bad precision/device),
 * NB_ENOMEM, NB_ECUDA.  On error *out is NULL.
 */
int nb_create(nb_ctx** out, int64_t n_max, int precision, int device, void* cuda_stream);

/* nb_destroy -- free the context and everything it allocated (NULL is a no-op). */
void nb_destroy(nb_ctx* ctx);

/*
 * nb_set_params -- softening length eps >= 0 (Plummer softening, the
 * "softening parameter" of Sec. 2), accuracy parameter eta > 0 of the
 * Aarseth step criterion, and the block-step range dt_min <= dt_max, both
 * powers of two (Sec. 2: powers of two between 2^-22 and 2^-3).  dt_min ==
 * dt_max gives shared (equal) steps.  Errors: NB_EINVAL.
 */
int nb_set_params(nb_ctx* ctx, double eps, double eta, double dt_min, double dt_max);

/* nb_get_params -- the context's eps, eta, dt_min, dt_max (any pointer may be
 * NULL; no GPU work).  Errors: NB_EINVAL (ctx NULL). */
int nb_get_params(nb_ctx* ctx, double* eps, double* eta, double* dt_min, double* dt_max);

/* nb_default_params -- the paper's defaults (no context needed, no GPU). */
void nb_default_params(double* eps, double* eta, double* dt_min, double* dt_max);

/* nb_set_precision -- switch the force path (NB_FP64 / NB_MIXED).  Errors: NB_EINVAL. */
int nb_set_precision(nb_ctx* ctx, int precision);

/*
 * nb_set_j_particles -- Sec. 4.1 step 1 (read the snapshot): write particles
 * [first, first + count) of the j-store.  m[count]; x, v, a, jerk [count][3];
 * t, dt [count].  a, jerk, t, dt may be NULL (zero; call
 * nb_initial_forces_and_dt before stepping).  The particle count N becomes
 * max(N, first + count).  Errors: NB_EINVAL (range beyond n_max, NULL m/x/v,
 * count < 0, non-finite value), NB_ECUDA.
 */
int nb_set_j_particles(nb_ctx* ctx, int64_t first, int64_t count, const double* m, const double* x,
                       const double* v, const double* a, const double* jerk, const double* t,
                       const double* dt, int ptr_kind);

/* nb_set_n -- set the particle count N (<= n_max); particles >= N are ignored. */
int nb_set_n(nb_ctx* ctx, int64_t n);

/* nb_get_n -- current particle count N. */
int nb_get_n(nb_ctx* ctx, int64_t* n);

/*
 * nb_get_particles -- Sec. 4.1 step 7 (write the output): copy particles
 * [first, first + count) out.  Any output pointer may be NULL (skipped).
 * pot is the potential from the last force evaluation of each particle.
 * Errors: NB_EINVAL (range), NB_ECUDA.
 */
int nb_get_particles(nb_ctx* ctx, int64_t first, int64_t count, double* m, double* x, double* v,
                     double* a, double* jerk, double* pot, double* t, double* dt, int ptr_kind);

/*
 * nb_next_block -- Sec. 4.1 step 2: the next system time
 * t = min_i (t_i + dt_i) and the active block {i : t_i + dt_i == t} in
 * ascending index order.  *t_next and *n_active are written (host);
 * active_idx (host, capacity >= N, may be NULL) receives the indices.  The
 * block also stays on the device for nb_step / nb_correct_block.
 * Errors: NB_ESTATE (N == 0), NB_ECUDA.
 */
int nb_next_block(nb_ctx* ctx, double* t_next, int32_t* active_idx, int64_t* n_active);

/*
 * nb_predict -- Sec. 4.1 step 3 (Sec. 4.4 step 4 on GRAPE): Taylor-predict
 * positions and velocities of all N particles to time t from (x, v, a,
 * jerk, t_i).  FP64; the mixed path also gets double-single positions.
 * Asynchronous on the context's stream.  Errors: NB_ESTATE, NB_ECUDA.
 */
int nb_predict(nb_ctx* ctx, double t);

/*
 * nb_compute_forces -- Sec. 4.1 step 4, Eq. 3 (t_force = tau_force n N):
 * for each of the n active particles i_idx[k] (ascending, unique, < N),
 * the Plummer-softened acceleration, jerk and potential summed over all
 * j != i at the predicted positions/velocities of the last nb_predict:
 *   acc_i  = sum_j m_j r_ij / s^3,
 *   jerk_i = sum_j m_j [ v_ij / s^3 - 3 (r_ij . v_ij) r_ij / s^5 ],
 *   pot_i  = - sum_j m_j / s,
 * r_ij = x_j - x_i, v_ij = v_j - v_i, s^2 = |r_ij|^2 + eps^2.
 * Outputs acc, jerk [n][3] and pot [n] (any may be NULL); the results are
 * also kept for nb_correct.  i_idx and outputs are host or device per
 * ptr_kind.  n == 0 is a no-op.  Errors: NB_EINVAL (n > N, index out of
 * range or not ascending -- checked on the host for host indices),
 * NB_ESTATE (no prediction), NB_ECUDA.
 */
int nb_compute_forces(nb_ctx* ctx, const int32_t* i_idx, int64_t n, double* acc, double* jerk,
                      double* pot, int ptr_kind);

/*
 * nb_compute_forces_at -- GRAPE's split of steps 3-5 (Sec. 4.4 steps 3-5):
 * the n listed particles i_idx (ascending, unique, < N) are predicted to t
 * alone (step 3, in FP64 as nb_predict does), every j-particle is predicted
 * to t inside the force kernel as its tile is loaded (step 4, the board's
 * on-the-fly prediction), and the forces on the list are summed as in
 * nb_compute_forces (step 5).  No nb_predict of all N is needed; t must lie
 * within every particle's current step (t_j <= t <= t_j + dt_j, as any block
 * time of the particles' schedule does).  Outputs and errors as
 * nb_compute_forces; the results are kept for nb_correct(t).
 *
 * Mixed path: the kernel predicts from a "j-memory" of double-single records
 * (80 bytes per particle, allocated on the first call and kept current
 * through the context's own corrections): x + v h is carried in
 * double-single FP32 (~2^-48), the acceleration and jerk terms in FP32
 * (error <= 2^-24 |a| h^2/2 + ...), velocities in FP32.  NB_FP64: there is
 * no on-the-fly prediction; all N are predicted first (as nb_predict).
 */
int nb_compute_forces_at(nb_ctx* ctx, double t, const int32_t* i_idx, int64_t n, double* acc, double* jerk,
                         double* pot, int ptr_kind);

/*
 * nb_set_jpredict -- which block steps of the host-driven loop (nb_step,
 * nb_integrate with NB_LOOP_HOST) take the on-the-fly j prediction of
 * nb_compute_forces_at instead of predicting all N first (mixed path, single
 * system): blocks of n <= max_n active particles.  max_n = 0 never,
 * NB_JPREDICT_AUTO (the default) the measured crossover on GB300, n <= 1024
 * (the in-kernel prediction costs ~5% of the force kernel, the separate
 * predictor of all N a fixed pass over the state).  The block steps are the
 * same; the predicted j differ from the FP64 predictor's in the last bits
 * (see nb_compute_forces_at).  The j-memory is allocated on the first block
 * that takes this path.  Errors: NB_EINVAL (max_n < -1).
 */
#define NB_JPREDICT_AUTO (-1)
int nb_set_jpredict(nb_ctx* ctx, int64_t max_n);

/* nb_get_jpredict -- the largest block that takes the on-the-fly prediction. */
int nb_get_jpredict(nb_ctx* ctx, int64_t* max_n);

/* ---- exchange between ranks: the copy (Sec. 4.2) and ring (Sec. 4.3)
 * algorithms, one context per rank, driven by the package's distributed
 * module.  These calls share the list staging of nb_compute_forces and
 * nb_correct: make them between block steps, not between a force call and
 * its nb_correct (except nb_set_forces, which feeds nb_correct). ---------- */

/*
 * nb_get_particles_idx -- particles idx[0..n) (ascending, unique, < N) out
 * of the state, in list order: m[n], x, v, a, jerk [n][3], pot, t, dt [n]
 * (any output NULL = skipped).  The copy algorithm gathers its corrected
 * block with it before the all-gather.  Errors: NB_EINVAL, NB_ECUDA.
 */
int nb_get_particles_idx(nb_ctx* ctx, const int32_t* idx, int64_t n, double* m, double* x, double* v, double* a,
                         double* jerk, double* pot, double* t, double* dt, int ptr_kind);

/*
 * nb_set_particles_idx -- write particles idx[0..n) (ascending, unique,
 * < N) of the state from the list-ordered arrays (NULL = unchanged): the copy
 * algorithm's update of every rank's full copy with the blocks the other
 * ranks corrected.  Invalidates the prediction.  Errors: NB_EINVAL
 * (non-finite host value, bad list), NB_ECUDA.
 */
int nb_set_particles_idx(nb_ctx* ctx, const int32_t* idx, int64_t n, const double* m, const double* x,
                         const double* v, const double* a, const double* jerk, const double* pot, const double* t,
                         const double* dt, int ptr_kind);

/*
 * nb_get_predicted -- predicted positions and velocities xp, vp [n][3] of
 * particles idx[0..n) at the time of the last nb_predict: the ring
 * algorithm's active block leaves its rank with them.  Errors: NB_EINVAL,
 * NB_ESTATE (no current prediction), NB_ECUDA.
 */
int nb_get_predicted(nb_ctx* ctx, const int32_t* idx, int64_t n, double* xp, double* vp, int ptr_kind);

/*
 * nb_forces_on -- Eq. 3 on n particles held elsewhere (the ring algorithm's
 * visiting block, Sec. 4.3): positions xi and velocities vi [n][3] at the
 * block time, summed over this context's j-particles at their last
 * nb_predict (the same arithmetic as nb_compute_forces, in the context's
 * precision).  gid[k] (nullable) is particle k's global index; a j-particle
 * whose global index gid_base + (its index here) equals it is the self pair
 * and is excluded.  Outputs acc, jerk [n][3], pot [n] (any may be NULL),
 * overwritten, or with accumulate != 0 added onto what they hold (the
 * block's running sums).  n <= the context's padded capacity (n_max rounded
 * up to 1024).  Errors: NB_EINVAL, NB_ESTATE (no prediction), NB_ENOMEM,
 * NB_ECUDA.
 */
int nb_forces_on(nb_ctx* ctx, int64_t n, const double* xi, const double* vi, const int64_t* gid, int64_t gid_base,
                 double* acc, double* jerk, double* pot, int accumulate, int ptr_kind);

/*
 * nb_set_forces -- install forces computed elsewhere (the ring algorithm's
 * sums, back home after the last shift) as the results for the particles
 * idx[0..n) (ascending, unique), for the nb_correct(idx, t) that follows;
 * needs the prediction to t of these particles (nb_predict).  Errors:
 * NB_EINVAL (NULL or non-finite value), NB_ESTATE, NB_ECUDA.
 */
int nb_set_forces(nb_ctx* ctx, const int32_t* idx, int64_t n, const double* acc, const double* jerk,
                  const double* pot, int ptr_kind);

/*
 * nb_set_initial_forces -- Sec. 4.1 step 1 with forces summed elsewhere (the
 * ring algorithm's first circuit, when no rank holds all N): every
 * particle's acceleration, jerk and potential from acc, jerk [N][3], pot [N]
 * (particle order), t_i = 0, and the initial steps of
 * nb_initial_forces_and_dt.  Errors: NB_EINVAL, NB_ESTATE (N == 0),
 * NB_ENUMERIC, NB_ECUDA.
 */
int nb_set_initial_forces(nb_ctx* ctx, const double* acc, const double* jerk, const double* pot, int ptr_kind);

/*
 * nb_correct -- Sec. 4.1 step 5: 4th-order Hermite correction of the n
 * particles i_idx (the list of the preceding nb_compute_forces or
 * nb_compute_forces_at(t)) to time t,
 * using their old (a, jerk) and the new ones; stores the new a, jerk, pot,
 * t_i = t and a new block step dt_i: the Aarseth criterion with eta,
 * rounded down to a power of two, clamped to [dt_min, dt_max], growing at
 * most x2 and only when t is a multiple of 2 dt_old (Sec. 2 block steps).
 * Errors: NB_EINVAL, NB_ESTATE (list differs from the force call), NB_ECUDA.
 * NaN/Inf results and criterion underflows are recorded on the device and
 * reported by nb_check_device_status.
 */
int nb_correct(nb_ctx* ctx, const int32_t* i_idx, int64_t n, double t, int ptr_kind);

/*
 * nb_initial_forces_and_dt -- Sec. 4.1 step 1 (initialise the N-body
 * system): forces of all N at their current positions (t_i = 0), and
 * initial steps dt_i = largest power of two <= eta |a| / |jerk|, clamped.
 */
int nb_initial_forces_and_dt(nb_ctx* ctx);

/*
 * nb_step -- one block step entirely on the device: next block (step 2),
 * predict (3), forces (4), correct (5).  Writes the block time and size
 * (host).  Errors as the calls it makes.
 */
int nb_step(nb_ctx* ctx, double* t_out, int64_t* n_active_out);

/*
 * nb_integrate -- Sec. 4.1 steps 2-6: block steps until every particle has
 * reached t_end (t_end must be a multiple of dt_max).  loop selects who
 * drives the steps:
 *   NB_LOOP_HOST        the host, one launch sequence per block step;
 *   NB_LOOP_GRAPH       one CUDA graph whose body sits in a device-side while
 *                       node (no host round trip per step);
 *   NB_LOOP_PERSISTENT  one cooperative kernel that stays resident for the
 *                       whole run (a few CTAs per SM, three grid barriers per
 *                       block step, each wait bounded), for systems whose
 *                       block steps are latency-bound: N <= NB_PERSISTENT_MAX_N
 *                       on the mixed path, N <= NB_PERSISTENT_MAX_N_FP64 on
 *                       the FP64 path (a full-block force phase must stay
 *                       far inside the 4 s barrier wait: ~70 ms for 2^18
 *                       mixed particles, ~0.3 s for 2^16 in FP64).
 *   NB_LOOP_CLUSTER     one thread-block cluster (16 CTAs, one per SM; 8 where
 *                       the GPU cannot co-schedule 16) for the whole run, the
 *                       ring algorithm of Sec. 4.3 on one chip: each CTA holds
 *                       N/16 particles in shared memory, predicted on the fly
 *                       (Sec. 4.4 step 4), the active block visits every CTA
 *                       through distributed shared memory, and the cluster's
 *                       hardware barrier separates the phases (three per
 *                       step; no spin wait).  Mixed path only, N <=
 *                       NB_CLUSTER_MAX_N (8192 on an 8-CTA cluster).
 *   NB_LOOP_AUTO        the driver measured fastest per block step on a GB300
 *                       for the context's precision and N: the cluster loop
 *                       for mixed systems of N <= 2048 (where the GPU
 *                       co-schedules the cluster), the persistent loop up to
 *                       N = 131072 (mixed) or 2048 (FP64, whose force phase
 *                       outweighs the step overhead sooner), the host loop
 *                       beyond.
 * All of them take the same block steps with the same per-particle arithmetic;
 * sums over j-splits may group differently.  The mixed path renews its
 * spatial order between launches (graph and persistent loops run segments of
 * at most the sort interval).  Errors: NB_EINVAL (t_end, loop, N too large
 * for the persistent loop at the context's precision), NB_ENUMERIC, NB_ETIMEOUT (a bounded device wait
 * gave up, or the graph loop reached t_end / dt_min + 2 iterations; the state
 * is then undefined), NB_ESTATE (the block time stopped increasing: a state
 * without valid steps, e.g. dt = 0 because nb_initial_forces_and_dt was not
 * called; every loop stops within two block steps), NB_ECUDA.  NB_LOOP_CLUSTER: NB_EINVAL
 * also for the FP64 path or N beyond what the cluster holds.
 */
#define NB_LOOP_HOST        0
#define NB_LOOP_GRAPH       1
#define NB_LOOP_PERSISTENT  2
#define NB_LOOP_CLUSTER     3
#define NB_LOOP_AUTO        4
#define NB_PERSISTENT_MAX_N 262144
#define NB_PERSISTENT_MAX_N_FP64 65536
#define NB_CLUSTER_MAX_N    16384
int nb_integrate(nb_ctx* ctx, double t_end, int loop);

/*
 * nb_energy -- kinetic and potential energy of the current state (the paper
 * is silent on diagnostics): K = sum m v^2/2, W = (1/2) sum m_i phi_i with
 * phi from a full i = j force evaluation in the context's precision.  Uses
 * the state as stored (call when all t_i are equal).  Host outputs.
 */
int nb_energy(nb_ctx* ctx, double* ekin, double* epot);

/*
 * nb_get_timings -- accumulated device time (ms) of the predict, force and
 * correct phases (Eq. 1: t_pred + t_force + t_corr per step) and the number
 * of pairwise interactions (sum of n N over force calls) since the last
 * reset; reset != 0 zeroes them after reading.  Any pointer may be NULL.
 */
int nb_get_timings(nb_ctx* ctx, double* ms_pred, double* ms_force, double* ms_corr,
                   double* interactions, int reset);

/*
 * nb_get_counters -- kernels this context has launched (every library kernel,
 * counted at launch) and block steps taken, since creation.  Host-only.
 */
int nb_get_counters(nb_ctx* ctx, int64_t* kernel_launches, int64_t* block_steps);

/*
 * nb_check_device_status -- synchronise and read the device-side status
 * word: NaN/Inf seen (NB_ENUMERIC), step criterion below dt_min (count in
 * *dt_underflows, may be NULL), bounded wait timeout (NB_ETIMEOUT), a
 * device-driven loop whose block time stopped increasing (NB_ESTATE), a bad
 * device list (NB_EINVAL).  Bits stay set until nb_clear_error.
 */
int nb_check_device_status(nb_ctx* ctx, int64_t* dt_underflows);

/*
 * nb_check_grid_barrier -- exercises the bounded wait of the persistent
 * loop's grid barrier on the device: one CTA per SM, three barriers.  With
 * phantom = 0 every wait completes (NB_OK); with phantom != 0 the barrier
 * waits for one CTA more than were launched, every CTA gives up after
 * wait_ms (0 < wait_ms <= 4000) and the call returns NB_ETIMEOUT with the
 * timeout bit set in the device status (clear it with nb_clear_error); the
 * context stays usable.  Errors: NB_EINVAL, NB_ENOMEM, NB_ECUDA.
 */
int nb_check_grid_barrier(nb_ctx* ctx, int phantom, double wait_ms);

/* nb_last_error / nb_clear_error -- the sticky first error of a context. */
int nb_last_error(nb_ctx* ctx);
void nb_clear_error(nb_ctx* ctx);

/*
 * nb_set_tuning -- override the force launch: i per thread (1,2,4),
 * threads per CTA (64..512), j-tile (32..1024), split-j factor (0 = auto).
 * 0 for any argument restores the automatic choice (autotuner table).
 * Errors: NB_EINVAL (unsupported combination).
 */
int nb_set_tuning(nb_ctx* ctx, int i_per_thread, int threads, int j_tile, int n_split);

/*
 * nb_set_far_tiles -- the mixed path's far-tile pass (not in the paper).
 * With the particles kept in spatial order, a (warp of i, j-tile) pair in
 * which every i of the warp is at least theta (|x_i| + |x|max_j) from the
 * tile's bounding box (theta = 1/8) forms each position difference from the
 * FP32 "hi" parts alone, with
 * relative error <= 2^-24 (1/theta + 1) ~ 5.4e-7 per pair; every other pair,
 * and every pair when the pass is off, uses the double-single difference
 * (x_j.hi - x_i.hi) + (x_j.lo - x_i.lo).  enable != 0 turns the pass on (the
 * default), 0 off ("strict": double-single differences on every tile, at
 * about 6 more FP32 operations per pair).  Applies to every later force
 * launch of the context (host, graph and persistent loops, ensembles); the
 * FP64 path ignores it.  Errors: NB_EINVAL (ctx NULL).
 */
int nb_set_far_tiles(nb_ctx* ctx, int enable);

/* nb_get_far_tiles -- whether the far-tile pass is on (1) or off (0). */
int nb_get_far_tiles(nb_ctx* ctx, int* enabled);

/*
 * nb_selftest_corrector -- device self-check of the corrector's exact
 * shortcuts (Sec. 4.1 step 5): the powers of a power-of-two step and the
 * power-of-two step rule taken from exponent bits instead of FP64 products,
 * division and square root.  On `samples` seeded random operand sets (steps,
 * norms, times, step bounds; boundary, zero, subnormal, infinite and NaN
 * cases included) each shortcut is compared bit for bit with its FP64
 * expression on `device`; *mismatches receives the number of differences
 * (0 expected).  Errors: NB_EINVAL (samples < 0, NULL output), NB_ENOMEM,
 * NB_ECUDA.
 */
int nb_selftest_corrector(int device, int64_t samples, uint64_t seed, int64_t* mismatches);

/*
 * nb_autotune -- time the supported force launches of the host-driven path
 * (i per thread, threads per CTA, j-tile, split-j factor) for the current N
 * and active-block size n on the current state (needs a prediction) and keep
 * the fastest in the context's tuning table for systems and blocks within a
 * factor sqrt(2) of (N, n); every later force call of such a size takes it
 * (unless nb_set_tuning overrides).  Writes the chosen configuration (any
 * pointer may be NULL; *n_split = 0 means the automatic split).
 */
int nb_autotune(nb_ctx* ctx, int64_t n, int* i_per_thread, int* threads, int* j_tile, int* n_split);

/*
 * nb_autotune_list -- nb_autotune timed on the caller's active list (n
 * particle indices, ascending, in host or device memory per ptr_kind) instead
 * of the first n particles of the resident spatial order, so that the launch
 * shapes are compared on the block that will run: a block scattered over the
 * system finds fewer far tiles than a compact one and favours other shapes.
 * The entry is kept for (N, n) like nb_autotune's.  Errors: NB_EINVAL (n out
 * of [1, N], NULL list, bad ptr_kind; a device list that is not ascending is
 * reported as NB_EINVAL by the next call that checks the status word),
 * NB_ESTATE (no prediction), NB_ECUDA.
 */
int nb_autotune_list(nb_ctx* ctx, const int32_t* i_idx, int64_t n, int ptr_kind, int* i_per_thread, int* threads,
                     int* j_tile, int* n_split);

/*
 * nb_ensemble_autotune -- the item shape of the device-driven block steps
 * (the CUDA-graph loop of one system, or the batched ensemble): i-tile 32, 64
 * or 128 particles and 2, 4, 8 or 16 force items planned per resident CTA
 * (which sets the split-j length), each timed on `steps` block steps
 * (1..4096) of the context's own state, which is restored after every trial
 * and at the end (the particles, the counters and the schedule are as
 * before the call).  The fastest goes into the tuning table for batches of
 * about the same median cluster size (factor sqrt(2)) and cluster count
 * (factor 2); later nb_ensemble_integrate / nb_integrate(NB_LOOP_GRAPH) calls
 * use it.  Outputs (any may be NULL): the chosen i-tile and items per CTA,
 * its time and the time of the default shape (ms for the `steps` steps).
 * Errors: NB_EINVAL, NB_ESTATE (no particles), NB_ENOMEM, NB_ECUDA,
 * NB_ENUMERIC (a trial produced NaN/Inf).
 */
int nb_ensemble_autotune(nb_ctx* ctx, int64_t steps, int* i_tile, int* item_waves, double* ms_best,
                         double* ms_default);

/*
 * nb_tune_save / nb_tune_load -- the context's tuning table as a JSON file:
 *   {"format": "libnbody tuning table 1", "device": "<name>", "sm_count": S,
 *    "entries": [{"kind": "single"|"batched", "precision": "fp64"|"mixed",
 *                 "N_lo", "N_hi", "n_lo", "n_hi", "i_per_thread", "threads",
 *                 "j_tile", "n_split", "item_waves", "ms"}, ...]}
 * (for "batched" entries N is the median cluster size, n the cluster count
 * and "threads" the i-tile).  Loading replaces the table; a file measured on
 * a GPU with another SM count, or not in this format, is refused with
 * NB_EINVAL and leaves the table as it was.  nb_create and
 * nb_ensemble_create load the file named by the environment variable
 * NB_TUNE_FILE when it is set (silently skipped when it cannot be used).
 */
int nb_tune_save(nb_ctx* ctx, const char* path);
int nb_tune_load(nb_ctx* ctx, const char* path);

/* nb_tune_count / nb_tune_clear -- entries in the tuning table; empty it. */
int nb_tune_count(nb_ctx* ctx, int* count);
int nb_tune_clear(nb_ctx* ctx);

/*
 * nb_measure_peaks -- measured arithmetic throughput of the context's GPU:
 * dependent FMA chains in FP32 and FP64 (TFLOP/s, 2 flop per FMA) and the
 * hardware rsqrt (T results/s).  Roofline denominators for the force paths
 * (not in the paper).  Uses the context's scratch; any pointer may be NULL.
 */
int nb_measure_peaks(nb_ctx* ctx, double* fp32_tflops, double* fp64_tflops, double* rsqrt_tops);

/*
 * nb_measure_fp64_issue -- how the context's GPU issues FP64 instructions, in
 * SM cycles per FP64 FMA (clock64 around chains of 4096 FMAs in one CTA):
 * *dep32 one warp, all 32 lanes, a dependent chain; *dep1 the same with one
 * lane active; *indep4 one warp, four independent chains (per instruction);
 * *sm16 sixteen warps on one SM, SM cycles per warp instruction.  On GB300
 * each is ~64, ~64, ~64 and ~19: a warp issues one FP64 instruction per ~64
 * cycles whatever its active lanes, which is why the small-block paths keep
 * FP64 off their critical paths (not in the paper).  Uses the context's
 * scratch; any pointer may be NULL.  Errors: NB_EINVAL, NB_ECUDA.
 */
int nb_measure_fp64_issue(nb_ctx* ctx, double* dep32, double* dep1, double* indep4, double* sm16);

/* ---- batched ensemble of independent clusters --------------------------- */
/*
 * nb_ensemble_create -- a context for n_clusters independent systems stored
 * back to back: cluster c owns particles [offsets[c], offsets[c+1]) of one
 * j-store (offsets host, ascending, offsets[0] == 0).  eps[c] is each
 * cluster's softening (host).  Fill it with nb_set_j_particles on the whole
 * range, then nb_initial_forces_and_dt.  Errors: NB_EINVAL, NB_ENOMEM.
 */
int nb_ensemble_create(nb_ctx** out, int32_t n_clusters, const int64_t* offsets, const double* eps,
                       int precision, int device, void* cuda_stream);

#define NB_ENSEMBLE_PERSISTENT   0  /* one graph launch: every cluster's block
                                       steps as device-driven batched steps   */
#define NB_ENSEMBLE_PER_CLUSTER  1  /* reference: clusters one after another,
                                       host-driven per-step kernel launches   */

/*
 * nb_ensemble_initial_forces_and_dt -- Sec. 4.1 step 1 for every cluster:
 * forces of all particles within their own cluster at t = 0, initial steps.
 * (nb_initial_forces_and_dt on an ensemble context calls this.)
 */
int nb_ensemble_initial_forces_and_dt(nb_ctx* ctx);

/*
 * nb_ensemble_integrate -- integrate every cluster to t_end with its own
 * block steps (Sec. 4.1 steps 2-6 per cluster; t_end a multiple of dt_max).
 * mode: NB_ENSEMBLE_*.  Both modes give the same block schedule.
 */
int nb_ensemble_integrate(nb_ctx* ctx, double t_end, int mode);

/*
 * nb_ensemble_energy -- kinetic and potential energy of every cluster (host
 * arrays of n_clusters), each cluster's potential from its own particles.
 */
int nb_ensemble_energy(nb_ctx* ctx, double* ekin, double* epot);

/* ---- forces without any device allocation ------------------------------- */
#define NB_NOALLOC_SCRATCH_DOUBLES (1 << 22)   /* fixed scratch: 32 MiB per GPU  */
#define NB_NOALLOC_MAX_ACTIVE      (1 << 19)   /* largest active block accepted  */

/*
 * nb_forces_fp64_noalloc -- the paper has no counterpart to this call; it is
 * a service for callers that cannot allocate device memory: applications
 * that own all device memory themselves (their own pool, no cudaMalloc from
 * libraries) and latency-critical loops where an allocation could stall or
 * fail mid-run.  Such callers cannot use nb_create, which allocates.
 *
 * Computes the same FP64 acceleration, jerk and potential as
 * nb_compute_forces with NB_FP64 (softening eps >= 0, j == i excluded) for
 * the n active particles i_idx[0..n) from all N particles, with every buffer
 * owned by the caller and resident on the current CUDA device: m[N],
 * x[N][3], v[N][3] (positions/velocities at the common time), i_idx[n]
 * (int32, each in [0, N); the list need not be sorted), outputs acc[n][3],
 * jerk[n][3], pot[n] (any may be NULL).  The indices are not checked (that
 * would need a status word the caller reads back): an index below 0 or
 * >= N is clamped to 0 or N - 1 for every read, so no access leaves the
 * caller's arrays, and the outputs at that list position are unspecified.
 * Work is enqueued on cuda_stream (a cudaStream_t, NULL = default stream);
 * the call returns without synchronising.  It calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *
 * Split-j partial sums use one fixed array inside the library
 * (NB_NOALLOC_SCRATCH_DOUBLES doubles, kept on every GPU that loads the
 * library until the process exits).  The first call on a device does a
 * one-time set-up: it looks up that array's device address
 * (cudaGetSymbolAddress) with the device current.  Make that first call
 * before any stream capture.  The address is remembered with the id of the
 * CUDA context it belongs to; after a device reset the next call repeats the
 * look-up (so, after a reset, make one call before any capture again).  All
 * calls share the array, which keeps the previous call's contents (every
 * partial is written before it is read, so nothing needs clearing): calls
 * whose work may overlap on the GPU race and must be ordered by the caller
 * (one stream, or events).
 * Errors: NB_EINVAL (N < 1, n < 0, n > N, n > NB_NOALLOC_MAX_ACTIVE -- the
 * partial sums would not fit --, NULL inputs, eps < 0), NB_ECUDA.
 */
int nb_forces_fp64_noalloc(int64_t N, const double* m, const double* x, const double* v, double eps,
                           const int32_t* i_idx, int64_t n, double* acc, double* jerk, double* pot,
                           void* cuda_stream);

/* nb_strerror -- static text for a status code (never NULL). */
const char* nb_strerror(int code);

/* nb_version -- library version string (never NULL). */
const char* nb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
