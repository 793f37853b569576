/*
 * mdlg.h -- C-ABI of libmdlg.so, the GB300 (sm_103a) hot path of the
 * molecular-dynamics lattice-gas (MDLG) equilibrium analysis of
 * Pachalieva & Wagner, arXiv 2101.01160.
 *
 * What the library computes
 *   * 2D Lennard-Jones molecular dynamics (Sec. 4): V = 4 eps [(s/r)^12 -
 *     (s/r)^6] truncated at rc and shifted to zero there (force not shifted),
 *     periodic square box, NVE velocity Verlet.
 *   * The MDLG coarse-graining fused into the time step (Sec. 2): every S MD
 *     steps each particle's lattice cell at t and t - S dt is compared and
 *     the integer displacement v_i is counted, i.e. the occupation numbers
 *     n_i(x,t) of Eq. (n_i) summed over all lattice sites x, accumulated over
 *     windows into the global histogram behind f_i^eq of Eq. (theory_feq);
 *     the displacement moments mu2, mu4 of Sec. 3(b) are accumulated beside.
 *   * The analytic equilibria of Sec. 3: the single-Gaussian f^{eq,G}
 *     (Eqs. feq_prod, feq_gaussian), the Poisson weighted sum of Gaussians
 *     f^{eq,WSG} (Eq. f_eq_wsg) and its collision rate lambda from the
 *     moments (Eq. lambda_eq), and the comparison measures of Eq. (k_Xi) /
 *     Eq. (kullback_leibler).
 *
 * Conventions
 *   * Every function returns MD_OK (0) or a negative MD_E_* code; no C++
 *     exception crosses the ABI.  md_last_error() gives a message for the
 *     calling thread's last failure.
 *   * "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it unless a function says
 *     it synchronises.
 *   * Pointers documented "host or device" may be either (the copy uses
 *     unified addressing); "device" means device memory the caller owns.
 *     The library never frees caller memory.  A md_system owns only its own
 *     state and scratch, released by md_destroy.
 *   * Lattice-velocity tables have (2W+1)^2 entries, entry (vy+W)(2W+1) +
 *     (vx+W) for the displacement (vx, vy), |vx|,|vy| <= W.
 *   * Positions are in sigma units on [0, L); the library stores them as a
 *     cell index plus an offset (FP32 or FP64) and reports L_eff = ncell*h,
 *     the box edge it actually simulates (equal to the requested L to FP64
 *     rounding for MD_FP64, to FP32 rounding of h for MD_FP32_CELLOFF).
 */
#ifndef MDLG_H
#define MDLG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MD_OK 0
#define MD_E_ARG -1        /* invalid argument (message says which)          */
#define MD_E_CUDA -2       /* CUDA runtime error                            */
#define MD_E_TIMEOUT -3    /* a bounded device-side wait gave up            */
#define MD_E_SKIN -4       /* a particle moved more than skin/2 between two  */
                           /* cell-list rebuilds (forces may have missed     */
                           /* pairs); raise skin                            */
#define MD_E_NONFINITE -5  /* a non-finite position or velocity was seen     */
#define MD_E_DOMAIN -6     /* kurtosis outside the range with a real lambda  */
#define MD_E_NOMEM -7      /* device allocation failed                      */
#define MD_E_LIMIT -8      /* a size exceeds a documented maximum           */

/* ---- precision of the MD state ----------------------------------------- */
#define MD_FP64 0          /* FP64 offsets, velocities and forces            */
#define MD_FP32_CELLOFF 1  /* integer cell + FP32 in-cell offset, FP32 forces */
                           /* and velocities; lattice mapping, moments and   */
                           /* reductions stay FP64                           */

#define MD_MAX_LG 8        /* sampling intervals per system                 */
#define MD_MAX_DX 4        /* lattice spacings per system                   */
#define MD_MAX_W 10        /* largest displacement window half-width        */
#define MD_NBLK 32         /* error-bar blocks per histogram                */
#define MD_MAX_REP 4096    /* replicas per batch                            */

/* Parameters of one system (one replica of a batch).  Units: LJ (sigma,
 * eps, m, tau).  The sampling interval of slot k is Delta t_LG =
 * lg_every[k]*dt (Sec. 4, "output frequency" times the MD step); lattice d
 * has lx[d] cells per edge, spacing L_eff/lx[d]. */
typedef struct md_params {
    int64_t n;             /* particles, >= 2                               */
    double box_L;          /* requested periodic box edge                   */
    double dt;             /* MD time step                                  */
    double rc;             /* LJ cutoff (2.5 in the configured workloads)    */
    double eps, sigma, mass;
    double skin;           /* Verlet skin: neighbour lists hold all pairs   */
                           /* within rc + skin (cell edge >= rc + skin) and */
                           /* are rebuilt once the accumulated bound on     */
                           /* any displacement reaches skin/2                */
    int32_t precision;     /* MD_FP64 or MD_FP32_CELLOFF                     */
    int32_t W;             /* displacement window half-width, 1..MD_MAX_W   */
    int64_t n_equil;       /* MD steps before the first snapshot            */
    int32_t n_lg;          /* sampling intervals in use, 0..MD_MAX_LG       */
    int32_t lg_every[MD_MAX_LG];
    int32_t n_dx;          /* lattices in use, 1..MD_MAX_DX                 */
    int32_t lx[MD_MAX_DX]; /* lattice cells per box edge                    */
    int32_t block_windows; /* windows per error-bar block (>= 1)            */
    int32_t nbr_max;       /* neighbour-list capacity per particle (0 =     */
                           /* automatic: 3x the mean count within rc+skin   */
                           /* plus 8 standard deviations); overflow is      */
                           /* reported as MD_E_LIMIT by md_sync              */
} md_params;

typedef struct md_system md_system;   /* opaque, library-owned */

/* Snapshot of positions in the (cell, offset) encoding: the position of
 * particle j is x = cx*h + off_x[j], y = cy*h + off_y[j] (FP64 arithmetic,
 * each product and sum rounded separately), with cell[j] = cy*ncell + cx.
 * Offsets may lie outside [0, h) (a stale cell list); positions are taken
 * modulo the box edge ncell*h. */
typedef struct md_snapshot {
    const int32_t *cell;   /* device, [n]                                   */
    const void *off_x;     /* device, [n] float or double                   */
    const void *off_y;     /* device, [n] float or double                   */
    int32_t off_is_f64;    /* 0: float offsets, 1: double offsets           */
    int32_t ncell;         /* cells per box edge                            */
    double h;              /* cell edge; box edge L = ncell*h               */
} md_snapshot;

/* Information about a system, filled by md_info. */
typedef struct md_info_t {
    int64_t n_total;       /* particles over all replicas                   */
    int64_t step;          /* completed MD steps                            */
    int64_t n_rebuilds;    /* cell-list rebuilds so far                     */
    int32_t n_rep;
    int32_t precision;
    int32_t grid_blocks;   /* persistent-kernel CTAs                        */
    int32_t block_threads;
} md_info_t;

typedef struct md_rep_info_t {
    int64_t n;
    double L_eff;          /* ncell*h                                       */
    double h;              /* MD cell edge                                  */
    int32_t ncell;
    int32_t reserved;
    double dx_eff[MD_MAX_DX]; /* L_eff / lx[d]                              */
} md_rep_info_t;

/* Measured equilibrium of one (replica, interval, lattice), see feq_measured. */
typedef struct md_feq_stats {
    double mu2;            /* <dx_alpha^2> per axis over all samples         */
    double mu4;            /* <dx_alpha^4>                                  */
    double a2;             /* mu2 / dx_eff^2 (Eq. a2_n_ua)                  */
    double dx_eff;
    int64_t n_windows;     /* sampling windows accumulated                  */
    int64_t n_samples;     /* particle-windows = sum(hist) + n_overflow     */
    int64_t n_overflow;    /* displacements outside the window             */
    int64_t n_blocks_used; /* error-bar blocks holding data                 */
} md_feq_stats;

/* ---- system lifecycle ---------------------------------------------------- */

/* Creates a system of one replica from an initial state (Sec. 4: homogeneous
 * positions, kinetic energy at the target temperature, zero momentum; the
 * caller generates it).  x, y, vx, vy: host or device, FP64, [p->n],
 * particle-id order; positions are wrapped into the box.  Velocities are
 * taken as the velocities at step 0.  Synchronises the stream.  On success
 * *out owns device memory until md_destroy. */
int md_init(const md_params *p, const double *x, const double *y, const double *vx,
            const double *vy, void *stream, md_system **out);

/* Creates a batch of n_rep independent replicas advanced together by one
 * persistent kernel.  p[r] are the per-replica parameters; precision, W,
 * n_equil, n_lg, lg_every, n_dx and block_windows must agree over all
 * replicas (lx, L, n, dt, ... may differ).  The state arrays hold the
 * replicas back to back in replica order (sum of p[r].n entries). */
int md_init_batch(const md_params *p, int32_t n_rep, const double *x, const double *y,
                  const double *vx, const double *vy, void *stream, md_system **out);

void md_destroy(md_system *s);

/* Advances every replica by nsteps velocity-Verlet steps (Sec. 4) in one
 * persistent cooperative kernel, sampling the MDLG histograms (Sec. 2) on
 * every step t = n_equil + m*lg_every[k] and rebuilding cell lists as
 * needed.  Asynchronous on the system's stream; device-side failures
 * (MD_E_TIMEOUT, MD_E_SKIN, MD_E_NONFINITE) are reported by md_sync. */
int md_step(md_system *s, int64_t nsteps);

/* Launch shape of the persistent kernel: block_threads in {128, 256} (0 =
 * 256), per_thread in [1, 8] particles per thread per chunk (0 = 1),
 * staging 1 = each chunk's neighbour positions, velocities and first list
 * entries are copied to shared memory (double buffered) before its forces
 * are computed, 2 = neighbours are read from global memory through L1,
 * 3 = as 2 with the register budget of full occupancy (8 CTAs of 256
 * threads per SM; FP32 only, in FP64 the same as 2) (0 = 1).
 * staging 4 selects the shared-memory-resident engine instead (FP32 only):
 * every replica is cut into slabs of whole MD-cell rows, each slab held in
 * one CTA's shared memory (state and Verlet lists) for the whole md_step,
 * the slabs of a replica exchanging their boundary rows through L2 and
 * meeting at a bounded per-replica barrier once per step; block_threads and
 * per_thread are ignored; MD_E_LIMIT if a replica fits no slab plan.
 * Results do not depend on the shape or the engine: particle order, force
 * summation order, every reduction order and the rebuild schedule (per
 * replica) are fixed by the data, not by the launch; only the FP64 moment
 * sums are grouped differently by the two engines (their last bits may
 * differ).  Used by md_autotune. */
int md_tune(md_system *s, int32_t block_threads, int32_t per_thread, int32_t staging);

/* Autotuner: times md_step(steps_per_trial) twice for every launch shape
 * (block {256,128} x per_thread {1,2,4} x staging {1,2,3}; 3 skipped in
 * FP64; then staging 4 for FP32 batches of >= 2 replicas) and keeps the
 * fastest; the choice is cached for the process by (precision, replicas,
 * particle count rounded up to a power of two, list capacity) and reused
 * without trials.  The trial steps are real MD steps: the system advances
 * by them (the trajectory itself does not depend on the shape).  best3
 * (host, may be NULL) receives {block_threads, per_thread, staging}.
 * Synchronises. */
int md_autotune(md_system *s, int64_t steps_per_trial, int32_t *best3);

/* Host-only dry run of the resident engine's plan (md_tune staging 4) for
 * the replicas p[0 .. n_rep) on `grid` CTAs with smem_bytes of dynamic
 * shared memory each (no GPU call; a project addition, no counterpart in
 * the paper).  Each replica is cut into g slabs of whole MD-cell rows; the
 * slabs are dealt to the CTAs.  jobs_out (host, [max_jobs][8]) receives per
 * slab {replica, g, k, first row, end row, particle capacity, halo capacity,
 * CTA of slab 0}, grouped by CTA in execution order; start_out (host,
 * [grid + 1]) the first slab of each CTA; *makespan (may be NULL) the
 * plan's estimated time in its cost units.  MD_E_LIMIT when a replica fits
 * no plan or there are more than max_jobs slabs. */
int md_resident_plan(const md_params *p, int32_t n_rep, int32_t grid, int64_t smem_bytes, int32_t *jobs_out,
                     int32_t max_jobs, int32_t *start_out, double *makespan);

/* Waits for the system's stream and returns the device status word (and
 * clears it). */
int md_sync(md_system *s);

/* Failure-detection self-test of the bounded grid barrier (no counterpart in
 * the paper).  Runs one MD step launch in which CTA 0 leaves the kernel
 * instead of arriving at the step's grid barrier, with the barrier wait
 * limited to limit_s seconds (0 < limit_s <= 4): the other CTAs give up
 * after limit_s, flag the timeout and leave, and the call returns
 * MD_E_TIMEOUT (MD_OK would mean the limit failed).  Nothing faults or
 * hangs; the barrier's arrival count is cleared afterwards, but the
 * particle state is that of an aborted step: destroy the system.  Needs a
 * launch of at least 2 CTAs.  Synchronises. */
int md_barrier_selftest(md_system *s, double limit_s);

int md_info(md_system *s, md_info_t *out);
int md_rep_info(md_system *s, int32_t rep, md_rep_info_t *out);

/* Positions (wrapped into [0, L_eff)) and velocities at the current step, in
 * particle-id order over all replicas; host or device outputs, FP64.
 * Completes the half kick if needed (the trajectory continues bit for bit
 * as if not called).  Synchronises. */
int md_get_state(md_system *s, double *x, double *y, double *vx, double *vy);

/* Replaces positions and velocities (same layout as md_init; host or device
 * FP64 arrays, read in stream order on the system's stream); keeps the
 * histograms and the step counter.  Synchronises. */
int md_set_state(md_system *s, const double *x, const double *y, const double *vx,
                 const double *vy);

/* Exact checkpoint of a system (no counterpart in the paper): everything
 * that decides its future trajectory and statistics -- step counter,
 * half-step flag, displacement bounds, the particle state slot by slot
 * (cells, offsets, velocities, ids), the sampling snapshots, the integer
 * histograms of every error-bar block, the overflow counts and the FP64
 * moment partials.  md_checkpoint_bytes gives the size; md_checkpoint_save
 * writes it to host memory `buf` (synchronises); md_checkpoint_load
 * restores it into a system created by md_init / md_init_batch with the
 * same parameters (any initial state; MD_E_ARG for a checkpoint of other
 * sizes) and synchronises.  Running k steps, saving, loading into a fresh
 * system and running m more steps gives the same bits as k + m steps
 * straight: positions, velocities, snapshots, histograms and overflow on
 * either engine, the FP64 moment sums too on the global engine (the
 * resident engine sums a slab's moment terms in its slot order, which a
 * load resets, so their last bits may differ).  The buffer format is that
 * of this library build only. */
int md_checkpoint_bytes(md_system *s, int64_t *bytes);
int md_checkpoint_save(md_system *s, void *buf);
int md_checkpoint_load(md_system *s, const void *buf);

/* Raw current positions in the snapshot encoding, particle-id order:
 * cell (linear cy*ncell+cx), offsets as float (MD_FP32_CELLOFF) or double
 * (MD_FP64).  Device outputs.  Synchronises. */
int md_get_raw(md_system *s, int32_t *cell, void *off_x, void *off_y);

/* The snapshot held for sampling interval lg (positions at the last
 * sampling time), same encoding as md_get_raw. Device outputs. Synchronises. */
int md_get_snapshot(md_system *s, int32_t lg, int32_t *cell, void *off_x, void *off_y);

/* Forces at the current positions, FP64, particle-id order, host or device
 * outputs; fabs_sum (may be NULL) receives sum_j |F_ij| per particle.
 * Synchronises. */
int md_forces(md_system *s, double *fx, double *fy, double *fabs_sum);

/* Advances nsteps >= 1 steps exactly as md_step(s, nsteps) does (the same
 * kernel and launch shape, the same trajectory bit for bit) and returns, by
 * particle id, the Lennard-Jones force (Sec. 4) that the last step's force
 * pass summed over the Verlet neighbour lists at the positions of step
 * nsteps - 1 (those that md_get_raw returned just before the call when
 * nsteps = 1).  This is the arithmetic of every ordinary step, including
 * lists built several steps earlier; md_forces instead evaluates the force
 * from the current cell list.  fx, fy: host or device, FP64, [n_total].
 * Synchronises. */
int md_step_forces(md_system *s, int64_t nsteps, double *fx, double *fy);

/* Energy of replica rep at the current step: out4 = {kinetic, shifted
 * potential, P_x, P_y} (host, FP64).  Synchronises. */
int md_energy(md_system *s, int32_t rep, double *out4);

/* Energies (Sec. 4: kinetic, shifted Lennard-Jones potential, momentum) of
 * every replica from one evaluation of the current state: out[4 r + k] =
 * component k of md_energy(s, r, .) for replica r, bit for bit (the same
 * partial sums in the same order).  out: host or device, FP64, [n_rep][4],
 * caller-owned.  The kinetic temperature of replica r in two dimensions with
 * zero total momentum is out[4 r] / (N_r - 1).  MD_E_ARG for a null handle
 * or out.  Synchronises. */
int md_energy_batch(md_system *s, double *out);

/* Raw integer histogram totals of (rep, lg, dxi): hist (host, int64,
 * (2W+1)^2), *overflow, *n_windows (host).  Synchronises. */
int md_hist_raw(md_system *s, int32_t rep, int32_t lg, int32_t dxi, int64_t *hist,
                int64_t *overflow, int64_t *n_windows);

/* Measured equilibrium distribution (Eq. theory_feq, normalised per
 * particle): P_out[i] = H_i / (N * n_windows), the probability that a
 * particle's lattice displacement over one interval is v_i; sum(P) = 1 -
 * overflow fraction.  If symmetrize != 0 each value is replaced by its
 * symmetric-set average (Sec. 5).  stderr_out (may be NULL) receives the
 * batch-means standard error over error-bar blocks.  Normalisation runs on
 * the device in FP64; outputs are host memory.  Synchronises. */
int feq_measured(md_system *s, int32_t rep, int32_t lg, int32_t dxi, int32_t symmetrize,
                 double *P_out, double *stderr_out, md_feq_stats *stats);

/* The integer histogram of (rep, lg, dxi) per error-bar block: hist (host,
 * int32, [MD_NBLK][(2W+1)^2]) and wblk (host, int64, [MD_NBLK]) the windows
 * each block holds.  Synchronises. */
int md_hist_blocks(md_system *s, int32_t rep, int32_t lg, int32_t dxi, int32_t *hist, int64_t *wblk);

/* Block-bootstrap standard error of the measured equilibrium (Eq.
 * theory_feq as feq_measured normalises it; the paper's averages over
 * iterations come from a finite run) for every replica: the error-bar
 * blocks of windows holding data are resampled with replacement, as many
 * draws as used blocks, n_resamples times (2 .. 2^20); each resample's P_i
 * is its drawn counts over n * its drawn windows (symmetric-set averaged if
 * symmetrize != 0); sigma_out[r*(2W+1)^2 + i] is the sample standard
 * deviation of P_i over the resamples (divisor n_resamples - 1).  Draws:
 * SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator,
 * draw c = ((r * 2^20 + b) * 64 + k) of `seed` for slot k of resample b:
 * the output function of seed + (c + 1) * 0x9e3779b97f4a7c15, block index
 * = (draw >> 32) * used >> 32.  sigma_out: host (synchronises) or device
 * (asynchronous on the stream). */
int feq_bootstrap(md_system *s, int32_t lg, int32_t dxi, int32_t symmetrize, int32_t n_resamples, uint64_t seed,
                  double *sigma_out);

/* The whole f_eq stage for every replica in one launch (no host round
 * trip): per replica r, out[r*(3*nb+16) + ...] holds
 *   [0, nb)      measured P_i (as feq_measured, symmetric-set averaged if
 *                symmetrize != 0),
 *   [nb, 2nb)    Gaussian equilibrium (Eq. feq_gaussian) at the measured a^2,
 *   [2nb, 3nb)   WSG equilibrium (Eq. f_eq_wsg) at a^2 and lambda,
 *   3nb + 0..13  mu2, mu4, a^2, lambda (root 2 of Eq. lambda_eq; 0 when the
 *                kurtosis is <= 3, 1 when > 3.75, capped at 1e5),
 *                max|P-G|, D_KL(P||G), max|P-WSG|, D_KL(P||WSG), windows,
 *                samples, overflow, dx_eff, lambda status (0 ok, 1 k<=3,
 *                2 k>3.75, 3 capped), sum(P).
 * nb = (2W+1)^2.  out: host or device; with host memory the call
 * synchronises, with device memory it is asynchronous on the stream. */
int feq_batch(md_system *s, int32_t lg, int32_t dxi, int32_t symmetrize, double *out);

/* ---- MDLG binning of two snapshots (Sec. 2, Eq. n_i) -------------------- */

/* Lattice displacement histogram of n particles between snapshots t0 and t1
 * (same ncell and h): lattice index l = floor(x / dxl) mod lx per axis,
 * dxl = ncell*h/lx, displacement = nearest periodic image of l1 - l0; inside
 * the window it counts in hist_out, else in *overflow_out.  mom_out[0] =
 * sum of delta^2, mom_out[1] = sum of delta^4 over particles and both axes
 * for the continuous nearest-image displacement delta.  Outputs (device)
 * are overwritten.  Bit-exact integer results: the FP64 arithmetic is
 * rounded operation by operation.  n < 2^31. */
int mdlg_bin(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx, int32_t W,
             int32_t *hist_out, int64_t *overflow_out, double *mom_out, void *stream);

/* mdlg_bin without any device allocation.  The paper has no counterpart;
 * this is for callers that cannot allocate device memory while they run:
 * a process whose device memory is all handed to a framework's caching
 * allocator or to a fixed budget at start-up (a cudaMalloc there fails or
 * forces a device-wide synchronisation), or an analysis loop binning many
 * snapshot pairs that must not stall on allocator calls.  Same arguments,
 * same results bit for bit (same launch shape).  The per-CTA moment
 * partials go to one fixed 32 KiB device array inside the library (every
 * GPU that loads the library holds it until the process exits), room for
 * 2048 CTAs; the grid is
 * min(ceil(n/256), 8 x SM count), 1216 CTAs on a 152-SM GPU, and a call
 * that would need more returns MD_E_LIMIT.  The outputs are cleared with
 * cudaMemsetAsync on `stream`; the array needs no clearing.  The array is
 * shared by every call on a device: calls that may run at the same time on
 * the device (other streams, other host threads, without ordering between
 * them) race on it and can return wrong moments, so order them.  The first
 * call on each device looks up the array's address (cudaGetSymbolAddress);
 * make that first call before any stream capture. */
int mdlg_bin_noalloc(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx, int32_t W,
                     int32_t *hist_out, int64_t *overflow_out, double *mom_out, void *stream);

/* ---- arithmetic peaks (measurement; no counterpart in the paper) -------- */

/* Measured fused multiply-add throughput of the current GPU, FP32 (f64 = 0)
 * or FP64 (f64 = 1): the full resident grid runs 8 independent FFMA / DFMA
 * chains per thread for `iters` rounds (1 <= iters <= 2^32) after a short
 * warm-up, timed with CUDA events on `stream`.  *flops_per_s (host)
 * receives 2 flops per multiply-add over the elapsed time, *ms_out (host,
 * may be NULL) the time.  The denominator of the FP64 MD path's roofline
 * and of the shared-memory-resident FP32 path's.  Synchronises. */
int mdlg_fma_peak(int32_t f64, int64_t iters, double *flops_per_s, double *ms_out, void *stream);

/* ---- local MDLG fields (Sec. 2, Eqs. n_i and mdlg_evolution) ------------ */

/* Local occupation numbers of Eq. (n_i): n_i(x, t1) is the number of
 * particles in lattice site x at t1 that were in site x - v_i at t0.  Sites
 * and the lattice displacement v_i are those of mdlg_bin (l = floor(x /
 * dxl) mod lx per axis, dxl = ncell*h/lx, nearest periodic image of
 * l1 - l0), so the field summed over its sites is mdlg_bin's histogram and
 * its overflow summed is mdlg_bin's overflow, bit for bit.
 * n_out: device int32 [(2W+1)^2][lx][lx], class-major, entry
 * ((vy+W)(2W+1) + (vx+W)) lx^2 + ly lx + lx_ at the arrival site (lx_, ly);
 * overflow_out: device int32 [lx][lx], particles arriving at a site whose
 * displacement leaves the window.  Both are ADDED TO (clear them first): a
 * call over a snapshot pair that concatenates R replicas of one box, or R
 * calls, leave the ensemble sum, and f_i = <n_i> of the MDLB (Sec. 2) is
 * that sum over R.  Counts are exact; the caller keeps each entry below
 * 2^31.  n < 2^31, 1 <= lx, 0 <= W <= MD_MAX_W, (2W+1)^2 lx^2 < 2^31
 * (MD_E_LIMIT).  Asynchronous on stream. */
int mdlg_site_occupation(const md_snapshot *t0, const md_snapshot *t1, int64_t n, int32_t lx,
                         int32_t W, int32_t *n_out, int32_t *overflow_out, void *stream);

/* Lattice-gas collision operator of Eq. (mdlg_evolution):
 * Xi_i(x, t) = n_i(x + v_i, t + dt) - n_i(x, t), x + v_i periodic on the
 * lx x lx lattice, from the fields n_t = n(., t) and n_next = n(., t + dt)
 * in the layout of mdlg_site_occupation (the window t -> t + dt must start
 * at the snapshot that ended the window of n_t).  xi_out (int32) and/or
 * omega_out (double, scale * Xi; with fields summed over R replicas and
 * scale = 1/R this is the MDLB collision operator Omega_i = <Xi_i>) are
 * overwritten; either may be NULL, not both.  All device memory, same
 * shape as the fields.  Summed over i, Xi vanishes at every site when no
 * displacement of either window left the window W.  Asynchronous on
 * stream. */
int mdlg_collision(const int32_t *n_t, const int32_t *n_next, int32_t lx, int32_t W, double scale,
                   int32_t *xi_out, double *omega_out, void *stream);

/* ---- displacement-PDF diagnostics (Sec. 3(b), Fig. 2) -------------------- */

/* Histogram of the continuous one-dimensional displacement component between
 * snapshots t0 and t1 (same ncell and h): for every particle and both axes,
 * delta = wrap(c1 - c0) * h + (off1 - off0), the cell-index difference
 * wrapped to the nearest periodic image (into [-ncell/2, ncell/2]) -- the
 * continuous nearest-image displacement, evaluated in the cell frame with a
 * single rounding -- falls in bin floor(delta * (1/width)) + nbins/2 (each
 * operation rounded on its own; bin k covers about
 * [(k - nbins/2) width, (k - nbins/2 + 1) width)).  Values outside all bins
 * count in *outside_out, so sum(hist) + outside = 2n.  hist_out
 * (int64[nbins]) and outside_out are device memory, overwritten; exact
 * integers.  n < 2^31, 1 <= nbins <= 8192, width > 0, else MD_E_ARG.
 * Asynchronous on stream. */
int mdlg_disp_hist(const md_snapshot *t0, const md_snapshot *t1, int64_t n, double width,
                   int32_t nbins, int64_t *hist_out, int64_t *outside_out, void *stream);

/* Bin masses, over the bins of mdlg_disp_hist, of the one-dimensional
 * Gaussian displacement PDF of second moment mu2 (Eq. gaussian_df, d = 1,
 * u = 0) into pg_out, and of the Poisson weighted sum of Gaussians
 * (Eq. poisson_v2 with the Gaussians of Eq. p_wsg_one, variance
 * (c+1) mu2/(lambda+1), c over the window lambda +- (12 sqrt(lambda) + 20))
 * into pwsg_out.  Device outputs (double[nbins]).  mu2 > 0,
 * 0 <= lambda <= 1e5, width > 0, 1 <= nbins <= 8192, else MD_E_ARG. */
int disp_pdf_models(double mu2, double lambda, double width, int32_t nbins, double *pg_out,
                    double *pwsg_out, void *stream);

/* Element-wise Kullback-Leibler terms of Eq. k_Xi, K_out[i] =
 * R[i] log(R[i]/Q[i]) (0 where R[i] = 0); their sum is D_KL of
 * Eq. kullback_leibler.  R, Q, K_out: device double[n]. */
int kl_terms(const double *R, const double *Q, int32_t n, double *K_out, void *stream);

/* ---- analytic equilibria (Sec. 3) ---------------------------------------- */

/* Single-Gaussian equilibrium, Eqs. (feq_prod), (feq_gaussian): P_out[i] =
 * f_i^{eq,G}/rho = g(vx - ux) g(vy - uy), a2 = <dx^2>/dx^2, (ux, uy) the mean
 * velocity in lattice units.  P_out: device, (2W+1)^2 doubles. */
int feq_gaussian(double a2, double ux, double uy, int32_t W, double *P_out, void *stream);

/* Mean collision number lambda from the measured moments, Eq. (lambda_eq):
 * root 1 takes the '+' sign of the square root, root 2 (the paper's choice)
 * the '-' sign.  *lambda_out: device double.  If the kurtosis mu4/mu2^2 is
 * <= 3 (no excess: the mixture degenerates to one Gaussian) 0 is written; if
 * it exceeds 3.75 (no real root) 1 is written (the double root at 3.75);
 * both return MD_E_DOMAIN. */
int wsg_lambda(double mu2, double mu4, int32_t root, double *lambda_out, void *stream);

/* Poisson weighted sum of Gaussians equilibrium, Eq. (f_eq_wsg): P_out[i] =
 * sum_c Pois(c; lambda) f^c(vx-ux) f^c(vy-uy), N_c = sqrt(2 a2 (c+1) /
 * (lambda+1)); terms c with |c - lambda| <= 12 sqrt(lambda) + 20 (omitted
 * Poisson tails < 1e-16).  lambda < 1e6.  P_out: device, (2W+1)^2
 * doubles. */
int feq_wsg(double a2, double lambda, double ux, double uy, int32_t W, double *P_out,
            void *stream);

/* Comparison of two distributions over n classes (Sec. 3, Eqs. k_Xi,
 * kullback_leibler): out3 (device) = {max_i |R_i - Q_i|, D_KL(R||Q) with
 * 0 log 0 = 0, sum_i R_i}.  R, Q: device. */
int feq_compare(const double *R, const double *Q, int32_t n, double *out3, void *stream);

/* ---- f_eq surrogate (a project addition, not in the paper) -------------- */

/* A multilayer perceptron from the state point x = (phi, T, Delta t_LG,
 * Delta x) to the probabilities of n_classes (2..112) displacement classes:
 * features (x - shift)/scale, n_hidden (2..15) layers of width 256 with the
 * SiLU activation, a softmax output; trained on the mean Kullback-Leibler
 * divergence (Eq. kullback_leibler) to measured distributions with Adam.
 * Training runs layer 1 in FP32 on CUDA cores and the others as BF16
 * tensor-core GEMMs with FP32 accumulation.  Weights are FP32 masters with
 * BF16 copies for the tensor cores.  params (host or device, FP32) packs
 * W_1, b_1, W_2, b_2, ... with W_l row-major [out][in]; mlp_param_count
 * gives its length.  Device memory is owned by the model (workspace grows
 * with the largest batch seen).  MD_E_ARG for sizes outside these ranges. */
typedef struct mlp_model mlp_model;
int mlp_create(int32_t n_hidden, int32_t width, int32_t n_classes, const float *shift4,
               const float *scale4, const float *params, mlp_model **out);
void mlp_destroy(mlp_model *m);
int64_t mlp_param_count(mlp_model *m);
int mlp_set_params(mlp_model *m, const float *params);
int mlp_get_params(mlp_model *m, float *params);

/* P_out[M][n_classes] = model(X[M][4]); X (16-byte aligned), P_out device
 * FP32.  One fused persistent kernel; every layer runs on the tensor cores
 * with FP32 accumulation: layer 1 as one K = 16 product of split BF16
 * operands (x_hi W_hi + x_lo W_hi + x_hi W_lo, relative error ~2^-16), the
 * others BF16 x BF16; SiLU through the hardware tanh approximation (relative
 * error ~2^-11, below the BF16 rounding of the activations).  Asynchronous
 * on `stream`; MD_E_ARG for NULL pointers, M < 1 or misaligned X. */
int mlp_forward(mlp_model *m, const float *X, int64_t M, float *P_out, void *stream);

/* Gradient of the mean KL loss over a batch (X [B][4], targets T
 * [B][n_classes], device, B a multiple of 128) into grad_out (device or host,
 * packed like params; may be NULL) and the loss into *loss_out (device, may
 * be NULL).  Asynchronous. */
int mlp_grad(mlp_model *m, const float *X, const float *T, int32_t B, float *grad_out,
             float *loss_out, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on a
 * batch.  Asynchronous. */
int mlp_train_step(mlp_model *m, const float *X, const float *T, int32_t B, float lr,
                   float *loss_out, void *stream);

/* Waits for the device and reports a timed-out tensor-core wait
 * (MD_E_TIMEOUT). */
int mlp_status(mlp_model *m);

/* C[M][N] (FP32) = A[M][K] * B[N][K]^T on the tensor cores; A, B BF16
 * row-major device; M % 128 == 0, K % 64 == 0, N % 16 == 0 with N <= 256.
 * *status (device int) gets bit 0 set if a wait timed out.  Asynchronous. */
int bf16_gemm_tn(const void *A, const void *B, float *C, int32_t M, int32_t N, int32_t K,
                 int32_t *status, void *stream);

/* Failure-detection self-test of the bounded mbarrier waits of the
 * tensor-core kernels (no counterpart in the paper): bf16_gemm_tn on the
 * same arguments, except that CTA 0 withholds the completion signal of its
 * first K stage and every mbarrier wait is limited to limit_s seconds (0 <
 * limit_s <= 2; K >= 192, so that a later stage waits for that signal).
 * CTA 0's wait runs out, it waits (with the same limit) for the MMAs it
 * issued, frees its tensor memory, flags *status and leaves; the call
 * returns MD_E_TIMEOUT (MD_OK would mean the limit failed).  Nothing faults
 * or hangs; C is undefined.  Synchronises the stream. */
int bf16_gemm_selftest(const void *A, const void *B, float *C, int32_t M, int32_t N, int32_t K,
                       int32_t *status, double limit_s, void *stream);

/* Message of the calling thread's last failure ("" if none). */
const char *md_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MDLG_H */
