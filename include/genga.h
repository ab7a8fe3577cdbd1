/*
 * genga.h -- C ABI of the GB300 (sm_103a) hybrid symplectic N-body hot path of
 * GENGA II (Grimm et al., arXiv:2201.10058).
 *
 * One library object (genga_system_t) integrates N bodies around a central mass
 * in democratic heliocentric coordinates (Sec. 2, Eq. H = Ha + Hb + Hc):
 * heliocentric positions, barycentric velocities.  The caller owns the state
 * arrays (device memory, structure-of-arrays, component-major):
 *
 *     pos[0*n + i], pos[1*n + i], pos[2*n + i]   x, y, z of body i   (AU)
 *     vel[0*n + i], vel[1*n + i], vel[2*n + i]   barycentric velocity (AU/day)
 *     mass[i]                                    (solar masses)
 *
 * The library keeps these pointers and updates pos/vel in place on the stream
 * given at creation.  It owns all scratch (critical radii, candidate and
 * encounter pair lists, groups, pre-drift copies, kick partial sums,
 * Bulirsch-Stoer state) and frees it in genga_destroy.
 *
 * Calls are stream-ordered.  Unless a comment says otherwise a call returns
 * after enqueueing its kernels; errors detected on the device (non-converged
 * Kepler solve or Bulirsch-Stoer integration, capacity overflow, bad state)
 * are latched in a device error word and reported by the next call that
 * synchronises (genga_step, genga_build_encounters, genga_energy, the getters,
 * genga_sync).  Return value: 0 on success, a negative GENGA_E* code otherwise;
 * genga_last_error() gives a message.  No call falls back to the CPU.
 */
#ifndef GENGA_H
#define GENGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define GENGA_OK          0
#define GENGA_EINVAL     -1  /* bad argument (null pointer, n < 1, bad parameter) */
#define GENGA_ECAPACITY  -2  /* a fixed capacity was exceeded (see genga_get_stats) */
#define GENGA_ENONCONV   -3  /* Kepler or Bulirsch-Stoer iteration limit reached */
#define GENGA_ETIMEOUT   -4  /* a bounded device wait gave up */
#define GENGA_EBADSTATE  -5  /* NaN/Inf in the state, or a body at the origin */
#define GENGA_ECUDA      -6  /* a CUDA runtime call failed */
#define GENGA_ENOMEM     -7  /* device allocation failed */

/* ---- kick arithmetic --------------------------------------------------- */
#define GENGA_FP64   0   /* every pair term in FP64 (double rsqrt: CUDA's in the tiled
                            kick layout, an FP32 seed with an FP64 Newton step and
                            series of full double precision in the symmetric one) */
#define GENGA_MIXED  1   /* FP64 displacement and accumulation, FP32 rsqrt seed +
                            one FP64 Newton correction, compensated per-tile sums */

/* Integration parameters.  Units are the caller's; the defaults of
 * genga_default_params are Gaussian units (AU, day, solar mass).            */
typedef struct genga_params {
    double G;          /* gravitational constant */
    double m_star;     /* central mass */
    double dt;         /* base time step */
    double n1;         /* Eq. rcrit: Hill-radius factor (paper: 3) */
    double n2;         /* Eq. rcrit: velocity factor (paper: 0.4) */
    double f_pc;       /* pre-check factor: candidates have r_ij < f_pc * rc_ij (default 4) */
    double bs_tol;     /* Bulirsch-Stoer relative tolerance (default 1e-13) */
    int32_t slevels;   /* symplectic levels, Sec. 6.3 / Appendix A (1 = original method) */
    int32_t substeps;  /* sub-steps per level (time-step reduction factor per level) */
    int32_t precision; /* GENGA_FP64 or GENGA_MIXED for the all-pairs kick */
    int32_t kepler_max_iter; /* Newton iteration limit of the Kepler solve (default 50) */
    int32_t bs_max_steps;    /* limit on Bulirsch-Stoer step attempts per group (default 100000) */
    int32_t tp_mode;         /* Sec. 8.1 test-particle mode: 0 every pair interacts (default);
                                2 semi-active: bodies i >= n_massive are test particles and two
                                test particles have no interaction (no force, no candidate, no
                                encounter, no potential term).  Mode 1 (test particles that act
                                on nothing) is mode 2 with massless test particles.  The
                                adjoint calls refuse mode 2. */
    int64_t cand_capacity;   /* initial capacity of the candidate pair list (grows on demand) */
    int64_t pair_capacity;   /* initial capacity of each level's encounter list (grows) */
    int64_t n_massive;       /* tp_mode 2: the large bodies are 0..n_massive-1 (callers order the
                                bodies by a mass threshold); >= n means no test particles */
} genga_params_t;

/* Counters of the last genga_step call (summed over its steps). */
typedef struct genga_stats {
    int64_t n_candidates;    /* pre-check candidate pairs */
    int64_t n_pairs[8];      /* encounter pairs found per level (summed over sub-steps) */
    int64_t n_groups;        /* close-encounter groups integrated by Bulirsch-Stoer */
    int64_t max_group;       /* largest group */
    int64_t bs_steps;        /* accepted Bulirsch-Stoer sub-steps */
    int64_t bs_rejects;      /* rejected attempts (step halvings) */
    int64_t kepler_fail;     /* Kepler solves that hit kepler_max_iter */
    int64_t bs_fail;         /* groups that hit bs_max_steps */
    int64_t kernel_launches; /* CUDA kernels this library launched for these steps */
    int64_t bs_max_attempts; /* most step attempts any one group needed */
    int64_t host_syncs;      /* times the host waited for the stream inside these steps */
} genga_stats_t;

typedef struct genga_system genga_system_t;

/* Fills *p with the paper's defaults (n1 = 3, n2 = 0.4, Sec. 2) and this
 * library's defaults for the remaining fields; G is k^2 for the Gaussian k.  */
void genga_default_params(genga_params_t *p);

/* Creates a system of n bodies on the CUDA stream `stream` (a cudaStream_t;
 * NULL = legacy default stream) of the current device.  pos and vel (3n
 * doubles each) and mass (n doubles) are caller-owned device arrays that must
 * outlive the system.  Allocates all library scratch.  Errors: EINVAL, ENOMEM.
 * genga_create is the same call under its earlier name.                     */
int genga_init_system(genga_system_t **out, const genga_params_t *p, int64_t n, double *pos,
                      double *vel, const double *mass, void *stream);
int genga_create(genga_system_t **out, const genga_params_t *p, int64_t n, double *pos,
                 double *vel, const double *mass, void *stream);

/* Frees the library scratch (not the caller's arrays).  NULL is a no-op.   */
void genga_destroy(genga_system_t *sys);

/* Message of the last failed call on this system ("" if none).  The string is
 * owned by the system and valid until its next call.                       */
const char *genga_last_error(const genga_system_t *sys);

/* Changes the parameters (same n).  Levels beyond those the system already
 * holds get their arrays here; arrays of levels dropped are kept for reuse.
 * Errors: EINVAL (invalid parameters; nothing changed), ENOMEM, ECUDA.      */
int genga_set_params(genga_system_t *sys, const genga_params_t *p);

/* Blocks until the stream has finished; reports latched device errors.     */
int genga_sync(genga_system_t *sys);

/* Eq. rcrit (Sec. 2): rc_i = max(n1 R_H,i, n2 dt |v_i|) for every body, with
 * R_H,i = |x_i| (m_i / 3 m_star)^(1/3), stored as the level-0 critical radii
 * used by genga_kick, genga_build_encounters and genga_bs.                  */
int genga_rcrit(genga_system_t *sys, double dt);

/* Replaces the level-0 critical radii with the n values of the host array rc
 * (a test hook; the derived thresholds are recomputed).  Synchronises.      */
int genga_set_rcrit(genga_system_t *sys, const double *rc_host);

/* Kick of Eq. Hb (Appendix A "Kick(dt/2)"): for every body
 *     v_i += dt_half * G * sum_{j != i} m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3
 * with the changeover function K of Chambers (1999), Eq. 10 (Sec. 6.3 fn.),
 * rc_ij = max(rc_i, rc_j) from genga_rcrit, in the arithmetic selected by
 * params.precision.  If precheck != 0 a pass before the kick records the
 * close-encounter candidates at the same positions (i < j with
 * r_ij^2 < (f_pc rc_ij)^2, decided exactly in FP64) for genga_build_encounters.
 * If acc_out (device, 3n doubles, SoA) is not NULL the accelerations
 * G sum_j ... are written there and, when dt_half == 0, v is left unchanged. */
int genga_kick(genga_system_t *sys, double dt_half, int precheck, double *acc_out);

/* ---- kick layout ---------------------------------------------------------- */
#define GENGA_KICK_AUTO       0  /* the symmetric layout where it is predicted faster */
#define GENGA_KICK_TILED      1  /* every ordered pair (i, j): grid of i-tiles x j-chunks */
#define GENGA_KICK_SYMMETRIC  2  /* every unordered pair once, its force to both bodies */

/* Selects how the all-pairs kick (genga_kick and the kicks of genga_step)
 * traverses the pairs.  The symmetric layout applies Newton's third law: it
 * evaluates each unordered pair once, in super-tile pairs of P x P tiles of
 * 128 bodies taken by persistent blocks, and writes one compensated partial
 * sum per body and super-range, folded in a fixed order (deterministic).
 * P = 0 lets the library choose P in 1..6 for N (by a schedule of the work
 * items over the resident blocks); 1..6 fixes it.  With test particles
 * (tp_mode 2, n_massive < n) the symmetric layout leaves out the work items
 * made of test particles only and masks the pairs of two test particles.  The
 * layouts give the same sums up to the rounding of a different summation
 * order.  Errors: EINVAL.                                                    */
int genga_set_kick_layout(genga_system_t *sys, int32_t layout, int32_t P);

/* The layout of the next kick: *layout (GENGA_KICK_TILED or
 * GENGA_KICK_SYMMETRIC), *P (0 for tiled), *slots partial sums per body and
 * *blocks blocks launched.  Any pointer may be NULL.  May allocate.         */
int genga_get_kick_layout(genga_system_t *sys, int32_t *layout, int32_t *P, int32_t *slots,
                          int32_t *blocks);

/* ---- derivative form of the batched Bulirsch-Stoer (Sec. 6.1, groups of
 * more than 32 members) ------------------------------------------------------ */
#define GENGA_BS_PAIRS_AUTO  0  /* pair-centric where a sub-step phase takes several passes */
#define GENGA_BS_PAIRS_OFF   1  /* every member evaluates its partner terms */
#define GENGA_BS_PAIRS_ON    2  /* every pair once per column, its terms to both members */

/* Selects how the persistent Bulirsch-Stoer kernel forms the group ODE's
 * derivative (forward integration without collisions; the adjoint and the
 * collision variant always take the member form).  The pair form evaluates
 * each partner pair once per extrapolation column and writes its two terms
 * into the two partner-list entries, which the members then sum with the
 * member form's lanes and order: the results are bit-identical in every mode,
 * only the time differs.  Errors: EINVAL.                                    */
int genga_set_bs_pair_mode(genga_system_t *sys, int32_t mode);

/* Eq. Hc (Appendix A "HC(dt/2)"): x_i += dt_half * (sum_j m_j v_j) / m_star,
 * the momentum summed in a fixed order.                                     */
int genga_hc(genga_system_t *sys, double dt_half);

/* Eq. Ha Kepler part (Appendix A "FG(dt)"): saves the pre-drift state, then
 * drifts every body on its Kepler orbit about mu = G m_star for dt
 * (universal variables, Stumpff functions by series and argument quartering). */
int genga_drift(genga_system_t *sys, double dt);

/* Appendix A "close-encounter detection" and "grouping" at level 0: keeps the
 * candidates of the last pre-check whose distance before (saved pre-drift
 * state) or after (current state) the drift is below rc_ij, then forms the
 * connected components of these pairs (group label = smallest member index).
 * Synchronises; any output pointer may be NULL.                             */
int genga_build_encounters(genga_system_t *sys, int64_t *n_pairs, int64_t *n_groups,
                           int64_t *max_group);

/* Appendix A "Bulirsch-Stoer(dt)": restores every member of the level-0 groups
 * from the pre-drift state and integrates each group over dt (Sec. 6.1) with
 * the pair forces scaled by 1 - K.  Synchronises.                           */
int genga_bs(genga_system_t *sys, double dt);

/* nsteps full steps of Appendix A (SEnc recursion when slevels > 1): Rcrit,
 * Kick + pre-check, HC, FG, detection, grouping, BS or SEnc, HC, Kick.
 * Synchronises at the end; stats of these steps via genga_get_stats.        */
int genga_step(genga_system_t *sys, int64_t nsteps);

/* Self-tuning of the level scheme (Sec. 6.3: the best number of symplectic
 * levels and sub-steps depends on N and the GPU, so the paper recommends
 * trying configurations before a long run): from the current state, each
 * candidate (slevels[c], substeps[c]), c < ncand, takes one untimed step and
 * then trial_steps timed steps (CUDA events on the system's stream), the state
 * being restored bit for bit before each; the fastest candidate becomes the
 * system's setting.  On return the positions, velocities and stats are those
 * of before the call, so later steps are exactly those of a system created
 * with the chosen setting.  best_out (may be NULL) receives the chosen index,
 * ms_out (may be NULL, ncand doubles) each candidate's time per step.
 * Synchronises.  Errors: EINVAL (bad candidate or counts; nothing run), and
 * any error of a trial step (the state and the previous setting restored).  */
int genga_tune_levels(genga_system_t *sys, const int32_t *slevels, const int32_t *substeps,
                      int32_t ncand, int64_t trial_steps, int32_t *best_out, double *ms_out);

/* genga_step from host buffers: copies pos_host/vel_host (3n doubles each,
 * same layout, ideally pinned) to the device arrays, runs nsteps, copies the
 * result back.  Synchronises.                                               */
int genga_step_host(genga_system_t *sys, double *pos_host, double *vel_host, int64_t nsteps);

/* Total energy (Eq. H with the K terms summing to the full pair potential)
 * and angular momentum sum_i m_i x_i x v_i, FP64 with compensated sums.
 * E and L are host pointers (1 and 3 doubles).  Synchronises.               */
int genga_energy(genga_system_t *sys, double *E, double *L);

/* Host copies, sorted ascending by (i, j), of the last pre-check candidates
 * or of the encounter pairs found at `level` (0 = from genga_build_encounters
 * or the last step's first detection).  ij receives up to cap pairs as
 * interleaved uint32 (i, j); *n the total count.  Synchronises.             */
int genga_get_candidates(genga_system_t *sys, uint32_t *ij, int64_t cap, int64_t *n);
int genga_get_pairs(genga_system_t *sys, int level, uint32_t *ij, int64_t cap, int64_t *n);

/* Host copy of the level-0 group label of every body (smallest member index,
 * -1 for bodies in no encounter), n int64 values.  Synchronises.            */
int genga_get_groups(genga_system_t *sys, int64_t *label);

/* Host copy of the level-`level` critical radii (n doubles).  Synchronises. */
int genga_get_rcrit(genga_system_t *sys, int level, double *rc_host);

/* Replaces the saved pre-drift state (3n doubles each, host, SoA) that
 * genga_build_encounters and genga_bs read (a test hook).  Synchronises.    */
int genga_set_predrift(genga_system_t *sys, const double *pos_host, const double *vel_host);

/* Counters of the last genga_step (or of the last build_encounters / bs).   */
int genga_get_stats(genga_system_t *sys, genga_stats_t *st);

/* ---- collisions (Sec. 7.1-7.2) -------------------------------------------- */
/* Switches collision handling on.  Collisions are found inside the
 * Bulirsch-Stoer integration of the close-encounter groups, at the end of
 * every accepted step, over the group's encounter pairs whose bodies are both
 * alive: bodies i and j collide when r_ij < R_i + R_j.  With a collision
 * precision p > 0 (Sec. 7.2, in units of the radius sum) a step that ends with
 * an overlap (R_i + R_j - r_ij)/(R_i + R_j) >= p is rejected and halved, so a
 * merger happens at an overlap below p; p = 0 merges at the first overlapping
 * step.  Pairs overlapping when a group's integration starts merge at once;
 * overlapping pairs merge in ascending (i, j) order, each seeing the mergers
 * before it.  A merger is perfectly inelastic (Sec. 7.1): the survivor is the
 * more massive body (equal masses: the lower index), it takes the
 * mass-weighted position and velocity, the summed mass and R^3, and the spin
 * S_i + S_j + mu (r_ij x v_ij) (mu = m_i m_j / (m_i + m_j)); the collision
 * energy U grows by mu |v_ij|^2 / 2 - G m_i m_j / r_ij.  The other body keeps its
 * position and velocity with mass, radius and spin 0 and is no longer alive:
 * it exerts no force, inside a group it feels only the star, and it never
 * collides again (genga_remove_merged takes such bodies out).
 *   mass    the system's mass array (the same pointer as at creation), now
 *           written by mergers;
 *   radius  n radii (device, caller-owned, written by mergers);
 *   spin    3n spin vectors, component-major like pos (device, caller-owned,
 *           written by mergers; may hold zeros).
 * All bodies start alive.  Errors: EINVAL (mass is not the system's, NULL
 * radius or spin, p < 0), ENOMEM.                                            */
int genga_set_collisions(genga_system_t *sys, double *mass, double *radius, double *spin,
                         double precision);

/* The mergers since the previous call (or since genga_set_collisions), in the
 * order of the integration (Bulirsch-Stoer calls in time order; within one
 * call, groups by ascending smallest member, each group's mergers in time
 * order), 6 doubles each: time within its Bulirsch-Stoer call, i, j, r_ij,
 * R_i + R_j, Delta U.  log (host, 6 cap doubles) may be NULL; *n (may be NULL)
 * receives the count, *dU (may be NULL) the sum of their Delta U, added in that
 * order.  When log is not NULL the records are copied and the device log is
 * cleared; with log NULL the call only reports (a size query).
 * Synchronises.  Errors: EINVAL, ECAPACITY (cap too small: nothing copied or
 * cleared, *n set).                                                         */
int genga_get_mergers(genga_system_t *sys, double *log, int64_t cap, int64_t *n, double *dU);

/* Host copy of the alive flags (n bytes, 1 alive, 0 merged away).  Synchronises. */
int genga_get_alive(genga_system_t *sys, uint8_t *alive);

/* Takes the merged-away bodies out: pos, vel, mass, radius and spin are
 * compacted in place on the device (alive bodies keep their order) and the
 * system's body count becomes the number of alive bodies, *n_new.  old_index
 * (host, may be NULL, n_new int64 values) receives each new body's former
 * index.  The critical radii and encounter lists are recomputed by the next
 * step.  Synchronises.  Errors: EINVAL (collisions not on).                 */
int genga_remove_merged(genga_system_t *sys, int64_t *n_new, int64_t *old_index);

/* ---- bounded device waits ------------------------------------------------ */
/* Every wait and loop on the device is bounded, so that a stuck integration
 * returns an error instead of holding the GPU.  Two of the bounds are wall
 * clock limits:
 *   bs_group_seconds  one group's in-block Bulirsch-Stoer integration over a
 *                     (sub-)step (groups of up to 32 members); default 10 s;
 *   barrier_seconds   one grid-barrier wait of the persistent Bulirsch-Stoer
 *                     kernel (groups of more than 32 members); default 2 s.
 * A negative value restores the default; 0 makes the first check run out.
 * When a limit is reached the call returns GENGA_ETIMEOUT with a message, the
 * integration of that step stops (the state is left partly advanced), and
 * the system stays usable.  barrier_absent_blocks is a test hook: with n > 0
 * every grid barrier waits for n blocks that do not exist, so every wait
 * runs out after barrier_seconds (0 in normal use).  Errors: EINVAL.        */
int genga_set_wait_limits(genga_system_t *sys, double bs_group_seconds, double barrier_seconds,
                          int32_t barrier_absent_blocks);

/* ---- detection log (verification) --------------------------------------- */
/* With the log on, every close-encounter detection of genga_step and
 * genga_build_encounters (Appendix A "close-encounter detection": level 0
 * once per step, level l >= 1 once per sub-step) appends its level and its
 * encounter pairs, sorted ascending by (i, j), to a host-side log -- for
 * comparing the pair lists of whole steps with another implementation.
 * Logging copies each list to the host and synchronises; it does not change
 * the integration.  genga_set_pair_log clears the log.                      */
int genga_set_pair_log(genga_system_t *sys, int enable);

/* Copies the log: level (max_events int32), off (max_events + 1 int64: the
 * pairs of event k are ij[2 off[k]] .. ij[2 off[k+1] - 1]) and ij (max_pairs
 * interleaved uint32 pairs); *n_events and *n_pairs (may be NULL) receive the
 * sizes.  NULL buffers: sizes only.  Errors: EINVAL, ECAPACITY (buffers too
 * small; sizes still set).                                                  */
int genga_get_pair_log(genga_system_t *sys, int32_t *level, int64_t *off, uint32_t *ij,
                       int64_t max_events, int64_t max_pairs, int64_t *n_events, int64_t *n_pairs);

/* ---- phase timing ------------------------------------------------------ */
/* Where a step's time goes, by the phases of Appendix A.  With timing on,
 * genga_step records a CUDA event on the system's stream at every phase
 * boundary and, after each step, adds the device time between consecutive
 * boundaries to that phase's sum.  An interval includes any time the GPU
 * waited for the host inside it (a count read, the next launch), so the
 * phase sums add up to the step's device time.  The Bulirsch-Stoer kernels on
 * the library's side streams are inside the interval that joins them.
 * Phases of the higher levels (SEnc) are summed over levels and sub-steps;
 * with one level, grouping and Bulirsch-Stoer of level 0 go to the same
 * phases.  Timing synchronises once per step.                               */
#define GENGA_NPHASES 18
#define GENGA_PH_RCRIT        0   /* Rcrit(dt) at level 0 */
#define GENGA_PH_KICK1        1   /* pre-check + first Kick(dt/2) */
#define GENGA_PH_CANDCOUNT    2   /* candidate count (list regrown on overflow) */
#define GENGA_PH_HC_DRIFT     3   /* HC(dt/2) + FG(dt) */
#define GENGA_PH_DETECT0      4   /* level-0 detection + its count */
#define GENGA_PH_CSR0         5   /* level-0 partner lists */
#define GENGA_PH_LEVELSETUP   6   /* groupS: level bodies + restore from pre-drift state */
#define GENGA_PH_RCRITS       7   /* RcritS(dt_l) */
#define GENGA_PH_KICKS        8   /* KickS(dt_l/2), both halves */
#define GENGA_PH_FGS          9   /* FGS(dt_l) */
#define GENGA_PH_DETECTS     10   /* level-l detection + its count */
#define GENGA_PH_CSRS        11   /* level-l partner lists */
#define GENGA_PH_GROUPING    12   /* connected components */
#define GENGA_PH_BUCKETS     13   /* group size buckets + their counts */
#define GENGA_PH_BS_SMALL    14   /* in-block Bulirsch-Stoer (groups <= 32) */
#define GENGA_PH_BS_LARGE    15   /* persistent Bulirsch-Stoer (groups > 32) */
#define GENGA_PH_HC2         16   /* second HC(dt/2) */
#define GENGA_PH_KICK2       17   /* second Kick(dt/2) */

/* Switches phase timing on (enable != 0) or off; either way the sums are
 * cleared.  Errors: EINVAL, ECUDA.                                          */
int genga_set_timing(genga_system_t *sys, int enable);

/* ms (host, GENGA_NPHASES doubles) receives each phase's device time summed
 * over the steps timed since timing was switched on, *nsteps (may be NULL)
 * the number of those steps.                                               */
int genga_get_phase_ms(genga_system_t *sys, double *ms, int64_t *nsteps);

/* Short name of a phase ("kick1", "bs_small", ...); NULL outside [0, GENGA_NPHASES). */
const char *genga_phase_name(int phase);

/* ---- adjoint of kick-drift-kick steps with frozen encounters ------------ */
/* Reverse-mode derivative of nsteps steps of the original scheme (Appendix A,
 * slevels = 1) with every step's level-0 critical radii and encounter pairs
 * frozen to those of a recorded forward run (no derivative through rc).  The
 * kick and Bulirsch-Stoer force derivatives include dK/dr of the changeover
 * function; the Kepler drift uses its exact state-transition matrix; each
 * encounter group's Bulirsch-Stoer step is differentiated through its
 * continuous adjoint, integrated backwards by the same scheme.  Checkpoints
 * of the state every `checkpoint_every` steps bound the memory; the backward
 * pass recomputes each segment from its checkpoint.                          */

/* Records a forward run: saves the current state as the initial state, runs
 * nsteps normal steps (leaving the final state in pos/vel) and keeps each
 * step's rc and pairs and a checkpoint every checkpoint_every steps.
 * genga_get_stats then reports the whole run (sums; maxima for max_group and
 * bs_max_attempts).  Errors: EINVAL (slevels != 1 or tp_mode != 0), the errors
 * of genga_step.                                                             */
int genga_adjoint_forward(genga_system_t *sys, int64_t nsteps, int64_t checkpoint_every);

/* Uses a recording made elsewhere: rc_hist (host, nsteps x n doubles, step
 * major), pair_offsets (host, nsteps + 1) and pairs (host, interleaved uint32
 * i < j, step k's pairs at pair_offsets[k] .. pair_offsets[k+1]-1).  The
 * current state is the initial state; the steps are replayed with the frozen
 * rc and pairs, leaving the final state in pos/vel.  Synchronises.  Errors:
 * EINVAL (as genga_adjoint_forward).                                        */
int genga_adjoint_load(genga_system_t *sys, int64_t nsteps, int64_t checkpoint_every,
                       const double *rc_hist, const int64_t *pair_offsets, const uint32_t *pairs);

/* Given lam_x, lam_v (device, 3n each: dL/d final positions and velocities)
 * writes grad_x0, grad_v0 (device, 3n: dL/d initial state) and grad_m
 * (device, n: dL/d masses).  pos/vel are used as work space and hold the
 * final state again on return.  Synchronises.                              */
int genga_adjoint_backward(genga_system_t *sys, const double *lam_x, const double *lam_v,
                           double *grad_x0, double *grad_v0, double *grad_m);
/* The same call under the boundary's name for the backward step.           */
int genga_step_backward(genga_system_t *sys, const double *lam_x, const double *lam_v,
                        double *grad_x0, double *grad_v0, double *grad_m);

/* Host copies of the current recording: rc_hist (nsteps x n doubles),
 * pair_offsets (nsteps + 1), pairs (up to cap interleaved uint32 pairs, in
 * each step's detection order); any output may be NULL.  Synchronises.      */
int genga_adjoint_export(genga_system_t *sys, double *rc_hist, int64_t *pair_offsets,
                         uint32_t *pairs, int64_t cap, int64_t *n_steps, int64_t *n_pairs);

/* ---- batched ensemble (multi-simulation mode) --------------------------- */
/* Many independent small systems integrated together by the original hybrid
 * method (Appendix A, slevels = 1) with the post-Newtonian GR acceleration of
 * Sec. 3 (Eq. apn) and the constant-time-lag tidal force and spin evolution of
 * Sec. 4.1-4.2, both applied after each half kick by the implicit midpoint
 * rule of Sec. 2.3 on heliocentric velocities.  All arrays are device memory
 * owned by the caller, concatenated over systems (system s = bodies
 * offsets[s] .. offsets[s+1]-1), vectors component-major over all bodies.     */
#define GENGA_ENSEMBLE_MAX_N 64
typedef struct genga_ensemble_desc {
    int64_t n_systems;
    const int64_t *offsets;   /* host, n_systems + 1; each system 1..GENGA_ENSEMBLE_MAX_N bodies */
    double *pos, *vel;        /* 3 x n_total each (heliocentric x, barycentric v per system) */
    const double *mass;       /* n_total */
    double *spin;             /* 3 x n_total planet spin vectors (rad / time unit), updated */
    const double *radius, *k2, *tau, *rg2;  /* n_total: radius, Love number k2, time lag, I/(m R^2) */
    const double *m_star, *dt;              /* n_systems: central mass, time step */
    double *star;             /* 8 x n_systems, per system: R, k2, tau, rg2, spin x, y, z, unused;
                                 the spin is updated */
    double c_light;           /* speed of light in the caller's units */
    int32_t gr;               /* 0 off; GENGA_GR_IMPLICIT: Eq. apn by the implicit midpoint rule
                                 (Sec. 3); GENGA_GR_SPLIT: the Hamiltonian splitting of Sec. 3.1
                                 (sun kick with the kick, gamma term with HC, drift time of each
                                 body scaled by 1 - 3 mu / (2 a c^2), the same factor on the star
                                 term inside Bulirsch-Stoer; pseudovelocities between the
                                 conversions around them, real velocities outside) */
    int32_t tides;            /* switch (Sec. 4.1-4.2) */
} genga_ensemble_desc_t;
#define GENGA_GR_IMPLICIT 1
#define GENGA_GR_SPLIT    2
typedef struct genga_ensemble genga_ensemble_t;

/* Creates the ensemble on `stream` (cudaStream_t).  params supplies G, n1, n2,
 * f_pc, bs_tol and the iteration limits (slevels must be 1).  Errors: EINVAL
 * (bad sizes or pointers), ENOMEM, ECUDA.                                    */
int genga_ensemble_create(genga_ensemble_t **out, const genga_params_t *params,
                          const genga_ensemble_desc_t *desc, void *stream);
/* The same call under the boundary's name (genga_init_ensemble).            */
int genga_init_ensemble(genga_ensemble_t **out, const genga_params_t *params,
                        const genga_ensemble_desc_t *desc, void *stream);
void genga_ensemble_destroy(genga_ensemble_t *ens);
const char *genga_ensemble_last_error(const genga_ensemble_t *ens);

/* Advances every system by nsteps of its own dt in one persistent launch
 * (captured in a CUDA graph on first use for each nsteps and tile shape, then
 * replayed).  Synchronises; counters via genga_ensemble_get_stats.          */
int genga_ensemble_step(genga_ensemble_t *ens, int64_t nsteps);
/* The same call under the boundary's name (genga_step_ensemble).            */
int genga_step_ensemble(genga_ensemble_t *ens, int64_t nsteps);

/* Tile shape: threads per CTA (32 only when every system has <= 32 bodies, 64
 * or 128) and resident CTAs per SM (1..8).                                   */
int genga_ensemble_set_tile(genga_ensemble_t *ens, int threads, int ctas_per_sm);

/* Self-tuning (Sec. 8.3's kernel-parameter search): times trial_steps with
 * each tile shape from the same saved state, restores the state and keeps the
 * fastest.  threads_out / ctas_out (may be NULL) receive the choice.         */
int genga_ensemble_autotune(genga_ensemble_t *ens, int64_t trial_steps, int *threads_out,
                            int *ctas_out);

/* Per-system total angular momentum (orbit + planet spins + star spin), 3
 * doubles per system into the host array L.  Synchronises.                  */
int genga_ensemble_angmom(genga_ensemble_t *ens, double *L);
int genga_ensemble_get_stats(genga_ensemble_t *ens, genga_stats_t *st);

/* ---- allocation-free kick ---------------------------------------------- */
/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: a caller whose framework's caching allocator
 * already holds the device's free memory (a cudaMalloc would fail or fragment
 * that pool), or one on a latency-critical loop where cudaMalloc/cudaFree
 * would stall every stream of the device.  It performs the same kick as
 * genga_kick without the pre-check, on arrays the caller passes (device
 * pointers, layout as in genga_create): pos (3n), mass (n), rc (n critical
 * radii), vel (3n, updated by dt_half * a when dt_half != 0), acc_out (3n or
 * NULL; receives the accelerations).  It calls no cudaMalloc/cudaFree: its
 * scratch is one fixed device array of 16 MiB inside the library, held by
 * every GPU that loads the library until the process exits.  n may be at most
 * GENGA_KICK_STATIC_MAX_N (larger n returns GENGA_ECAPACITY before any launch).
 * The first call on a device looks up that array's device address (with that
 * device current); make that first call before any stream capture.  After a
 * cudaDeviceReset the next call looks the address up again (the device's new
 * context loads the library's device code anew), so that call too should
 * come before any capture.  All calls
 * share the array and it keeps the last call's contents (every call rewrites
 * what it reads); calls that overlap on the GPU race with each other -- issue
 * them on one stream or synchronise between them.  Returns GENGA_OK, EINVAL,
 * ECAPACITY or ECUDA.  Enqueued on `stream` (a cudaStream_t, NULL = default). */
#define GENGA_KICK_STATIC_MAX_N 279616
int genga_kick_static(int64_t n, const double *pos, const double *mass, const double *rc,
                      double G, double dt_half, int precision, double *vel, double *acc_out,
                      void *stream);

/* ---- pipe-rate probe ---------------------------------------------------- */
/* The paper has no counterpart: a measurement utility for the roofline of the
 * kernels above.  On the current device, runs one block of 1024 threads per
 * SM issuing independent chains of FP64 FMA, add and multiply, FP32 FMA and
 * MUFU reciprocal square root, and reports the thread-level operations per
 * clock per SM of each (cycle counts of the SMs themselves, so independent of
 * the clock frequency); multiply by the SM count and the SM clock for a peak
 * rate.  Any output may be NULL.  Allocates and frees a few KB, synchronises,
 * takes about 50 ms.  Errors: ECUDA, ENOMEM.                                */
int genga_measure_pipe_rates(double *dfma_per_clk_sm, double *dadd_per_clk_sm,
                             double *dmul_per_clk_sm, double *ffma_per_clk_sm,
                             double *rsqrt_per_clk_sm);

/* Latency of dependent FP64 arithmetic: one block alone on the device runs a
 * chain of dependent FP64 FMAs, as a full warp (*warp_cycles) and as a single
 * thread (*lane_cycles); each is the SM cycles per instruction of the chain --
 * the time an instruction on the critical path of a latency-bound kernel (a
 * Bulirsch-Stoer group integrated alone) costs.  Any output may be NULL.
 * Synchronises, a few ms.  Errors: ECUDA, ENOMEM.                           */
int genga_measure_fp64_latency(double *warp_cycles, double *lane_cycles);

#ifdef __cplusplus
}
#endif
#endif /* GENGA_H */
