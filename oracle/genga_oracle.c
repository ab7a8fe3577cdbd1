/*
 * genga_oracle.c -- plain, slow, FP64 CPU oracle of the hybrid symplectic step of
 * GENGA II (Grimm et al., arXiv:2201.10058).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Compile with -O2 -ffp-contract=off so that every a*b+c below is rounded twice,
 * exactly as written.  All arithmetic is IEEE binary64 unless a comment says
 * otherwise (energy uses long double with Kahan summation).
 *
 * Coordinates: democratic heliocentric (Sec. 2, Eq. H): positions x_i are
 * heliocentric, velocities v_i barycentric.  Arrays are row-major (n,3).
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *  R1  Hill radius in Eq. rcrit: R_H,i = |x_i| (m_i/(3 m_star))^(1/3).
 *  R2  v_i in Eq. rcrit is the stored (barycentric) speed.
 *  R3  Pair critical radius rc_ij = max(rc_i, rc_j).
 *  R4  Changeover function K (Sec. 6.3, footnote on Chambers 1999 Eq. 10):
 *      y = (r/rc - 0.1)/0.9 clamped to [0,1], K = y^2 / (2y^2 - 2y + 1).
 *  R5  Force scaling: the kick applies K times the Newtonian pair force and the
 *      close-encounter part applies (1-K) times it (no dK/dr term).
 *  R6  Pre-check (Appendix A): candidate pairs i<j with r_ij^2 < (f_pc rc_ij)^2,
 *      evaluated on the positions of the first half kick.
 *  R7  Detection (Appendix A): a candidate is an encounter when its distance
 *      before or after the drift is below rc_ij (r^2 < rc_ij^2).
 *  R8  Grouping: connected components of the encounter pairs; group label is the
 *      smallest member index; members ascending (Serial Grouping, App. B).
 *  R9  Bulirsch-Stoer: modified midpoint with n = 2,4,...,16, polynomial
 *      extrapolation in h^2; pair forces summed over the group's encounter pairs
 *      (the partner lists of the BS-A kernel, Sec. 6.1); step halving on failure.
 *  R10 Higher levels (Sec. 6.3, Appendix A): level bodies restart from the
 *      pre-drift state of the enclosing level; level-l kicks use the factor
 *      prod_{k<l}(1-K_k) K_l over the enclosing level's encounter pairs; BS uses
 *      prod_{k<=l}(1-K_k).
 *  R11 Kepler drift with mu = G m_star (Eq. Ha), universal variables with
 *      Stumpff functions evaluated by series and argument quartering.
 *  R24 Semi-active test particles (Sec. 8.1, TP 2): the bodies are ordered
 *      with the large ones first; bodies i >= n_massive are test particles,
 *      and a pair of two test particles has no interaction at all (no force,
 *      no candidate, no encounter, no potential term); every other pair is
 *      treated as in the fully interactive mode.
 *  R25 Collisions (Sec. 7.1-7.2): checked at the end of every accepted
 *      Bulirsch-Stoer step over the group's encounter pairs whose bodies are
 *      both alive, r_ij < R_i + R_j; with a collision precision tol > 0 a step
 *      that ends with an overlap (R_i + R_j - r_ij)/(R_i + R_j) >= tol is
 *      rejected and halved, so a merger happens at an overlap below tol; pairs
 *      overlapping when a group's integration starts merge at once; overlapping
 *      pairs merge in ascending pair order.  A merger follows Sec. 7.1: the
 *      survivor is the more massive body (equal masses: the lower index),
 *      position and velocity are mass-weighted, m and R^3 add, the spin is
 *      S_i + S_j + mu (r_ij x v_ij), U grows by mu v_ij^2/2 - G m_i m_j/r_ij;
 *      the other body keeps its position and velocity with m = R = S = 0 and
 *      is no longer alive: it exerts no force, feels only the star inside a
 *      group integration, and never collides again.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Parameters of one integration (own definition; not shared with the GPU).  */
typedef struct orc_params {
    double G;          /* gravitational constant */
    double m_star;     /* central mass */
    double dt;         /* base time step */
    double n1, n2;     /* Eq. rcrit constants */
    double f_pc;       /* pre-check factor (R6) */
    double bs_tol;     /* Bulirsch-Stoer relative tolerance */
    int32_t slevels;   /* number of symplectic levels (1 = original method) */
    int32_t substeps;  /* sub-steps per level */
    int32_t kepler_max_iter;
    int32_t bs_max_steps; /* limit on BS sub-step attempts per group call */
    int32_t nthreads;  /* OpenMP threads for the O(N^2) loops (1 = serial) */
    int32_t tp_mode;   /* Sec. 8.1: 0 fully interactive; 2 semi-active test particles */
    int64_t n_massive; /* tp_mode 2: bodies i >= n_massive are test particles */
} orc_params;

/* Statistics of the last step (for tests and reports). */
typedef struct orc_stats {
    int64_t n_candidates;
    int64_t n_pairs[8];      /* encounter pairs found at each level (summed over sub-steps) */
    int64_t n_groups;        /* BS groups integrated */
    int64_t max_group;       /* largest BS group */
    int64_t bs_steps;        /* accepted BS sub-steps */
    int64_t bs_rejects;      /* rejected BS attempts (step halvings) */
    int64_t kepler_fail;     /* Kepler solves that hit the iteration limit */
    int64_t bs_fail;         /* groups that hit bs_max_steps */
    int64_t bs_max_attempts; /* most step attempts any one group needed */
} orc_stats;

#define ORC_MAX_LEVELS 8

/* ------------------------------------------------------------------------- */
/* R4: the changeover function of Chambers (1999), Eq. 10, as read here.      */
double orc_changeover(double r, double rc)
{
    double y = (r / rc - 0.1) / 0.9;
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    double y2 = y * y;
    return y2 / (2.0 * y2 - 2.0 * y + 1.0);
}

/* ------------------------------------------------------------------------- */
/* Eq. rcrit with readings R1, R2: rc_i = max(n1 R_H,i, n2 dt |v_i|).         */
void orc_rcrit(int64_t n, const double *x, const double *v, const double *m,
               double m_star, double dt, double n1, double n2, double *rc)
{
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i, *vi = v + 3 * i;
        double r = sqrt((xi[0] * xi[0] + xi[1] * xi[1]) + xi[2] * xi[2]);
        double vabs = sqrt((vi[0] * vi[0] + vi[1] * vi[1]) + vi[2] * vi[2]);
        double hill = r * cbrt(m[i] / (3.0 * m_star));
        double a = n1 * hill;
        double b = n2 * dt * vabs;
        rc[i] = a > b ? a : b;
    }
}

/* R3 */
static double pair_rc(const double *rc, int64_t i, int64_t j)
{
    return rc[i] > rc[j] ? rc[i] : rc[j];
}

/* Squared distance in the prescribed order (dx^2 + dy^2) + dz^2, dx = x_j - x_i. */
static double dist2(const double *xi, const double *xj)
{
    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* ------------------------------------------------------------------------- */
/* Eq. Hb kick acceleration of particle i:
 *   a_i = G sum_{j != i} m_j K(r_ij) (x_j - x_i) / r_ij^3, j ascending;
 * with test particles (R24) a test particle i takes only j < nm.             */
static void accel_one(int64_t n, int64_t nm, const double *x, const double *m, const double *rc,
                      double G, int64_t i, double *ai)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const double *xi = x + 3 * i;
    const int64_t jend = i >= nm ? nm : n;
    for (int64_t j = 0; j < jend; j++) {
        if (j == i) continue;
        const double *xj = x + 3 * j;
        double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
        double r2 = (dx * dx + dy * dy) + dz * dz;
        double r = sqrt(r2);
        double K = orc_changeover(r, pair_rc(rc, i, j));
        double f = m[j] * K / (r2 * r);
        s0 += f * dx;
        s1 += f * dy;
        s2 += f * dz;
    }
    ai[0] = G * s0;
    ai[1] = G * s1;
    ai[2] = G * s2;
}

/* nm = n: fully interactive; nm < n: bodies i >= nm are test particles (R24). */
void orc_accel_tp(int64_t n, int64_t nm, const double *x, const double *m, const double *rc,
                  double G, double *acc, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t i = 0; i < n; i++) accel_one(n, nm, x, m, rc, G, i, acc + 3 * i);
}

void orc_accel(int64_t n, const double *x, const double *m, const double *rc,
               double G, double *acc, int nthreads)
{
    orc_accel_tp(n, n, x, m, rc, G, acc, nthreads);
}

/* Acceleration of a subset of rows (for sampled checks at large N). */
void orc_accel_rows(int64_t n, const double *x, const double *m, const double *rc,
                    double G, const int64_t *rows, int64_t nrows, double *acc, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t k = 0; k < nrows; k++) accel_one(n, n, x, m, rc, G, rows[k], acc + 3 * k);
}

/* Kick(dt/2): v_i += dt_half a_i. */
static void kick_tp(int64_t n, int64_t nm, const double *x, const double *m, const double *rc,
                    double G, double dt_half, double *v, int nthreads)
{
    double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_accel_tp(n, nm, x, m, rc, G, acc, nthreads);
    for (int64_t i = 0; i < 3 * n; i++) v[i] += dt_half * acc[i];
    free(acc);
}

void orc_kick(int64_t n, const double *x, const double *m, const double *rc,
              double G, double dt_half, double *v, int nthreads)
{
    kick_tp(n, n, x, m, rc, G, dt_half, v, nthreads);
}

/* R6 pre-check: candidates i<j with r_ij^2 < (f_pc rc_ij)^2, ascending (i,j).
 * Returns the number of candidates; writes at most cap of them.             */
int64_t orc_precheck_tp(int64_t n, int64_t nm, const double *x, const double *rc, double f_pc,
                        uint32_t *cand, int64_t cap)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        const int64_t jend = i >= nm ? i + 1 : n;   /* no pair of two test particles (R24) */
        for (int64_t j = i + 1; j < jend; j++) {
            double t = f_pc * pair_rc(rc, i, j);
            if (dist2(x + 3 * i, x + 3 * j) < t * t) {
                if (c < cap) { cand[2 * c] = (uint32_t)i; cand[2 * c + 1] = (uint32_t)j; }
                c++;
            }
        }
    }
    return c;
}

int64_t orc_precheck(int64_t n, const double *x, const double *rc, double f_pc,
                     uint32_t *cand, int64_t cap)
{
    return orc_precheck_tp(n, n, x, rc, f_pc, cand, cap);
}

/* ------------------------------------------------------------------------- */
/* Eq. Hc: x_i += dt_half P / m_star, P = sum_j m_j v_j (j ascending).         */
void orc_hc(int64_t n, double *x, const double *v, const double *m, double m_star,
            double dt_half)
{
    double P[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; j++)
        for (int k = 0; k < 3; k++) P[k] += m[j] * v[3 * j + k];
    double c[3];
    for (int k = 0; k < 3; k++) c[k] = dt_half * P[k] / m_star;
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) x[3 * i + k] += c[k];
}

/* ------------------------------------------------------------------------- */
/* Kepler drift (Eq. Ha, Kepler term), universal variables.
 * Stumpff functions c_k(z) = sum_{m>=0} (-z)^m / (2m+k)!; for |z| large the
 * argument is quartered until small, the series is used, and the quadrupling
 * relations c0(4z)=2c0^2-1, c1(4z)=c0 c1, c2(4z)=c1^2/2, c3(4z)=(c2+c0 c3)/4
 * map back.  With s the universal variable and beta = 2mu/r0 - v0^2:
 *   G_k(s) = s^k c_k(beta s^2),
 *   t(s) = r0 G1 + u G2 + mu G3,    u = x0.v0,
 *   r(s) = r0 G0 + u G1 + mu G2 = dt/ds,
 *   f = 1 - mu G2/r0,  g = t - mu G3,  fdot = -mu G1/(r r0),  gdot = 1 - mu G2/r.  */
static void stumpff(double z, double *c0, double *c1, double *c2, double *c3)
{
    int q = 0;
    while (fabs(z) > 0.1 && q < 60) { z *= 0.25; q++; }
    /* series for c2 and c3 (|z| <= 0.1: 9 terms reach below 1e-20) */
    double s2 = 0.0, s3 = 0.0;
    double fact2[10], fact3[10];
    {   /* 1/(2m+2)! and 1/(2m+3)! for m = 0..9 */
        double f = 1.0; /* running factorial */
        int k = 1;
        for (int mm = 0; mm < 10; mm++) {
            while (k < 2 * mm + 2) { k++; f *= k; }
            fact2[mm] = 1.0 / f;
            k++; f *= k;
            fact3[mm] = 1.0 / f;
        }
    }
    for (int mm = 9; mm >= 0; mm--) {
        s2 = fact2[mm] - z * s2;
        s3 = fact3[mm] - z * s3;
    }
    double C2 = s2, C3 = s3;
    double C0 = 1.0 - z * C2;
    double C1 = 1.0 - z * C3;
    for (int k = 0; k < q; k++) {
        double n3 = 0.25 * (C2 + C0 * C3);
        double n2 = 0.5 * C1 * C1;
        double n1 = C0 * C1;
        double n0 = 2.0 * C0 * C0 - 1.0;
        C0 = n0; C1 = n1; C2 = n2; C3 = n3;
    }
    *c0 = C0; *c1 = C1; *c2 = C2; *c3 = C3;
}

/* Drift one body; returns 0 on success, 1 if Newton hit max_iter. */
static int kepler_one(double *x, double *v, double mu, double dt, int max_iter)
{
    double r0 = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    double u = (x[0] * v[0] + x[1] * v[1]) + x[2] * v[2];
    double beta = 2.0 * mu / r0 - v2;
    /* second-order initial guess of s */
    double s = dt / r0 - (u * dt * dt) / (2.0 * r0 * r0 * r0);
    double c0, c1, c2, c3;
    double ds_prev = 0.0;
    int it, ok = 0;
    /* Newton on t(s) = dt.  Converged when |ds| <= 1e-15 |s|, or when the
     * quadratic phase is over and rounding of t(s) stalls the update at
     * |ds| <= 1e-12 |s| without halving it any more.                        */
    for (it = 0; it < max_iter; it++) {
        double z = beta * s * s;
        stumpff(z, &c0, &c1, &c2, &c3);
        double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
        double G0 = c0;
        double t = r0 * G1 + u * G2 + mu * G3;
        double rr = r0 * G0 + u * G1 + mu * G2;
        double ds = (t - dt) / rr;
        s -= ds;
        double ads = fabs(ds), as = fabs(s);
        if (ads <= 1e-15 * as) { ok = 1; break; }
        if (it > 0 && ads <= 1e-12 * as && ads > 0.5 * ds_prev) { ok = 1; break; }
        ds_prev = ads;
    }
    double z = beta * s * s;
    stumpff(z, &c0, &c1, &c2, &c3);
    double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
    double r = r0 * c0 + u * G1 + mu * G2;
    double fm1 = -mu * G2 / r0;
    double g = dt - mu * G3;
    double fd = -mu * G1 / (r * r0);
    double gdm1 = -mu * G2 / r;
    double x0[3] = {x[0], x[1], x[2]}, v0[3] = {v[0], v[1], v[2]};
    for (int k = 0; k < 3; k++) {
        x[k] = x0[k] + (fm1 * x0[k] + g * v0[k]);
        v[k] = v0[k] + (fd * x0[k] + gdm1 * v0[k]);
    }
    return ok ? 0 : 1;
}

/* FG(dt) for all bodies, or for the listed ones.  Returns the failure count. */
int64_t orc_fg(int64_t n, double *x, double *v, double mu, double dt, int max_iter)
{
    int64_t fails = 0;
    for (int64_t i = 0; i < n; i++) fails += kepler_one(x + 3 * i, v + 3 * i, mu, dt, max_iter);
    return fails;
}

static int64_t fg_list(const int64_t *idx, int64_t nb, double *x, double *v, double mu,
                       double dt, int max_iter)
{
    int64_t fails = 0;
    for (int64_t k = 0; k < nb; k++)
        fails += kepler_one(x + 3 * idx[k], v + 3 * idx[k], mu, dt, max_iter);
    return fails;
}

/* ------------------------------------------------------------------------- */
/* R7 detection: keep candidate (i,j) if r^2 < rc_ij^2 before or after the drift.
 * Output keeps the candidate order (ascending when the input is ascending).  */
int64_t orc_detect(int64_t ncand, const uint32_t *cand, const double *xpre,
                   const double *xpost, const double *rc, uint32_t *pairs)
{
    int64_t c = 0;
    for (int64_t k = 0; k < ncand; k++) {
        int64_t i = cand[2 * k], j = cand[2 * k + 1];
        double rcij = pair_rc(rc, i, j);
        double rc2 = rcij * rcij;
        if (dist2(xpre + 3 * i, xpre + 3 * j) < rc2 || dist2(xpost + 3 * i, xpost + 3 * j) < rc2) {
            pairs[2 * c] = (uint32_t)i;
            pairs[2 * c + 1] = (uint32_t)j;
            c++;
        }
    }
    return c;
}

/* Detection log (verification only: switched on by orc_pair_log, no effect
 * on the integration).  Every detection inside a step appends its level, the
 * encounter pairs it found (in its output order) and the candidates whose
 * separation before or after the drift lies within PAIR_LOG_REL of rc_ij
 * relative -- the pairs whose decision a rounding difference could flip.    */
#define PAIR_LOG_REL 1e-12
static struct {
    int on;
    int64_t nev, npairs, nborder, cap_ev, cap_pairs, cap_border;
    int32_t *level;
    int64_t *off, *boff;     /* nev + 1 each */
    uint32_t *pairs, *border;
} plog;

static void plog_reserve(void **buf, int64_t *cap, int64_t need, size_t elem)
{
    if (need <= *cap) return;
    int64_t c = *cap > 0 ? *cap : 64;
    while (c < need) c *= 2;
    *buf = realloc(*buf, elem * (size_t)c);
    *cap = c;
}

static void plog_near(const double *x, int64_t i, int64_t j, double rcij, int *near)
{
    double r = sqrt(dist2(x + 3 * i, x + 3 * j));
    if (fabs(r / rcij - 1.0) <= PAIR_LOG_REL) *near = 1;
}

static void plog_detection(int level, int64_t ncand, const uint32_t *cand, const double *xpre,
                           const double *xpost, const double *rc, int64_t ne, const uint32_t *enc)
{
    if (!plog.on) return;
    int64_t ev = plog.nev;
    /* level holds cap_ev >= ev + 2 entries; off and boff (one more than the
     * events) are kept at the same length */
    plog_reserve((void **)&plog.level, &plog.cap_ev, ev + 2, sizeof(int32_t));
    plog.off = (int64_t *)realloc(plog.off, sizeof(int64_t) * (size_t)plog.cap_ev);
    plog.boff = (int64_t *)realloc(plog.boff, sizeof(int64_t) * (size_t)plog.cap_ev);
    if (ev == 0) { plog.off[0] = 0; plog.boff[0] = 0; }
    plog.level[ev] = level;
    plog_reserve((void **)&plog.pairs, &plog.cap_pairs, 2 * (plog.npairs + ne), sizeof(uint32_t));
    memcpy(plog.pairs + 2 * plog.npairs, enc, sizeof(uint32_t) * 2 * (size_t)ne);
    plog.npairs += ne;
    for (int64_t k = 0; k < ncand; k++) {
        int64_t i = cand[2 * k], j = cand[2 * k + 1];
        double rcij = pair_rc(rc, i, j);
        int near = 0;
        plog_near(xpre, i, j, rcij, &near);
        plog_near(xpost, i, j, rcij, &near);
        if (!near) continue;
        plog_reserve((void **)&plog.border, &plog.cap_border, 2 * (plog.nborder + 1), sizeof(uint32_t));
        plog.border[2 * plog.nborder] = (uint32_t)i;
        plog.border[2 * plog.nborder + 1] = (uint32_t)j;
        plog.nborder++;
    }
    plog.off[ev + 1] = plog.npairs;
    plog.boff[ev + 1] = plog.nborder;
    plog.nev = ev + 1;
}

/* Switches the detection log on (enable != 0) or off; either way it is cleared. */
void orc_pair_log(int enable)
{
    free(plog.level); free(plog.off); free(plog.boff); free(plog.pairs); free(plog.border);
    memset(&plog, 0, sizeof(plog));
    plog.on = enable != 0;
}

void orc_pair_log_size(int64_t *nev, int64_t *npairs, int64_t *nborder)
{
    *nev = plog.nev; *npairs = plog.npairs; *nborder = plog.nborder;
}

/* level (nev), off and boff (nev + 1), pairs (2 npairs), border (2 nborder). */
void orc_pair_log_get(int32_t *level, int64_t *off, uint32_t *pairs, int64_t *boff, uint32_t *border)
{
    if (plog.nev == 0) { off[0] = 0; boff[0] = 0; return; }
    memcpy(level, plog.level, sizeof(int32_t) * (size_t)plog.nev);
    memcpy(off, plog.off, sizeof(int64_t) * (size_t)(plog.nev + 1));
    memcpy(boff, plog.boff, sizeof(int64_t) * (size_t)(plog.nev + 1));
    memcpy(pairs, plog.pairs, sizeof(uint32_t) * 2 * (size_t)plog.npairs);
    memcpy(border, plog.border, sizeof(uint32_t) * 2 * (size_t)plog.nborder);
}

/* ------------------------------------------------------------------------- */
/* R8 grouping: union-find, label = smallest index in the component; bodies in
 * no pair get label -1.                                                     */
static int64_t uf_find(int64_t *p, int64_t a)
{
    while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
    return a;
}

void orc_group(int64_t n, int64_t npairs, const uint32_t *pairs, int64_t *label)
{
    int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    char *in = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t i = 0; i < n; i++) p[i] = i;
    for (int64_t k = 0; k < npairs; k++) {
        int64_t a = uf_find(p, pairs[2 * k]), b = uf_find(p, pairs[2 * k + 1]);
        in[pairs[2 * k]] = 1; in[pairs[2 * k + 1]] = 1;
        if (a == b) continue;
        if (a < b) p[b] = a; else p[a] = b;
    }
    for (int64_t i = 0; i < n; i++) label[i] = in[i] ? uf_find(p, i) : -1;
    free(p);
    free(in);
}

/* ------------------------------------------------------------------------- */
/* Collisions (R25).                                                          */
typedef struct coll_ctx {
    double *m, *R, *S;        /* masses, physical radii, spins (3 per body), updated by mergers */
    unsigned char *alive;     /* 0 once merged away */
    double tol;               /* collision precision (0: merge at the first overlapping step) */
    double G;
    double U;                 /* energy moved into U by the mergers so far */
    int64_t ncoll;
    double *log;              /* per merger: t, i, j, r_ij, R_i + R_j, Delta U (or NULL) */
    int64_t log_cap;          /* mergers the log can hold */
    double t0;                /* time of the current BS call's start */
} coll_ctx;

/* Sec. 7.1 merger of bodies i and j at positions xi, xj with velocities vi, vj:
 * the merged position and velocity go to xo, vo; m, R and S of the survivor
 * are updated and those of the other body zeroed.  Returns the survivor;
 * *other the removed body, *dU the energy moved into U.                      */
static int64_t merge_core(int64_t i, int64_t j, const double *xi, const double *vi,
                          const double *xj, const double *vj, double *m, double *R, double *S,
                          double G, double *xo, double *vo, int64_t *other, double *dU)
{
    const double mi = m[i], mj = m[j], M = mi + mj;
    double r[3], w[3];
    for (int k = 0; k < 3; k++) { r[k] = xi[k] - xj[k]; w[k] = vi[k] - vj[k]; }
    const double rr = sqrt((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
    const double w2 = (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2];
    double mu = 0.0;
    if (M > 0.0) {
        mu = mi * mj / M;
        for (int k = 0; k < 3; k++) {
            xo[k] = (xi[k] * mi + xj[k] * mj) / M;
            vo[k] = (vi[k] * mi + vj[k] * mj) / M;
        }
    } else {
        for (int k = 0; k < 3; k++) { xo[k] = 0.5 * (xi[k] + xj[k]); vo[k] = 0.5 * (vi[k] + vj[k]); }
    }
    *dU = 0.5 * mu * w2 - (rr > 0.0 ? G * mi * mj / rr : 0.0);
    const double L[3] = {mu * (r[1] * w[2] - r[2] * w[1]), mu * (r[2] * w[0] - r[0] * w[2]),
                         mu * (r[0] * w[1] - r[1] * w[0])};
    const int64_t sv = (mi > mj || (mi == mj && i < j)) ? i : j, ot = sv == i ? j : i;
    const double R3 = R[i] * R[i] * R[i] + R[j] * R[j] * R[j];
    double Sn[3];
    for (int k = 0; k < 3; k++) Sn[k] = S[3 * i + k] + S[3 * j + k] + L[k];
    m[sv] = M;
    R[sv] = cbrt(R3);
    for (int k = 0; k < 3; k++) S[3 * sv + k] = Sn[k];
    m[ot] = 0.0;
    R[ot] = 0.0;
    for (int k = 0; k < 3; k++) S[3 * ot + k] = 0.0;
    *other = ot;
    return sv;
}

/* Merger of bodies i and j of the row-major arrays x, v (n x 3): the survivor
 * takes the merged position and velocity, the other keeps its own.  Returns
 * Delta U; *survivor receives the surviving index.                           */
double orc_merge(int64_t i, int64_t j, double *x, double *v, double *m, double *R, double *S,
                 double G, int64_t *survivor)
{
    double xo[3], vo[3], dU;
    int64_t ot;
    const int64_t sv = merge_core(i, j, x + 3 * i, v + 3 * i, x + 3 * j, v + 3 * j, m, R, S, G,
                                  xo, vo, &ot, &dU);
    for (int k = 0; k < 3; k++) { x[3 * sv + k] = xo[k]; v[3 * sv + k] = vo[k]; }
    if (survivor) *survivor = sv;
    return dU;
}

/* ------------------------------------------------------------------------- */
/* Bulirsch-Stoer integration of one close-encounter group (R9, R10).
 * The group's ODE (Eq. Ha restricted to the group):
 *   dx_i/dt = v_i
 *   dv_i/dt = -mu x_i/|x_i|^3
 *             + G sum_{j in partners(i)} m_j W_ij (x_j - x_i)/r_ij^3,
 *   W_ij = prod_{k=0..L} (1 - K(r_ij; rc_k,ij)).                             */
typedef struct bs_group {
    int64_t nm;            /* members */
    const int64_t *mem;    /* global indices, ascending */
    const int64_t *poff;   /* partner offsets, nm+1 */
    const int64_t *plist;  /* partner local indices, ascending per member */
    const double *m;       /* masses (global) */
    const double *const *rcl; /* rc of levels 0..L (global arrays) */
    int nlev;              /* L+1 */
    double G, mu;
    const unsigned char *alive; /* collisions (R25): bodies merged away feel only the star; or NULL */
    double gr_inv_c2;      /* GR splitting (R28): 1/c^2, or 0 when off */
} bs_group;

static void bs_deriv(const bs_group *g, const double *y, double *f)
{
    /* y[6*k .. 6*k+5] = x, v of member k */
    for (int64_t a = 0; a < g->nm; a++) {
        const double *xa = y + 6 * a;
        double r2 = (xa[0] * xa[0] + xa[1] * xa[1]) + xa[2] * xa[2];
        double r = sqrt(r2);
        double s = -g->mu / (r2 * r);
        double ax = s * xa[0], ay = s * xa[1], az = s * xa[2];
        double px = 0.0, py = 0.0, pz = 0.0;
        int64_t ia = g->mem[a];
        const int64_t q1 = (g->alive && !g->alive[ia]) ? g->poff[a] : g->poff[a + 1];
        for (int64_t q = g->poff[a]; q < q1; q++) {
            int64_t b = g->plist[q];
            int64_t ib = g->mem[b];
            if (g->alive && !g->alive[ib]) continue;   /* merged away: no mass */
            const double *xb = y + 6 * b;
            double dx = xb[0] - xa[0], dy = xb[1] - xa[1], dz = xb[2] - xa[2];
            double d2 = (dx * dx + dy * dy) + dz * dz;
            double d = sqrt(d2);
            double W = 1.0;
            for (int l = 0; l < g->nlev; l++) {
                const double *rc = g->rcl[l];
                double rcij = rc[ia] > rc[ib] ? rc[ia] : rc[ib];
                W *= 1.0 - orc_changeover(d, rcij);
            }
            double c = g->m[ib] * W / (d2 * d);
            px += c * dx; py += c * dy; pz += c * dz;
        }
        /* GR splitting (R28): the alpha term rescales the member's own Kepler
         * motion -- its velocity term and the star's acceleration -- by
         * 1 + 3 (u^2/2 - mu/r) / c^2 at the current state; pair terms are not
         * rescaled (Sec. 3.1) */
        double fac = 1.0;
        if (g->gr_inv_c2 > 0.0) {
            const double u2 = (xa[3] * xa[3] + xa[4] * xa[4]) + xa[5] * xa[5];
            fac = 1.0 + 3.0 * (0.5 * u2 - g->mu / r) * g->gr_inv_c2;
        }
        f[6 * a + 0] = fac * xa[3];
        f[6 * a + 1] = fac * xa[4];
        f[6 * a + 2] = fac * xa[5];
        f[6 * a + 3] = fac * ax + g->G * px;
        f[6 * a + 4] = fac * ay + g->G * py;
        f[6 * a + 5] = fac * az + g->G * pz;
    }
}

/* Modified midpoint over H with nsub steps, starting from y0 with f0 = f(y0). */
static void bs_midpoint(const bs_group *g, const double *y0, const double *f0, double H,
                        int nsub, double *out, double *zm, double *zn, double *fz)
{
    int64_t d = 6 * g->nm;
    double h = H / nsub;
    for (int64_t c = 0; c < d; c++) { zm[c] = y0[c]; zn[c] = y0[c] + h * f0[c]; }
    for (int m = 1; m < nsub; m++) {
        bs_deriv(g, zn, fz);
        for (int64_t c = 0; c < d; c++) {
            double t = zm[c] + 2.0 * h * fz[c];
            zm[c] = zn[c];
            zn[c] = t;
        }
    }
    bs_deriv(g, zn, fz);
    for (int64_t c = 0; c < d; c++) out[c] = 0.5 * (zn[c] + zm[c] + h * fz[c]);
}

#define BS_KMAX 8

/* Deepest overlap (R_i + R_j - r_ij)/(R_i + R_j) over the group's pairs of
 * alive bodies in state y; *any = 1 if some pair overlaps (R25).              */
static double group_overlap(const bs_group *g, const coll_ctx *cc, const double *y, int *any)
{
    double deepest = 0.0;
    *any = 0;
    for (int64_t a = 0; a < g->nm; a++) {
        const int64_t ia = g->mem[a];
        if (!cc->alive[ia]) continue;
        for (int64_t q = g->poff[a]; q < g->poff[a + 1]; q++) {
            const int64_t b = g->plist[q], ib = g->mem[b];
            if (b <= a || !cc->alive[ib]) continue;
            const double dx = y[6 * b] - y[6 * a], dy = y[6 * b + 1] - y[6 * a + 1],
                         dz = y[6 * b + 2] - y[6 * a + 2];
            const double r = sqrt((dx * dx + dy * dy) + dz * dz);
            const double Rs = cc->R[ia] + cc->R[ib];
            if (r < Rs) {
                *any = 1;
                const double f = (Rs - r) / Rs;
                if (f > deepest) deepest = f;
            }
        }
    }
    return deepest;
}

/* Mergers of the overlapping pairs of alive bodies in state y at time t of the
 * BS call, in ascending pair order, each seeing the mergers before it (R25). */
static void group_merge(const bs_group *g, coll_ctx *cc, double *y, double t)
{
    for (int64_t a = 0; a < g->nm; a++) {
        for (int64_t q = g->poff[a]; q < g->poff[a + 1]; q++) {
            const int64_t ia = g->mem[a];
            const int64_t b = g->plist[q], ib = g->mem[b];
            if (b <= a || !cc->alive[ia] || !cc->alive[ib]) continue;
            const double dx = y[6 * b] - y[6 * a], dy = y[6 * b + 1] - y[6 * a + 1],
                         dz = y[6 * b + 2] - y[6 * a + 2];
            const double r = sqrt((dx * dx + dy * dy) + dz * dz);
            const double Rs = cc->R[ia] + cc->R[ib];
            if (!(r < Rs)) continue;
            double xo[3], vo[3], dU;
            int64_t ot;
            const int64_t sv = merge_core(ia, ib, y + 6 * a, y + 6 * a + 3, y + 6 * b, y + 6 * b + 3,
                                          cc->m, cc->R, cc->S, cc->G, xo, vo, &ot, &dU);
            double *ys = y + 6 * (sv == ia ? a : b);
            for (int k = 0; k < 3; k++) { ys[k] = xo[k]; ys[3 + k] = vo[k]; }
            if (cc->log && cc->ncoll < cc->log_cap) {
                double *e = cc->log + 6 * cc->ncoll;
                e[0] = cc->t0 + t; e[1] = (double)ia; e[2] = (double)ib; e[3] = r; e[4] = Rs; e[5] = dU;
            }
            cc->alive[ot] = 0;
            cc->U += dU;
            cc->ncoll++;
        }
    }
}

/* Integrates y (6 nm values) over dt.  Returns 0, or 1 on hitting max_steps.
 * With cc, collisions (R25) are resolved on the way.                         */
static int bs_integrate(const bs_group *g, double *y, double dt, double tol, int max_steps,
                        int64_t *n_acc, int64_t *n_rej, int64_t *max_att, coll_ctx *cc)
{
    int64_t d = 6 * g->nm;
    double *f0 = (double *)malloc(sizeof(double) * (size_t)d);
    double *T = (double *)malloc(sizeof(double) * (size_t)d * BS_KMAX);
    double *yk = (double *)malloc(sizeof(double) * (size_t)d);
    double *zm = (double *)malloc(sizeof(double) * (size_t)d);
    double *zn = (double *)malloc(sizeof(double) * (size_t)d);
    double *fz = (double *)malloc(sizeof(double) * (size_t)d);
    double *sc = (double *)malloc(sizeof(double) * (size_t)d);
    double t = 0.0, H = dt;
    int attempts = 0, status = 0;
    if (cc) group_merge(g, cc, y, 0.0);       /* pairs overlapping at the start */
    while (t < dt) {
        if (attempts >= max_steps) { status = 1; break; }
        attempts++;
        if (H > dt - t) H = dt - t;
        bs_deriv(g, y, f0);
        for (int64_t c = 0; c < d; c++) sc[c] = fabs(y[c]) + fabs(H * f0[c]) + 1e-300;
        int accepted = 0, kconv = 0;
        /* T[(j)*d + c] holds column j of the current row (Neville, in place) */
        for (int k = 0; k < BS_KMAX; k++) {
            int nk = 2 * (k + 1);
            bs_midpoint(g, y, f0, H, nk, yk, zm, zn, fz);
            double err = 0.0;
            /* new row: R[0] = yk; R[j] = R[j-1] + (R[j-1] - Tprev[j-1]) / ((nk/n_{k-j})^2 - 1) */
            for (int64_t c = 0; c < d; c++) {
                double prev = T[0 * d + c];
                double cur = yk[c];
                T[0 * d + c] = cur;
                for (int j = 1; j <= k; j++) {
                    double ratio = (double)nk / (double)(2 * (k - j + 1));
                    double nxt = cur + (cur - prev) / (ratio * ratio - 1.0);
                    prev = T[j * d + c];
                    T[j * d + c] = nxt;
                    cur = nxt;
                }
                if (k >= 1) {
                    double e = fabs(T[k * d + c] - T[(k - 1) * d + c]) / sc[c];
                    if (e > err) err = e;
                }
            }
            if (k >= 1 && err <= tol) { accepted = 1; kconv = k; break; }
        }
        if (accepted && cc && cc->tol > 0.0) {
            /* collision precision: an overlap of tol or more ends the step too late */
            int any = 0;
            const double f = group_overlap(g, cc, T + (size_t)kconv * (size_t)d, &any);
            if (any && f >= cc->tol) accepted = 0;
        }
        if (accepted) {
            for (int64_t c = 0; c < d; c++) y[c] = T[kconv * d + c];
            t += H;
            (*n_acc)++;
            if (kconv < 4) H *= 1.5;
            if (cc) group_merge(g, cc, y, t);
        } else {
            (*n_rej)++;
            H *= 0.5;
        }
    }
    if (attempts > *max_att) *max_att = attempts;
    free(f0); free(T); free(yk); free(zm); free(zn); free(fz); free(sc);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Level machinery (Sec. 6.3, Appendix A).                                    */
typedef struct step_ctx {
    int64_t n;
    double *x, *v;
    const double *m;
    const orc_params *p;
    double *rcl[ORC_MAX_LEVELS];  /* rc of each level (full-length arrays) */
    orc_stats *st;
    int status;
    coll_ctx *cc;                 /* collisions (R25), or NULL */
    double gr_inv_c2;             /* GR splitting (R28): 1/c^2 in the BS groups, or 0 */
} step_ctx;

/* Partner lists (CSR) of a pair list that is ascending in (i,j): appending j to
 * i's list and i to j's list in pair order gives every list in ascending order
 * (a body's smaller partners come from earlier pairs than its larger ones).
 * Returns 0, or -1 if the pairs are not strictly ascending.                 */
static int build_partners(int64_t n, int64_t npairs, const uint32_t *pairs, int64_t *off,
                          int64_t *list)
{
    for (int64_t k = 1; k < npairs; k++) {
        uint64_t a = ((uint64_t)pairs[2 * k - 2] << 32) | pairs[2 * k - 1];
        uint64_t b = ((uint64_t)pairs[2 * k] << 32) | pairs[2 * k + 1];
        if (!(a < b)) return -1;
    }
    for (int64_t i = 0; i <= n; i++) off[i] = 0;
    for (int64_t k = 0; k < npairs; k++) { off[pairs[2 * k] + 1]++; off[pairs[2 * k + 1] + 1]++; }
    for (int64_t i = 0; i < n; i++) off[i + 1] += off[i];
    int64_t *fill = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    for (int64_t k = 0; k < npairs; k++) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        list[off[i] + fill[i]++] = j;
        list[off[j] + fill[j]++] = i;
    }
    free(fill);
    return 0;
}

/* Integrate every group of the pair list (ascending pairs) by BS over dt_l,
 * starting from the saved pre-drift state (xs, vs) of the members.          */
static void bs_all_groups(step_ctx *cx, int64_t npairs, const uint32_t *pairs, int level,
                          double dt_l, const double *xs, const double *vs)
{
    int64_t n = cx->n;
    int64_t *label = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    orc_group(n, npairs, pairs, label);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * npairs + 1));
    if (build_partners(n, npairs, pairs, off, list) != 0) cx->status |= 4;
    /* local index of each body inside its group; members ascending */
    int64_t *loc = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *gsize = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    for (int64_t i = 0; i < n; i++)
        if (label[i] >= 0) loc[i] = gsize[label[i]]++;
    for (int64_t g0 = 0; g0 < n; g0++) {
        if (gsize[g0] == 0) continue;          /* g0 is a label iff its group is non-empty */
        int64_t nm = gsize[g0];
        int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)nm);
        int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nm + 1));
        for (int64_t i = g0, c = 0; c < nm; i++)
            if (label[i] == g0) mem[c++] = i;
        poff[0] = 0;
        for (int64_t a = 0; a < nm; a++) poff[a + 1] = poff[a] + (off[mem[a] + 1] - off[mem[a]]);
        int64_t *plist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(poff[nm] > 0 ? poff[nm] : 1));
        for (int64_t a = 0; a < nm; a++)
            for (int64_t q = off[mem[a]], c = 0; q < off[mem[a] + 1]; q++, c++)
                plist[poff[a] + c] = loc[list[q]];
        double *y = (double *)malloc(sizeof(double) * 6 * (size_t)nm);
        for (int64_t a = 0; a < nm; a++)
            for (int k = 0; k < 3; k++) {
                y[6 * a + k] = xs[3 * mem[a] + k];
                y[6 * a + 3 + k] = vs[3 * mem[a] + k];
            }
        bs_group g;
        g.nm = nm; g.mem = mem; g.poff = poff; g.plist = plist; g.m = cx->cc ? cx->cc->m : cx->m;
        g.rcl = (const double *const *)cx->rcl; g.nlev = level + 1;
        g.G = cx->p->G; g.mu = cx->p->G * cx->p->m_star;
        g.alive = cx->cc ? cx->cc->alive : NULL;
        g.gr_inv_c2 = cx->gr_inv_c2;
        int fail = bs_integrate(&g, y, dt_l, cx->p->bs_tol, cx->p->bs_max_steps,
                                &cx->st->bs_steps, &cx->st->bs_rejects, &cx->st->bs_max_attempts,
                                cx->cc);
        if (fail) { cx->st->bs_fail++; cx->status |= 2; }
        for (int64_t a = 0; a < nm; a++)
            for (int k = 0; k < 3; k++) {
                cx->x[3 * mem[a] + k] = y[6 * a + k];
                cx->v[3 * mem[a] + k] = y[6 * a + 3 + k];
            }
        cx->st->n_groups++;
        if (nm > cx->st->max_group) cx->st->max_group = nm;
        free(y); free(plist); free(poff); free(mem);
    }
    free(gsize); free(loc); free(list); free(off); free(label);
}

/* KickS over a pair list at level l (1..): factor prod_{k<l}(1-K_k) K_l.
 * Accelerations of all bodies first (partners ascending), then the update.  */
static void kick_pairs(step_ctx *cx, int64_t nb, const int64_t *bodies, const int64_t *poff,
                       const int64_t *plist, int level, double dt_half)
{
    double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    const double *rcL = cx->rcl[level];
    for (int64_t a = 0; a < nb; a++) {
        int64_t i = bodies[a];
        const double *xi = cx->x + 3 * i;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int64_t q = poff[a]; q < poff[a + 1]; q++) {
            int64_t j = plist[q];
            const double *xj = cx->x + 3 * j;
            double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
            double r2 = (dx * dx + dy * dy) + dz * dz;
            double r = sqrt(r2);
            double W = 1.0;
            for (int l = 0; l < level; l++) {
                const double *rc = cx->rcl[l];
                W *= 1.0 - orc_changeover(r, rc[i] > rc[j] ? rc[i] : rc[j]);
            }
            W *= orc_changeover(r, rcL[i] > rcL[j] ? rcL[i] : rcL[j]);
            double f = cx->m[j] * W / (r2 * r);
            s0 += f * dx; s1 += f * dy; s2 += f * dz;
        }
        acc[3 * a + 0] = cx->p->G * s0;
        acc[3 * a + 1] = cx->p->G * s1;
        acc[3 * a + 2] = cx->p->G * s2;
    }
    for (int64_t a = 0; a < nb; a++)
        for (int k = 0; k < 3; k++) cx->v[3 * bodies[a] + k] += dt_half * acc[3 * a + k];
    free(acc);
}

/* SEnc (Appendix A) at level `level` >= 1 over the pairs of level-1. */
static void senc(step_ctx *cx, int64_t npairs, const uint32_t *pairs, int level, double dt_l,
                 const double *xs_up, const double *vs_up)
{
    int64_t n = cx->n;
    const orc_params *p = cx->p;
    /* groupS: bodies of this level = members of the upper level's pairs, and
     * each body's partner list (ascending global index).                     */
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * npairs + 1));
    if (build_partners(n, npairs, pairs, off, list) != 0) cx->status |= 4;
    int64_t nb = 0;
    for (int64_t i = 0; i < n; i++) nb += off[i + 1] > off[i];
    int64_t *bodies = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb + 1));
    for (int64_t i = 0, c = 0; i < n; i++) if (off[i + 1] > off[i]) bodies[c++] = i;
    poff[0] = 0;
    for (int64_t a = 0; a < nb; a++) poff[a + 1] = poff[a] + (off[bodies[a] + 1] - off[bodies[a]]);
    int64_t *plist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(poff[nb] > 0 ? poff[nb] : 1));
    for (int64_t a = 0; a < nb; a++)
        for (int64_t q = off[bodies[a]], c = 0; q < off[bodies[a] + 1]; q++, c++)
            plist[poff[a] + c] = list[q];
    free(list);
    free(off);
    /* R10: restart the level bodies from the enclosing level's pre-drift state */
    for (int64_t a = 0; a < nb; a++)
        for (int k = 0; k < 3; k++) {
            cx->x[3 * bodies[a] + k] = xs_up[3 * bodies[a] + k];
            cx->v[3 * bodies[a] + k] = vs_up[3 * bodies[a] + k];
        }
    double *xs = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *vs = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    uint32_t *enc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)(npairs > 0 ? npairs : 1));
    double *rcL = cx->rcl[level];
    for (int s = 0; s < p->substeps; s++) {
        /* RcritS(dt_l) on the level bodies */
        for (int64_t a = 0; a < nb; a++) {
            int64_t i = bodies[a];
            orc_rcrit(1, cx->x + 3 * i, cx->v + 3 * i, cx->m + i, p->m_star, dt_l, p->n1, p->n2,
                      rcL + i);
        }
        kick_pairs(cx, nb, bodies, poff, plist, level, 0.5 * dt_l);
        for (int64_t a = 0; a < nb; a++)
            for (int k = 0; k < 3; k++) {
                xs[3 * bodies[a] + k] = cx->x[3 * bodies[a] + k];
                vs[3 * bodies[a] + k] = cx->v[3 * bodies[a] + k];
            }
        cx->st->kepler_fail += fg_list(bodies, nb, cx->x, cx->v, p->G * p->m_star, dt_l,
                                       p->kepler_max_iter);
        int64_t ne = orc_detect(npairs, pairs, xs, cx->x, rcL, enc);
        plog_detection(level, npairs, pairs, xs, cx->x, rcL, ne, enc);
        cx->st->n_pairs[level] += ne;
        if (ne > 0) {
            if (level < p->slevels - 1)
                senc(cx, ne, enc, level + 1, dt_l / p->substeps, xs, vs);
            else
                bs_all_groups(cx, ne, enc, level, dt_l, xs, vs);
        }
        kick_pairs(cx, nb, bodies, poff, plist, level, 0.5 * dt_l);
    }
    free(enc); free(vs); free(xs); free(plist); free(poff); free(bodies);
}

/* ------------------------------------------------------------------------- */
/* Non-Newtonian forces (Sec. 3 GR, Sec. 4.1-4.2 tides) applied with the implicit
 * midpoint rule of Sec. 2.3 (Eq. implicit) over each half kick.
 *
 * Readings (the paper gives the formulas, not where they enter the step):
 *  R15 after each level-0 gravitational half kick, velocities are converted to
 *      heliocentric u_i = v_i + P/m_star (P = sum m_j v_j), the forces act on u for
 *      dt/2 by the implicit midpoint rule, and u is converted back with
 *      v_i = u_i - sum_j m_j u_j / (m_star + sum_j m_j);
 *  R16 GR: a_PN,i of Eq. apn with mu = G (m_star + m_i), r-dot = x.u/|x|;
 *  R17 tides: the force F_T of Eq. (Bolmont 2015 Eq. 6, corrected) gives the
 *      heliocentric acceleration F_T / m_i; spins follow
 *      d(I_i W_i)/dt = -(m_star/(m_star+m_i)) N_Ti and
 *      d(I_star W_star)/dt = -sum_j (m_star/(m_star+m_j)) N_Tstar,j, I = rg2 m R^2;
 *      with this reading total angular momentum (orbit + spins) is conserved
 *      exactly for one planet;
 *  R18 the implicit iteration updates u, W_i and W_star together from their
 *      midpoint values until no component changes by more than 1e-16 of its
 *      size, at most implicit_max_iter (10) times.                           */
typedef struct orc_nn {
    int32_t gr, tides;
    int32_t implicit_max_iter;
    int32_t gr_split;  /* GR by the Hamiltonian splitting of Sec. 3.1 (R28) instead of Eq. apn */
    double c_light;
    double R_star, k2_star, tau_star, rg2_star;
} orc_nn;

/* GR (Eq. apn) and tidal (F_T / m_i) heliocentric acceleration of one body and
 * the tidal torques N_Ti, N_Tstar (Sec. 4.2), from position x, heliocentric
 * velocity u and spins W (body) and Ws (star).                              */
static void nn_terms(const double *x, const double *u, const double *W, const double *Ws,
                     double mi, double Ri, double k2i, double taui, double G, double m_star,
                     const orc_nn *nn, double *acc, double *Ni, double *Ns)
{
    double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
    double r = sqrt(r2);
    double er[3] = {x[0] / r, x[1] / r, x[2] / r};
    double rdot = ((x[0] * u[0] + x[1] * u[1]) + x[2] * u[2]) / r;
    double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    for (int k = 0; k < 3; k++) { acc[k] = 0.0; Ni[k] = 0.0; Ns[k] = 0.0; }
    if (nn->gr) {
        double mu = G * (m_star + mi);
        double eta = m_star * mi / ((m_star + mi) * (m_star + mi));
        double c2 = nn->c_light * nn->c_light;
        double pre = -mu / (r2 * c2);
        double cv = -2.0 * (2.0 - eta) * rdot;
        double cr = (1.0 + 3.0 * eta) * u2 - 1.5 * eta * rdot * rdot - 2.0 * (2.0 + eta) * mu / r;
        for (int k = 0; k < 3; k++) acc[k] += pre * (cv * u[k] + cr * er[k]);
    }
    if (nn->tides) {
        double r5 = r2 * r2 * r;
        double r7 = r5 * r2;
        double Ri5 = Ri * Ri * Ri * Ri * Ri;
        double Rs5 = nn->R_star * nn->R_star * nn->R_star * nn->R_star * nn->R_star;
        double Dti = 3.0 * G * m_star * m_star * Ri5 / r7 * k2i;
        double Dts = 3.0 * G * mi * mi * Rs5 / r7 * nn->k2_star;
        double Pti = Dti * taui;
        double Pts = Dts * nn->tau_star;
        /* F_T = [-(Dts + Dti) - 2 rdot/r (Pts + Pti)] e_r + Pti (W x e_r) + Pts (Ws x e_r)
         *       - (Pti + Pts) u / r                                              */
        double fr = -(Dts + Dti) - 2.0 * rdot / r * (Pts + Pti);
        double wxe[3] = {W[1] * er[2] - W[2] * er[1], W[2] * er[0] - W[0] * er[2],
                         W[0] * er[1] - W[1] * er[0]};
        double sxe[3] = {Ws[1] * er[2] - Ws[2] * er[1], Ws[2] * er[0] - Ws[0] * er[2],
                         Ws[0] * er[1] - Ws[1] * er[0]};
        double exu[3] = {er[1] * u[2] - er[2] * u[1], er[2] * u[0] - er[0] * u[2],
                         er[0] * u[1] - er[1] * u[0]};
        double rW = (x[0] * W[0] + x[1] * W[1]) + x[2] * W[2];
        double rWs = (x[0] * Ws[0] + x[1] * Ws[1]) + x[2] * Ws[2];
        for (int k = 0; k < 3; k++) {
            double F = fr * er[k] + Pti * wxe[k] + Pts * sxe[k] - (Pti + Pts) * u[k] / r;
            acc[k] += F / mi;
            /* N = P [W r - (r.W) e_r - e_r x u] */
            Ni[k] = Pti * (W[k] * r - rW * er[k] - exu[k]);
            Ns[k] = Pts * (Ws[k] * r - rWs * er[k] - exu[k]);
        }
    }
}

/* Implicit midpoint of the non-Newtonian forces over dt for all bodies. */
static void nn_implicit(int64_t n, const double *x, double *v, const double *m, double G,
                        double m_star, const orc_nn *nn, const double *R, const double *k2,
                        const double *tau, const double *rg2, double *spin, double *spin_star,
                        double dt)
{
    if (!nn || (!nn->gr && !nn->tides) || n == 0) return;
    double P[3] = {0.0, 0.0, 0.0}, Mp = 0.0;
    for (int64_t j = 0; j < n; j++) {
        for (int k = 0; k < 3; k++) P[k] += m[j] * v[3 * j + k];
        Mp += m[j];
    }
    double *u0 = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *u1 = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *W0 = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *W1 = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            u0[3 * i + k] = v[3 * i + k] + P[k] / m_star;
            u1[3 * i + k] = u0[3 * i + k];
            W0[3 * i + k] = spin[3 * i + k];
            W1[3 * i + k] = spin[3 * i + k];
        }
    double Ws0[3] = {spin_star[0], spin_star[1], spin_star[2]};
    double Ws1[3] = {Ws0[0], Ws0[1], Ws0[2]};
    double Is = nn->rg2_star * m_star * nn->R_star * nn->R_star;
    for (int it = 0; it < nn->implicit_max_iter; it++) {
        int changed = 0;
        double dLs[3] = {0.0, 0.0, 0.0};
        double Wsm[3];
        for (int k = 0; k < 3; k++) Wsm[k] = 0.5 * (Ws0[k] + Ws1[k]);
        for (int64_t i = 0; i < n; i++) {
            double um[3], Wm[3], acc[3], Ni[3], Ns[3];
            for (int k = 0; k < 3; k++) {
                um[k] = 0.5 * (u0[3 * i + k] + u1[3 * i + k]);
                Wm[k] = 0.5 * (W0[3 * i + k] + W1[3 * i + k]);
            }
            nn_terms(x + 3 * i, um, Wm, Wsm, m[i], R ? R[i] : 0.0, k2 ? k2[i] : 0.0,
                     tau ? tau[i] : 0.0, G, m_star, nn, acc, Ni, Ns);
            double fac = m_star / (m_star + m[i]);
            double Ii = rg2 ? rg2[i] * m[i] * R[i] * R[i] : 0.0;
            for (int k = 0; k < 3; k++) {
                double un = u0[3 * i + k] + dt * acc[k];
                if (fabs(un - u1[3 * i + k]) > 1e-16 * fabs(un)) changed = 1;
                u1[3 * i + k] = un;
                if (nn->tides && Ii > 0.0) {
                    double Wn = W0[3 * i + k] - dt * fac * Ni[k] / Ii;
                    if (fabs(Wn - W1[3 * i + k]) > 1e-16 * fabs(Wn)) changed = 1;
                    W1[3 * i + k] = Wn;
                }
                dLs[k] += fac * Ns[k];
            }
        }
        if (nn->tides && Is > 0.0)
            for (int k = 0; k < 3; k++) {
                double Wn = Ws0[k] - dt * dLs[k] / Is;
                if (fabs(Wn - Ws1[k]) > 1e-16 * fabs(Wn)) changed = 1;
                Ws1[k] = Wn;
            }
        if (!changed) break;
    }
    double Q[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; j++)
        for (int k = 0; k < 3; k++) Q[k] += m[j] * u1[3 * j + k];
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            v[3 * i + k] = u1[3 * i + k] - Q[k] / (m_star + Mp);
            spin[3 * i + k] = W1[3 * i + k];
        }
    for (int k = 0; k < 3; k++) spin_star[k] = Ws1[k];
    free(u0); free(u1); free(W0); free(W1);
}

/* ------------------------------------------------------------------------- */
/* GR by Hamiltonian splitting (Sec. 3.1, after Saha & Tremaine 1994; reading
 * R28).  H_PN = sum_i alpha_i H_Kep,i^2 + beta_i / r_i^2 + gamma_i p_i^4 acts on
 * the canonical momenta p_i = m_i u_i (u: pseudovelocities):
 *   beta:  u_i += -dt 2 mu_i^2 / (c^2 r_i^4) x_i, mu_i = G (m_star + m_i), with
 *          the kick ("sun kick"; no changeover factor);
 *   gamma: x_i += -dt 2 (u_i^2 / c^2) u_i, with HC;
 *   alpha: the Kepler drift of body i over dt (1 + 2 alpha_i H_Kep,i / m_i) =
 *          dt (1 + 3 (u_i^2/2 - mu/r_i) / c^2) = dt (1 - 3 mu / (2 a_i c^2)),
 *          mu = G m_star as in the drift; in a close-encounter group the same
 *          factor multiplies the member's velocity term and the star's
 *          acceleration, not the pair terms.
 * The real velocity is dx/dt = dH/dp without the HC term:
 *   v = u (1 - (u^2/2 + 3 mu / r) / c^2);
 * the step converts v -> u before the sun kick, HC and the drift, and back
 * after them, so the pair kicks and the tides act on real velocities.      */
static double gr_alpha_factor(const double *x, const double *u, double mu, double inv_c2)
{
    double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    return 1.0 + 3.0 * (0.5 * u2 - mu / r) * inv_c2;
}

static double gr_real_factor(const double *x, const double *u, double mu, double inv_c2)
{
    double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    return 1.0 - (0.5 * u2 + 3.0 * mu / r) * inv_c2;
}

/* v -> u: u = v / (1 - (u^2/2 + 3 mu/r)/c^2) by fixed-point iteration from
 * u = v (the correction is ~v^2/c^2; 4 iterations reach rounding).           */
static void gr_to_pseudo(int64_t n, const double *x, double *v, double mu, double inv_c2)
{
    for (int64_t i = 0; i < n; i++) {
        double u[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
        for (int it = 0; it < 4; it++) {
            double f = gr_real_factor(x + 3 * i, u, mu, inv_c2);
            for (int k = 0; k < 3; k++) u[k] = v[3 * i + k] / f;
        }
        for (int k = 0; k < 3; k++) v[3 * i + k] = u[k];
    }
}

static void gr_to_real(int64_t n, const double *x, double *v, double mu, double inv_c2)
{
    for (int64_t i = 0; i < n; i++) {
        double f = gr_real_factor(x + 3 * i, v + 3 * i, mu, inv_c2);
        for (int k = 0; k < 3; k++) v[3 * i + k] *= f;
    }
}

static void gr_beta_kick(int64_t n, const double *x, double *u, const double *m, double G,
                         double m_star, double inv_c2, double dt)
{
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i;
        double r2 = (xi[0] * xi[0] + xi[1] * xi[1]) + xi[2] * xi[2];
        double mui = G * (m_star + m[i]);
        double s = -dt * 2.0 * mui * mui * inv_c2 / (r2 * r2);
        for (int k = 0; k < 3; k++) u[3 * i + k] += s * xi[k];
    }
}

/* HC(dt) with the gamma term: x_i += dt P/m_star - dt 2 (u_i^2/c^2) u_i (the
 * HC shift formed as orc_hc forms it). */
static void gr_hc_gamma(int64_t n, double *x, const double *u, const double *m, double m_star,
                        double inv_c2, double dt)
{
    double P[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; j++)
        for (int k = 0; k < 3; k++) P[k] += m[j] * u[3 * j + k];
    double c[3];
    for (int k = 0; k < 3; k++) c[k] = dt * P[k] / m_star;
    for (int64_t i = 0; i < n; i++) {
        const double *ui = u + 3 * i;
        double u2 = (ui[0] * ui[0] + ui[1] * ui[1]) + ui[2] * ui[2];
        double g = dt * 2.0 * u2 * inv_c2;
        for (int k = 0; k < 3; k++) x[3 * i + k] += c[k] - g * ui[k];
    }
}

/* FG with each body's drift time rescaled by the alpha factor. */
static int64_t gr_fg(int64_t n, double *x, double *u, double mu, double inv_c2, double dt, int max_iter)
{
    int64_t fails = 0;
    for (int64_t i = 0; i < n; i++) {
        double dti = dt * gr_alpha_factor(x + 3 * i, u + 3 * i, mu, inv_c2);
        if (kepler_one(x + 3 * i, u + 3 * i, mu, dti, max_iter)) fails++;
    }
    return fails;
}

/* ------------------------------------------------------------------------- */
/* Direct entry for tests: group the ascending pair list and integrate every
 * group by BS over dt from (x, v) in place, with nlev levels of critical radii
 * rc_levels[l*n + i].  Returns 0, or 2 when a group hit bs_max_steps.        */
int orc_bs_groups(int64_t n, double *x, double *v, const double *m, const double *rc_levels,
                  int nlev, int64_t npairs, const uint32_t *pairs, double G, double m_star,
                  double dt, double tol, int max_steps, orc_stats *st)
{
    orc_params p;
    memset(&p, 0, sizeof(p));
    p.G = G; p.m_star = m_star; p.bs_tol = tol; p.bs_max_steps = max_steps;
    step_ctx cx;
    memset(&cx, 0, sizeof(cx));
    memset(st, 0, sizeof(*st));
    cx.n = n; cx.x = x; cx.v = v; cx.m = m; cx.p = &p; cx.st = st;
    if (nlev < 1 || nlev > ORC_MAX_LEVELS) return -1;
    for (int l = 0; l < nlev; l++) cx.rcl[l] = (double *)(rc_levels + (size_t)l * (size_t)n);
    double *xs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *vs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    memcpy(xs, x, sizeof(double) * 3 * (size_t)n);
    memcpy(vs, v, sizeof(double) * 3 * (size_t)n);
    bs_all_groups(&cx, npairs, pairs, nlev - 1, dt, xs, vs);
    free(xs); free(vs);
    return cx.status;
}

/* Test hook for the level split of the pair forces (Sec. 6.3, Appendix A):
 * with one ascending pair list used at every level, the parts of each body's
 * acceleration that the step's own routines give --
 *   acc_kick  (3n): the level-0 Kick over all pairs (factor K_0; orc_accel),
 *   acc_kicks ((nlev-1) x 3n): KickS at levels l = 1..nlev-1 over the list
 *             (factor prod_{k<l} (1 - K_k) K_l; kick_pairs, from v = 0 with
 *             dt_half = 1),
 *   acc_bs    (3n): the pair part of the Bulirsch-Stoer derivative at the
 *             deepest level (factor prod_{k<nlev} (1 - K_k); bs_deriv with the
 *             star term off, all bodies one group).
 * rc_levels: nlev x n.  When the list holds every pair, the parts sum to the
 * Newtonian pair acceleration.  Returns 0, or -1 for a bad list or nlev.     */
int orc_level_force_parts(int64_t n, const double *x, const double *m, const double *rc_levels,
                          int nlev, int64_t npairs, const uint32_t *pairs, double G,
                          double *acc_kick, double *acc_kicks, double *acc_bs)
{
    if (nlev < 1 || nlev > ORC_MAX_LEVELS || n < 1) return -1;
    orc_accel(n, x, m, rc_levels, G, acc_kick, 1);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * npairs + 1));
    if (build_partners(n, npairs, pairs, off, list) != 0) { free(off); free(list); return -1; }
    orc_params p;
    memset(&p, 0, sizeof(p));
    p.G = G;
    orc_stats st;
    memset(&st, 0, sizeof(st));
    step_ctx cx;
    memset(&cx, 0, sizeof(cx));
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *vw = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(xw, x, sizeof(double) * 3 * (size_t)n);
    cx.n = n; cx.x = xw; cx.v = vw; cx.m = m; cx.p = &p; cx.st = &st;
    for (int l = 0; l < nlev; l++) cx.rcl[l] = (double *)(rc_levels + (size_t)l * (size_t)n);
    /* KickS bodies and partner lists as groupS builds them */
    int64_t nb = 0;
    for (int64_t i = 0; i < n; i++) nb += off[i + 1] > off[i];
    int64_t *bodies = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb + 1));
    for (int64_t i = 0, c = 0; i < n; i++) if (off[i + 1] > off[i]) bodies[c++] = i;
    poff[0] = 0;
    for (int64_t a = 0; a < nb; a++) poff[a + 1] = poff[a] + (off[bodies[a] + 1] - off[bodies[a]]);
    int64_t *plist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(poff[nb] > 0 ? poff[nb] : 1));
    for (int64_t a = 0; a < nb; a++)
        for (int64_t q = off[bodies[a]], c = 0; q < off[bodies[a] + 1]; q++, c++)
            plist[poff[a] + c] = list[q];
    for (int l = 1; l < nlev; l++) {
        memset(vw, 0, sizeof(double) * 3 * (size_t)n);
        kick_pairs(&cx, nb, bodies, poff, plist, l, 1.0);
        memcpy(acc_kicks + (size_t)(l - 1) * 3 * (size_t)n, vw, sizeof(double) * 3 * (size_t)n);
    }
    /* Bulirsch-Stoer derivative: every body a member (local = global index) */
    int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; i++) mem[i] = i;
    double *y = (double *)calloc(6 * (size_t)n, sizeof(double));
    double *f = (double *)malloc(sizeof(double) * 6 * (size_t)n);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) y[6 * i + k] = x[3 * i + k];
    bs_group g;
    g.nm = n; g.mem = mem; g.poff = off; g.plist = list; g.m = m;
    g.rcl = (const double *const *)cx.rcl; g.nlev = nlev;
    g.G = G; g.mu = 0.0; g.alive = NULL; g.gr_inv_c2 = 0.0;
    bs_deriv(&g, y, f);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) acc_bs[3 * i + k] = f[6 * i + 3 + k];
    free(f); free(y); free(mem); free(plist); free(poff); free(bodies);
    free(vw); free(xw); free(list); free(off);
    return 0;
}

/* orc_bs_groups with collisions (R25): m, R, S (3 per body) and alive are
 * updated by the mergers; *U and *ncoll accumulate; log (may be NULL) takes
 * up to log_cap mergers, 6 doubles each: time in the call, i, j, r_ij,
 * R_i + R_j, Delta U.                                                        */
int orc_bs_groups_coll(int64_t n, double *x, double *v, double *m, double *R, double *S,
                       unsigned char *alive, const double *rc_levels, int nlev, int64_t npairs,
                       const uint32_t *pairs, double G, double m_star, double dt, double tol,
                       int max_steps, double coll_tol, double *U, int64_t *ncoll, double *log,
                       int64_t log_cap, orc_stats *st)
{
    orc_params p;
    memset(&p, 0, sizeof(p));
    p.G = G; p.m_star = m_star; p.bs_tol = tol; p.bs_max_steps = max_steps;
    coll_ctx cc;
    cc.m = m; cc.R = R; cc.S = S; cc.alive = alive; cc.tol = coll_tol; cc.G = G;
    cc.U = *U; cc.ncoll = *ncoll; cc.log = log; cc.log_cap = log_cap; cc.t0 = 0.0;
    step_ctx cx;
    memset(&cx, 0, sizeof(cx));
    memset(st, 0, sizeof(*st));
    cx.n = n; cx.x = x; cx.v = v; cx.m = m; cx.p = &p; cx.st = st; cx.cc = &cc;
    if (nlev < 1 || nlev > ORC_MAX_LEVELS) return -1;
    for (int l = 0; l < nlev; l++) cx.rcl[l] = (double *)(rc_levels + (size_t)l * (size_t)n);
    double *xs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *vs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    memcpy(xs, x, sizeof(double) * 3 * (size_t)n);
    memcpy(vs, v, sizeof(double) * 3 * (size_t)n);
    bs_all_groups(&cx, npairs, pairs, nlev - 1, dt, xs, vs);
    free(xs); free(vs);
    *U = cc.U;
    *ncoll = cc.ncoll;
    return cx.status;
}

/* ------------------------------------------------------------------------- */
/* One step of Appendix A (original scheme for slevels == 1, SEnc otherwise).
 * Returns 0, or a bit mask: 1 Kepler non-convergence, 2 BS limit reached.    */
static int step_impl(int64_t n, double *x, double *v, const double *m, const orc_params *p,
                     int64_t nsteps, orc_stats *st, const orc_nn *nn, const double *R,
                     const double *k2, const double *tau, const double *rg2, double *spin,
                     double *spin_star, coll_ctx *cc)
{
    step_ctx cx;
    memset(&cx, 0, sizeof(cx));
    cx.n = n; cx.x = x; cx.v = v; cx.m = cc ? cc->m : m; cx.p = p; cx.st = st; cx.cc = cc;
    if (cc) m = cc->m;
    memset(st, 0, sizeof(*st));
    int L = p->slevels < 1 ? 1 : p->slevels;
    if (L > ORC_MAX_LEVELS) L = ORC_MAX_LEVELS;
    for (int l = 0; l < L; l++) cx.rcl[l] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *xs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *vs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double dt = p->dt, mu = p->G * p->m_star;
    /* R28: GR by Hamiltonian splitting (original scheme, one level) */
    const int split = nn && nn->gr && nn->gr_split && L == 1;
    const double inv_c2 = split ? 1.0 / (nn->c_light * nn->c_light) : 0.0;
    orc_nn nn_tides;
    if (nn) { nn_tides = *nn; nn_tides.gr = 0; }
    cx.gr_inv_c2 = inv_c2;
    /* R24: bodies i >= nm are semi-active test particles */
    const int64_t nm = (p->tp_mode == 2 && p->n_massive >= 0 && p->n_massive < n) ? p->n_massive : n;
    for (int64_t s = 0; s < nsteps; s++) {
        orc_rcrit(n, x, v, m, p->m_star, dt, p->n1, p->n2, cx.rcl[0]);
        int64_t cap = 1024;
        uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)cap);
        int64_t nc = orc_precheck_tp(n, nm, x, cx.rcl[0], p->f_pc, cand, cap);
        if (nc > cap) {
            free(cand);
            cap = nc;
            cand = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)cap);
            nc = orc_precheck_tp(n, nm, x, cx.rcl[0], p->f_pc, cand, cap);
        }
        st->n_candidates += nc;
        kick_tp(n, nm, x, m, cx.rcl[0], p->G, 0.5 * dt, v, p->nthreads);
        if (split) {
            /* R28: tides by the implicit midpoint rule on real velocities,
             * then sun kick, HC + gamma and the alpha-scaled drift in
             * pseudovelocities */
            nn_implicit(n, x, v, m, p->G, p->m_star, &nn_tides, R, k2, tau, rg2, spin, spin_star, 0.5 * dt);
            gr_to_pseudo(n, x, v, mu, inv_c2);
            gr_beta_kick(n, x, v, m, p->G, p->m_star, inv_c2, 0.5 * dt);
            gr_hc_gamma(n, x, v, m, p->m_star, inv_c2, 0.5 * dt);
            memcpy(xs, x, sizeof(double) * 3 * (size_t)n);
            memcpy(vs, v, sizeof(double) * 3 * (size_t)n);
            st->kepler_fail += gr_fg(n, x, v, mu, inv_c2, dt, p->kepler_max_iter);
        } else {
            nn_implicit(n, x, v, m, p->G, p->m_star, nn, R, k2, tau, rg2, spin, spin_star, 0.5 * dt);
            orc_hc(n, x, v, m, p->m_star, 0.5 * dt);
            memcpy(xs, x, sizeof(double) * 3 * (size_t)n);
            memcpy(vs, v, sizeof(double) * 3 * (size_t)n);
            st->kepler_fail += orc_fg(n, x, v, mu, dt, p->kepler_max_iter);
        }
        if (nc > 0) {
            uint32_t *enc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)nc);
            int64_t ne = orc_detect(nc, cand, xs, x, cx.rcl[0], enc);
            plog_detection(0, nc, cand, xs, x, cx.rcl[0], ne, enc);
            st->n_pairs[0] += ne;
            if (ne > 0) {
                if (L > 1)
                    senc(&cx, ne, enc, 1, dt / p->substeps, xs, vs);
                else
                    bs_all_groups(&cx, ne, enc, 0, dt, xs, vs);
            }
            free(enc);
        }
        free(cand);
        if (split) {
            gr_hc_gamma(n, x, v, m, p->m_star, inv_c2, 0.5 * dt);
            gr_beta_kick(n, x, v, m, p->G, p->m_star, inv_c2, 0.5 * dt);
            gr_to_real(n, x, v, mu, inv_c2);
            kick_tp(n, nm, x, m, cx.rcl[0], p->G, 0.5 * dt, v, p->nthreads);
            nn_implicit(n, x, v, m, p->G, p->m_star, &nn_tides, R, k2, tau, rg2, spin, spin_star, 0.5 * dt);
        } else {
            orc_hc(n, x, v, m, p->m_star, 0.5 * dt);
            kick_tp(n, nm, x, m, cx.rcl[0], p->G, 0.5 * dt, v, p->nthreads);
            nn_implicit(n, x, v, m, p->G, p->m_star, nn, R, k2, tau, rg2, spin, spin_star, 0.5 * dt);
        }
    }
    if (st->kepler_fail) cx.status |= 1;
    for (int l = 0; l < L; l++) free(cx.rcl[l]);
    free(xs); free(vs);
    return cx.status;
}

int orc_step(int64_t n, double *x, double *v, const double *m, const orc_params *p,
             int64_t nsteps, orc_stats *st)
{
    return step_impl(n, x, v, m, p, nsteps, st, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* One system with GR and/or tides (R15-R18); spin (3n) and spin_star (3) are
 * updated in place; R, k2, tau, rg2 are per-body arrays (n).                 */
/* Steps with collisions (R25): m, R, S (3 per body) and alive are updated by
 * the mergers; *U and *ncoll accumulate; log as for orc_bs_groups_coll, the
 * time measured from the start of the BS call of the merger.                */
int orc_step_coll(int64_t n, double *x, double *v, double *m, double *R, double *S,
                  unsigned char *alive, const orc_params *p, int64_t nsteps, double coll_tol,
                  double *U, int64_t *ncoll, double *log, int64_t log_cap, orc_stats *st)
{
    coll_ctx cc;
    cc.m = m; cc.R = R; cc.S = S; cc.alive = alive; cc.tol = coll_tol; cc.G = p->G;
    cc.U = *U; cc.ncoll = *ncoll; cc.log = log; cc.log_cap = log_cap; cc.t0 = 0.0;
    const int status = step_impl(n, x, v, m, p, nsteps, st, NULL, NULL, NULL, NULL, NULL, NULL, NULL, &cc);
    *U = cc.U;
    *ncoll = cc.ncoll;
    return status;
}

int orc_step_nn(int64_t n, double *x, double *v, const double *m, const orc_params *p,
                const orc_nn *nn, const double *R, const double *k2, const double *tau,
                const double *rg2, double *spin, double *spin_star, int64_t nsteps, orc_stats *st)
{
    return step_impl(n, x, v, m, p, nsteps, st, nn, R, k2, tau, rg2, spin, spin_star, NULL);
}

/* Total angular momentum with spins: sum m_i x_i x v_i + sum I_i W_i + I_s W_s. */
void orc_angmom_spin(int64_t n, const double *x, const double *v, const double *m,
                     const double *R, const double *rg2, const double *spin, double m_star,
                     double R_star, double rg2_star, const double *spin_star, double *L)
{
    long double Lx = 0.0L, Ly = 0.0L, Lz = 0.0L;
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i, *vi = v + 3 * i;
        Lx += (long double)m[i] * ((long double)xi[1] * vi[2] - (long double)xi[2] * vi[1]);
        Ly += (long double)m[i] * ((long double)xi[2] * vi[0] - (long double)xi[0] * vi[2]);
        Lz += (long double)m[i] * ((long double)xi[0] * vi[1] - (long double)xi[1] * vi[0]);
        long double I = (long double)rg2[i] * m[i] * R[i] * R[i];
        Lx += I * spin[3 * i + 0]; Ly += I * spin[3 * i + 1]; Lz += I * spin[3 * i + 2];
    }
    long double Is = (long double)rg2_star * m_star * R_star * R_star;
    L[0] = (double)(Lx + Is * spin_star[0]);
    L[1] = (double)(Ly + Is * spin_star[1]);
    L[2] = (double)(Lz + Is * spin_star[2]);
}

/* ------------------------------------------------------------------------- */
/* Frozen-encounter steps and their tangent-linear (forward-mode) derivative,
 * for the adjoint configuration.  Readings:
 *  R20 a step with frozen encounters uses a given level-0 rc array and a given
 *      ascending pair list instead of Rcrit, pre-check and detection (the
 *      original scheme, slevels = 1); there is no derivative through rc;
 *  R21 the derivative of the changeover function is taken (dK/dr), i.e. the
 *      derivative of the kick and BS forces as defined by R4/R5;
 *  R22 the tangent of the Kepler drift and of each BS group is the solution of
 *      the variational equations integrated alongside the state by the same
 *      Bulirsch-Stoer scheme, with error control on the state only.          */

/* dK/dr of the changeover function R4 (0 outside the band). */
static double changeover_dr(double r, double rc)
{
    double y = (r / rc - 0.1) / 0.9;
    if (y <= 0.0 || y >= 1.0) return 0.0;
    double D = 2.0 * y * y - 2.0 * y + 1.0;
    return 2.0 * y * (1.0 - y) / (D * D) / (0.9 * rc);
}

/* M = w (I/r^3 - 3 d d^T / r^5) + w' d d^T / r^4 applied to e (3-vector). */
static void pair_tensor_apply(const double *d, double r, double w, double wp, const double *e,
                              double *out)
{
    double r2 = r * r, r3 = r2 * r;
    double de = (d[0] * e[0] + d[1] * e[1]) + d[2] * e[2];
    for (int k = 0; k < 3; k++)
        out[k] = w * (e[k] / r3 - 3.0 * d[k] * de / (r3 * r2)) + wp * d[k] * de / (r2 * r2);
}

/* Tangent of the kick acceleration: da_i = G sum_j [m_j M_ij (dx_j - dx_i) + dm_j K d/r^3]. */
static void kick_tl(int64_t n, const double *x, const double *m, const double *rc, double G,
                    const double *dx, const double *dm, double *da)
{
    for (int64_t i = 0; i < n; i++) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            double rcij = pair_rc(rc, i, j);
            double K = orc_changeover(r, rcij);
            double Kp = changeover_dr(r, rcij);
            double e[3] = {dx[3 * j] - dx[3 * i], dx[3 * j + 1] - dx[3 * i + 1], dx[3 * j + 2] - dx[3 * i + 2]};
            double Me[3];
            pair_tensor_apply(d, r, K, Kp, e, Me);
            double r3 = r * r * r;
            for (int k = 0; k < 3; k++) s[k] += m[j] * Me[k] + dm[j] * K * d[k] / r3;
        }
        for (int k = 0; k < 3; k++) da[3 * i + k] = G * s[k];
    }
}

/* Generic Bulirsch-Stoer (same scheme as bs_integrate) for dim values, of
 * which the first nerr enter the error norm.                                */
typedef void (*bs_fn)(const void *ctx, const double *y, double *f);

static int bs_generic(bs_fn fn, const void *ctx, double *y, int64_t dim, int64_t nerr, double dt,
                      double tol, int max_steps)
{
    double *f0 = (double *)malloc(sizeof(double) * (size_t)dim);
    double *T = (double *)malloc(sizeof(double) * (size_t)dim * BS_KMAX);
    double *yk = (double *)malloc(sizeof(double) * (size_t)dim);
    double *zm = (double *)malloc(sizeof(double) * (size_t)dim);
    double *zn = (double *)malloc(sizeof(double) * (size_t)dim);
    double *fz = (double *)malloc(sizeof(double) * (size_t)dim);
    double *sc = (double *)malloc(sizeof(double) * (size_t)dim);
    double t = 0.0, H = dt;
    int attempts = 0, status = 0;
    while (t < dt) {
        if (attempts >= max_steps) { status = 1; break; }
        attempts++;
        if (H > dt - t) H = dt - t;
        fn(ctx, y, f0);
        for (int64_t c = 0; c < dim; c++) sc[c] = fabs(y[c]) + fabs(H * f0[c]) + 1e-300;
        int accepted = 0, kconv = 0;
        for (int k = 0; k < BS_KMAX; k++) {
            int nk = 2 * (k + 1);
            double h = H / nk;
            for (int64_t c = 0; c < dim; c++) { zm[c] = y[c]; zn[c] = y[c] + h * f0[c]; }
            for (int mm = 1; mm < nk; mm++) {
                fn(ctx, zn, fz);
                for (int64_t c = 0; c < dim; c++) {
                    double tt = zm[c] + 2.0 * h * fz[c];
                    zm[c] = zn[c];
                    zn[c] = tt;
                }
            }
            fn(ctx, zn, fz);
            for (int64_t c = 0; c < dim; c++) yk[c] = 0.5 * (zn[c] + zm[c] + h * fz[c]);
            double err = 0.0;
            for (int64_t c = 0; c < dim; c++) {
                double prev = T[c];
                double cur = yk[c];
                T[c] = cur;
                for (int j = 1; j <= k; j++) {
                    double ratio = (double)nk / (double)(2 * (k - j + 1));
                    double nxt = cur + (cur - prev) / (ratio * ratio - 1.0);
                    prev = T[j * dim + c];
                    T[j * dim + c] = nxt;
                    cur = nxt;
                }
                if (k >= 1 && c < nerr) {
                    double e = fabs(T[k * dim + c] - T[(k - 1) * dim + c]) / sc[c];
                    if (e > err) err = e;
                }
            }
            if (k >= 1 && err <= tol) { accepted = 1; kconv = k; break; }
        }
        if (accepted) {
            for (int64_t c = 0; c < dim; c++) y[c] = T[kconv * dim + c];
            t += H;
            if (kconv < 4) H *= 1.5;
        } else {
            H *= 0.5;
        }
    }
    free(f0); free(T); free(yk); free(zm); free(zn); free(fz); free(sc);
    return status;
}

/* Group state and its tangent: y = [6 nm state | 6 nm tangent]. */
typedef struct tl_group {
    bs_group g;             /* members, partners, masses, rc (level 0), G, mu */
    const double *dm;       /* mass tangents (global) */
} tl_group;

static void tl_group_deriv(const void *ctxp, const double *y, double *f)
{
    const tl_group *ctx = (const tl_group *)ctxp;
    const bs_group *g = &ctx->g;
    int64_t nm = g->nm;
    bs_deriv(g, y, f);                           /* state part */
    const double *ty = y + 6 * nm;
    double *tf = f + 6 * nm;
    for (int64_t a = 0; a < nm; a++) {
        const double *xa = y + 6 * a;
        double r = sqrt((xa[0] * xa[0] + xa[1] * xa[1]) + xa[2] * xa[2]);
        double acc[3];
        /* star: d(-mu x/r^3) = -mu (I/r^3 - 3 x x^T / r^5) dx */
        double xs[3] = {xa[0], xa[1], xa[2]};
        pair_tensor_apply(xs, r, -g->mu, 0.0, ty + 6 * a, acc);
        int64_t ia = g->mem[a];
        double s[3] = {0.0, 0.0, 0.0};
        for (int64_t q = g->poff[a]; q < g->poff[a + 1]; q++) {
            int64_t b = g->plist[q], ib = g->mem[b];
            const double *xb = y + 6 * b;
            double d[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
            double dd = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            double rcij = g->rcl[0][ia] > g->rcl[0][ib] ? g->rcl[0][ia] : g->rcl[0][ib];
            double W = 1.0 - orc_changeover(dd, rcij);
            double Wp = -changeover_dr(dd, rcij);
            double e[3] = {ty[6 * b] - ty[6 * a], ty[6 * b + 1] - ty[6 * a + 1], ty[6 * b + 2] - ty[6 * a + 2]};
            double Me[3];
            pair_tensor_apply(d, dd, W, Wp, e, Me);
            double r3 = dd * dd * dd;
            for (int k = 0; k < 3; k++) s[k] += g->m[ib] * Me[k] + ctx->dm[ib] * W * d[k] / r3;
        }
        for (int k = 0; k < 3; k++) {
            tf[6 * a + k] = ty[6 * a + 3 + k];
            tf[6 * a + 3 + k] = acc[k] + g->G * s[k];
        }
    }
}

/* One step of the original scheme with frozen rc and pairs (R20); with the
 * tangent (dx, dv, dm) when dx != NULL (R21, R22).  rc: n; pairs ascending.  */
static int frozen_step(int64_t n, double *x, double *v, const double *m, const orc_params *p,
                       const double *rc, int64_t npairs, const uint32_t *pairs, double *dx,
                       double *dv, const double *dm)
{
    double dt = p->dt, h = 0.5 * dt, G = p->G, mu = p->G * p->m_star;
    size_t N3 = 3 * (size_t)(n > 0 ? n : 1);
    double *acc = (double *)malloc(sizeof(double) * N3);
    double *da = (double *)malloc(sizeof(double) * N3);
    double *xs = (double *)malloc(sizeof(double) * N3);
    double *vs = (double *)malloc(sizeof(double) * N3);
    int status = 0;
    /* Kick(dt/2) */
    orc_accel(n, x, m, rc, G, acc, p->nthreads);
    if (dx) {
        kick_tl(n, x, m, rc, G, dx, dm, da);
        for (size_t c = 0; c < 3 * (size_t)n; c++) dv[c] += h * da[c];
    }
    for (size_t c = 0; c < 3 * (size_t)n; c++) v[c] += h * acc[c];
    /* HC(dt/2) */
    if (dx) {
        double Q[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++)
            for (int k = 0; k < 3; k++) Q[k] += dm[j] * v[3 * j + k] + m[j] * dv[3 * j + k];
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < 3; k++) dx[3 * i + k] += h * Q[k] / p->m_star;
    }
    orc_hc(n, x, v, m, p->m_star, h);
    memcpy(xs, x, sizeof(double) * 3 * (size_t)n);
    memcpy(vs, v, sizeof(double) * 3 * (size_t)n);
    /* FG(dt) for everybody (members are overwritten by BS below) */
    int64_t *label = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    orc_group(n, npairs, pairs, label);
    if (orc_fg(n, x, v, mu, dt, p->kepler_max_iter)) status |= 1;
    if (dx) {
        /* tangent of the Kepler drift of non-members: variational equations */
        for (int64_t i = 0; i < n; i++) {
            if (label[i] >= 0) continue;
            int64_t mem = i, poff[2] = {0, 0}, plist = 0;
            bs_group g;
            g.nm = 1; g.mem = &mem; g.poff = poff; g.plist = &plist; g.m = m;
            const double *rcl[1] = {rc};
            g.rcl = rcl; g.nlev = 1; g.G = G; g.mu = mu; g.alive = NULL; g.gr_inv_c2 = 0.0;
            tl_group ctx; ctx.g = g; ctx.dm = dm;
            double y[12];
            for (int k = 0; k < 3; k++) {
                y[k] = xs[3 * i + k]; y[3 + k] = vs[3 * i + k];
                y[6 + k] = dx[3 * i + k]; y[9 + k] = dv[3 * i + k];
            }
            if (bs_generic(tl_group_deriv, &ctx, y, 12, 6, dt, p->bs_tol, p->bs_max_steps)) status |= 2;
            for (int k = 0; k < 3; k++) { dx[3 * i + k] = y[6 + k]; dv[3 * i + k] = y[9 + k]; }
        }
    }
    /* BS groups from the pre-drift state (with tangents) */
    if (npairs > 0) {
        int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
        int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * npairs + 1));
        if (build_partners(n, npairs, pairs, off, list) != 0) status |= 4;
        int64_t *loc = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *gsize = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        for (int64_t i = 0; i < n; i++)
            if (label[i] >= 0) loc[i] = gsize[label[i]]++;
        for (int64_t g0 = 0; g0 < n; g0++) {
            if (gsize[g0] == 0) continue;
            int64_t nm = gsize[g0];
            int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)nm);
            int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nm + 1));
            for (int64_t i = g0, c = 0; c < nm; i++)
                if (label[i] == g0) mem[c++] = i;
            poff[0] = 0;
            for (int64_t a = 0; a < nm; a++) poff[a + 1] = poff[a] + (off[mem[a] + 1] - off[mem[a]]);
            int64_t *plist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(poff[nm] > 0 ? poff[nm] : 1));
            for (int64_t a = 0; a < nm; a++)
                for (int64_t q = off[mem[a]], c = 0; q < off[mem[a] + 1]; q++, c++)
                    plist[poff[a] + c] = loc[list[q]];
            bs_group g;
            const double *rcl[1] = {rc};
            g.nm = nm; g.mem = mem; g.poff = poff; g.plist = plist; g.m = m;
            g.rcl = rcl; g.nlev = 1; g.G = G; g.mu = mu; g.alive = NULL; g.gr_inv_c2 = 0.0;
            int64_t dim = dx ? 12 * nm : 6 * nm;
            double *y = (double *)malloc(sizeof(double) * (size_t)dim);
            for (int64_t a = 0; a < nm; a++)
                for (int k = 0; k < 3; k++) {
                    y[6 * a + k] = xs[3 * mem[a] + k];
                    y[6 * a + 3 + k] = vs[3 * mem[a] + k];
                    if (dx) {
                        y[6 * nm + 6 * a + k] = dx[3 * mem[a] + k];
                        y[6 * nm + 6 * a + 3 + k] = dv[3 * mem[a] + k];
                    }
                }
            int fail;
            if (dx) {
                tl_group ctx; ctx.g = g; ctx.dm = dm;
                fail = bs_generic(tl_group_deriv, &ctx, y, dim, 6 * nm, dt, p->bs_tol, p->bs_max_steps);
            } else {
                int64_t a1 = 0, r1 = 0, m1 = 0;
                fail = bs_integrate(&g, y, dt, p->bs_tol, p->bs_max_steps, &a1, &r1, &m1, NULL);
            }
            if (fail) status |= 2;
            for (int64_t a = 0; a < nm; a++)
                for (int k = 0; k < 3; k++) {
                    x[3 * mem[a] + k] = y[6 * a + k];
                    v[3 * mem[a] + k] = y[6 * a + 3 + k];
                    if (dx) {
                        dx[3 * mem[a] + k] = y[6 * nm + 6 * a + k];
                        dv[3 * mem[a] + k] = y[6 * nm + 6 * a + 3 + k];
                    }
                }
            free(y); free(plist); free(poff); free(mem);
        }
        free(gsize); free(loc); free(list); free(off);
    }
    free(label);
    /* HC(dt/2) */
    if (dx) {
        double Q[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++)
            for (int k = 0; k < 3; k++) Q[k] += dm[j] * v[3 * j + k] + m[j] * dv[3 * j + k];
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < 3; k++) dx[3 * i + k] += h * Q[k] / p->m_star;
    }
    orc_hc(n, x, v, m, p->m_star, h);
    /* Kick(dt/2) */
    orc_accel(n, x, m, rc, G, acc, p->nthreads);
    if (dx) {
        kick_tl(n, x, m, rc, G, dx, dm, da);
        for (size_t c = 0; c < 3 * (size_t)n; c++) dv[c] += h * da[c];
    }
    for (size_t c = 0; c < 3 * (size_t)n; c++) v[c] += h * acc[c];
    free(acc); free(da); free(xs); free(vs);
    return status;
}

/* One normal step (slevels = 1) that also reports its level-0 rc (n values)
 * and encounter pairs (ascending, at most cap; *npairs = total).            */
int orc_step_record(int64_t n, double *x, double *v, const double *m, const orc_params *p,
                    double *rc_out, uint32_t *pairs_out, int64_t cap, int64_t *npairs)
{
    double dt = p->dt;
    orc_rcrit(n, x, v, m, p->m_star, dt, p->n1, p->n2, rc_out);
    int64_t nc = orc_precheck(n, x, rc_out, p->f_pc, NULL, 0);
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)(nc > 0 ? nc : 1));
    orc_precheck(n, x, rc_out, p->f_pc, cand, nc);
    /* detection needs the pre- and post-drift positions of this step */
    double *xa = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *va = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(xa, x, sizeof(double) * 3 * (size_t)n);
    memcpy(va, v, sizeof(double) * 3 * (size_t)n);
    orc_kick(n, xa, m, rc_out, p->G, 0.5 * dt, va, p->nthreads);
    orc_hc(n, xa, va, m, p->m_star, 0.5 * dt);
    double *xb = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *vb = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(xb, xa, sizeof(double) * 3 * (size_t)n);
    memcpy(vb, va, sizeof(double) * 3 * (size_t)n);
    orc_fg(n, xb, vb, p->G * p->m_star, dt, p->kepler_max_iter);
    uint32_t *enc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)(nc > 0 ? nc : 1));
    int64_t ne = orc_detect(nc, cand, xa, xb, rc_out, enc);
    *npairs = ne;
    for (int64_t k = 0; k < ne && k < cap; k++) { pairs_out[2 * k] = enc[2 * k]; pairs_out[2 * k + 1] = enc[2 * k + 1]; }
    int st = frozen_step(n, x, v, m, p, rc_out, ne, enc, NULL, NULL, NULL);
    free(cand); free(xa); free(va); free(xb); free(vb); free(enc);
    return st;
}

/* One step with frozen rc and pairs; with the tangent when dx != NULL.       */
int orc_step_frozen(int64_t n, double *x, double *v, const double *m, const orc_params *p,
                    const double *rc, int64_t npairs, const uint32_t *pairs, double *dx,
                    double *dv, const double *dm)
{
    return frozen_step(n, x, v, m, p, rc, npairs, pairs, dx, dv, dm);
}

/* ------------------------------------------------------------------------- */
/* Total energy (Eq. H = Ha + Hb + Hc, the K terms summing to the full pair
 * potential) and angular momentum sum_i m_i x_i x v_i, in long double with
 * Kahan summation.                                                          */
void orc_energy_tp(int64_t n, int64_t nm, const double *x, const double *v, const double *m,
                   double m_star, double G, double *E, double *L)
{
    long double sum = 0.0L, comp = 0.0L;
#define KAHAN_ADD(term) do { long double y_ = (term) - comp; long double t_ = sum + y_; \
        comp = (t_ - sum) - y_; sum = t_; } while (0)
    long double P[3] = {0.0L, 0.0L, 0.0L};
    long double Lx = 0.0L, Ly = 0.0L, Lz = 0.0L;
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i, *vi = v + 3 * i;
        long double v2 = (long double)vi[0] * vi[0] + (long double)vi[1] * vi[1] +
                         (long double)vi[2] * vi[2];
        long double r = sqrtl((long double)xi[0] * xi[0] + (long double)xi[1] * xi[1] +
                              (long double)xi[2] * xi[2]);
        KAHAN_ADD(0.5L * m[i] * v2);
        KAHAN_ADD(-(long double)G * m_star * m[i] / r);
        for (int k = 0; k < 3; k++) P[k] += (long double)m[i] * vi[k];
        Lx += (long double)m[i] * ((long double)xi[1] * vi[2] - (long double)xi[2] * vi[1]);
        Ly += (long double)m[i] * ((long double)xi[2] * vi[0] - (long double)xi[0] * vi[2]);
        Lz += (long double)m[i] * ((long double)xi[0] * vi[1] - (long double)xi[1] * vi[0]);
    }
    for (int64_t i = 0; i < n; i++) {
        const double *xi = x + 3 * i;
        long double part = 0.0L;
        const int64_t jend = i >= nm ? i + 1 : n;   /* no test-particle pair term (R24) */
        for (int64_t j = i + 1; j < jend; j++) {
            const double *xj = x + 3 * j;
            long double dx = (long double)xj[0] - xi[0], dy = (long double)xj[1] - xi[1],
                        dz = (long double)xj[2] - xi[2];
            part += (long double)m[j] / sqrtl(dx * dx + dy * dy + dz * dz);
        }
        KAHAN_ADD(-(long double)G * m[i] * part);
    }
    KAHAN_ADD((P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0L * m_star));
#undef KAHAN_ADD
    *E = (double)sum;
    L[0] = (double)Lx; L[1] = (double)Ly; L[2] = (double)Lz;
}

void orc_energy(int64_t n, const double *x, const double *v, const double *m, double m_star,
                double G, double *E, double *L)
{
    orc_energy_tp(n, n, x, v, m, m_star, G, E, L);
}

/* Size of the parameter and statistics structs, for the loader's layout check. */
int64_t orc_sizeof_params(void) { return (int64_t)sizeof(orc_params); }
int64_t orc_sizeof_stats(void) { return (int64_t)sizeof(orc_stats); }
int64_t orc_sizeof_nn(void) { return (int64_t)sizeof(orc_nn); }
