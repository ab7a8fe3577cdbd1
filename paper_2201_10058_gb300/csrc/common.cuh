// common.cuh -- internal declarations of the GB300 hybrid symplectic library.
// Device helpers, the system object and the kernel launchers shared by the
// translation units.  Nothing here is part of the public ABI (include/genga.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/genga.h"

namespace genga {

constexpr int kMaxLevels = 8;
// All-pairs kicks split the sources into at most this many chunks: the chunk
// partial sums take nchunk x (4 or 6) doubles per body, so beyond it a larger N
// widens the chunks instead of adding chunks.
constexpr int kMaxKickChunks = 64;
// Close-encounter groups with more members than this are integrated by the
// batched grid-wide Bulirsch-Stoer driver (bsm.cu) instead of one thread block.
constexpr int kBlockGroupMax = 32;
// Group size buckets: up to 4, 8, 16 and 32 members (in-block kernels), larger.
constexpr int kBuckets = 5;

// Device error word bits (latched; read by the host after synchronising).
enum : unsigned {
    kErrKepler = 1u,      // Kepler Newton iteration limit
    kErrBS = 2u,          // Bulirsch-Stoer step-attempt limit
    kErrCandCap = 4u,     // candidate list overflow (recovered by the host)
    kErrPairCap = 8u,     // encounter list overflow (recovered by the host)
    kErrBadState = 16u,   // NaN / Inf / body at the origin
    kErrUnionFind = 32u,  // bounded union-find retry loop gave up
    kErrTimeout = 64u,    // an in-block Bulirsch-Stoer group call hit its time limit
    kErrMergeLog = 128u,  // the merger log is full
};

// One merger record of the device log: Bulirsch-Stoer call, group label,
// sequence number in the group, time in the call, i, j, r_ij, R_i + R_j, dU.
constexpr int kMergeRec = 9;

// Counters that live in device memory.
struct DevCounters {
    unsigned long long cand_count;
    unsigned long long pair_count[kMaxLevels];
    unsigned long long nbodies[kMaxLevels];
    unsigned long long kepler_fail;
    unsigned long long bs_steps;
    unsigned long long bs_rejects;
    unsigned long long bs_fail;
    unsigned long long groups_total;     // groups formed since the last reset
    unsigned long long max_group_total;  // largest of them
    unsigned long long bs_max_attempts;  // most step attempts of one group
    unsigned long long pair_total[kMaxLevels];   // pairs found at levels whose count stays on the device
    unsigned int err;
    unsigned int ngroups;
    unsigned int max_group;
    unsigned int hc_done;                  // blocks of hc_reduce_kernel finished (reset by the last)
    double hc_shift[3];
    unsigned int bucket_count[kBuckets];   // groups per size bucket (bucket_groups)
    unsigned int pad2[8 - kBuckets];
    unsigned int bucket_next[kBuckets];    // next group of each bucket to claim (persistent BS kernels)
    unsigned int pad3[8 - kBuckets];
    unsigned long long merge_count;        // records written to the merger log
};

// Collision state handed to the Bulirsch-Stoer kernels (Sec. 7.1-7.2).
struct CollArgs {
    int on;                       // collisions switched on
    double tol;                   // collision precision (0: merge at the first overlapping step)
    double *mass;                 // = the system's masses, written by mergers
    double *radius, *spin;        // radii (n), spins (3n, component-major)
    unsigned char *alive;         // n
    double *log;                  // merger records (kMergeRec doubles each)
    unsigned long long log_cap;   // records
    long long call;               // index of this Bulirsch-Stoer call
    double G;
    int64_t n;                    // bodies (the stride of spin)
};

// Level-independent per-body data of the critical radius (level 0 uses all).
struct RcritArrays {
    double *rc = nullptr;    // rc_i
    double *rc2 = nullptr;   // rc_i^2 (pair value: max of the two, exact)
    double *pc2 = nullptr;   // (f_pc rc_i)^2 (level 0 only)
    float *thr_rc = nullptr; // conservative FP32 upper bound of rc_i^2 (level 0 only)
    double *irc = nullptr;   // 1 / rc_i, correctly rounded (so min(irc_i, irc_j) = 1 / rc_ij exactly)
};

// CSR partner lists (both directions) of one pair list.
struct Csr {
    int *deg = nullptr;    // n+1
    int *off = nullptr;    // n+1 (exclusive scan of deg)
    int *fill = nullptr;   // n
    int *list = nullptr;   // 2 * cap: partner of each entry
    int *lpair = nullptr;  // 2 * cap: 2 k + d for the entry of pair k in the row of its body d (0: pairs[k].x, 1: pairs[k].y)
    int *ent = nullptr;    // 2 * cap: the inverse, entry of 2 k + d in the sorted rows
    double *term = nullptr;  // 8 * cap: the mass-weighted KickS term (x, y, z, pad) of each entry
    int64_t cap = 0;       // pairs
};

struct Scratch {
    // scan temporaries
    int *scan_blocks = nullptr;
    int scan_blocks_cap = 0;
};

}  // namespace genga

struct genga_system {
    genga_params_t p;
    int64_t n = 0;
    double *pos = nullptr;         // caller-owned, 3n
    double *vel = nullptr;         // caller-owned, 3n
    const double *mass = nullptr;  // caller-owned, n
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;

    genga::DevCounters *ctr = nullptr;   // device
    genga::RcritArrays rcl[genga::kMaxLevels];
    double *pre_pos[genga::kMaxLevels] = {};  // pre-drift copies, 3n each
    double *pre_vel[genga::kMaxLevels] = {};

    // all-pairs kick
    double *kick_part = nullptr;   // [max(nchunk, ksym_nS)][6][n]
    size_t kick_part_cap = 0;      // doubles allocated
    int kick_nchunk = 0;
    int kick_chunk = 0;
    // symmetric kick (each unordered pair once): geometry for (ksym_n, ksym_prec)
    int64_t ksym_n = -1;
    int ksym_prec = -1;
    int ksym_nm = -1;              // large bodies (tp_bound) the geometry was chosen for
    int ksym_R = 0;                // super-ranges holding large bodies: slots a test particle has
    int ksym_layout = 0;           // GENGA_KICK_AUTO / _TILED / _SYMMETRIC requested
    int ksym_req_P = 0;            // requested P (0: chosen)
    int ksym_P = 0;                // super-range in tiles; 0: not used at this N
    int ksym_nS = 0;               // partial slots per body
    int ksym_blocks = 0;           // persistent blocks
    int ksym_items = 0;
    int2 *ksym_list = nullptr;     // dispatch order of the super-tile pairs
    size_t ksym_list_cap = 0;
    unsigned *ksym_ctr = nullptr;  // dispatch counter
    double *ksym_irc = nullptr;    // 1 / rc per body
    float2 *ksym_ircf = nullptr;   // the same as two floats
    float2 *ksym_mhl = nullptr;    // mass as two floats
    float *ksym_thrpc = nullptr;   // FP32 upper bound of (f_pc rc)^2
    float2 *ksym_pcf = nullptr;    // (f_pc rc)^2 as two floats
    size_t ksym_body_cap = 0;

    // candidates and encounter lists
    uint2 *cand = nullptr;
    int64_t cand_cap = 0;
    uint2 *pairs[genga::kMaxLevels] = {};
    int64_t pair_cap[genga::kMaxLevels] = {};
    int64_t npairs_host[genga::kMaxLevels] = {};
    genga::Csr csr[genga::kMaxLevels];
    int *bodies[genga::kMaxLevels] = {};   // level body lists (ascending)
    int *flags = nullptr;                  // n+1 scan input

    // grouping
    int *parent = nullptr;   // n
    int *label = nullptr;    // n
    int *gsize = nullptr;    // n+1
    int *goff = nullptr;     // n+1
    int *gfill = nullptr;    // n
    int *glist = nullptr;    // n
    int *member = nullptr;   // n
    int *slotof = nullptr;   // n
    int *bucket_list = nullptr;  // kBuckets x bucket_stride group labels per size bucket
    int bucket_stride = 0;       // n / 2 + 1 (groups have at least 2 members)
    unsigned *bucket_host = nullptr;  // pinned copy of the bucket counts
    unsigned long long *np_host = nullptr;  // pinned copies of the levels' last pair counts (kMaxLevels)
    cudaEvent_t ev_counts = nullptr;  // recorded after that copy
    int label_level = -1;    // level whose grouping `label` holds

    // batched grid-wide Bulirsch-Stoer buffers (bsm.cu), grown on demand
    void *bsm = nullptr;

    // HC / energy reductions
    double *red = nullptr;   // reduction scratch

    genga::Scratch scr;
    cudaStream_t side[4] = {};     // library-owned streams for concurrent BS buckets
    cudaEvent_t ev_fork = nullptr, ev_join[4] = {};
    genga_stats_t stats;
    void *adj = nullptr;           // adjoint recording (adjoint.cu)
    // collisions (genga_set_collisions)
    bool coll_on = false;
    double coll_tol = 0.0;
    double *radius = nullptr;          // caller-owned, n
    double *spin = nullptr;            // caller-owned, 3n
    unsigned char *alive = nullptr;    // library-owned, n
    double *mlog = nullptr;            // library-owned merger records
    int64_t mlog_cap = 0;
    long long bs_call = 0;             // Bulirsch-Stoer calls since collisions were switched on
    // bounded device waits (genga_set_wait_limits)
    unsigned long long bs_group_limit_ns = 10000000000ull;   // in-block BS, per group call
    unsigned long long barrier_limit_ns = 2000000000ull;     // persistent BS, per grid-barrier wait
    unsigned barrier_absent = 0;   // test hook: blocks every grid barrier waits for in vain
    int bs_pairs = 0;              // GENGA_BS_PAIRS_*: derivative form of the persistent BS kernel
    int64_t launches = 0;          // kernels launched by this system (host-side count)
    int64_t host_syncs = 0;        // host waits on the stream inside steps
    // phase timing (genga_set_timing): an event on the stream at each phase
    // boundary; after a step the intervals are added to the phase sums
    bool timing = false;
    std::vector<cudaEvent_t> mark_ev;
    std::vector<int> mark_phase;
    size_t nmarks = 0;
    double phase_ms[GENGA_NPHASES] = {};
    int64_t timed_steps = 0;
    // detection log (genga_set_pair_log): level and sorted pairs of every detection
    bool pair_log = false;
    std::vector<int32_t> log_level;
    std::vector<int64_t> log_off;
    std::vector<uint32_t> log_pairs;
    char err[512] = {0};
};

// Test-particle boundary (Sec. 8.1 semi-active mode): bodies i >= the bound are
// test particles that do not interact with one another; n when there are none.
inline int tp_bound(const genga_system *s) {
    if (s->p.tp_mode != 2) return (int)s->n;
    return (int)std::min<int64_t>(std::max<int64_t>(s->p.n_massive, 0), s->n);
}

namespace genga {

// ---------------------------------------------------------------------------
// Device helpers.

// Changeover function of Chambers (1999) Eq. 10 as used in Sec. 6.3:
// y = (r/rc - 0.1)/0.9 clamped to [0,1], K = y^2/(2y^2 - 2y + 1).  Written with
// explicit round-to-nearest operations (no contraction).
__device__ __forceinline__ double changeover(double r, double rc) {
    double y = __ddiv_rn(__dsub_rn(__ddiv_rn(r, rc), 0.1), 0.9);
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    double y2 = __dmul_rn(y, y);
    double den = __dadd_rn(__dsub_rn(__dmul_rn(2.0, y2), __dmul_rn(2.0, y)), 1.0);
    return __ddiv_rn(y2, den);
}

// Squared distance in the detection order (dx^2 + dy^2) + dz^2, no contraction.
__device__ __forceinline__ double dist2_rn(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Error-free sum: s + e = a + b exactly (Knuth TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// The same error-free sum in 3 FP64 operations: Dekker's Fast2Sum on the
// operands ordered by exponent.  The high words with the sign cleared compare
// as unsigned integers in the order of the exponents (ties: equal exponents,
// where either order is exact), so the ordering costs no FP64 operation.  For
// finite a and b the rounding error is representable and unique, so s and e
// equal two_sum()'s (up to the sign of a zero e).
__device__ __forceinline__ void two_sum_ordered(double a, double b, double &s, double &e) {
    const unsigned ha = (unsigned)__double2hiint(a) & 0x7fffffffu;
    const unsigned hb = (unsigned)__double2hiint(b) & 0x7fffffffu;
    const bool ge = ha >= hb;
    const double big = ge ? a : b, small = ge ? b : a;
    s = __dadd_rn(big, small);
    e = __dsub_rn(small, __dsub_rn(s, big));
}

__device__ __forceinline__ void latch_error(DevCounters *c, unsigned bit) { atomicOr(&c->err, bit); }

// ---------------------------------------------------------------------------
// Host launchers (defined in the .cu files).  All take the system's stream.

// particle.cu
cudaError_t launch_rcrit(genga_system *s, int level, double dt, const int *bodies, int nb);
cudaError_t launch_rcrit_derive(genga_system *s);   // thresholds from rcl[0].rc
cudaError_t launch_hc(genga_system *s, double dt_half);
cudaError_t launch_drift(genga_system *s, int level, double dt, const int *bodies, int nb);
cudaError_t launch_restore(genga_system *s, int from_level, const int *bodies, int nb);
cudaError_t launch_energy(genga_system *s, double *E_host, double *L_host);

// kick.cu
cudaError_t launch_kick(genga_system *s, double dt_half, bool precheck, double *acc_out);
cudaError_t kick_reserve(genga_system *s);
cudaError_t launch_precheck_only(genga_system *s);
int kick_nchunk_for(int n, int num_sms);

// Kick on caller-provided arrays (no system object, no pre-check).
struct KickRaw {
    const double *pos, *mass, *rc, *rc2;
    const float *thr;
    double *part;        // partial sums, [nchunk][6][n]
    int n;
    double G, dt_half;
    double *vel, *acc_out;
    bool mixed;
};
cudaError_t launch_kick_raw(const KickRaw &k, int num_sms, int max_nchunk, cudaStream_t stream);

// encounter.cu
cudaError_t launch_detect(genga_system *s, const uint2 *in, int64_t nin, int level,
                          uint2 *out, int64_t cap, unsigned long long *count);
// npairs: the pair count, or, with npd (the count the detection left on the
// device), a bound on it that sizes the grids; total: a device sum the count
// is added to (levels whose count the host does not read); np_hint: with npd,
// a recent count of the level that picks the row sort.
cudaError_t build_csr(genga_system *s, int level, int64_t npairs, const unsigned long long *npd = nullptr,
                      unsigned long long *total = nullptr, int64_t np_hint = 0);
cudaError_t build_bodies(genga_system *s, int level_pairs, int out_level, int *nb_host);
cudaError_t build_groups(genga_system *s, int level, int64_t npairs, const unsigned long long *npd = nullptr);
cudaError_t exclusive_scan(genga_system *s, const int *in, int *out, int64_t len);

// genga.cu
int ensure_pair_capacity(genga_system *s, int level, int64_t np);
// collide.cu: the collision arguments of the system for the next
// Bulirsch-Stoer call (on = 0 when collisions are off)
CollArgs coll_args(const genga_system *s);
// Phase timing: from here on, stream time counts for `phase` (no-op when off).
int phase_mark(genga_system *s, int phase);
// adjoint.cu
void adjoint_free(genga_system *s);

// bs.cu
// Batched grid-wide Bulirsch-Stoer of the groups larger than kBlockGroupMax
// (bsm.cu); genga error codes.
int bsm_forward_groups(genga_system *s, int level, double dt_l);
void bsm_release(genga_system *s);
// launch_bs and join_bs, then bsm_forward_groups.
int run_bs(genga_system *s, int level, double dt_l, int64_t np);
// The same without reading the group counts first: the in-block kernels take
// the device counts; the host waits only for the counts' copy (made before the
// kernels run) to decide on the groups larger than kBlockGroupMax.
int run_bs_dev(genga_system *s, int level, double dt_l);
int bsm_adjoint_groups(genga_system *s, const double *x2, const double *v2, double *lx, double *lv,
                       double *lm, double dt);
// Sorts the current groups into the size buckets (device lists + counts) and
// copies the kBuckets counts to the host (synchronises).
cudaError_t bucket_groups(genga_system *s, unsigned counts[kBuckets]);
// The same, the counts copied to s->bucket_host behind the event s->ev_counts
// (no wait).
cudaError_t bucket_groups_async(genga_system *s);
// Launches the in-block BS kernels on the side streams (forked from the
// system stream) for the first four buckets: with counts, one block per group
// (up to the resident capacity); without, the resident capacity, the blocks
// claiming the device counts.  join_bs makes the system stream wait for them.
cudaError_t launch_bs(genga_system *s, int level, double dt_l, const unsigned *counts);
cudaError_t join_bs(genga_system *s);
cudaError_t launch_kick_pairs(genga_system *s, int level, double dt_half, int nb);

// ---------------------------------------------------------------------------
// Kepler drift (Eq. Ha, Kepler term).
// Stumpff functions c_k(z) = sum_m (-z)^m/(2m+k)!: quarter z until |z| <= 0.1,
// sum the series for c2 and c3 (ten terms), c0 = 1 - z c2, c1 = 1 - z c3, then
// undo the quartering with c0(4z) = 2c0^2 - 1, c1(4z) = c0 c1,
// c2(4z) = c1^2/2, c3(4z) = (c2 + c0 c3)/4.
__device__ __forceinline__ void stumpff(double z, double &c0, double &c1, double &c2, double &c3) {
    int q = 0;
    while (fabs(z) > 0.1 && q < 60) { z *= 0.25; q++; }
    // 1/(2m+2)! and 1/(2m+3)!, m = 0..9
    const double ic2[10] = {1.0 / 2.0, 1.0 / 24.0, 1.0 / 720.0, 1.0 / 40320.0, 1.0 / 3628800.0,
                            1.0 / 479001600.0, 1.0 / 87178291200.0, 1.0 / 20922789888000.0,
                            1.0 / 6402373705728000.0, 1.0 / 2432902008176640000.0};
    const double ic3[10] = {1.0 / 6.0, 1.0 / 120.0, 1.0 / 5040.0, 1.0 / 362880.0,
                            1.0 / 39916800.0, 1.0 / 6227020800.0, 1.0 / 1307674368000.0,
                            1.0 / 355687428096000.0, 1.0 / 121645100408832000.0,
                            1.0 / 51090942171709440000.0};
    double s2 = 0.0, s3 = 0.0;
#pragma unroll
    for (int m = 9; m >= 0; m--) {
        s2 = ic2[m] - z * s2;
        s3 = ic3[m] - z * s3;
    }
    double C2 = s2, C3 = s3, C0 = 1.0 - z * C2, C1 = 1.0 - z * C3;
    for (int k = 0; k < q; k++) {
        const double n3 = 0.25 * (C2 + C0 * C3);
        const double n2 = 0.5 * C1 * C1;
        const double n1 = C0 * C1;
        const double n0 = 2.0 * C0 * C0 - 1.0;
        C0 = n0; C1 = n1; C2 = n2; C3 = n3;
    }
    c0 = C0; c1 = C1; c2 = C2; c3 = C3;
}

// Kepler drift of one body over dt about mu.  Universal variable s with
// beta = 2 mu / r0 - v0^2, G_k = s^k c_k(beta s^2):
//   t(s) = r0 G1 + u G2 + mu G3 (u = x0.v0),  dt/ds = r(s) = r0 G0 + u G1 + mu G2,
//   f - 1 = -mu G2 / r0, g = dt - mu G3, fdot = -mu G1/(r r0), gdot - 1 = -mu G2 / r.
// Newton from s = dt/r0 - u dt^2/(2 r0^3); converged when |ds| <= 1e-15 |s|, or
// when rounding stalls the update at |ds| <= 1e-12 |s| without halving it.
__device__ __forceinline__ bool kepler_solve_s(double r0, double u, double beta, double mu,
                                               double dt, int max_iter, double &s_out) {
    double s = dt / r0 - (u * dt * dt) / (2.0 * r0 * r0 * r0);
    double c0, c1, c2, c3, ds_prev = 0.0;
    bool ok = false;
    for (int it = 0; it < max_iter; it++) {
        stumpff(beta * s * s, c0, c1, c2, c3);
        const double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
        const double t = r0 * G1 + u * G2 + mu * G3;
        const double rr = r0 * c0 + u * G1 + mu * G2;
        const double ds = (t - dt) / rr;
        s -= ds;
        const double ads = fabs(ds), as = fabs(s);
        if (ads <= 1e-15 * as) { ok = true; break; }
        if (it > 0 && ads <= 1e-12 * as && ads > 0.5 * ds_prev) { ok = true; break; }
        ds_prev = ads;
    }
    s_out = s;
    return ok;
}

__device__ __forceinline__ bool kepler_drift(double &x, double &y, double &z, double &vx, double &vy, double &vz,
                                             double mu, double dt, int max_iter) {
    const double r0 = sqrt(x * x + y * y + z * z);
    const double v2 = vx * vx + vy * vy + vz * vz;
    const double u = x * vx + y * vy + z * vz;
    const double beta = 2.0 * mu / r0 - v2;
    double s;
    const bool ok = kepler_solve_s(r0, u, beta, mu, dt, max_iter, s);
    double c0, c1, c2, c3;
    stumpff(beta * s * s, c0, c1, c2, c3);
    const double G1 = s * c1, G2 = s * s * c2, G3 = s * s * s * c3;
    const double r = r0 * c0 + u * G1 + mu * G2;
    const double fm1 = -mu * G2 / r0;
    const double g = dt - mu * G3;
    const double fd = -mu * G1 / (r * r0);
    const double gdm1 = -mu * G2 / r;
    const double x0 = x, y0 = y, z0 = z, vx0 = vx, vy0 = vy, vz0 = vz;
    x = x0 + (fm1 * x0 + g * vx0);
    y = y0 + (fm1 * y0 + g * vy0);
    z = z0 + (fm1 * z0 + g * vz0);
    vx = vx0 + (fd * x0 + gdm1 * vx0);
    vy = vy0 + (fd * y0 + gdm1 * vy0);
    vz = vz0 + (fd * z0 + gdm1 * vz0);
    return ok;
}

// dK/dr of changeover() (zero outside the transition band 0.1 rc < r < rc).
__device__ __forceinline__ double changeover_dr_dev(double r, double rc) {
    const double y = (r / rc - 0.1) / 0.9;
    if (y <= 0.0 || y >= 1.0) return 0.0;
    const double D = 2.0 * y * y - 2.0 * y + 1.0;
    return 2.0 * y * (1.0 - y) / (D * D) / (0.9 * rc);
}

// ---------------------------------------------------------------------------
// FP64 reciprocal square root and reciprocal from an FP32 hardware seed plus
// Newton steps in FP64 (two steps reach full double precision).  The seed's
// conversions use integer bit manipulation (no FP64 pipe work); inputs must be
// positive normal doubles within the FP32 exponent range.
__device__ __forceinline__ float f32_of_f64_trunc(double v) {
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    return __uint_as_float(((hi - 0x38000000u) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f64_of_f32(float f) {
    const unsigned fb = __float_as_uint(f);
    return __hiloint2double((int)((fb >> 3) + 0x38000000u), (int)(fb << 29));
}
__device__ __forceinline__ double half_of(double y) {   // y / 2 for positive normal y
    return __hiloint2double(__double2hiint(y) - 0x00100000, __double2loint(y));
}
// Float nearest (ties away from zero) to a double of magnitude in
// [2^-126, 2^128), any sign; smaller magnitudes give a signed zero.  Integer
// operations only.
__device__ __forceinline__ float f32_of_f64_rn(double v) {
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const unsigned mag = hi & 0x7fffffffu, sgn = hi & 0x80000000u;
    const unsigned fb = (mag >= 0x38100000u)
                            ? (sgn | ((((mag - 0x38000000u) << 3) | (lo >> 29)) + ((lo >> 28) & 1u)))
                            : sgn;
    return __uint_as_float(fb);
}
__device__ __forceinline__ double rsqrt_newton(double x) {
    // one residual e = 1 - x y0^2 of the ~2^-22 seed and the series
    // x^-1/2 = y0 (1 - e)^-1/2 = y0 (1 + e/2 + 3 e^2/8 + O(e^3)): a chain of 5
    // dependent FP64 operations (two Newton steps take 6), error ~2^-64 + rounding
    const double y0 = f64_of_f32(rsqrtf(f32_of_f64_trunc(x)));
    const double t = x * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(0.375, e, 0.5);
    return fma(y0, e * p, y0);
}
__device__ __forceinline__ double rcp_newton(double d) {
    float s;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(f32_of_f64_trunc(d)));
    double x = f64_of_f32(s);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const double e = fma(-d, x, 1.0);
        x = fma(x, e, x);
    }
    return x;
}
// Changeover function with the reciprocal 1/rc supplied; same definition as
// changeover() (y = (r/rc - 0.1)/0.9, K = y^2/(2y^2 - 2y + 1)), evaluated with
// contracted FP64 arithmetic for force terms (not for decisions).
__device__ __forceinline__ double changeover_fast(double r, double irc) {
    const double y = fma(r, irc, -0.1) * (1.0 / 0.9);
    if (y <= 0.0) return 0.0;
    if (y >= 1.0) return 1.0;
    const double y2 = y * y;
    const double w = 1.0 - y;
    return y2 * rcp_newton(fma(w, w, y2));
}
// Side of the changeover band from FP32 copies of r (f32_of_f64_trunc of a
// positive normal double in the FP32 range) and of 1/rc (__double2float_rz):
// -1 when r/rc < 0.1 for certain (K = 0 exactly in changeover_fast), +1 when
// r/rc > 1 for certain (K = 1 exactly), 0 otherwise (evaluate K).  Both copies
// are truncations, < 2^-23 low each, and the product rounds by <= 2^-24, so the
// float product lies in [x (1 - 2^-22), x (1 + 2^-24)] of x = r/rc; the
// margins 0.09999 and 1.0001 are far wider, so both decisions are exact.  An
// infinite 1/rc (rc = 0) gives +1, as K = 1 there.
__device__ __forceinline__ int changeover_side_f32(float rf, float ircf) {
    const float p = rf * ircf;
    return p < 0.09999f ? -1 : (p > 1.0001f ? 1 : 0);
}

// K and dK/dr with 1/rc supplied: the definitions of changeover() and
// changeover_dr_dev() (dK/dy = 2y(1 - y)/D^2, D = y^2 + (1 - y)^2, dy/dr = 1/(0.9 rc)),
// in contracted FP64 arithmetic for force terms.
__device__ __forceinline__ void changeover_fast_dr(double r, double irc, double &K, double &dK) {
    const double y = fma(r, irc, -0.1) * (1.0 / 0.9);
    if (y <= 0.0) { K = 0.0; dK = 0.0; return; }
    if (y >= 1.0) { K = 1.0; dK = 0.0; return; }
    const double y2 = y * y;
    const double w = 1.0 - y;
    const double iD = rcp_newton(fma(w, w, y2));
    K = y2 * iD;
    dK = 2.0 * y * w * (iD * iD) * (irc * (1.0 / 0.9));
}

// ---------------------------------------------------------------------------
// Float-float helpers of the mixed-precision pair kicks (kick.cu, ensemble.cu).
// (hi, lo) += v in float-float: TwoSum of hi and v, the rounding error into lo.
__device__ __forceinline__ void float_two_sum_acc(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

// Double with the value of a float (exact), for any sign; zero and subnormal
// floats give a signed zero.  Integer operations only.
__device__ __forceinline__ double f64_of_f32_any(float f) {
    const unsigned fb = __float_as_uint(f);
    const unsigned mag = fb & 0x7fffffffu, sgn = fb & 0x80000000u;
    const unsigned hi = (mag >= 0x00800000u) ? (sgn | ((mag >> 3) + 0x38000000u)) : sgn;
    const unsigned lo = (mag >= 0x00800000u) ? (mag << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// 1/rc as two floats (an infinite 1/rc keeps a zero low part).
__device__ __forceinline__ float2 ff_of_irc(double ir) {
    const float h = __double2float_rn(ir);
    return make_float2(h, isinf(h) ? 0.0f : __double2float_rn(ir - (double)h));
}

// Float-float helpers of the mixed kicks' changeover band (kick.cu, bs.cu).
__device__ __forceinline__ void ff_fast2sum(float &h, float &l) {      // |h| >= |l|
    const float s = h + l;
    l = l - (s - h);
    h = s;
}
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (ah, al) *= (bh, bl)
__device__ __forceinline__ void ff_mul(float &ah, float &al, float bh, float bl) {
    const float ph = ah * bh;
    float pl = fmaf(ah, bh, -ph);
    pl = fmaf(ah, bl, pl);
    pl = fmaf(al, bh, pl);
    ah = ph;
    al = pl;
    ff_fast2sum(ah, al);
}

// The changeover function K of Sec. 6.3 (y = (r/rc - 0.1)/0.9 clamped to
// [0, 1], K = y^2 / (y^2 + (1 - y)^2)) in float-float, from what the mixed kick
// already holds: r = r^2 r^-1 with r^2 = Rh + Rl, Rh y0 = u + ue exactly and
// r^-1 = y0 (1 + e/2 + 3e^2/8) for the residual e, and 1/rc_ij as two floats.
// Absolute error of K ~2^-44 (the FP64 form's to rounding), on the FP32 pipe:
// the band's pairs are few and scattered, and the FP64 pipe would charge each
// one's whole warp.
__device__ __forceinline__ void changeover_ff(float u, float ue, float Rl, float y0f, float ef, float ih, float il,
                                              float &Kh, float &Kl) {
    // 0.1 and 1/0.9 (the doubles of the FP64 form) as float pairs
    constexpr float c01h = 0.100000001490116119384765625f, c01l = -1.4901161415892261e-09f;
    constexpr float c9h = 1.1111111640930176f, c9l = -5.298190686175985e-08f;
    float rh = u;
    float rl = ue + fmaf(Rl, y0f, u * fmaf(0.375f * ef, ef, 0.5f * ef));
    ff_fast2sum(rh, rl);
    ff_mul(rh, rl, ih, il);                                       // r / rc
    float dh, dl;
    ff_two_sum(rh, -c01h, dh, dl);
    dl += rl - c01l;
    ff_fast2sum(dh, dl);
    ff_mul(dh, dl, c9h, c9l);                                     // y
    if (dh <= 0.0f) { Kh = 0.0f; Kl = 0.0f; return; }
    if (dh >= 1.0f) { Kh = 1.0f; Kl = 0.0f; return; }
    float ah = dh, al = dl;
    ff_mul(ah, al, dh, dl);                                       // y^2
    float wh, wl;
    ff_two_sum(1.0f, -dh, wh, wl);
    wl -= dl;
    ff_fast2sum(wh, wl);
    ff_mul(wh, wl, wh, wl);                                       // (1 - y)^2
    float Dh, Dl;
    ff_two_sum(ah, wh, Dh, Dl);
    Dl += al + wl;
    ff_fast2sum(Dh, Dl);                                          // D in [1/2, 1]
    float qh = ah / Dh;
    const float ph = qh * Dh;
    float pl = fmaf(qh, Dh, -ph);
    pl = fmaf(qh, Dl, pl);
    float ql = (((ah - ph) - pl) + al) / Dh;
    ff_fast2sum(qh, ql);
    Kh = qh;
    Kl = ql;
}

// v = hi + lo exactly up to 2^-47 |v|: hi is v with the mantissa truncated
// to float precision, lo the 29 discarded mantissa bits rounded to a float.
// Integer operations, one integer-to-float conversion and one FP32 scale;
// |v| < 2^-74 gives lo = 0, |v| < 2^-126 also hi = 0 (signed zeros).
__device__ __forceinline__ void split_f64(double v, float &hi, float &lo) {
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned mag = hw & 0x7fffffffu, sgn = hw & 0x80000000u;
    const bool normal = mag >= 0x38100000u;
    hi = __uint_as_float(normal ? (sgn | ((mag - 0x38000000u) << 3) | (lw >> 29)) : sgn);
    const unsigned E = mag >> 20;                       // biased double exponent
    float l = 0.0f;
    if (E >= 949u) l = __uint2float_rn(lw & 0x1fffffffu) * __uint_as_float((E - 948u) << 23);
    lo = __uint_as_float(__float_as_uint(l) | sgn);
}

// ---------------------------------------------------------------------------
// Collisions (Sec. 7.1): one perfectly inelastic merger of bodies i < j with
// states (xi, vi), (xj, vj), in the operations and order of the definition
// without contraction.  The survivor (the more massive body; equal masses:
// the lower index) gets the summed mass, the radius of the summed R^3 and the
// spin S_i + S_j + mu (r_ij x v_ij), and its new position and velocity go to
// xo, vo (the other body keeps its own); the other body gets mass, radius and
// spin 0 and is marked not alive.  Returns the survivor; *dU receives
// mu |v_ij|^2 / 2 - G m_i m_j / r_ij, *r the separation.
__device__ __forceinline__ int merge_bodies(const CollArgs &C, size_t N, int i, int j, const double *xi,
                                            const double *vi, const double *xj, const double *vj,
                                            double *xo, double *vo, double *dU, double *r_out) {
    const double mi = C.mass[i], mj = C.mass[j], M = __dadd_rn(mi, mj);
    double r[3], w[3];
    for (int k = 0; k < 3; k++) {
        r[k] = __dsub_rn(xi[k], xj[k]);
        w[k] = __dsub_rn(vi[k], vj[k]);
    }
    const double rr = __dsqrt_rn(dist2_rn(r[0], r[1], r[2]));
    const double w2 = dist2_rn(w[0], w[1], w[2]);
    double mu = 0.0;
    if (M > 0.0) {
        mu = __ddiv_rn(__dmul_rn(mi, mj), M);
        for (int k = 0; k < 3; k++) {
            xo[k] = __ddiv_rn(__dadd_rn(__dmul_rn(xi[k], mi), __dmul_rn(xj[k], mj)), M);
            vo[k] = __ddiv_rn(__dadd_rn(__dmul_rn(vi[k], mi), __dmul_rn(vj[k], mj)), M);
        }
    } else {
        for (int k = 0; k < 3; k++) {
            xo[k] = __dmul_rn(0.5, __dadd_rn(xi[k], xj[k]));
            vo[k] = __dmul_rn(0.5, __dadd_rn(vi[k], vj[k]));
        }
    }
    *dU = __dsub_rn(__dmul_rn(__dmul_rn(0.5, mu), w2),
                    rr > 0.0 ? __ddiv_rn(__dmul_rn(__dmul_rn(C.G, mi), mj), rr) : 0.0);
    *r_out = rr;
    const double L[3] = {__dmul_rn(mu, __dsub_rn(__dmul_rn(r[1], w[2]), __dmul_rn(r[2], w[1]))),
                         __dmul_rn(mu, __dsub_rn(__dmul_rn(r[2], w[0]), __dmul_rn(r[0], w[2]))),
                         __dmul_rn(mu, __dsub_rn(__dmul_rn(r[0], w[1]), __dmul_rn(r[1], w[0])))};
    const int sv = (mi > mj || (mi == mj && i < j)) ? i : j, ot = sv == i ? j : i;
    const double Ri = C.radius[i], Rj = C.radius[j];
    const double R3 = __dadd_rn(__dmul_rn(__dmul_rn(Ri, Ri), Ri), __dmul_rn(__dmul_rn(Rj, Rj), Rj));
    double Sn[3];
    for (int k = 0; k < 3; k++)
        Sn[k] = __dadd_rn(__dadd_rn(C.spin[k * N + i], C.spin[k * N + j]), L[k]);
    C.mass[sv] = M;
    C.radius[sv] = cbrt(R3);
    for (int k = 0; k < 3; k++) C.spin[k * N + sv] = Sn[k];
    C.mass[ot] = 0.0;
    C.radius[ot] = 0.0;
    for (int k = 0; k < 3; k++) C.spin[k * N + ot] = 0.0;
    C.alive[ot] = 0;
    return sv;
}

// Appends one record to the merger log (latches kErrMergeLog when full).
__device__ __forceinline__ void log_merger(const CollArgs &C, DevCounters *ctr, int label, int seq, double t,
                                           int i, int j, double r, double Rs, double dU) {
    const unsigned long long k = atomicAdd(&ctr->merge_count, 1ull);
    if (k >= C.log_cap) {
        latch_error(ctr, kErrMergeLog);
        return;
    }
    double *e = C.log + (size_t)k * kMergeRec;
    e[0] = (double)C.call; e[1] = (double)label; e[2] = (double)seq; e[3] = t;
    e[4] = (double)i; e[5] = (double)j; e[6] = r; e[7] = Rs; e[8] = dU;
}

}  // namespace genga

#define GENGA_CUDA_TRY(expr)                                  \
    do {                                                      \
        cudaError_t e__ = (expr);                             \
        if (e__ != cudaSuccess) return e__;                   \
    } while (0)
