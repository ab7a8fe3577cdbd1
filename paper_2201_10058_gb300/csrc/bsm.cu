// bsm.cu -- Bulirsch-Stoer for close-encounter groups of more than
// kBlockGroupMax members, spread over the whole GPU (the role of the paper's
// BS-M, Sec. 6.1), with every such group of the current grouping advanced
// together by one persistent cooperative kernel.
//
// One round is one attempt of every still-running group, at its own step H,
// in phases separated by grid-wide barriers:
//   start      derivative at the attempt's start, error scale, first
//              midpoint sub-step of all 8 extrapolation columns;
//   sub-step   it = 1..16 moves every column whose n_k = 2(k+1) still has
//              sub-steps left, over all (column, member) pairs (ping-pong
//              state buffers, so partner reads never race with writes);
//              for large batches of the forward ODE a pair phase first
//              evaluates each partner pair once per column and writes its two
//              terms to the pair's partner-list entries, which the sub-step
//              then sums per member (the same values, in the same order);
//   Neville    per (component, member): the extrapolation table, its
//              diagonal, and each column's error folded into the group's 8
//              error words (atomic max on the bits of non-negative doubles);
//   decide     one thread per group: first column k >= 1 under tolerance
//              -> accept (grow H by 1.5 if k < 4), else halve H; attempt
//              and time bookkeeping; done / failed status;
//   accept     members of accepting groups take the accepted column.
// Step control and iteration stay on the device: the host launches once and
// reads the result.  A group fails after bs_max_steps attempts, so at most
// bs_max_steps rounds run; every barrier wait has a time limit (2 s unless
// genga_set_wait_limits sets another) after which the kernel records a
// timeout and returns.  Scheme and acceptance rule
// are those of the in-block kernels (modified midpoint n = 2..16, Neville in
// h^2, error scale |y| + |H dy/dt| + 1e-300, the same force arithmetic).
// Data written by one block and read by another inside the kernel is read
// through L2 (ld.global.cg), never from a possibly stale L1 line.
//
// The ODE is a template policy: the group's forward ODE (6 values per member)
// or the adjoint's augmented backward ODE (13 values per member).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace genga {
namespace {

constexpr int kPThreads = 128;

struct GridBarrier {
    unsigned count;     // blocks arrived at the current barrier
    unsigned gen;       // barrier generation
    unsigned err;       // a wait ran out
    unsigned running;   // groups still integrating
};

// Batch of groups: compact member index m in [0, M) over the groups.
struct BsmArgs {
    int M;                         // members over all batched groups
    int ng;                        // batched groups
    int nlev;                      // levels whose (1 - K) factors apply
    // per member, written before the persistent launch
    const int *mgroup;             // [M] batched group of m
    const int *mq0, *mq1;          // [M] partner range in the level CSR
    const int *pidx;               // [CSR entries] compact index of each partner
    const double *mmass;           // [M] mass
    const double *irc;             // [nlev][M] 1/rc per level
    double G, mu, dt, tol;
    int max_steps;
    // state, component-major over members ([..][D][M])
    double *Y, *F0, *SC;           // attempt start, its derivative, error scale
    double *ZM, *ZA, *ZB;          // [8] per column: previous midpoint state, two current buffers
    double *OUT, *DIAG;            // [8] column results, Neville diagonal T_kk
    // per-group step control
    double *gt, *gH;
    int *gstat;                    // 0 running, 1 done, 2 failed
    int *gkconv;                   // accepted column of the last round, -1 none
    long long *gatt, *gacc, *grej;
    unsigned long long *gerr;      // [ng][8]
    GridBarrier *bar;
    unsigned long long barrier_ns; // limit of one grid-barrier wait
    unsigned barrier_absent;       // test hook: arrivals every barrier waits for in vain (0)
    // collisions (Sec. 7.1-7.2), used by the collision ODE instance
    CollArgs coll;
    const int *mbody;              // [M] body of each member
    const int *gbase;              // [ng + 1] first member of each group
    int *morder;                   // [M] members of each group by ascending body index
    int *malive;                   // [M] alive flags of the members
    double *mmass_rw;              // = mmass, written by mergers
    int *gseq;                     // [ng] mergers of each group so far
    DevCounters *ctr;
    // pair-centric derivative (forward ODE without collisions, large batches):
    // each unordered pair once per column, its two terms written to the two
    // partner-list entries, then summed per member
    int pairs;                     // 1: this mode
    const int *pcount;             // pairs listed
    const int *pq, *pm;            // [pairs] entry q (member m -> partner) and member m, partner > m
    const int *prev;               // [entries] the reverse entry of each entry of a batched member
    double2 *rec;                  // [8][entries][2]: (c, dx), (dy, dz) of each entry per column
    size_t nq;                     // entries (the stride of rec per column)
};

__device__ __forceinline__ double ldc(const double *p) { return __ldcg(p); }
__device__ __forceinline__ int ldc(const int *p) { return __ldcg(p); }

__device__ __forceinline__ double step_of(const BsmArgs &A, int g) {
    const double H = ldc(&A.gH[g]);
    const double left = A.dt - ldc(&A.gt[g]);
    return H > left ? left : H;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier (all blocks co-resident: cooperative launch).  One
// thread per block arrives with an atomic and polls the generation word with
// volatile loads (served by L2); a wait longer than limit_ns records a
// timeout, and a wait also ends once another block has recorded one.  The
// barrier completes when gridDim.x + absent blocks have arrived (absent = 0
// in normal use; a test makes every wait run out with absent > 0).  Returns
// false if this or another block's wait ran out.
__device__ bool grid_barrier(GridBarrier *b, unsigned long long limit_ns, unsigned absent) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        volatile unsigned *gen = &b->gen;
        volatile unsigned *err = &b->err;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x + absent - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned polls = 0;
            while (*gen == g) {
                if ((++polls & 63u) == 0u && (*err != 0u || global_ns() - t0 >= limit_ns)) {
                    atomicExch(&b->err, 1u);
                    good = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok = good && *(volatile unsigned *)&b->err == 0u;
    }
    __syncthreads();
    return ok != 0;
}

// Lanes per item in the derivative phases: the partner loop of one (column,
// member) item is split over kLanes adjacent lanes (partner q to lane
// q mod kLanes) and the partial sums are combined by an xor butterfly, which
// gives every lane the same bits (IEEE addition commutes).
constexpr int kLanes = 4;

__device__ __forceinline__ unsigned lane_mask() {
    return 0xfu << ((threadIdx.x & 31u) & ~3u);
}
__device__ __forceinline__ double lane_sum(double v) {
    const unsigned mk = lane_mask();
    v += __shfl_xor_sync(mk, v, 1);
    v += __shfl_xor_sync(mk, v, 2);
    return v;
}

// Forward group ODE: y = (x, v); a = -mu x/r^3 + G sum_p m_p W (x_p - x)/r^3,
// W = prod_{levels} (1 - K).  Every lane of the item returns f.  With
// collisions (COLL) the members' masses and alive flags change inside the
// kernel (read through L2); a member merged away feels only the star, and a
// partner merged away has mass 0.
template <bool COLL_>
struct FwdOdeT {
    static constexpr int D = 6;
    static constexpr int NERR = 6;
    static constexpr bool COLL = COLL_;
    __device__ static void deriv(const BsmArgs &A, const double *Z, int m, int lane, double *f) {
        const size_t ld = (size_t)A.M;
        const double x = ldc(&Z[0 * ld + m]), y = ldc(&Z[1 * ld + m]), z = ldc(&Z[2 * ld + m]);
        double px = 0.0, py = 0.0, pz = 0.0;
        const int q1 = (COLL && !ldc(&A.malive[m])) ? A.mq0[m] : A.mq1[m];
        for (int q = A.mq0[m] + lane; q < q1; q += kLanes) {
            const int sp = A.pidx[q];
            const double dx = ldc(&Z[0 * ld + sp]) - x, dy = ldc(&Z[1 * ld + sp]) - y,
                         dz = ldc(&Z[2 * ld + sp]) - z;
            const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double yv = rsqrt_newton(d2);
            const double d = d2 * yv;
            double W = 1.0;
            for (int l = 0; l < A.nlev; l++)
                W *= 1.0 - changeover_fast(d, fmin(A.irc[(size_t)l * ld + m], A.irc[(size_t)l * ld + sp]));
            const double ms = COLL ? ldc(&A.mmass[sp]) : A.mmass[sp];
            const double c = ms * W * (yv * yv * yv);
            px = fma(c, dx, px); py = fma(c, dy, py); pz = fma(c, dz, pz);
        }
        px = lane_sum(px); py = lane_sum(py); pz = lane_sum(pz);
        const double r2 = fma(z, z, fma(y, y, x * x));
        const double ys = rsqrt_newton(r2);
        const double sst = -A.mu * (ys * ys * ys);
        f[0] = ldc(&Z[3 * ld + m]); f[1] = ldc(&Z[4 * ld + m]); f[2] = ldc(&Z[5 * ld + m]);
        f[3] = fma(sst, x, A.G * px); f[4] = fma(sst, y, A.G * py); f[5] = fma(sst, z, A.G * pz);
    }
};
// The forward derivative of member m in column k from the entries' records
// (pair-centric mode): the same terms, summed in the same lane split and order.
__device__ __forceinline__ void fwd_deriv_rec(const BsmArgs &A, const double *Z, int k, int m, int lane,
                                              double *f) {
    const size_t ld = (size_t)A.M;
    const double x = ldc(&Z[0 * ld + m]), y = ldc(&Z[1 * ld + m]), z = ldc(&Z[2 * ld + m]);
    const double2 *R = A.rec + (size_t)k * 2 * A.nq;
    double px = 0.0, py = 0.0, pz = 0.0;
    for (int q = A.mq0[m] + lane; q < A.mq1[m]; q += kLanes) {
        const double2 u = __ldcg(&R[2 * (size_t)q]), w = __ldcg(&R[2 * (size_t)q + 1]);
        px = fma(u.x, u.y, px); py = fma(u.x, w.x, py); pz = fma(u.x, w.y, pz);
    }
    px = lane_sum(px); py = lane_sum(py); pz = lane_sum(pz);
    const double r2 = fma(z, z, fma(y, y, x * x));
    const double ys = rsqrt_newton(r2);
    const double sst = -A.mu * (ys * ys * ys);
    f[0] = ldc(&Z[3 * ld + m]); f[1] = ldc(&Z[4 * ld + m]); f[2] = ldc(&Z[5 * ld + m]);
    f[3] = fma(sst, x, A.G * px); f[4] = fma(sst, y, A.G * py); f[5] = fma(sst, z, A.G * pz);
}

using FwdOde = FwdOdeT<false>;
using FwdCollOde = FwdOdeT<true>;

// Adjoint augmented ODE in reversed time (level 0): y (6), lambda (6), the
// mass-gradient integral (1); with A = da/dx:
//   dy/dtau = -f(y),  dlx/dtau = A^T lv,  dlv/dtau = lx,
//   dg_a/dtau = G sum_p W lv_p . (x_a - x_p)/r^3   (da_p/dm_a).
struct AdjOde {
    static constexpr int D = 13;
    static constexpr int NERR = 6;
    static constexpr bool COLL = false;
    __device__ static void deriv(const BsmArgs &A, const double *Z, int m, int lane, double *f) {
        const size_t ld = (size_t)A.M;
        const double x = ldc(&Z[0 * ld + m]), y = ldc(&Z[1 * ld + m]), z = ldc(&Z[2 * ld + m]);
        const double lvx = ldc(&Z[9 * ld + m]), lvy = ldc(&Z[10 * ld + m]), lvz = ldc(&Z[11 * ld + m]);
        const double mb = A.mmass[m];
        double px = 0.0, py = 0.0, pz = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, gm = 0.0;
        const int q1 = A.mq1[m];
        for (int q = A.mq0[m] + lane; q < q1; q += kLanes) {
            const int sp = A.pidx[q];
            const double dx = ldc(&Z[0 * ld + sp]) - x, dy = ldc(&Z[1 * ld + sp]) - y,
                         dz = ldc(&Z[2 * ld + sp]) - z;
            const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double yv = rsqrt_newton(d2);
            const double d = d2 * yv, id2 = yv * yv, id3 = id2 * yv;
            double K, dK;
            changeover_fast_dr(d, fmin(A.irc[m], A.irc[sp]), K, dK);
            const double W = 1.0 - K;
            const double Wp = -dK;
            const double mp = A.mmass[sp];
            const double cw = mp * W * id3;
            px = fma(cw, dx, px); py = fma(cw, dy, py); pz = fma(cw, dz, pz);
            const double qx = ldc(&Z[9 * ld + sp]), qy = ldc(&Z[10 * ld + sp]), qz = ldc(&Z[11 * ld + sp]);
            const double e0 = mb * qx - mp * lvx, e1 = mb * qy - mp * lvy, e2 = mb * qz - mp * lvz;
            const double de = dx * e0 + dy * e1 + dz * e2;
            const double aa = W * id3;
            const double bb = de * id2 * (Wp * id2 - 3.0 * W * id3);
            gx += aa * e0 + bb * dx; gy += aa * e1 + bb * dy; gz += aa * e2 + bb * dz;
            gm -= W * (qx * dx + qy * dy + qz * dz) * id3;
        }
        px = lane_sum(px); py = lane_sum(py); pz = lane_sum(pz);
        gx = lane_sum(gx); gy = lane_sum(gy); gz = lane_sum(gz); gm = lane_sum(gm);
        const double r2 = fma(z, z, fma(y, y, x * x));
        const double ys = rsqrt_newton(r2);
        const double ir2 = ys * ys, ir3 = ir2 * ys;
        const double xl = x * lvx + y * lvy + z * lvz;
        const double tx = -A.mu * ir3 * (lvx - 3.0 * x * xl * ir2);
        const double ty = -A.mu * ir3 * (lvy - 3.0 * y * xl * ir2);
        const double tz = -A.mu * ir3 * (lvz - 3.0 * z * xl * ir2);
        const double ax = -A.mu * x * ir3 + A.G * px, ay = -A.mu * y * ir3 + A.G * py,
                     az = -A.mu * z * ir3 + A.G * pz;
        f[0] = -ldc(&Z[3 * ld + m]); f[1] = -ldc(&Z[4 * ld + m]); f[2] = -ldc(&Z[5 * ld + m]);
        f[3] = -ax; f[4] = -ay; f[5] = -az;
        f[6] = tx + A.G * gx; f[7] = ty + A.G * gy; f[8] = tz + A.G * gz;
        f[9] = ldc(&Z[6 * ld + m]); f[10] = ldc(&Z[7 * ld + m]); f[11] = ldc(&Z[8 * ld + m]);
        f[12] = A.G * gm;
    }
};

// ---------------------------------------------------------------- phases
// start and sub-step: item = kLanes adjacent lanes; lane 0 writes.
template <class Ode>
__device__ void phase_start(const BsmArgs &A, int m, int lane) {
    const int g = A.mgroup[m];
    if (ldc(&A.gstat[g]) != 0) return;
    constexpr int D = Ode::D;
    const size_t ld = (size_t)A.M, blk = (size_t)D * ld;
    const double H = step_of(A, g);
    double f[D];
    Ode::deriv(A, A.Y, m, lane, f);
    if (lane != 0) return;
    for (int c = 0; c < D; c++) {
        const double y = ldc(&A.Y[c * ld + m]);
        A.F0[c * ld + m] = f[c];
        A.SC[c * ld + m] = fabs(y) + fabs(H * f[c]) + 1e-300;
        for (int k = 0; k < 8; k++) {
            const double h = H / (2 * (k + 1));
            A.ZM[k * blk + c * ld + m] = y;
            A.ZA[k * blk + c * ld + m] = y + h * f[c];
        }
    }
}

template <class Ode>
__device__ void phase_substep(const BsmArgs &A, long long t, int it, int lane) {
    const int k = (int)(t / A.M), m = (int)(t % A.M);
    const int nk = 2 * (k + 1);
    if (it > nk) return;
    const int g = A.mgroup[m];
    if (ldc(&A.gstat[g]) != 0) return;
    constexpr int D = Ode::D;
    const size_t ld = (size_t)A.M, blk = (size_t)D * ld;
    const double *Zcur = ((it & 1) ? A.ZA : A.ZB) + k * blk;
    double *Znext = ((it & 1) ? A.ZB : A.ZA) + k * blk;
    double *ZM = A.ZM + k * blk;
    const double h = step_of(A, g) / nk;
    double f[D];
    if constexpr (D == 6 && !Ode::COLL) {
        if (A.pairs) fwd_deriv_rec(A, Zcur, k, m, lane, f);
        else Ode::deriv(A, Zcur, m, lane, f);
    } else {
        Ode::deriv(A, Zcur, m, lane, f);
    }
    if (lane != 0) return;
    if (it < nk) {
        for (int c = 0; c < D; c++) {
            const double zc = ldc(&Zcur[c * ld + m]);
            const double tt = ldc(&ZM[c * ld + m]) + 2.0 * h * f[c];
            ZM[c * ld + m] = zc;
            Znext[c * ld + m] = tt;
        }
    } else {
        for (int c = 0; c < D; c++)
            A.OUT[k * blk + c * ld + m] = 0.5 * (ldc(&Zcur[c * ld + m]) + ldc(&ZM[c * ld + m]) + h * f[c]);
    }
}

// Pair-centric mode, before each sub-step: pair t of column k computes the
// terms member m's partner loop would (displacement from m to its partner p,
// W, m_p W / r^3) and those p's would (the displacement negated, exactly, and
// m_m W / r^3), into the records of entries m -> p and p -> m.
__device__ void phase_pairs(const BsmArgs &A, long long t, long long P, int it) {
    const int k = (int)(t / P);
    const long long pi = t - (long long)k * P;
    if (it > 2 * (k + 1)) return;
    const int q = A.pq[pi], m = A.pm[pi];
    if (ldc(&A.gstat[A.mgroup[m]]) != 0) return;
    const int sp = A.pidx[q], q2 = A.prev[q];
    const size_t ld = (size_t)A.M, blk = 6 * ld;
    const double *Z = ((it & 1) ? A.ZA : A.ZB) + k * blk;
    const double x = ldc(&Z[0 * ld + m]), y = ldc(&Z[1 * ld + m]), z = ldc(&Z[2 * ld + m]);
    const double dx = ldc(&Z[0 * ld + sp]) - x, dy = ldc(&Z[1 * ld + sp]) - y, dz = ldc(&Z[2 * ld + sp]) - z;
    const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double yv = rsqrt_newton(d2);
    const double d = d2 * yv;
    double W = 1.0;
    for (int l = 0; l < A.nlev; l++)
        W *= 1.0 - changeover_fast(d, fmin(A.irc[(size_t)l * ld + m], A.irc[(size_t)l * ld + sp]));
    const double cm = A.mmass[sp] * W * (yv * yv * yv);
    const double cp = A.mmass[m] * W * (yv * yv * yv);
    double2 *R = A.rec + (size_t)k * 2 * A.nq;
    R[2 * (size_t)q] = make_double2(cm, dx);
    R[2 * (size_t)q + 1] = make_double2(dy, dz);
    R[2 * (size_t)q2] = make_double2(cp, -dx);
    R[2 * (size_t)q2 + 1] = make_double2(-dy, -dz);
}

// Neville for item t; called by every lane of a warp (the reductions need all
// lanes), items past the end contribute nothing.
template <class Ode>
__device__ void phase_neville(const BsmArgs &A, long long t) {
    constexpr int D = Ode::D;
    const size_t ld = (size_t)A.M, blk = (size_t)D * ld;
    double e[8];
    for (int k = 0; k < 8; k++) e[k] = 0.0;
    int g = -1;
    if (t < (long long)D * A.M) {
        const int c = (int)(t / A.M), m = (int)(t % A.M);
        g = A.mgroup[m];
        if (ldc(&A.gstat[g]) == 0) {
            double T[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            const double sc = ldc(&A.SC[c * ld + m]);
            for (int k = 0; k < 8; k++) {
                double cur = ldc(&A.OUT[k * blk + c * ld + m]);
                double prev = T[0];
                T[0] = cur;
                for (int j = 1; j <= k; j++) {
                    const double coef = (double)((k - j + 1) * (k - j + 1)) / (double)(j * (2 * k + 2 - j));
                    const double nxt = fma(cur - prev, coef, cur);
                    prev = T[j];
                    T[j] = nxt;
                    cur = nxt;
                }
                A.DIAG[k * blk + c * ld + m] = T[k];
                if (k >= 1 && c < Ode::NERR) e[k] = fabs(T[k] - T[k - 1]) / sc;
            }
        } else {
            g = -1;
        }
    }
    // one atomic per warp when all its lanes belong to one running group
    const int g0 = __shfl_sync(0xffffffffu, g, 0);
    const bool uniform = __all_sync(0xffffffffu, g == g0);
    for (int k = 1; k < 8; k++) {
        double v = e[k];
        if (uniform) {
            for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0 && g0 >= 0)
                atomicMax(&A.gerr[(size_t)g0 * 8 + k], (unsigned long long)__double_as_longlong(v));
        } else if (g >= 0) {
            atomicMax(&A.gerr[(size_t)g * 8 + k], (unsigned long long)__double_as_longlong(v));
        }
    }
}

// Collisions (reading R25) of group g, by one thread: the separation of two
// members in the state Z (component-major over members, stride M).
__device__ __forceinline__ double member_dist(const BsmArgs &A, const double *Z, int a, int b) {
    const size_t ld = (size_t)A.M;
    return __dsqrt_rn(dist2_rn(__dsub_rn(ldc(&Z[0 * ld + b]), ldc(&Z[0 * ld + a])),
                               __dsub_rn(ldc(&Z[1 * ld + b]), ldc(&Z[1 * ld + a])),
                               __dsub_rn(ldc(&Z[2 * ld + b]), ldc(&Z[2 * ld + a]))));
}

// Deepest overlap fraction over the group's pairs of alive members in Z.
__device__ double group_overlap(const BsmArgs &A, int g, const double *Z) {
    double deepest = 0.0;
    for (int m = A.gbase[g]; m < A.gbase[g + 1]; m++) {
        if (!ldc(&A.malive[m])) continue;
        for (int q = A.mq0[m]; q < A.mq1[m]; q++) {
            const int p = A.pidx[q];
            if (A.mbody[p] <= A.mbody[m] || !ldc(&A.malive[p])) continue;
            const double r = member_dist(A, Z, m, p);
            const double Rs = __dadd_rn(ldc(&A.coll.radius[A.mbody[m]]), ldc(&A.coll.radius[A.mbody[p]]));
            if (r < Rs) deepest = fmax(deepest, __ddiv_rn(__dsub_rn(Rs, r), Rs));
        }
    }
    return deepest;
}

// Mergers of the overlapping pairs of alive members of group g in the state
// Y at time t of the call, in ascending (i, j) order (members by rank, partner
// lists ascending), each seeing the mergers before it.
__device__ void group_merge(const BsmArgs &A, int g, double t) {
    const size_t ld = (size_t)A.M;
    const int label = A.mbody[A.morder[A.gbase[g]]];
    int seq = A.gseq[g];
    for (int rk = A.gbase[g]; rk < A.gbase[g + 1]; rk++) {
        const int m = A.morder[rk];
        for (int q = A.mq0[m]; q < A.mq1[m]; q++) {
            const int p = A.pidx[q];
            const int im = A.mbody[m], ip = A.mbody[p];
            if (ip <= im || !ldc(&A.malive[m]) || !ldc(&A.malive[p])) continue;
            const double r = member_dist(A, A.Y, m, p);
            const double Rs = __dadd_rn(ldc(&A.coll.radius[im]), ldc(&A.coll.radius[ip]));
            if (!(r < Rs)) continue;
            double xa[3], va[3], xb[3], vb[3], xo[3], vo[3], dU, rr;
            for (int k = 0; k < 3; k++) {
                xa[k] = ldc(&A.Y[k * ld + m]); va[k] = ldc(&A.Y[(3 + k) * ld + m]);
                xb[k] = ldc(&A.Y[k * ld + p]); vb[k] = ldc(&A.Y[(3 + k) * ld + p]);
            }
            const int sv = merge_bodies(A.coll, (size_t)A.coll.n, im, ip, xa, va, xb, vb, xo, vo, &dU, &rr);
            const int ms = sv == im ? m : p, mo = sv == im ? p : m;
            for (int k = 0; k < 3; k++) { A.Y[k * ld + ms] = xo[k]; A.Y[(3 + k) * ld + ms] = vo[k]; }
            A.mmass_rw[ms] = A.coll.mass[sv];
            A.mmass_rw[mo] = 0.0;
            A.malive[mo] = 0;
            log_merger(A.coll, A.ctr, label, seq++, t, im, ip, r, Rs, dU);
        }
    }
    A.gseq[g] = seq;
}

// Step control of group g (the in-block kernels' rule).  The group's
// counters are touched only by this thread, so plain accesses suffice for
// them; the words other blocks read go through L2.
template <class Ode>
__device__ void phase_decide(const BsmArgs &A, int g) {
    A.gkconv[g] = -1;
    if (ldc(&A.gstat[g]) != 0) return;
    double H = step_of(A, g);
    int kconv = -1;
    for (int k = 1; k < 8 && kconv < 0; k++) {
        const double e = __longlong_as_double((long long)atomicAdd(&A.gerr[(size_t)g * 8 + k], 0ull));
        if (e <= A.tol) kconv = k;
    }
    // collision precision (Sec. 7.2): a step that ends with an overlap of
    // tol or more of the radius sum ends too late
    if (Ode::COLL && kconv >= 0 && A.coll.tol > 0.0 &&
        group_overlap(A, g, A.DIAG + (size_t)kconv * Ode::D * A.M) >= A.coll.tol)
        kconv = -1;
    for (int k = 0; k < 8; k++) atomicExch(&A.gerr[(size_t)g * 8 + k], 0ull);
    const long long att = A.gatt[g] + 1;
    A.gatt[g] = att;
    double t = ldc(&A.gt[g]);
    if (kconv >= 0) {
        t += H;
        A.gacc[g] += 1;
        if (kconv < 4) H *= 1.5;
    } else {
        A.grej[g] += 1;
        H *= 0.5;
    }
    A.gt[g] = t;
    A.gH[g] = H;
    A.gkconv[g] = kconv;
    int st = 0;
    if (!(t < A.dt)) st = 1;
    else if (att >= A.max_steps) st = 2;
    if (st) {
        A.gstat[g] = st;
        atomicSub(&A.bar->running, 1u);
    }
}

template <class Ode>
__device__ void phase_accept(const BsmArgs &A, long long t) {
    constexpr int D = Ode::D;
    const size_t blk = (size_t)D * A.M;
    const int m = (int)(t % A.M);
    const int k = ldc(&A.gkconv[A.mgroup[m]]);
    if (k >= 0) A.Y[t] = ldc(&A.DIAG[k * blk + t]);
}

template <class Ode>
__global__ void __launch_bounds__(kPThreads)
bsm_persistent_kernel(BsmArgs A) {
    constexpr int D = Ode::D;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long M = A.M;
    // derivative phases: kLanes adjacent lanes per item (blockDim is a multiple of 32)
    const long long item0 = tid / kLanes, nitem = nth / kLanes;
    const int lane = (int)(threadIdx.x % kLanes);
    // pairs of the pair-centric mode (listed by bsm_pairs_kernel before the launch)
    const long long P = (D == 6 && !Ode::COLL && A.pairs) ? (long long)*A.pcount : 0;
    __shared__ unsigned running;
    if (Ode::COLL) {
        // pairs already overlapping when the integration starts merge at once
        for (long long g = tid; g < A.ng; g += nth) group_merge(A, (int)g, 0.0);
        if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
    }
    for (int round = 0; round < A.max_steps; round++) {
        // one read per block; the previous round ended with a barrier
        if (threadIdx.x == 0) running = atomicAdd(&A.bar->running, 0u);
        __syncthreads();
        if (running == 0u) break;
        for (long long t = item0; t < M; t += nitem) phase_start<Ode>(A, (int)t, lane);
        if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
        for (int it = 1; it <= 16; it++) {
            if (P > 0) {
                for (long long t = tid; t < 8 * P; t += nth) phase_pairs(A, t, P, it);
                if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
            }
            for (long long t = item0; t < 8 * M; t += nitem) phase_substep<Ode>(A, t, it, lane);
            if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
        }
        for (long long base = (long long)blockIdx.x * blockDim.x; base < D * M; base += nth)
            phase_neville<Ode>(A, base + threadIdx.x);
        if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
        for (long long g = tid; g < A.ng; g += nth) phase_decide<Ode>(A, (int)g);
        if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
        for (long long t = tid; t < D * M; t += nth) phase_accept<Ode>(A, t);
        if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
        if (Ode::COLL) {
            // mergers at the end of every accepted step (same thread per group
            // as the decision, which wrote gkconv and gt)
            for (long long g = tid; g < A.ng; g += nth)
                if (A.gkconv[g] >= 0) group_merge(A, (int)g, ldc(&A.gt[g]));
            if (!grid_barrier(A.bar, A.barrier_ns, A.barrier_absent)) return;
        }
    }
}

// ---------------------------------------------------------------- set-up
struct RcPtrs {
    const double *p[kMaxLevels];
};

// Per member: group, body, partner range, compact partner indices, mass, 1/rc.
__global__ void bsm_members_kernel(int ng, const int *gbase, const int *gslot0, const int *member,
                                   const int *slotof, const int *off, const int *list, const double *mass,
                                   RcPtrs rc, int nlev, int M, int *mbody, int *mgroup, int *mq0, int *mq1,
                                   int *pidx, double *mmass, double *irc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int lo = 0, hi = ng - 1;                     // last group with gbase <= m
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gbase[mid] <= m) lo = mid; else hi = mid - 1;
    }
    mgroup[m] = lo;
    const int b = member[gslot0[lo] + (m - gbase[lo])];
    mbody[m] = b;
    mmass[m] = mass[b];
    const int q0 = off[b], q1 = off[b + 1];
    mq0[m] = q0;
    mq1[m] = q1;
    // partners belong to the same group (connected components of the pair graph)
    for (int q = q0; q < q1; q++) pidx[q] = gbase[lo] + (slotof[list[q]] - gslot0[lo]);
    for (int l = 0; l < nlev; l++) irc[(size_t)l * M + m] = 1.0 / rc.p[l][b];
}

// Pair-centric mode: the unordered pairs of the batched members (each listed
// from its lower member, in any order) and every entry's reverse entry (the
// rows are ascending in body index, so a binary search finds it).
__global__ void bsm_pairs_kernel(int M, const int *mq0, const int *mq1, const int *pidx, const int *mbody,
                                 const int *list, int *pcount, int *pq, int *pm, int *prev) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int bm = mbody[m];
    for (int q = mq0[m]; q < mq1[m]; q++) {
        const int p = pidx[q];
        int lo = mq0[p], hi = mq1[p] - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (list[mid] < bm) lo = mid + 1; else hi = mid;
        }
        prev[q] = lo;
        if (p > m) {
            const int k = atomicAdd(pcount, 1);
            pq[k] = q;
            pm[k] = m;
        }
    }
}

// Collisions: each member's alive flag, and the members of each group by
// ascending body index (rank = members of the group with a smaller body).
__global__ void bsm_coll_init_kernel(BsmArgs A) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.M) return;
    const int b = A.mbody[m];
    A.malive[m] = A.coll.alive[b];
    const int g = A.mgroup[m];
    int rank = 0;
    for (int q = A.gbase[g]; q < A.gbase[g + 1]; q++) rank += A.mbody[q] < b;
    A.morder[A.gbase[g] + rank] = m;
}

__global__ void bsm_init_groups_kernel(BsmArgs A) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) {
        A.bar->count = 0u;
        A.bar->gen = 0u;
        A.bar->err = 0u;
        A.bar->running = (unsigned)A.ng;
    }
    if (g >= A.ng) return;
    A.gt[g] = 0.0;
    A.gH[g] = A.dt;
    A.gstat[g] = 0;
    A.gkconv[g] = -1;
    A.gatt[g] = 0;
    A.gacc[g] = 0;
    A.grej[g] = 0;
    if (A.gseq) A.gseq[g] = 0;
    for (int k = 0; k < 8; k++) A.gerr[(size_t)g * 8 + k] = 0ull;
}

__global__ void bsm_gather_fwd(int n, int M, const int *mbody, const double *pos, const double *vel, double *Y) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int b = mbody[m];
    for (int c = 0; c < 3; c++) {
        Y[c * (size_t)M + m] = pos[c * (size_t)n + b];
        Y[(3 + c) * (size_t)M + m] = vel[c * (size_t)n + b];
    }
}
__global__ void bsm_scatter_fwd(int n, int M, const int *mbody, const double *Y, double *pos, double *vel) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int b = mbody[m];
    for (int c = 0; c < 3; c++) {
        pos[c * (size_t)n + b] = Y[c * (size_t)M + m];
        vel[c * (size_t)n + b] = Y[(3 + c) * (size_t)M + m];
    }
}
__global__ void bsm_gather_adj(int n, int M, const int *mbody, const double *x2, const double *v2,
                               const double *lx, const double *lv, double *Y) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int b = mbody[m];
    const size_t ld = (size_t)M;
    for (int c = 0; c < 3; c++) {
        Y[c * ld + m] = x2[c * (size_t)n + b];
        Y[(3 + c) * ld + m] = v2[c * (size_t)n + b];
        Y[(6 + c) * ld + m] = lx[c * (size_t)n + b];
        Y[(9 + c) * ld + m] = lv[c * (size_t)n + b];
    }
    Y[12 * ld + m] = 0.0;
}
__global__ void bsm_scatter_adj(int n, int M, const int *mbody, const double *Y, double *lx, double *lv,
                                double *lm) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int b = mbody[m];
    const size_t ld = (size_t)M;
    for (int c = 0; c < 3; c++) {
        lx[c * (size_t)n + b] = Y[(6 + c) * ld + m];
        lv[c * (size_t)n + b] = Y[(9 + c) * ld + m];
    }
    lm[b] += Y[12 * ld + m];
}

// Folds the groups' counters into the system's (one thread, group order).
__global__ void bsm_stats_kernel(BsmArgs A, DevCounters *ctr, int count_steps) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    unsigned long long acc = 0, rej = 0, att = 0, fail = 0;
    for (int g = 0; g < A.ng; g++) {
        acc += (unsigned long long)A.gacc[g];
        rej += (unsigned long long)A.grej[g];
        if ((unsigned long long)A.gatt[g] > att) att = (unsigned long long)A.gatt[g];
        fail += A.gstat[g] == 2 ? 1ull : 0ull;
    }
    if (count_steps) {
        atomicAdd(&ctr->bs_steps, acc);
        atomicAdd(&ctr->bs_rejects, rej);
        atomicMax(&ctr->bs_max_attempts, att);
    }
    if (fail) {
        atomicAdd(&ctr->bs_fail, fail);
        latch_error(ctr, kErrBS);
    }
}

// Device buffers of the batch, grown on demand, kept by the system.
struct BsmBuffers {
    void *raw = nullptr;
    size_t bytes = 0;
};

void *bsm_reserve(genga_system *s, size_t bytes) {
    BsmBuffers *b = static_cast<BsmBuffers *>(s->bsm);
    if (!b) {
        b = new BsmBuffers;
        s->bsm = b;
    }
    if (b->bytes < bytes) {
        if (b->raw) cudaFree(b->raw);
        b->raw = nullptr;
        b->bytes = 0;
        if (cudaMalloc(&b->raw, bytes) != cudaSuccess) return nullptr;
        b->bytes = bytes;
    }
    return b->raw;
}

// Host list of the groups with more than kBlockGroupMax members: (slot0, nm),
// ascending slot.
int batched_groups(genga_system *s, std::vector<int2> &out) {
    out.clear();
    DevCounters c;
    if (cudaMemcpyAsync(&c, s->ctr, sizeof(c), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return -1;
    ++s->host_syncs;
    if ((int)c.max_group <= kBlockGroupMax || c.ngroups == 0) return 0;
    std::vector<int> glist(c.ngroups), goff((size_t)s->n + 1);
    if (cudaMemcpyAsync(glist.data(), s->glist, sizeof(int) * c.ngroups, cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(goff.data(), s->goff, sizeof(int) * goff.size(), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return -1;
    ++s->host_syncs;
    for (int g : glist) {
        const int nm = goff[(size_t)g + 1] - goff[(size_t)g];
        if (nm > kBlockGroupMax) out.push_back(make_int2(goff[(size_t)g], nm));
    }
    std::sort(out.begin(), out.end(), [](const int2 &a, const int2 &b) { return a.x < b.x; });
    return 0;
}

size_t aligned(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

template <typename T>
T *carve(char *&p, size_t count) {
    T *r = reinterpret_cast<T *>(p);
    p += aligned(sizeof(T) * count);
    return r;
}

// Runs every batched group over dt from the state `gather` writes into Y;
// `scatter` takes Y back.  Returns a genga error code.
template <class Ode, class Gather, class Scatter>
int bsm_run(genga_system *s, int level, double dt, const std::vector<int2> &groups, bool count_steps,
            Gather gather, Scatter scatter) {
    constexpr int D = Ode::D;
    const int ng = (int)groups.size();
    const int nlev = level + 1;
    std::vector<int> gbase(ng + 1), gslot0(ng);
    int M = 0;
    for (int g = 0; g < ng; g++) {
        gbase[g] = M;
        gslot0[g] = groups[g].x;
        M += groups[g].y;
    }
    gbase[ng] = M;
    const size_t blk = (size_t)D * M;
    const size_t nq = 2 * (size_t)s->csr[level].cap;
    // one persistent cooperative launch: as many blocks as fit on the GPU (more
    // warps to hide the partner reads from L2 outweigh the barrier's extra
    // arrivals), and no more than the (column, member) items need
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bsm_persistent_kernel<Ode>, kPThreads, 0) !=
            cudaSuccess || per_sm < 1)
        return GENGA_ECUDA;
    const long long want = (8LL * M * kLanes + kPThreads - 1) / kPThreads;
    const long long cap = (long long)per_sm * s->num_sms;
    const unsigned grid = (unsigned)std::max(1LL, std::min(want, cap));
    // pair-centric derivative where a sub-step phase takes more than two passes
    // over its (column, member) items: there the FP64 work of the partner
    // terms, halved, outweighs a second barrier per sub-step
    const bool pairs = D == 6 && !Ode::COLL &&
                       (s->bs_pairs == GENGA_BS_PAIRS_ON ||
                        (s->bs_pairs == GENGA_BS_PAIRS_AUTO && 8LL * M > 2LL * grid * (kPThreads / kLanes)));
    const size_t pbytes = pairs ? aligned(sizeof(double2) * 2 * 8 * nq) + aligned(sizeof(int) * nq) * 3 +
                                      aligned(sizeof(int))
                                : 0;
    const size_t bytes = pbytes + aligned(sizeof(double) * blk) * 3 + aligned(sizeof(double) * 8 * blk) * 5 +
                         aligned(sizeof(double) * (size_t)nlev * M) + aligned(sizeof(double) * M) +
                         aligned(sizeof(int) * M) * 4 + aligned(sizeof(int) * nq) +
                         aligned(sizeof(int) * (ng + 1)) + aligned(sizeof(int) * ng) * 4 +
                         aligned(sizeof(double) * ng) * 2 +
                         aligned(sizeof(long long) * ng) * 3 + aligned(sizeof(unsigned long long) * 8 * ng) +
                         aligned(sizeof(GridBarrier)) +
                         (Ode::COLL ? aligned(sizeof(int) * M) * 2 : 0);
    char *p = static_cast<char *>(bsm_reserve(s, bytes));
    if (!p) return GENGA_ENOMEM;
    BsmArgs A;
    A.M = M; A.ng = ng; A.nlev = nlev;
    A.pairs = pairs ? 1 : 0;
    A.nq = nq;
    int *pcount = nullptr, *pq = nullptr, *pm = nullptr, *prev = nullptr;
    A.rec = nullptr;
    if (pairs) {
        A.rec = carve<double2>(p, 2 * 8 * nq);
        pq = carve<int>(p, nq);
        pm = carve<int>(p, nq);
        prev = carve<int>(p, nq);
        pcount = carve<int>(p, 1);
    }
    A.pcount = pcount; A.pq = pq; A.pm = pm; A.prev = prev;
    A.Y = carve<double>(p, blk); A.F0 = carve<double>(p, blk); A.SC = carve<double>(p, blk);
    A.ZM = carve<double>(p, 8 * blk); A.ZA = carve<double>(p, 8 * blk); A.ZB = carve<double>(p, 8 * blk);
    A.OUT = carve<double>(p, 8 * blk); A.DIAG = carve<double>(p, 8 * blk);
    double *irc = carve<double>(p, (size_t)nlev * M), *mmass = carve<double>(p, M);
    int *mbody = carve<int>(p, M), *mgroup = carve<int>(p, M), *mq0 = carve<int>(p, M), *mq1 = carve<int>(p, M);
    int *pidx = carve<int>(p, nq);
    int *d_gbase = carve<int>(p, ng + 1), *d_gslot0 = carve<int>(p, ng);
    int *gseq = carve<int>(p, ng);
    A.gstat = carve<int>(p, ng);
    A.gkconv = carve<int>(p, ng);
    A.gt = carve<double>(p, ng);
    A.gH = carve<double>(p, ng);
    A.gatt = carve<long long>(p, ng);
    A.gacc = carve<long long>(p, ng);
    A.grej = carve<long long>(p, ng);
    A.gerr = carve<unsigned long long>(p, 8 * (size_t)ng);
    A.bar = carve<GridBarrier>(p, 1);
    A.mgroup = mgroup; A.mq0 = mq0; A.mq1 = mq1; A.pidx = pidx; A.mmass = mmass; A.irc = irc;
    A.mbody = mbody; A.gbase = d_gbase; A.mmass_rw = mmass; A.ctr = s->ctr;
    A.coll = coll_args(s);
    A.gseq = Ode::COLL ? gseq : nullptr;
    A.morder = Ode::COLL ? carve<int>(p, M) : nullptr;
    A.malive = Ode::COLL ? carve<int>(p, M) : nullptr;
    A.G = s->p.G; A.mu = s->p.G * s->p.m_star; A.dt = dt; A.tol = s->p.bs_tol;
    A.max_steps = s->p.bs_max_steps;
    A.barrier_ns = s->barrier_limit_ns;
    A.barrier_absent = s->barrier_absent;

    cudaStream_t st = s->stream;
    if (cudaMemcpyAsync(d_gbase, gbase.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_gslot0, gslot0.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GENGA_ECUDA;
    RcPtrs rcp;
    for (int l = 0; l < kMaxLevels; l++) rcp.p[l] = s->rcl[l].rc;
    const unsigned gm = (unsigned)((M + 127) / 128);
    bsm_members_kernel<<<gm, 128, 0, st>>>(ng, d_gbase, d_gslot0, s->member, s->slotof, s->csr[level].off,
                                          s->csr[level].list, s->mass, rcp, nlev, M, mbody, mgroup, mq0, mq1,
                                          pidx, mmass, irc);
    bsm_init_groups_kernel<<<(unsigned)((ng + 127) / 128), 128, 0, st>>>(A);
    if (pairs) {
        if (cudaMemsetAsync(pcount, 0, sizeof(int), st) != cudaSuccess) return GENGA_ECUDA;
        bsm_pairs_kernel<<<gm, 128, 0, st>>>(M, mq0, mq1, pidx, mbody, s->csr[level].list, pcount, pq, pm, prev);
        ++s->launches;
    }
    if (Ode::COLL) {
        bsm_coll_init_kernel<<<gm, 128, 0, st>>>(A);
        ++s->launches;
    }
    gather(st, mbody, A.Y);
    s->launches += 3;
    if (cudaGetLastError() != cudaSuccess) return GENGA_ECUDA;

    void *args[] = {&A};
    if (cudaLaunchCooperativeKernel((const void *)bsm_persistent_kernel<Ode>, dim3(grid), dim3(kPThreads), args,
                                    0, st) != cudaSuccess)
        return GENGA_ECUDA;
    ++s->launches;
    GridBarrier hb;
    if (cudaMemcpyAsync(&hb, A.bar, sizeof(hb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GENGA_ECUDA;
    ++s->host_syncs;
    if (hb.err) {
        snprintf(s->err, sizeof(s->err),
                 "persistent Bulirsch-Stoer: a grid-barrier wait exceeded its limit of %.3g s",
                 1e-9 * (double)s->barrier_limit_ns);
        return GENGA_ETIMEOUT;
    }
    scatter(st, mbody, A.Y);
    bsm_stats_kernel<<<1, 1, 0, st>>>(A, s->ctr, count_steps ? 1 : 0);
    s->launches += 2;
    return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}

int members_of(const std::vector<int2> &groups) {
    int t = 0;
    for (const int2 &g : groups) t += g.y;
    return t;
}

}  // namespace

void bsm_release(genga_system *s) {
    BsmBuffers *b = static_cast<BsmBuffers *>(s->bsm);
    if (!b) return;
    if (b->raw) cudaFree(b->raw);
    delete b;
    s->bsm = nullptr;
}

// Forward BS of every group larger than kBlockGroupMax, from the level's
// pre-drift state into pos/vel.
int bsm_forward_groups(genga_system *s, int level, double dt_l) {
    std::vector<int2> groups;
    if (batched_groups(s, groups) != 0) return GENGA_ECUDA;
    if (groups.empty()) return GENGA_OK;
    const double *pre_pos = s->pre_pos[level], *pre_vel = s->pre_vel[level];
    double *pos = s->pos, *vel = s->vel;
    const int n = (int)s->n;
    const int M = members_of(groups);
    const unsigned gr = (unsigned)((M + 127) / 128);
    auto gather = [&](cudaStream_t st, const int *mbody, double *Y) {
        bsm_gather_fwd<<<gr, 128, 0, st>>>(n, M, mbody, pre_pos, pre_vel, Y);
    };
    auto scatter = [&](cudaStream_t st, const int *mbody, const double *Y) {
        bsm_scatter_fwd<<<gr, 128, 0, st>>>(n, M, mbody, Y, pos, vel);
    };
    if (s->coll_on) return bsm_run<FwdCollOde>(s, level, dt_l, groups, true, gather, scatter);
    return bsm_run<FwdOde>(s, level, dt_l, groups, true, gather, scatter);
}

// Bulirsch-Stoer of every group of the current grouping at `level`: the
// in-block kernels for groups of up to kBlockGroupMax members on the side
// streams, then (joined, so that the cooperative launch has the GPU to
// itself) the persistent driver for the larger ones.
int run_bs(genga_system *s, int level, double dt_l, int64_t np) {
    if (np <= 0) return GENGA_OK;
    ++s->bs_call;                         // orders the merger records of the calls
    unsigned counts[kBuckets];
    int rc = phase_mark(s, GENGA_PH_BUCKETS);
    if (rc != GENGA_OK) return rc;
    if (bucket_groups(s, counts) != cudaSuccess) return GENGA_ECUDA;
    if ((rc = phase_mark(s, GENGA_PH_BS_SMALL)) != GENGA_OK) return rc;
    const cudaError_t e = launch_bs(s, level, dt_l, counts);
    if (join_bs(s) != cudaSuccess || e != cudaSuccess) return GENGA_ECUDA;
    if (!counts[kBuckets - 1]) return GENGA_OK;
    if ((rc = phase_mark(s, GENGA_PH_BS_LARGE)) != GENGA_OK) return rc;
    return bsm_forward_groups(s, level, dt_l);
}

extern "C" int genga_set_bs_pair_mode(genga_system_t *s, int32_t mode) {
    if (!s || mode < GENGA_BS_PAIRS_AUTO || mode > GENGA_BS_PAIRS_ON) return GENGA_EINVAL;
    s->bs_pairs = mode;
    return GENGA_OK;
}

int run_bs_dev(genga_system *s, int level, double dt_l) {
    ++s->bs_call;
    int rc = phase_mark(s, GENGA_PH_BUCKETS);
    if (rc != GENGA_OK) return rc;
    if (bucket_groups_async(s) != cudaSuccess) return GENGA_ECUDA;
    if ((rc = phase_mark(s, GENGA_PH_BS_SMALL)) != GENGA_OK) return rc;
    const cudaError_t e = launch_bs(s, level, dt_l, nullptr);
    if (join_bs(s) != cudaSuccess || e != cudaSuccess) return GENGA_ECUDA;
    // the counts were copied before the kernels above run: the GPU keeps
    // working while the host reads them
    if (cudaEventSynchronize(s->ev_counts) != cudaSuccess) return GENGA_ECUDA;
    ++s->host_syncs;
    if (!s->bucket_host[kBuckets - 1]) return GENGA_OK;
    if ((rc = phase_mark(s, GENGA_PH_BS_LARGE)) != GENGA_OK) return rc;
    return bsm_forward_groups(s, level, dt_l);
}

// Adjoint BS (backward, augmented) of every group larger than kBlockGroupMax.
int bsm_adjoint_groups(genga_system *s, const double *x2, const double *v2, double *lx, double *lv,
                       double *lm, double dt) {
    std::vector<int2> groups;
    if (batched_groups(s, groups) != 0) return GENGA_ECUDA;
    if (groups.empty()) return GENGA_OK;
    const int n = (int)s->n;
    const int M = members_of(groups);
    const unsigned gr = (unsigned)((M + 127) / 128);
    return bsm_run<AdjOde>(
        s, 0, dt, groups, false,
        [&](cudaStream_t st, const int *mbody, double *Y) {
            bsm_gather_adj<<<gr, 128, 0, st>>>(n, M, mbody, x2, v2, lx, lv, Y);
        },
        [&](cudaStream_t st, const int *mbody, const double *Y) {
            bsm_scatter_adj<<<gr, 128, 0, st>>>(n, M, mbody, Y, lx, lv, lm);
        });
}

}  // namespace genga
