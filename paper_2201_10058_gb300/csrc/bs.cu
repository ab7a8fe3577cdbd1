// bs.cu -- Bulirsch-Stoer integration of close-encounter groups (Sec. 6.1,
// Appendix A "Bulirsch-Stoer(dt)") and the level kick KickS of the
// higher-level changeover scheme (Sec. 6.3, Appendix A).
//
// BS for groups of at most kBlockGroupMax (32) members: one CTA per group at a
// time (the CTAs claim their bucket's groups) with the 8 extrapolation columns
// advanced at once (bs_cols_kernel below; larger groups go to the batched
// grid-wide driver in bsm.cu).  Each member
// integrates
//     dx/dt = v,   dv/dt = -mu x/|x|^3 + G sum_{partners j} m_j W_ij (x_j - x)/r^3,
//     W_ij = prod_{k=0..level} (1 - K(r_ij; rc_k,ij)),
// with partners taken from the ascending partner list of the level's
// encounter pairs (the BS-A partner-list scheme of Sec. 6.1; the sum order is
// fixed, so results do not depend on member layout).  Modified midpoint with
// n = 2, 4, ..., 16 and polynomial extrapolation in h^2 (Neville); error =
// max over members and components of |T_kk - T_k,k-1| / scale with
// scale = |y| + |H dy/dt| + 1e-300; accept at the first column k >= 1 with
// error <= tol, grow H by 1.5 if k < 4, otherwise halve H.  The step control is
// evaluated identically by every thread after a CTA-wide max reduction.
#include "common.cuh"

namespace genga {
namespace {


struct BsArgs {
    int n;
    const double *pre_pos, *pre_vel;
    double *pos, *vel;
    const double *mass;
    const double *rc[kMaxLevels];
    int nlev;
    const int *off, *list;
    const int *glist, *goff, *member, *slotof;
    const int *blist;      // this kernel's bucket: group labels
    int bucket;            // its index (device count and claim counter)
    double G, mu, dt, tol;
    int max_steps;
    unsigned long long time_limit_ns;
    DevCounters *ctr;
    CollArgs coll;         // collisions (Sec. 7.1-7.2), used by the COLL instances
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// KickS at level l >= 1 over the level-(l-1) encounter pairs:
//   v_b += dt_half G sum_p m_p prod_{k<l}(1 - K_k) K_l (x_p - x_b)/r^3.
// Phase 1, one thread per undirected pair (i < j): g = prod_{k<l}(1 - K_k) K_l / r^3
// (0 when the pair is beyond rc_0, where 1 - K_0 = 0) and the pair's two
// mass-weighted terms m_j g (x_j - x_i) (for i) and -m_i g (x_j - x_i) (for j),
// each a 32-byte record written to the pair's entry in the row of its body
// (ent), so that phase 2 reads every row as one contiguous run.  Factors
// outside their changeover band (K = 0 or 1 exactly) are decided from FP32
// copies, so they cost no FP64 operation.
// Phase 2, one body per kApplyLanes lanes: the records of its row, in
// ascending partner order per lane, lanes combined in a fixed butterfly -- a
// fixed summation order.
struct KickPairsArgs {
    int n, nb, level;
    long long np;
    const uint2 *pairs;
    const int *bodies;
    const int *off, *ent;
    double4_32a *term;     // one record per entry
    const double *pos;
    double *vel;
    const double *mass;
    const double *irc[kMaxLevels];   // 1 / rc per level and body
    const float *thr_rc0;            // FP32 upper bound of rc_0^2 per body
    double G, dt_half;
};

// Float copy of a positive double, truncated, saturating: +inf at or above
// 2^128, 0 below 2^-126 (integer operations only).  Monotone, and never above
// its argument except where that is >= 2^128.
__device__ __forceinline__ float f32_of_f64_trunc_sat(double v) {
    const unsigned hi = (unsigned)__double2hiint(v);
    if (hi >= 0x47f00000u) return __int_as_float(0x7f800000);
    if (hi < 0x38100000u) return 0.0f;
    return __uint_as_float(((hi - 0x38000000u) << 3) | ((unsigned)__double2loint(v) >> 29));
}

__global__ void kick_pairs_terms_kernel(KickPairsArgs A) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.np) return;
    const uint2 pr = A.pairs[k];
    const int i = (int)pr.x, j = (int)pr.y;
    const size_t N = (size_t)A.n;
    const double dx = A.pos[j] - A.pos[i], dy = A.pos[N + j] - A.pos[N + i],
                 dz = A.pos[2 * N + j] - A.pos[2 * N + i];
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    double g = 0.0;
    // beyond the FP32 bound of rc_0^2 (> rc_0^2 (1 + 2^-16)) the factor 1 - K_0
    // is exactly zero
    if (f32_of_f64_trunc_sat(r2) <= fmaxf(A.thr_rc0[i], A.thr_rc0[j])) {
        const double yv = rsqrt_newton(r2);
        const double r = r2 * yv;
        const float rf = f32_of_f64_trunc_sat(r);
        double W = 1.0;
        bool zero = false;
        // 1 / rc_ij = 1 / max(rc_i, rc_j) = min(1/rc_i, 1/rc_j), bit for bit
        for (int l = 0; l < A.level; l++) {
            const int side = changeover_side_f32(
                rf, fminf(f32_of_f64_trunc_sat(A.irc[l][i]), f32_of_f64_trunc_sat(A.irc[l][j])));
            if (side < 0) continue;
            if (side > 0) { zero = true; break; }
            W *= 1.0 - changeover_fast(r, fmin(A.irc[l][i], A.irc[l][j]));
        }
        if (!zero) {
            const int l = A.level;
            const int side = changeover_side_f32(
                rf, fminf(f32_of_f64_trunc_sat(A.irc[l][i]), f32_of_f64_trunc_sat(A.irc[l][j])));
            if (side == 0) W *= changeover_fast(r, fmin(A.irc[l][i], A.irc[l][j]));
            if (side >= 0) g = W * (yv * yv * yv);
        }
    }
    const double ci = A.mass[j] * g, cj = -A.mass[i] * g;
    const int2 e = reinterpret_cast<const int2 *>(A.ent)[k];
    A.term[e.x] = make_double4_32a(ci * dx, ci * dy, ci * dz, 0.0);
    A.term[e.y] = make_double4_32a(cj * dx, cj * dy, cj * dz, 0.0);
}

constexpr int kApplyLanes = 8;

__global__ void kick_pairs_apply_kernel(KickPairsArgs A) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / kApplyLanes, sub = gt % kApplyLanes;
    const size_t N = (size_t)A.n;
    int b = 0, q0 = 0, q1 = 0;
    if (t < A.nb) {
        b = A.bodies[t];
        q0 = A.off[b];
        q1 = A.off[b + 1];
    }
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int q = q0 + sub; q < q1; q += kApplyLanes) {
        const double4_32a w = A.term[q];
        sx += w.x;
        sy += w.y;
        sz += w.z;
    }
#pragma unroll
    for (int o = kApplyLanes / 2; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (t < A.nb && sub == 0) {
        A.vel[b] += A.dt_half * (A.G * sx);
        A.vel[N + b] += A.dt_half * (A.G * sy);
        A.vel[2 * N + b] += A.dt_half * (A.G * sz);
    }
}

// ---------------------------------------------------------------------------
// Column-parallel Bulirsch-Stoer for groups of at most 32 members.  The 8
// extrapolation columns of one step attempt (modified midpoint with n = 2, 4,
// ..., 16 sub-steps) are independent integrations from the same start, so a CTA
// of 8 x M threads runs them at once: thread (k, a) integrates column k for
// member a (M = 4, 8, 16 or 32 member slots).  One attempt then costs 16
// sequential derivative evaluations instead of 2 + 4 + ... + 16 + 8 = 80; the
// Neville table is built per (member, component) afterwards and the first
// column k >= 1 under tolerance is accepted -- the same arithmetic and the same
// acceptance rule as the serial scheme.  FP64 throughout.
// Pairs of a group of M member slots evaluated once each (M <= 16), listed
// in (a, q) order with a < q; at most M (M - 1) / 2.
template <int M>
constexpr int kColsPairs = (M <= 16) ? M * (M - 1) / 2 : 1;

template <int M>
struct ColsShared {
    double zx[8 * M + 1], zy[8 * M + 1], zz[8 * M + 1];   // current positions, per (column, member); + a zero
    double pt[3][8][kColsPairs<M>];              // W r^-3 (x_q - x_a) per column and pair a < q
    unsigned char pa[kColsPairs<M>], pq[kColsPairs<M>];   // the group's pairs (a < q), by a then q
    unsigned char pidx[M <= 16 ? M * M : 1];     // (a, q) -> pair index, both orders
    unsigned pmask[M];                           // partner ranks of each member
    int npairs;
    double m[M];
    double irc[kMaxLevels][M];
    float ircf[kMaxLevels][M];                   // 1/rc rounded to float towards zero (band side tests)
    double y[6][M], f0[6][M];                    // attempt start and its derivative
    double zf[3][6][M];                          // the completing column's z_n, z_{n-1}, f(z_n)
    double hcol[8];                              // sub-step H / n_k of each column
    double ynew[6][M];                           // accepted state
    int rank_of_slot[M];
    int flag;
    // collisions: radius, alive flag and body index of each member rank
    double R[M];
    int alive[M];
    int body[M];
};

template <int M, bool COLL>
__device__ __forceinline__ void cols_deriv(const BsArgs &A, ColsShared<M> &S, int tid, int col,
                                           bool active, unsigned mask, const double *irc_self,
                                           const double z[6], double f[6]) {
    __syncthreads();
    S.zx[tid] = z[0]; S.zy[tid] = z[1]; S.zz[tid] = z[2];
    __syncthreads();
    f[0] = z[3]; f[1] = z[4]; f[2] = z[5];
    if constexpr (M == 4) {
        if (S.npairs == 1) {
            // two members and their pair in one instruction stream: lane a
            // (a = 0, 1) takes the star term of member a as the displacement
            // from a zero slot, lane 2 the pair (0, 1) -- the operations of the
            // general form below on the same values, so the same results
            const int a = tid % M;
            const bool pl = a == 2;
            const int i1 = col * M + (pl ? 1 : a), i0 = pl ? col * M : 8 * M;
            const double ex = S.zx[i1] - S.zx[i0], ey = S.zy[i1] - S.zy[i0], ez = S.zz[i1] - S.zz[i0];
            const double r2 = fma(ez, ez, fma(ey, ey, ex * ex));
            const double yv = rsqrt_newton(r2);
            double sst = 0.0;
            if (pl) {
                const double d = r2 * yv;
                const float df = f32_of_f64_trunc(d);
                double W = 1.0;
                for (int l = 0; l < A.nlev; l++) {
                    const int side = changeover_side_f32(df, fminf(S.ircf[l][0], S.ircf[l][1]));
                    if (side < 0) continue;
                    if (side > 0) { W = 0.0; break; }
                    W *= 1.0 - changeover_fast(d, fmin(S.irc[l][0], S.irc[l][1]));
                }
                const double c = W * (yv * yv * yv);
                S.pt[0][col][0] = c * ex;
                S.pt[1][col][0] = c * ey;
                S.pt[2][col][0] = c * ez;
            } else if (active) {
                sst = -A.mu * (yv * yv * yv);
            }
            __syncthreads();
            if (!active) { f[3] = f[4] = f[5] = 0.0; return; }
            double px = 0.0, py = 0.0, pz = 0.0;
            if (!(COLL && !S.alive[a]) && mask) {
                const double w = a == 0 ? S.m[1] : -S.m[0];
                px = fma(w, S.pt[0][col][0], px);
                py = fma(w, S.pt[1][col][0], py);
                pz = fma(w, S.pt[2][col][0], pz);
            }
            f[3] = fma(sst, z[0], A.G * px);
            f[4] = fma(sst, z[1], A.G * py);
            f[5] = fma(sst, z[2], A.G * pz);
            return;
        }
    }
    if constexpr (M <= 16) {
        // each pair once; then every member sums its partners' terms in
        // ascending rank order (m_q t for q > a, -m_q t for q < a): exactly
        // antisymmetric pair forces
        const int a = tid % M;
        // own star term first: an independent dependency chain the compiler can
        // interleave with the first pair's (small-group BS is latency-bound)
        double sst = 0.0;
        if (active) {
            const double r2s = fma(z[2], z[2], fma(z[1], z[1], z[0] * z[0]));
            const double ys = rsqrt_newton(r2s);
            sst = -A.mu * (ys * ys * ys);
        }
        // the column's pairs round-robin over its M threads (short chains)
        for (int pi = a; pi < S.npairs; pi += M) {
            const int pa = S.pa[pi], pq = S.pq[pi];
            const int la = col * M + pa, lq = col * M + pq;
            const double dx = S.zx[lq] - S.zx[la], dy = S.zy[lq] - S.zy[la], dz = S.zz[lq] - S.zz[la];
            const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double yv = rsqrt_newton(d2);
            const double d = d2 * yv;
            const float df = f32_of_f64_trunc(d);
            double W = 1.0;
            // factors 1 - K outside the band (1 or 0) decided in FP32, exactly
            for (int l = 0; l < A.nlev; l++) {
                const int side = changeover_side_f32(df, fminf(S.ircf[l][pa], S.ircf[l][pq]));
                if (side < 0) continue;
                if (side > 0) { W = 0.0; break; }
                W *= 1.0 - changeover_fast(d, fmin(S.irc[l][pa], S.irc[l][pq]));
            }
            const double c = W * (yv * yv * yv);
            S.pt[0][col][pi] = c * dx;
            S.pt[1][col][pi] = c * dy;
            S.pt[2][col][pi] = c * dz;
        }
        __syncthreads();
        if (!active) { f[3] = f[4] = f[5] = 0.0; return; }
        double px = 0.0, py = 0.0, pz = 0.0;
        // a member merged away feels only the star (its partners' masses are
        // 0 after their mergers, so their terms vanish)
        unsigned mm = (COLL && !S.alive[a]) ? 0u : mask;
        while (mm) {
            const int q = __ffs(mm) - 1;
            mm &= mm - 1;
            const int pi = S.pidx[a * M + q];
            const double w = q > a ? S.m[q] : -S.m[q];
            px = fma(w, S.pt[0][col][pi], px);
            py = fma(w, S.pt[1][col][pi], py);
            pz = fma(w, S.pt[2][col][pi], pz);
        }
        f[3] = fma(sst, z[0], A.G * px);
        f[4] = fma(sst, z[1], A.G * py);
        f[5] = fma(sst, z[2], A.G * pz);
        return;
    }
    if (!active) { f[3] = f[4] = f[5] = 0.0; return; }
    const double r2s = fma(z[2], z[2], fma(z[1], z[1], z[0] * z[0]));
    const double ys = rsqrt_newton(r2s);
    const double sst = -A.mu * (ys * ys * ys);
    double px = 0.0, py = 0.0, pz = 0.0;
    unsigned mm = (COLL && !S.alive[tid % M]) ? 0u : mask;
    while (mm) {
        const int q = __ffs(mm) - 1;
        mm &= mm - 1;
        const int lq = col * M + q;
        const double dx = S.zx[lq] - z[0], dy = S.zy[lq] - z[1], dz = S.zz[lq] - z[2];
        const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double yv = rsqrt_newton(d2);
        const double d = d2 * yv;
        const float df = f32_of_f64_trunc(d);
        double W = 1.0;
        for (int l = 0; l < A.nlev; l++) {
            const int side = changeover_side_f32(df, fminf(S.ircf[l][tid % M], S.ircf[l][q]));
            if (side < 0) continue;
            if (side > 0) { W = 0.0; break; }
            W *= 1.0 - changeover_fast(d, fmin(irc_self[l], S.irc[l][q]));
        }
        const double c = S.m[q] * W * (yv * yv * yv);
        px = fma(c, dx, px); py = fma(c, dy, py); pz = fma(c, dz, pz);
    }
    f[3] = fma(sst, z[0], A.G * px);
    f[4] = fma(sst, z[1], A.G * py);
    f[5] = fma(sst, z[2], A.G * pz);
}

// Row k of the Neville table in h^2 (n_k = 2(k+1)), in place in T:
// T_k0 = cur, T_kj = T_k,j-1 + (T_k,j-1 - T_k-1,j-1) (n_k-j)^2 / (j (2k+2-j)) with the
// coefficients as exact compile-time doubles; returns T_kk and T_k,k-1.
template <int K>
__device__ __forceinline__ void neville_row_k(double (&T)[8], double cur, double &diag, double &prevdiag) {
    double prev = T[0];
    T[0] = cur;
#pragma unroll
    for (int j = 1; j <= K; j++) {
        const double coef = (double)((K - j + 1) * (K - j + 1)) / (double)(j * (2 * K + 2 - j));
        const double nxt = fma(cur - prev, coef, cur);
        prev = T[j];
        T[j] = nxt;
        cur = nxt;
    }
    diag = T[K];
    prevdiag = K >= 1 ? T[K >= 1 ? K - 1 : 0] : 0.0;
}
__device__ __forceinline__ void neville_row(int k, double (&T)[8], double cur, double &diag, double &prevdiag) {
    switch (k) {
    case 0: neville_row_k<0>(T, cur, diag, prevdiag); break;
    case 1: neville_row_k<1>(T, cur, diag, prevdiag); break;
    case 2: neville_row_k<2>(T, cur, diag, prevdiag); break;
    case 3: neville_row_k<3>(T, cur, diag, prevdiag); break;
    case 4: neville_row_k<4>(T, cur, diag, prevdiag); break;
    case 5: neville_row_k<5>(T, cur, diag, prevdiag); break;
    case 6: neville_row_k<6>(T, cur, diag, prevdiag); break;
    default: neville_row_k<7>(T, cur, diag, prevdiag); break;
    }
}

// Collisions (Sec. 7.1-7.2, reading R25) of one group, by its first thread on
// the state S.ynew (member rank a holds body S.body[a]; ranks ascend with the
// body index, so the pairs (a, q > a) taken rank by rank and partner by
// partner come in ascending (i, j) order).
// Deepest overlap fraction (R_a + R_q - r)/(R_a + R_q) over the group's pairs
// of alive bodies; 0 when no pair overlaps.
template <int M>
__device__ double cols_overlap(const ColsShared<M> &S, int nm) {
    double deepest = 0.0;
    for (int a = 0; a < nm; a++) {
        if (!S.alive[a]) continue;
        unsigned mm = S.pmask[a] & ~((2u << a) - 1u);
        while (mm) {
            const int q = __ffs(mm) - 1;
            mm &= mm - 1;
            if (!S.alive[q]) continue;
            const double r = __dsqrt_rn(dist2_rn(__dsub_rn(S.ynew[0][q], S.ynew[0][a]),
                                                 __dsub_rn(S.ynew[1][q], S.ynew[1][a]),
                                                 __dsub_rn(S.ynew[2][q], S.ynew[2][a])));
            const double Rs = __dadd_rn(S.R[a], S.R[q]);
            if (r < Rs) deepest = fmax(deepest, __ddiv_rn(__dsub_rn(Rs, r), Rs));
        }
    }
    return deepest;
}

// Mergers of the overlapping pairs of alive bodies at time t of the call, in
// ascending pair order, each seeing the mergers before it; logged with the
// group label and a running sequence number.
template <int M>
__device__ void cols_merge(const BsArgs &A, ColsShared<M> &S, int nm, double t, int label, int &seq) {
    const size_t N = (size_t)A.n;
    for (int a = 0; a < nm; a++) {
        unsigned mm = S.pmask[a] & ~((2u << a) - 1u);
        while (mm) {
            const int q = __ffs(mm) - 1;
            mm &= mm - 1;
            if (!S.alive[a] || !S.alive[q]) continue;
            const double r = __dsqrt_rn(dist2_rn(__dsub_rn(S.ynew[0][q], S.ynew[0][a]),
                                                 __dsub_rn(S.ynew[1][q], S.ynew[1][a]),
                                                 __dsub_rn(S.ynew[2][q], S.ynew[2][a])));
            const double Rs = __dadd_rn(S.R[a], S.R[q]);
            if (!(r < Rs)) continue;
            double xa[3], va[3], xq[3], vq[3], xo[3], vo[3], dU, rr;
            for (int k = 0; k < 3; k++) {
                xa[k] = S.ynew[k][a]; va[k] = S.ynew[3 + k][a];
                xq[k] = S.ynew[k][q]; vq[k] = S.ynew[3 + k][q];
            }
            const int ia = S.body[a], iq = S.body[q];
            const int sv = merge_bodies(A.coll, N, ia, iq, xa, va, xq, vq, xo, vo, &dU, &rr);
            const int ks = sv == ia ? a : q, ko = sv == ia ? q : a;
            for (int k = 0; k < 3; k++) { S.ynew[k][ks] = xo[k]; S.ynew[3 + k][ks] = vo[k]; }
            S.m[ks] = A.coll.mass[sv];
            S.R[ks] = A.coll.radius[sv];
            S.m[ko] = 0.0;
            S.R[ko] = 0.0;
            S.alive[ko] = 0;
            log_merger(A.coll, A.ctr, label, seq++, t, ia, iq, r, Rs, dU);
        }
    }
}

// One group g on the whole block.
template <int M, bool COLL>
__device__ __forceinline__ void cols_group(const BsArgs &A, ColsShared<M> &S, int g) {
    const int tid = threadIdx.x;
    const int col = tid / M, a = tid % M;
    const int s0 = A.goff[g], nm = A.goff[g + 1] - s0;
    if (nm > M || (M > 4 && nm <= M / 2)) return;          // not this bucket (never taken)
    const unsigned long long t_start = global_ns();
    const size_t N = (size_t)A.n;

    // member a of rank a (ascending body index), computed by the column-0 threads
    if (tid < M) {
        int mine = (a < nm) ? A.member[s0 + a] : 0x7fffffff;
        int rank = 0;
        for (int q = 0; q < nm; q++) rank += (A.member[s0 + q] < mine);
        if (a < nm) S.rank_of_slot[a] = rank;
    }
    __syncthreads();
    const bool active = a < nm;
    int b = 0;
    if (active)
        for (int q = 0; q < nm; q++)
            if (S.rank_of_slot[q] == a) b = A.member[s0 + q];
    double irc_self[kMaxLevels];
    unsigned pmask = 0;
    double y[6];
    for (int l = 0; l < kMaxLevels; l++) irc_self[l] = 0.0;
    for (int c = 0; c < 6; c++) y[c] = 0.0;
    if (active) {
        for (int l = 0; l < A.nlev; l++) irc_self[l] = 1.0 / A.rc[l][b];
        for (int q = A.off[b]; q < A.off[b + 1]; q++)
            pmask |= 1u << S.rank_of_slot[A.slotof[A.list[q]] - s0];
        for (int c = 0; c < 3; c++) { y[c] = A.pre_pos[c * N + b]; y[3 + c] = A.pre_vel[c * N + b]; }
        if (col == 0) {
            S.m[a] = A.mass[b];
            for (int l = 0; l < A.nlev; l++) {
                S.irc[l][a] = irc_self[l];
                S.ircf[l][a] = __double2float_rz(irc_self[l]);
            }
        }
    }
    if (COLL && col == 0) {
        S.R[a] = active ? A.coll.radius[b] : 0.0;
        S.alive[a] = active ? (int)A.coll.alive[b] : 0;
        S.body[a] = b;
    }
    if (COLL || M <= 16) {
        if (col == 0) S.pmask[a] = active ? pmask : 0u;
    }
    if constexpr (M <= 16) {
        __syncthreads();
        if (tid == 0) {                          // pair list in (a, q) order
            int np = 0;
            for (int aa = 0; aa < M; aa++) {
                unsigned mm = S.pmask[aa] & ~((2u << aa) - 1u);
                while (mm) {
                    const int q = __ffs(mm) - 1;
                    mm &= mm - 1;
                    S.pa[np] = (unsigned char)aa;
                    S.pq[np] = (unsigned char)q;
                    S.pidx[aa * M + q] = S.pidx[q * M + aa] = (unsigned char)np;
                    np++;
                }
            }
            S.npairs = np;
            S.zx[8 * M] = S.zy[8 * M] = S.zz[8 * M] = 0.0;   // the zero slot
        }
    }
    __syncthreads();

    int seq = 0;        // mergers of this group so far (log order)
    if (COLL) {
        // pairs already overlapping when the integration starts merge at once
        if (col == 0 && active)
            for (int c = 0; c < 6; c++) S.ynew[c][a] = y[c];
        __syncthreads();
        if (tid == 0) cols_merge<M>(A, S, nm, 0.0, g, seq);
        __syncthreads();
        if (active) for (int c = 0; c < 6; c++) y[c] = S.ynew[c][a];
    }

    const int nk = 2 * (col + 1);
    double t = 0.0, H = A.dt;
    int attempts = 0;
    long long acc = 0, rej = 0;
    int failed = 0;     // 1: attempt limit, 2: time limit
    double f0[6], zm[6], zn[6], fz[6];
    while (t < A.dt) {
        if (tid == 0)
            S.flag = attempts >= A.max_steps ? 1 : (global_ns() - t_start >= A.time_limit_ns ? 2 : 0);
        __syncthreads();
        if (S.flag) { failed = S.flag; break; }
        attempts++;
        if (H > A.dt - t) H = A.dt - t;
        cols_deriv<M, COLL>(A, S, tid, col, active, pmask, irc_self, y, f0);
        if (col == 0)
            for (int c = 0; c < 6; c++) { S.y[c][a] = y[c]; S.f0[c][a] = f0[c]; }
        // all 8 columns at once: column col takes nk midpoint sub-steps of H/nk.
        // Column k is complete after sub-step 2(k+1); its Neville row is built at
        // once (per component c = col < 6 and member a) and the attempt stops at
        // the first column k >= 1 under tolerance -- the columns beyond it are
        // never needed, so they are not computed to the end.
        const double h = H / nk;
        if (a == 0) S.hcol[col] = h;
        for (int c = 0; c < 6; c++) { zm[c] = y[c]; zn[c] = fma(h, f0[c], y[c]); }
        double T[8];
        double tsc = 0.0, diag = 0.0;
        int kconv = -1;
        for (int it = 1; it <= 16; it++) {
            cols_deriv<M, COLL>(A, S, tid, col, active, pmask, irc_self, zn, fz);
            if (it < nk) {
                for (int c = 0; c < 6; c++) {
                    const double tt = fma(2.0 * h, fz[c], zm[c]);
                    zm[c] = zn[c];
                    zn[c] = tt;
                }
            } else if (it == nk) {
                // the column's final smoothing step is formed by the Neville
                // lanes below (one component each), not by this column's lanes
                // while the others take midpoint sub-steps
                for (int c = 0; c < 6; c++) {
                    S.zf[0][c][a] = zn[c];
                    S.zf[1][c][a] = zm[c];
                    S.zf[2][c][a] = fz[c];
                }
            }
            if (it & 1) continue;
            const int k = it / 2 - 1;                    // column just completed
            __syncthreads();
            // error |T_kk - T_k,k-1| / scale <= tol for every member and
            // component, tested as |T_kk - T_k,k-1| <= tol scale and combined
            // by a block-wide vote
            bool ok = true;
            if (col < 6 && active) {
                if (k == 0) tsc = A.tol * (fabs(S.y[col][a]) + fabs(H * S.f0[col][a]) + 1e-300);
                double prevdiag = 0.0;
                const double yk = 0.5 * (S.zf[0][col][a] + S.zf[1][col][a] + S.hcol[k] * S.zf[2][col][a]);
                neville_row(k, T, yk, diag, prevdiag);
                ok = fabs(diag - prevdiag) <= tsc;
            }
            if (k >= 1 && __syncthreads_and(ok)) { kconv = k; break; }
        }
        bool accept = kconv >= 0;
        if (accept) {
            if (col < 6 && active) S.ynew[col][a] = diag;
            __syncthreads();
            if (COLL && A.coll.tol > 0.0) {
                // collision precision (Sec. 7.2): a step that ends with an
                // overlap of tol or more of the radius sum ends too late
                if (tid == 0) S.flag = cols_overlap<M>(S, nm) >= A.coll.tol ? 1 : 0;
                __syncthreads();
                accept = S.flag == 0;
                __syncthreads();
            }
        }
        if (accept) {
            t += H;
            acc++;
            if (kconv < 4) H *= 1.5;
            if (COLL) {
                if (tid == 0) cols_merge<M>(A, S, nm, t, g, seq);
                __syncthreads();
            }
            if (active) for (int c = 0; c < 6; c++) y[c] = S.ynew[c][a];
        } else {
            rej++;
            H *= 0.5;
        }
    }
    if (active && col == 0)
        for (int c = 0; c < 3; c++) { A.pos[c * N + b] = y[c]; A.vel[c * N + b] = y[3 + c]; }
    if (tid == 0) {
        atomicMax(&A.ctr->bs_max_attempts, (unsigned long long)attempts);
        atomicAdd(&A.ctr->bs_steps, (unsigned long long)acc);
        atomicAdd(&A.ctr->bs_rejects, (unsigned long long)rej);
        if (failed) {
            atomicAdd(&A.ctr->bs_fail, 1ull);
            latch_error(A.ctr, failed == 2 ? kErrTimeout : kErrBS);
        }
    }
}

// Block b takes group b of its bucket, then claims the groups beyond the grid
// one at a time, until the bucket's count (left on the device by
// bucket_groups) is reached: the grid need not match the count, so the host
// launches it without reading the count first.  The first groups keep the
// block order, which the hardware spreads over the SMs (claims in arrival
// order would pile some SMs up).  Groups are independent, so which block
// takes which group does not change any result.
template <int M, bool COLL>
__global__ void __launch_bounds__(8 * M)
bs_cols_kernel(BsArgs A) {
    __shared__ ColsShared<M> S;
    __shared__ int claim;
    for (bool first = true;; first = false) {
        if (threadIdx.x == 0) {
            const unsigned q = first ? blockIdx.x : gridDim.x + atomicAdd(&A.ctr->bucket_next[A.bucket], 1u);
            claim = q < A.ctr->bucket_count[A.bucket] ? A.blist[q] : -1;
        }
        __syncthreads();
        const int g = claim;
        __syncthreads();                  // claim read by all before it is rewritten
        if (g < 0) return;
        cols_group<M, COLL>(A, S, g);
        __syncthreads();                  // S free for the next group
    }
}


}  // namespace

// Resident blocks of one in-block BS instance on the whole GPU (the
// per-SM figure depends only on the kernel, so it is asked for once).
template <int M, bool COLL>
int cols_capacity(const genga_system *s) {
    static int per_sm = 0;
    if (per_sm < 1) {
        int q = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, bs_cols_kernel<M, COLL>, 8 * M, 0) != cudaSuccess)
            q = 0;
        per_sm = q < 1 ? 1 : q;
    }
    return per_sm * s->num_sms;
}

template <int M>
cudaError_t launch_cols(genga_system *s, BsArgs A, int q, const unsigned *counts, bool coll) {
    const int cap = coll ? cols_capacity<M, true>(s) : cols_capacity<M, false>(s);
    // with the counts known: one block per group up to the resident capacity;
    // without: the resident capacity, the blocks claiming the device count
    const unsigned grid = counts ? std::min<unsigned>(counts[q], (unsigned)cap) : (unsigned)cap;
    if (grid == 0) return cudaSuccess;
    A.blist = s->bucket_list + (size_t)q * s->bucket_stride;
    A.bucket = q;
    if (coll) bs_cols_kernel<M, true><<<grid, 8 * M, 0, s->side[q]>>>(A);
    else bs_cols_kernel<M, false><<<grid, 8 * M, 0, s->side[q]>>>(A);
    ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_bs(genga_system *s, int level, double dt_l, const unsigned *counts) {
    BsArgs A;
    A.n = (int)s->n;
    A.pre_pos = s->pre_pos[level];
    A.pre_vel = s->pre_vel[level];
    A.pos = s->pos; A.vel = s->vel; A.mass = s->mass;
    for (int l = 0; l < kMaxLevels; l++) A.rc[l] = s->rcl[l].rc;
    A.nlev = level + 1;
    A.off = s->csr[level].off; A.list = s->csr[level].list;
    A.glist = s->glist; A.goff = s->goff; A.member = s->member; A.slotof = s->slotof;
    A.G = s->p.G; A.mu = s->p.G * s->p.m_star; A.dt = dt_l; A.tol = s->p.bs_tol;
    A.max_steps = s->p.bs_max_steps;
    A.time_limit_ns = s->bs_group_limit_ns;   // per group call (default 10 s)
    A.ctr = s->ctr;
    A.coll = coll_args(s);
    const bool coll = s->coll_on;
    // the four size buckets run concurrently on library-owned streams so that
    // their slowest groups overlap
    GENGA_CUDA_TRY(cudaEventRecord(s->ev_fork, s->stream));
    for (int q = 0; q < 4; q++) GENGA_CUDA_TRY(cudaStreamWaitEvent(s->side[q], s->ev_fork, 0));
    GENGA_CUDA_TRY(launch_cols<4>(s, A, 0, counts, coll));
    GENGA_CUDA_TRY(launch_cols<8>(s, A, 1, counts, coll));
    GENGA_CUDA_TRY(launch_cols<16>(s, A, 2, counts, coll));
    GENGA_CUDA_TRY(launch_cols<32>(s, A, 3, counts, coll));
    return cudaGetLastError();
}

cudaError_t join_bs(genga_system *s) {
    for (int q = 0; q < 4; q++) {
        GENGA_CUDA_TRY(cudaEventRecord(s->ev_join[q], s->side[q]));
        GENGA_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->ev_join[q], 0));
    }
    return cudaGetLastError();
}

cudaError_t launch_kick_pairs(genga_system *s, int level, double dt_half, int nb) {
    if (nb <= 0) return cudaSuccess;
    KickPairsArgs A;
    A.n = (int)s->n; A.nb = nb; A.level = level;
    A.np = s->npairs_host[level - 1];
    A.pairs = s->pairs[level - 1];
    A.bodies = s->bodies[level];
    A.off = s->csr[level - 1].off; A.ent = s->csr[level - 1].ent;
    A.term = reinterpret_cast<double4_32a *>(s->csr[level - 1].term);
    A.pos = s->pos; A.vel = s->vel; A.mass = s->mass;
    for (int l = 0; l < kMaxLevels; l++) A.irc[l] = s->rcl[l].irc;
    A.thr_rc0 = s->rcl[0].thr_rc;
    A.G = s->p.G; A.dt_half = dt_half;
    if (A.np > 0) {
        kick_pairs_terms_kernel<<<(unsigned)((A.np + 255) / 256), 256, 0, s->stream>>>(A); ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
    }
    const long long nt = (long long)nb * kApplyLanes;
    kick_pairs_apply_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s->stream>>>(A); ++s->launches;
    return cudaGetLastError();
}

}  // namespace genga
