// ensemble.cu -- many small systems integrated at once (the paper's
// multi-simulation mode, Sec. 6/7), with the GR (Sec. 3, Eq. apn) and tidal
// (Sec. 4.1-4.2) forces applied by the implicit midpoint rule (Sec. 2.3).
//
// One persistent launch integrates every system for K steps.  Each CTA takes
// systems from a work queue (largest first) and keeps a whole system (N <= 64
// bodies) in shared memory for all K steps:
//   Rcrit; Kick(dt/2) with the changeover function and a bitmask pre-check;
//   GR + tides (dt/2, implicit midpoint, heliocentric velocities, spins);
//   HC(dt/2); FG(dt); detection; grouping + Bulirsch-Stoer per group;
//   HC(dt/2); Kick(dt/2); GR + tides (dt/2).
// Small sums (momentum, star torque) are taken by one thread in body order, so
// they match a sequential evaluation.  The kick's pair loop is spread over
// (body, j-slice) threads -- the slice count is the tile shape the autotuner
// picks (threads per CTA).  Bulirsch-Stoer, rare here, keeps its state in a
// per-CTA global scratch.
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace genga {
namespace {

constexpr int kEnsMaxN = GENGA_ENSEMBLE_MAX_N;
constexpr int kEnsBsRows = 84;          // BS scratch rows per member slot

struct EnsArgs {
    int n_systems;
    const long long *offsets;
    const int *order;
    double *pos, *vel, *spin;
    long long ntot;
    const double *mass, *radius, *k2, *tau, *rg2;
    const double *m_star, *dt;
    double *star;                       // [S][8]
    double c2, inv_c2;
    int gr, tides;                      // gr: 1 Eq. apn by the implicit midpoint rule, 2 splitting
    double G, n1, n2, f_pc, bs_tol;
    int kepler_max_iter, bs_max_steps, implicit_max_iter;
    long long nsteps;
    unsigned *work;
    double *bs_scr;                     // [gridDim][84][64]
    DevCounters *ctr;
    unsigned long long time_limit_ns;
};

struct EnsShared {
    double x[3][kEnsMaxN], v[3][kEnsMaxN];
    double x0[3][kEnsMaxN], v0[3][kEnsMaxN];
    double m[kEnsMaxN], R[kEnsMaxN], k2[kEnsMaxN], tau[kEnsMaxN], rg2[kEnsMaxN];
    double w[3][kEnsMaxN];
    double rc[kEnsMaxN], rc2[kEnsMaxN], pc2[kEnsMaxN];
    // mixed kick: masses as two floats, FP32 bounds of rc^2 (above) and of
    // (f_pc rc)^2 (below and above)
    float mh[kEnsMaxN], ml[kEnsMaxN], thr[kEnsMaxN], pclo[kEnsMaxN], pchi[kEnsMaxN];
    double u0[3][kEnsMaxN], u1[3][kEnsMaxN], w0[3][kEnsMaxN];
    double part[3][128];
    unsigned long long cand[kEnsMaxN], enc[kEnsMaxN];
    int parent[kEnsMaxN], slot[kEnsMaxN], mem[kEnsMaxN];
    int roots[kEnsMaxN];
    double ws0[3], ws1[3], wsm[3];
    double star_R, star_k2, star_tau, star_rg2, mstar, dt;
    int n, nroots, flag, sys;
    double bs_t, bs_H, bs_err;
    int bs_stop, bs_kconv;
    // per-body constants of the loaded system: cbrt(m/(3 m_star)) of Rcrit,
    // 1/m, eta = m_star m/(m_star + m)^2, mu = G(m_star + m), m_star/(m_star + m),
    // the moment of inertia rg^2 m R^2 and the tidal prefactors 3 G m_star^2 k2 R^5
    // (planet) and 3 G m^2 k2_star R_star^5 (star)
    double hf[kEnsMaxN], im[kEnsMaxN], eta[kEnsMaxN], mu[kEnsMaxN], fac[kEnsMaxN], Ii[kEnsMaxN];
    double fiI[kEnsMaxN];               // m_star / ((m_star + m) I): the spin update's factor
    double tdi[kEnsMaxN], tds[kEnsMaxN];
    double red[4][kEnsMaxN / 32];       // per-warp partial sums of ens_bsum
};

// Sums over the loaded system's bodies of K per-body values (thread t < n
// holds body t's), in a fixed order: a butterfly within each warp, then the
// warps in order.  Every thread receives the sums.  Called by all threads.
template <int K>
__device__ __forceinline__ void ens_bsum(EnsShared &S, const double (&v)[K], double (&out)[K]) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nw = (S.n + 31) >> 5;
    double a[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = t < S.n ? v[k] : 0.0;
    if (w < nw) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < K; k++) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < K; k++) S.red[k][w] = a[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double sum = S.red[k][0];
        for (int q = 1; q < nw; q++) sum += S.red[k][q];
        out[k] = sum;
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned long long ens_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------ kick (Eq. Hb)
// a_i = G sum_j m_j K r^-3 (x_j - x_i), thread (i, slice); pre-check bits.
// MIXED: the arithmetic of the main mixed kick (kick.cu) -- FP64 displacement
// and accumulation, r^2 in float-float from an exact split of the
// displacement, FP32 rsqrt seed with one Newton correction in float-float,
// the small correction terms summed in float-float and added once; the
// changeover band and the pre-check are decided in FP32 against rounded
// bounds, the pre-check with the exact FP64 test within 2^-20 of its
// threshold (so the candidates are those of the FP64 form).
template <int T, bool MIXED>
__device__ void ens_kick(const EnsArgs &A, EnsShared &S, double dt_half, bool precheck) {
    const int n = S.n;
    const int t = threadIdx.x;
    const int nsl = max(1, T / n);
    const int i = t % n, sl = t / n;
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (MIXED && sl < nsl && t < nsl * n) {
        const int per = (n + nsl - 1) / nsl;
        const int j0 = sl * per, j1 = min(n, j0 + per);
        const double xi = S.x[0][i], yi = S.x[1][i], zi = S.x[2][i];
        unsigned long long bits = 0;
        float cxh = 0.0f, cxl = 0.0f, cyh = 0.0f, cyl = 0.0f, czh = 0.0f, czl = 0.0f;
        for (int j = j0; j < j1; j++) {
            if (j == i) continue;
            const double dx = S.x[0][j] - xi, dy = S.x[1][j] - yi, dz = S.x[2][j] - zi;
            float hx, hy, hz, lx, ly, lz;
            split_f64(dx, hx, lx);
            split_f64(dy, hy, ly);
            split_f64(dz, hz, lz);
            const float px = hx * hx, py = hy * hy, pz = hz * hz;
            const float pxe = fmaf(hx, hx, -px), pye = fmaf(hy, hy, -py), pze = fmaf(hz, hz, -pz);
            const float s1 = px + py, b1 = s1 - px;
            const float e1s = (px - (s1 - b1)) + (py - b1);
            const float s2 = s1 + pz, b2 = s2 - s1;
            const float e2s = (s1 - (s2 - b2)) + (pz - b2);
            const float cross = 2.0f * fmaf(hx, lx, fmaf(hy, ly, hz * lz));
            const float tail = ((e1s + e2s) + (pxe + pye + pze)) + cross;
            const float Rh = s2 + tail;
            const float Rl = tail - (Rh - s2);
            float mh = S.mh[j], ml = S.ml[j];
            if (Rh < fmaxf(S.thr[i], S.thr[j])) {            // changeover band (rare)
                const double mk = S.m[j] * changeover(sqrt(fma(dz, dz, fma(dy, dy, dx * dx))),
                                                      fmax(S.rc[i], S.rc[j]));
                mh = __double2float_rn(mk);
                ml = __double2float_rn(mk - (double)mh);
            }
            if (precheck && j > i) {
                bool c;
                if (Rh < fmaxf(S.pclo[i], S.pclo[j])) c = true;
                else if (Rh > fmaxf(S.pchi[i], S.pchi[j])) c = false;
                else c = dist2_rn(dx, dy, dz) < fmax(S.pc2[i], S.pc2[j]);
                if (c) bits |= 1ull << j;
            }
            const float y0f = rsqrtf(Rh);
            const float u = Rh * y0f, ue = fmaf(Rh, y0f, -u);
            const float r1 = fmaf(-u, y0f, 1.0f);
            const float p = y0f * y0f, pe = fmaf(y0f, y0f, -p);
            const float q = p * y0f;
            float qe = fmaf(p, y0f, -q);
            qe = fmaf(pe, y0f, qe);
            const float ch = q * mh;
            float ce = fmaf(q, mh, -ch);
            ce = fmaf(q, ml, ce);
            ce = fmaf(qe, mh, ce);
            const float ef = r1 - fmaf(ue, y0f, Rl * p);
            const float corr = fmaf(ch, fmaf(1.875f * ef, ef, 1.5f * ef), ce);
            const double sd = f64_of_f32_any(ch);
            ax = fma(sd, dx, ax); ay = fma(sd, dy, ay); az = fma(sd, dz, az);
            float_two_sum_acc(cxh, cxl, corr * hx);
            float_two_sum_acc(cyh, cyl, corr * hy);
            float_two_sum_acc(czh, czl, corr * hz);
        }
        ax += f64_of_f32_any(cxh) + f64_of_f32_any(cxl);
        ay += f64_of_f32_any(cyh) + f64_of_f32_any(cyl);
        az += f64_of_f32_any(czh) + f64_of_f32_any(czl);
        if (precheck && bits) atomicOr(&S.cand[i], bits);
    } else if (!MIXED && sl < nsl && t < nsl * n) {
        const int per = (n + nsl - 1) / nsl;
        const int j0 = sl * per, j1 = min(n, j0 + per);
        const double xi = S.x[0][i], yi = S.x[1][i], zi = S.x[2][i];
        unsigned long long bits = 0;
        for (int j = j0; j < j1; j++) {
            if (j == i) continue;
            const double dx = S.x[0][j] - xi, dy = S.x[1][j] - yi, dz = S.x[2][j] - zi;
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double yv = rsqrt_newton(r2);
            double mk = S.m[j];
            if (r2 < 1.0000001 * fmax(S.rc2[i], S.rc2[j]))
                mk *= changeover(r2 * yv, fmax(S.rc[i], S.rc[j]));
            if (precheck && j > i && dist2_rn(dx, dy, dz) < fmax(S.pc2[i], S.pc2[j])) bits |= 1ull << j;
            const double s = mk * (yv * yv * yv);
            ax = fma(s, dx, ax); ay = fma(s, dy, ay); az = fma(s, dz, az);
        }
        if (precheck && bits) atomicOr(&S.cand[i], bits);
    }
    S.part[0][t] = ax; S.part[1][t] = ay; S.part[2][t] = az;
    __syncthreads();
    if (t < n) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int q = 0; q < nsl; q++) { sx += S.part[0][q * n + t]; sy += S.part[1][q * n + t]; sz += S.part[2][q * n + t]; }
        S.v[0][t] += dt_half * (A.G * sx);
        S.v[1][t] += dt_half * (A.G * sy);
        S.v[2][t] += dt_half * (A.G * sz);
    }
    __syncthreads();
}

// ------------------------------------------------------------ GR + tides
// GR (Eq. apn) and tidal (Sec. 4.1-4.2) acceleration of body i at velocity u
// (heliocentric) and spin W, with the torques on the body and on the star.
// Divisions by r are multiplications by 1/r (Newton rsqrt) and the per-body
// constants come with the system (EnsShared): the FP64 pipe bounds the kernel.
__device__ void nn_body(const EnsArgs &A, const EnsShared &S, int i, const double u[3],
                        const double W[3], double acc[3], double Ni[3], double Ns[3]) {
    const double x[3] = {S.x[0][i], S.x[1][i], S.x[2][i]};
    const double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
    const double ir = rsqrt_newton(r2);
    const double r = r2 * ir;
    const double er[3] = {x[0] * ir, x[1] * ir, x[2] * ir};
    const double rdot = ((x[0] * u[0] + x[1] * u[1]) + x[2] * u[2]) * ir;
    const double u2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
    for (int k = 0; k < 3; k++) { acc[k] = 0.0; Ni[k] = 0.0; Ns[k] = 0.0; }
    if (A.gr == 1) {
        const double mu = S.mu[i], eta = S.eta[i];
        const double pre = -mu * (ir * ir) * A.inv_c2;
        const double cv = -2.0 * (2.0 - eta) * rdot;
        const double cr = (1.0 + 3.0 * eta) * u2 - 1.5 * eta * rdot * rdot - 2.0 * (2.0 + eta) * mu * ir;
        for (int k = 0; k < 3; k++) acc[k] += pre * (cv * u[k] + cr * er[k]);
    }
    if (A.tides) {
        const double ir2 = ir * ir;
        const double ir7 = (ir2 * ir2) * (ir2 * ir);
        const double Dti = S.tdi[i] * ir7;
        const double Dts = S.tds[i] * ir7;
        const double Pti = Dti * S.tau[i], Pts = Dts * S.star_tau;
        const double fr = -(Dts + Dti) - 2.0 * rdot * ir * (Pts + Pti);
        const double *Ws = S.wsm;
        const double wxe[3] = {W[1] * er[2] - W[2] * er[1], W[2] * er[0] - W[0] * er[2], W[0] * er[1] - W[1] * er[0]};
        const double sxe[3] = {Ws[1] * er[2] - Ws[2] * er[1], Ws[2] * er[0] - Ws[0] * er[2], Ws[0] * er[1] - Ws[1] * er[0]};
        const double exu[3] = {er[1] * u[2] - er[2] * u[1], er[2] * u[0] - er[0] * u[2], er[0] * u[1] - er[1] * u[0]};
        const double rW = (x[0] * W[0] + x[1] * W[1]) + x[2] * W[2];
        const double rWs = (x[0] * Ws[0] + x[1] * Ws[1]) + x[2] * Ws[2];
        const double im = S.im[i], Ptot_ir = (Pti + Pts) * ir;
        for (int k = 0; k < 3; k++) {
            const double F = fr * er[k] + Pti * wxe[k] + Pts * sxe[k] - Ptot_ir * u[k];
            acc[k] += F * im;
            Ni[k] = Pti * (W[k] * r - rW * er[k] - exu[k]);
            Ns[k] = Pts * (Ws[k] * r - rWs * er[k] - exu[k]);
        }
    }
}

__device__ void ens_nn(const EnsArgs &A, EnsShared &S, double dt) {
    if (A.gr != 1 && !A.tides) return;
    const int n = S.n, t = threadIdx.x;
    const int b = t < n ? t : 0;
    double P[4];
    {
        const double mv[4] = {S.m[b] * S.v[0][b], S.m[b] * S.v[1][b], S.m[b] * S.v[2][b], S.m[b]};
        ens_bsum<4>(S, mv, P);
    }
    const double Mp = P[3];
    const double ims = 1.0 / S.mstar;
    if (t == 0)
        for (int k = 0; k < 3; k++) S.ws1[k] = S.ws0[k];
    if (t < n)
        for (int k = 0; k < 3; k++) {
            S.u0[k][t] = S.v[k][t] + P[k] * ims;
            S.u1[k][t] = S.u0[k][t];
            S.w0[k][t] = S.w[k][t];
        }
    const double Is = S.star_rg2 * S.mstar * S.star_R * S.star_R;
    for (int it = 0; it < A.implicit_max_iter; it++) {
        if (t == 0) {
            S.flag = 0;
            for (int k = 0; k < 3; k++) S.wsm[k] = 0.5 * (S.ws0[k] + S.ws1[k]);
        }
        __syncthreads();
        double nsv[3] = {0.0, 0.0, 0.0};
        if (t < n) {
            double um[3], Wm[3], acc[3], Ni[3], Ns[3];
            for (int k = 0; k < 3; k++) {
                um[k] = 0.5 * (S.u0[k][t] + S.u1[k][t]);
                Wm[k] = 0.5 * (S.w0[k][t] + S.w[k][t]);
            }
            nn_body(A, S, t, um, Wm, acc, Ni, Ns);
            const double fac = S.fac[t];
            const double Ii = S.Ii[t], fiI = S.fiI[t];
            bool changed = false;
            for (int k = 0; k < 3; k++) {
                const double un = S.u0[k][t] + dt * acc[k];
                if (fabs(un - S.u1[k][t]) > 1e-16 * fabs(un)) changed = true;
                S.u1[k][t] = un;
                if (A.tides && Ii > 0.0) {
                    const double Wn = S.w0[k][t] - dt * fiI * Ni[k];
                    if (fabs(Wn - S.w[k][t]) > 1e-16 * fabs(Wn)) changed = true;
                    S.w[k][t] = Wn;
                }
                nsv[k] = fac * Ns[k];
            }
            if (changed) S.flag = 1;
        }
        if (A.tides && Is > 0.0) {
            double d[3];
            ens_bsum<3>(S, nsv, d);
            if (t == 0)
                for (int k = 0; k < 3; k++) {
                    const double Wn = S.ws0[k] - dt * d[k] / Is;
                    if (fabs(Wn - S.ws1[k]) > 1e-16 * fabs(Wn)) S.flag = 1;
                    S.ws1[k] = Wn;
                }
        }
        __syncthreads();
        if (!S.flag) break;
        __syncthreads();
    }
    double Q[3];
    {
        const double mu1[3] = {S.m[b] * S.u1[0][b], S.m[b] * S.u1[1][b], S.m[b] * S.u1[2][b]};
        ens_bsum<3>(S, mu1, Q);
    }
    if (t == 0)
        for (int k = 0; k < 3; k++) S.ws0[k] = S.ws1[k];
    const double itot = 1.0 / (S.mstar + Mp);
    if (t < n)
        for (int k = 0; k < 3; k++) S.v[k][t] = S.u1[k][t] - Q[k] * itot;
    __syncthreads();
}

// ------------------------------------------------------------ HC (Eq. Hc)
__device__ void ens_hc(EnsShared &S, double dt_half) {
    const int n = S.n, t = threadIdx.x;
    double P[3];
    {
        const int b = t < n ? t : 0;
        const double mv[3] = {S.m[b] * S.v[0][b], S.m[b] * S.v[1][b], S.m[b] * S.v[2][b]};
        ens_bsum<3>(S, mv, P);
    }
    const double f = dt_half / S.mstar;
    if (t < n) for (int k = 0; k < 3; k++) S.x[k][t] += f * P[k];
    __syncthreads();
}

// ------------------------------------------------------------ GR by splitting
// Sec. 3.1 (reading R28): H_PN = sum alpha H_Kep^2 + beta/r^2 + gamma p^4 on the
// canonical velocities u (pseudovelocities): the sun kick
// u += -dt 2 mu_i^2/(c^2 r^4) x (mu_i = G (m_star + m_i)), the gamma term
// x += -dt 2 (u^2/c^2) u with HC, and the drift time of each body scaled by
// 1 + 3 (u^2/2 - mu/r)/c^2 (mu = G m_star); the real velocity is
// v = u (1 - (u^2/2 + 3 mu/r)/c^2).  The pair kicks and the tides act on real
// velocities.
__device__ __forceinline__ double ens_u2(const double u[3]) { return (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]; }

__device__ __forceinline__ double ens_real_factor(const double x[3], const double u[3], double mu, double inv_c2) {
    const double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    return 1.0 - (0.5 * ens_u2(u) + 3.0 * mu / r) * inv_c2;
}

__device__ __forceinline__ double ens_alpha_factor(const double x[3], const double u[3], double mu, double inv_c2) {
    const double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    return 1.0 + 3.0 * (0.5 * ens_u2(u) - mu / r) * inv_c2;
}

// v -> u by fixed-point iteration from u = v (4 iterations: the correction is ~v^2/c^2).
__device__ void ens_gr_to_pseudo(const EnsArgs &A, EnsShared &S) {
    const int t = threadIdx.x;
    if (t < S.n) {
        const double x[3] = {S.x[0][t], S.x[1][t], S.x[2][t]};
        const double v[3] = {S.v[0][t], S.v[1][t], S.v[2][t]};
        double u[3] = {v[0], v[1], v[2]};
        for (int it = 0; it < 4; it++) {
            const double f = ens_real_factor(x, u, A.G * S.mstar, A.inv_c2);
            for (int k = 0; k < 3; k++) u[k] = v[k] / f;
        }
        for (int k = 0; k < 3; k++) S.v[k][t] = u[k];
    }
    __syncthreads();
}

__device__ void ens_gr_to_real(const EnsArgs &A, EnsShared &S) {
    const int t = threadIdx.x;
    if (t < S.n) {
        const double x[3] = {S.x[0][t], S.x[1][t], S.x[2][t]};
        const double u[3] = {S.v[0][t], S.v[1][t], S.v[2][t]};
        const double f = ens_real_factor(x, u, A.G * S.mstar, A.inv_c2);
        for (int k = 0; k < 3; k++) S.v[k][t] = u[k] * f;
    }
    __syncthreads();
}

__device__ void ens_gr_beta(const EnsArgs &A, EnsShared &S, double dt) {
    const int t = threadIdx.x;
    if (t < S.n) {
        const double x[3] = {S.x[0][t], S.x[1][t], S.x[2][t]};
        const double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
        const double mui = A.G * (S.mstar + S.m[t]);
        const double s = -dt * 2.0 * mui * mui * A.inv_c2 / (r2 * r2);
        for (int k = 0; k < 3; k++) S.v[k][t] += s * x[k];
    }
    __syncthreads();
}

// HC(dt) with the gamma term: x += dt P/m_star - dt 2 (u^2/c^2) u.
__device__ void ens_hc_gamma(const EnsArgs &A, EnsShared &S, double dt) {
    const int n = S.n, t = threadIdx.x;
    double P[3];
    {
        const int b = t < n ? t : 0;
        const double mv[3] = {S.m[b] * S.v[0][b], S.m[b] * S.v[1][b], S.m[b] * S.v[2][b]};
        ens_bsum<3>(S, mv, P);
    }
    const double f = dt / S.mstar;
    if (t < n) {
        const double u[3] = {S.v[0][t], S.v[1][t], S.v[2][t]};
        const double g = dt * 2.0 * ens_u2(u) * A.inv_c2;
        for (int k = 0; k < 3; k++) S.x[k][t] += f * P[k] - g * u[k];
    }
    __syncthreads();
}

// ------------------------------------------------------------ BS of one group
__device__ __forceinline__ double &ebs(double *scr, int row, int slot) { return scr[row * kEnsMaxN + slot]; }

__device__ void ens_bs_deriv(const EnsArgs &A, EnsShared &S, double *scr, int z0, int f0, int s) {
    const int b = S.mem[s];
    const double x = ebs(scr, z0, s), y = ebs(scr, z0 + 1, s), z = ebs(scr, z0 + 2, s);
    const double r2 = x * x + y * y + z * z;
    const double sst = -A.G * S.mstar / (r2 * sqrt(r2));
    double px = 0.0, py = 0.0, pz = 0.0;
    unsigned long long bits = S.enc[b];
    while (bits) {
        const int p = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        const int sp = S.slot[p];
        const double dx = ebs(scr, z0, sp) - x, dy = ebs(scr, z0 + 1, sp) - y, dz = ebs(scr, z0 + 2, sp) - z;
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double d = sqrt(d2);
        const double W = 1.0 - changeover(d, fmax(S.rc[b], S.rc[p]));
        const double c = S.m[p] * W / (d2 * d);
        px += c * dx; py += c * dy; pz += c * dz;
    }
    // GR splitting: the member's Kepler motion (velocity term and star
    // acceleration, not the pair terms) runs at the alpha-scaled rate
    double fac = 1.0;
    if (A.gr == 2) {
        const double xx[3] = {x, y, z};
        const double uu[3] = {ebs(scr, z0 + 3, s), ebs(scr, z0 + 4, s), ebs(scr, z0 + 5, s)};
        fac = ens_alpha_factor(xx, uu, A.G * S.mstar, A.inv_c2);
    }
    ebs(scr, f0, s) = fac * ebs(scr, z0 + 3, s);
    ebs(scr, f0 + 1, s) = fac * ebs(scr, z0 + 4, s);
    ebs(scr, f0 + 2, s) = fac * ebs(scr, z0 + 5, s);
    ebs(scr, f0 + 3, s) = fac * (sst * x) + A.G * px;
    ebs(scr, f0 + 4, s) = fac * (sst * y) + A.G * py;
    ebs(scr, f0 + 5, s) = fac * (sst * z) + A.G * pz;
}

// Same integrator and step control as the large-system kernels: modified
// midpoint n = 2..16, Neville in h^2, accept at the first column k >= 1 under
// tolerance, grow 1.5x if k < 4, halve on failure.
__device__ void ens_bs_group(const EnsArgs &A, EnsShared &S, double *scr, int nm, double dt,
                             unsigned long long t_start) {
    enum { Y = 0, F0 = 6, ZM = 12, ZN = 18, FZ = 24, SC = 30, TT = 36 };
    const int t = threadIdx.x;
    for (int s = t; s < nm; s += blockDim.x) {
        const int b = S.mem[s];
        for (int c = 0; c < 3; c++) { ebs(scr, Y + c, s) = S.x0[c][b]; ebs(scr, Y + 3 + c, s) = S.v0[c][b]; }
    }
    if (t == 0) { S.bs_t = 0.0; S.bs_H = dt; }
    __syncthreads();
    int attempts = 0;
    long long acc = 0, rej = 0;
    bool failed = false;
    while (S.bs_t < dt) {
        if (t == 0) S.bs_stop = (attempts >= A.bs_max_steps) || (ens_now() - t_start > A.time_limit_ns);
        __syncthreads();
        if (S.bs_stop) { failed = true; break; }
        attempts++;
        double H = S.bs_H;
        if (H > dt - S.bs_t) H = dt - S.bs_t;
        for (int s = t; s < nm; s += blockDim.x) ens_bs_deriv(A, S, scr, Y, F0, s);
        for (int s = t; s < nm; s += blockDim.x)
            for (int c = 0; c < 6; c++) ebs(scr, SC + c, s) = fabs(ebs(scr, Y + c, s)) + fabs(H * ebs(scr, F0 + c, s)) + 1e-300;
        int kconv = -1;
        for (int k = 0; k < 8 && kconv < 0; k++) {
            const int nk = 2 * (k + 1);
            const double h = H / nk;
            for (int s = t; s < nm; s += blockDim.x)
                for (int c = 0; c < 6; c++) {
                    const double y0 = ebs(scr, Y + c, s);
                    ebs(scr, ZM + c, s) = y0;
                    ebs(scr, ZN + c, s) = y0 + h * ebs(scr, F0 + c, s);
                }
            for (int mm = 1; mm < nk; mm++) {
                __syncthreads();
                for (int s = t; s < nm; s += blockDim.x) ens_bs_deriv(A, S, scr, ZN, FZ, s);
                __syncthreads();
                for (int s = t; s < nm; s += blockDim.x)
                    for (int c = 0; c < 6; c++) {
                        const double tt = ebs(scr, ZM + c, s) + 2.0 * h * ebs(scr, FZ + c, s);
                        ebs(scr, ZM + c, s) = ebs(scr, ZN + c, s);
                        ebs(scr, ZN + c, s) = tt;
                    }
            }
            __syncthreads();
            for (int s = t; s < nm; s += blockDim.x) ens_bs_deriv(A, S, scr, ZN, FZ, s);
            if (t == 0) S.bs_err = 0.0;
            __syncthreads();
            double err = 0.0;
            for (int s = t; s < nm; s += blockDim.x)
                for (int c = 0; c < 6; c++) {
                    double cur = 0.5 * (ebs(scr, ZN + c, s) + ebs(scr, ZM + c, s) + h * ebs(scr, FZ + c, s));
                    double prev = ebs(scr, TT + c, s);
                    ebs(scr, TT + c, s) = cur;
                    for (int j = 1; j <= k; j++) {
                        const double coef = (double)((k - j + 1) * (k - j + 1)) / (double)(j * (2 * k + 2 - j));
                        const double nxt = fma(cur - prev, coef, cur);
                        prev = ebs(scr, TT + j * 6 + c, s);
                        ebs(scr, TT + j * 6 + c, s) = nxt;
                        cur = nxt;
                    }
                    if (k >= 1) err = fmax(err, fabs(ebs(scr, TT + k * 6 + c, s) - ebs(scr, TT + (k - 1) * 6 + c, s)) / ebs(scr, SC + c, s));
                }
            // max of non-negative doubles through their bit patterns
            atomicMax((unsigned long long *)&S.bs_err, (unsigned long long)__double_as_longlong(err));
            __syncthreads();
            if (k >= 1 && S.bs_err <= A.bs_tol) kconv = k;
            __syncthreads();
        }
        if (kconv >= 0) {
            for (int s = t; s < nm; s += blockDim.x)
                for (int c = 0; c < 6; c++) ebs(scr, Y + c, s) = ebs(scr, TT + kconv * 6 + c, s);
            if (t == 0) { S.bs_t += H; S.bs_H = (kconv < 4) ? 1.5 * H : H; }
            acc++;
        } else {
            if (t == 0) S.bs_H = 0.5 * H;
            rej++;
        }
        __syncthreads();
    }
    for (int s = t; s < nm; s += blockDim.x) {
        const int b = S.mem[s];
        for (int c = 0; c < 3; c++) { S.x[c][b] = ebs(scr, Y + c, s); S.v[c][b] = ebs(scr, Y + 3 + c, s); }
    }
    if (t == 0) {
        atomicAdd(&A.ctr->bs_steps, (unsigned long long)acc);
        atomicAdd(&A.ctr->bs_rejects, (unsigned long long)rej);
        atomicMax(&A.ctr->bs_max_attempts, (unsigned long long)attempts);
        atomicAdd(&A.ctr->groups_total, 1ull);
        atomicMax(&A.ctr->max_group_total, (unsigned long long)nm);
        if (failed) { atomicAdd(&A.ctr->bs_fail, 1ull); latch_error(A.ctr, kErrBS); }
    }
    __syncthreads();
}

__device__ int ens_find(int *p, int a) {
    while (p[a] != a) a = p[a];
    return a;
}

// ------------------------------------------------------------ one step
template <int T, bool MIXED>
__device__ void ens_step(const EnsArgs &A, EnsShared &S, double *scr, unsigned long long t_start) {
    const int n = S.n, t = threadIdx.x;
    const double dt = S.dt;
    // Rcrit (Eq. rcrit), pre-check thresholds
    if (t < n) {
        const double r = sqrt(dist2_rn(S.x[0][t], S.x[1][t], S.x[2][t]));
        const double va = sqrt(dist2_rn(S.v[0][t], S.v[1][t], S.v[2][t]));
        const double hill = r * S.hf[t];
        const double a1 = A.n1 * hill, b1 = A.n2 * dt * va;
        const double rc = a1 > b1 ? a1 : b1;
        S.rc[t] = rc;
        S.rc2[t] = __dmul_rn(rc, rc);
        const double tt = __dmul_rn(A.f_pc, rc);
        S.pc2[t] = __dmul_rn(tt, tt);
        if (MIXED) {
            // conservative float bounds: above rc^2, below and above (f_pc rc)^2,
            // each with a 2^-20 margin over the float errors of r^2 (~2^-23)
            S.thr[t] = fmaxf(__fmul_ru(__double2float_ru(S.rc2[t]), 1.00000095f), 1.17549435e-38f);
            S.pclo[t] = __fmul_rd(__double2float_rd(S.pc2[t]), 0.99999905f);
            S.pchi[t] = __fmul_ru(__double2float_ru(S.pc2[t]), 1.00000095f);
        }
        S.cand[t] = 0ull;
        S.enc[t] = 0ull;
    }
    __syncthreads();
    ens_kick<T, MIXED>(A, S, 0.5 * dt, true);
    ens_nn(A, S, 0.5 * dt);
    if (A.gr == 2) {
        ens_gr_to_pseudo(A, S);
        ens_gr_beta(A, S, 0.5 * dt);
        ens_hc_gamma(A, S, 0.5 * dt);
    } else {
        ens_hc(S, 0.5 * dt);
    }
    // FG (saves the pre-drift state); with GR splitting each body drifts for
    // its alpha-scaled time
    if (t < n) {
        double x = S.x[0][t], y = S.x[1][t], z = S.x[2][t], vx = S.v[0][t], vy = S.v[1][t], vz = S.v[2][t];
        S.x0[0][t] = x; S.x0[1][t] = y; S.x0[2][t] = z; S.v0[0][t] = vx; S.v0[1][t] = vy; S.v0[2][t] = vz;
        double dti = dt;
        if (A.gr == 2) {
            const double xx[3] = {x, y, z}, uu[3] = {vx, vy, vz};
            dti = dt * ens_alpha_factor(xx, uu, A.G * S.mstar, A.inv_c2);
        }
        if (!kepler_drift(x, y, z, vx, vy, vz, A.G * S.mstar, dti, A.kepler_max_iter)) {
            latch_error(A.ctr, kErrKepler);
            atomicAdd(&A.ctr->kepler_fail, 1ull);
        }
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) latch_error(A.ctr, kErrBadState);
        S.x[0][t] = x; S.x[1][t] = y; S.x[2][t] = z; S.v[0][t] = vx; S.v[1][t] = vy; S.v[2][t] = vz;
    }
    __syncthreads();
    // detection over the pre-check candidates
    if (t < n) {
        unsigned long long bits = S.cand[t];
        int nc = 0, ne = 0;
        while (bits) {
            const int j = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            nc++;
            const double lim = fmax(S.rc2[t], S.rc2[j]);
            const double d0 = dist2_rn(S.x0[0][j] - S.x0[0][t], S.x0[1][j] - S.x0[1][t], S.x0[2][j] - S.x0[2][t]);
            const double d1 = dist2_rn(S.x[0][j] - S.x[0][t], S.x[1][j] - S.x[1][t], S.x[2][j] - S.x[2][t]);
            if (d0 < lim || d1 < lim) {
                atomicOr(&S.enc[t], 1ull << j);
                atomicOr(&S.enc[j], 1ull << t);
                ne++;
            }
        }
        if (nc) atomicAdd(&A.ctr->cand_count, (unsigned long long)nc);
        if (ne) atomicAdd(&A.ctr->pair_count[0], (unsigned long long)ne);
    }
    __syncthreads();
    // grouping (union-find, root = smallest index) and BS per group
    if (t == 0) {
        for (int i = 0; i < n; i++) S.parent[i] = i;
        for (int i = 0; i < n; i++) {
            unsigned long long bits = S.enc[i] & ~((2ull << i) - 1ull);   // partners j > i
            while (bits) {
                const int j = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                const int a = ens_find(S.parent, i), b = ens_find(S.parent, j);
                if (a != b) { if (a < b) S.parent[b] = a; else S.parent[a] = b; }
            }
        }
        int nr = 0;
        for (int i = 0; i < n; i++)
            if (S.enc[i] && ens_find(S.parent, i) == i) S.roots[nr++] = i;
        S.nroots = nr;
    }
    __syncthreads();
    for (int gq = 0; gq < S.nroots; gq++) {
        if (t == 0) {
            const int g = S.roots[gq];
            int nm = 0;
            for (int i = 0; i < n; i++)
                if (S.enc[i] && ens_find(S.parent, i) == g) { S.slot[i] = nm; S.mem[nm++] = i; }
            S.flag = nm;
        }
        __syncthreads();
        ens_bs_group(A, S, scr, S.flag, dt, t_start);
    }
    if (A.gr == 2) {
        ens_hc_gamma(A, S, 0.5 * dt);
        ens_gr_beta(A, S, 0.5 * dt);
        ens_gr_to_real(A, S);
    } else {
        ens_hc(S, 0.5 * dt);
    }
    ens_kick<T, MIXED>(A, S, 0.5 * dt, false);
    ens_nn(A, S, 0.5 * dt);
}

template <int T, bool MIXED>
__global__ void __launch_bounds__(T) ensemble_kernel(EnsArgs A) {
    __shared__ EnsShared S;
    double *scr = A.bs_scr + (size_t)blockIdx.x * kEnsBsRows * kEnsMaxN;
    const int t = threadIdx.x;
    while (true) {
        if (t == 0) S.sys = (int)atomicAdd(A.work, 1u);
        __syncthreads();
        const int q = S.sys;
        if (q >= A.n_systems) break;
        const int s = A.order[q];
        const long long o = A.offsets[s];
        const int n = (int)(A.offsets[s + 1] - o);
        const size_t NT = (size_t)A.ntot;
        if (t == 0) {
            S.n = n; S.mstar = A.m_star[s]; S.dt = A.dt[s];
            const double *st = A.star + 8 * (size_t)s;
            S.star_R = st[0]; S.star_k2 = st[1]; S.star_tau = st[2]; S.star_rg2 = st[3];
            S.ws0[0] = st[4]; S.ws0[1] = st[5]; S.ws0[2] = st[6];
        }
        if (t < n) {
            const size_t g = (size_t)o + t;
            for (int c = 0; c < 3; c++) {
                S.x[c][t] = A.pos[c * NT + g]; S.v[c][t] = A.vel[c * NT + g]; S.w[c][t] = A.spin[c * NT + g];
            }
            S.m[t] = A.mass[g]; S.R[t] = A.radius[g]; S.k2[t] = A.k2[g]; S.tau[t] = A.tau[g]; S.rg2[t] = A.rg2[g];
            if (MIXED) {
                S.mh[t] = __double2float_rn(S.m[t]);
                S.ml[t] = __double2float_rn(S.m[t] - (double)S.mh[t]);
            }
        }
        __syncthreads();
        if (t < n) {
            const double ms = S.mstar, mi = S.m[t];
            const double Ri = S.R[t], Rs = S.star_R;
            S.hf[t] = cbrt(mi / (3.0 * ms));
            S.im[t] = mi > 0.0 ? 1.0 / mi : 0.0;
            S.eta[t] = ms * mi / ((ms + mi) * (ms + mi));
            S.mu[t] = A.G * (ms + mi);
            S.fac[t] = ms / (ms + mi);
            S.Ii[t] = S.rg2[t] * mi * Ri * Ri;
            S.fiI[t] = S.Ii[t] > 0.0 ? S.fac[t] / S.Ii[t] : 0.0;
            S.tdi[t] = 3.0 * A.G * ms * ms * (Ri * Ri * Ri * Ri * Ri) * S.k2[t];
            S.tds[t] = 3.0 * A.G * mi * mi * (Rs * Rs * Rs * Rs * Rs) * S.star_k2;
        }
        __syncthreads();
        const unsigned long long t_start = ens_now();
        for (long long k = 0; k < A.nsteps; k++) ens_step<T, MIXED>(A, S, scr, t_start);
        if (t < n) {
            const size_t g = (size_t)o + t;
            for (int c = 0; c < 3; c++) {
                A.pos[c * NT + g] = S.x[c][t]; A.vel[c * NT + g] = S.v[c][t]; A.spin[c * NT + g] = S.w[c][t];
            }
        }
        if (t == 0) {
            double *st = A.star + 8 * (size_t)s;
            st[4] = S.ws0[0]; st[5] = S.ws0[1]; st[6] = S.ws0[2];
        }
        __syncthreads();
    }
}

// Total angular momentum (orbit + spins) per system.
__global__ void ensemble_angmom_kernel(EnsArgs A, double *L) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.n_systems) return;
    const size_t NT = (size_t)A.ntot;
    double lx = 0.0, ly = 0.0, lz = 0.0;
    for (long long g = A.offsets[s]; g < A.offsets[s + 1]; g++) {
        const double x = A.pos[g], y = A.pos[NT + g], z = A.pos[2 * NT + g];
        const double vx = A.vel[g], vy = A.vel[NT + g], vz = A.vel[2 * NT + g];
        const double m = A.mass[g];
        const double I = A.rg2[g] * m * A.radius[g] * A.radius[g];
        lx += m * (y * vz - z * vy) + I * A.spin[g];
        ly += m * (z * vx - x * vz) + I * A.spin[NT + g];
        lz += m * (x * vy - y * vx) + I * A.spin[2 * NT + g];
    }
    const double *st = A.star + 8 * (size_t)s;
    const double Is = st[3] * A.m_star[s] * st[0] * st[0];
    L[3 * s] = lx + Is * st[4];
    L[3 * s + 1] = ly + Is * st[5];
    L[3 * s + 2] = lz + Is * st[6];
}

}  // namespace
}  // namespace genga

// ============================================================== ensemble ABI
using namespace genga;

struct genga_ensemble {
    genga_params_t p;
    genga_ensemble_desc_t d;
    int64_t ntot = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    long long *offsets = nullptr;
    int *order = nullptr;
    unsigned *work = nullptr;
    double *bs_scr = nullptr;
    int bs_ctas = 0;
    DevCounters *ctr = nullptr;
    int threads = 64;             // tile shape: threads per CTA (32, 64 or 128)
    int maxn = 0;                 // largest system
    int ctas_per_sm = 4;
    std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;
    genga_stats_t stats;
    int64_t launches = 0;
    char err[512] = {0};
};

namespace {

int efail(genga_ensemble *e, int code, const char *fmt, ...) {
    if (e) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(e->err, sizeof(e->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define ECU(expr)                                                                               \
    do {                                                                                        \
        cudaError_t e__ = (expr);                                                               \
        if (e__ != cudaSuccess)                                                                 \
            return efail(e, e__ == cudaErrorMemoryAllocation ? GENGA_ENOMEM : GENGA_ECUDA,      \
                         "%s: %s", #expr, cudaGetErrorString(e__));                             \
    } while (0)

EnsArgs ens_args(genga_ensemble *e, long long nsteps) {
    EnsArgs A;
    A.n_systems = (int)e->d.n_systems;
    A.offsets = e->offsets; A.order = e->order;
    A.pos = e->d.pos; A.vel = e->d.vel; A.spin = e->d.spin;
    A.ntot = e->ntot;
    A.mass = e->d.mass; A.radius = e->d.radius; A.k2 = e->d.k2; A.tau = e->d.tau; A.rg2 = e->d.rg2;
    A.m_star = e->d.m_star; A.dt = e->d.dt; A.star = e->d.star;
    A.c2 = e->d.c_light * e->d.c_light;
    A.inv_c2 = 1.0 / A.c2;
    A.gr = e->d.gr; A.tides = e->d.tides;
    A.G = e->p.G; A.n1 = e->p.n1; A.n2 = e->p.n2; A.f_pc = e->p.f_pc; A.bs_tol = e->p.bs_tol;
    A.kepler_max_iter = e->p.kepler_max_iter; A.bs_max_steps = e->p.bs_max_steps;
    A.implicit_max_iter = 10;
    A.nsteps = nsteps;
    A.work = e->work;
    A.bs_scr = e->bs_scr;
    A.ctr = e->ctr;
    A.time_limit_ns = 60000000000ull;   // 60 s per system call
    return A;
}

int grid_of(genga_ensemble *e) {
    return std::min<int>((int)e->d.n_systems, e->num_sms * e->ctas_per_sm);
}

cudaError_t launch_ensemble(genga_ensemble *e, long long nsteps, cudaStream_t st) {
    EnsArgs A = ens_args(e, nsteps);
    const int grid = grid_of(e);
    cudaError_t r = cudaMemsetAsync(e->work, 0, sizeof(unsigned), st);
    if (r != cudaSuccess) return r;
    const bool mixed = e->p.precision == GENGA_MIXED;
    if (e->threads == 32) {
        if (mixed) ensemble_kernel<32, true><<<grid, 32, 0, st>>>(A);
        else ensemble_kernel<32, false><<<grid, 32, 0, st>>>(A);
    } else if (e->threads == 128) {
        if (mixed) ensemble_kernel<128, true><<<grid, 128, 0, st>>>(A);
        else ensemble_kernel<128, false><<<grid, 128, 0, st>>>(A);
    } else {
        if (mixed) ensemble_kernel<64, true><<<grid, 64, 0, st>>>(A);
        else ensemble_kernel<64, false><<<grid, 64, 0, st>>>(A);
    }
    e->launches++;
    return cudaGetLastError();
}

int ens_errors(genga_ensemble *e) {
    DevCounters c;
    ECU(cudaMemcpyAsync(&c, e->ctr, sizeof(c), cudaMemcpyDeviceToHost, e->stream));
    ECU(cudaStreamSynchronize(e->stream));
    e->stats.n_candidates = (int64_t)c.cand_count;
    e->stats.n_pairs[0] = (int64_t)c.pair_count[0];
    e->stats.n_groups = (int64_t)c.groups_total;
    e->stats.max_group = (int64_t)c.max_group_total;
    e->stats.bs_steps = (int64_t)c.bs_steps;
    e->stats.bs_rejects = (int64_t)c.bs_rejects;
    e->stats.bs_fail = (int64_t)c.bs_fail;
    e->stats.kepler_fail = (int64_t)c.kepler_fail;
    e->stats.bs_max_attempts = (int64_t)c.bs_max_attempts;
    e->stats.kernel_launches = e->launches;
    if (!c.err) return GENGA_OK;
    ECU(cudaMemsetAsync(&e->ctr->err, 0, sizeof(unsigned), e->stream));
    if (c.err & kErrBadState) return efail(e, GENGA_EBADSTATE, "non-finite state");
    if (c.err & kErrKepler) return efail(e, GENGA_ENONCONV, "Kepler solve hit kepler_max_iter");
    if (c.err & kErrBS) return efail(e, GENGA_ENONCONV, "Bulirsch-Stoer hit its limit");
    return efail(e, GENGA_ECUDA, "device error word 0x%x", c.err);
}

}  // namespace

extern "C" {

int genga_ensemble_create(genga_ensemble_t **out, const genga_params_t *p,
                          const genga_ensemble_desc_t *d, void *stream) {
    if (!out || !p || !d) return GENGA_EINVAL;
    *out = nullptr;
    if (d->n_systems < 1 || !d->offsets || !d->pos || !d->vel || !d->mass || !d->spin || !d->radius ||
        !d->k2 || !d->tau || !d->rg2 || !d->m_star || !d->dt || !d->star)
        return GENGA_EINVAL;
    if (d->gr < 0 || d->gr > 2 || (d->gr && !(d->c_light > 0))) return GENGA_EINVAL;
    if (p->slevels != 1 || p->kepler_max_iter < 1 || p->bs_max_steps < 1 || !(p->bs_tol > 0) ||
        (p->precision != GENGA_FP64 && p->precision != GENGA_MIXED))
        return GENGA_EINVAL;
    std::vector<int> sizes((size_t)d->n_systems);
    for (int64_t s = 0; s < d->n_systems; s++) {
        const int64_t n = d->offsets[s + 1] - d->offsets[s];
        if (n < 1 || n > GENGA_ENSEMBLE_MAX_N) return GENGA_EINVAL;
        sizes[(size_t)s] = (int)n;
    }
    genga_ensemble *e = new (std::nothrow) genga_ensemble();
    if (!e) return GENGA_ENOMEM;
    e->p = *p;
    e->d = *d;
    e->d.offsets = nullptr;
    e->ntot = d->offsets[d->n_systems];
    e->stream = (cudaStream_t)stream;
    e->maxn = *std::max_element(sizes.begin(), sizes.end());
    if (e->maxn > 64) e->threads = 128;
    int dev = 0;
    auto bail = [&](int code) { genga_ensemble_destroy(e); return code; };
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(GENGA_ECUDA);
    // work order: largest systems first (better tail balance)
    std::vector<int> order((size_t)d->n_systems);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sizes[a] > sizes[b]; });
    std::vector<long long> offs((size_t)d->n_systems + 1);
    for (int64_t s = 0; s <= d->n_systems; s++) offs[(size_t)s] = (long long)d->offsets[s];
    e->bs_ctas = e->num_sms * 8;
    if (cudaMalloc(&e->offsets, sizeof(long long) * offs.size()) != cudaSuccess ||
        cudaMalloc(&e->order, sizeof(int) * order.size()) != cudaSuccess ||
        cudaMalloc(&e->work, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&e->ctr, sizeof(DevCounters)) != cudaSuccess ||
        cudaMalloc(&e->bs_scr, sizeof(double) * (size_t)e->bs_ctas * kEnsBsRows * kEnsMaxN) != cudaSuccess)
        return bail(GENGA_ENOMEM);
    if (cudaMemcpy(e->offsets, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->ctr, 0, sizeof(DevCounters)) != cudaSuccess)
        return bail(GENGA_ECUDA);
    *out = e;
    return GENGA_OK;
}

void genga_ensemble_destroy(genga_ensemble_t *e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    for (auto &kv : e->graphs) cudaGraphExecDestroy(kv.second);
    if (e->offsets) cudaFree(e->offsets);
    if (e->order) cudaFree(e->order);
    if (e->work) cudaFree(e->work);
    if (e->ctr) cudaFree(e->ctr);
    if (e->bs_scr) cudaFree(e->bs_scr);
    delete e;
}

const char *genga_ensemble_last_error(const genga_ensemble_t *e) { return e ? e->err : "null ensemble"; }

int genga_ensemble_set_tile(genga_ensemble_t *e, int threads, int ctas_per_sm) {
    if (!e || (threads != 32 && threads != 64 && threads != 128) || ctas_per_sm < 1 || ctas_per_sm > 8)
        return GENGA_EINVAL;
    if (threads < e->maxn) return efail(e, GENGA_EINVAL, "threads per CTA below the largest system");
    e->threads = threads;
    e->ctas_per_sm = ctas_per_sm;
    return GENGA_OK;
}

int genga_ensemble_step(genga_ensemble_t *e, int64_t nsteps) {
    if (!e || nsteps < 0) return GENGA_EINVAL;
    ECU(cudaMemsetAsync(e->ctr, 0, sizeof(DevCounters), e->stream));
    e->launches = 0;
    if (nsteps > 0) {
        // one persistent launch, captured once per (nsteps, tile) and replayed
        const auto key = std::make_pair((long long)nsteps, e->threads * 16 + e->ctas_per_sm);
        auto it = e->graphs.find(key);
        if (it == e->graphs.end()) {
            cudaStream_t cap = nullptr;
            ECU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t r = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (r == cudaSuccess) {
                r = launch_ensemble(e, (long long)nsteps, cap);
                cudaError_t r2 = cudaStreamEndCapture(cap, &graph);
                if (r == cudaSuccess) r = r2;
            }
            if (r == cudaSuccess) r = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            ECU(r);
            it = e->graphs.emplace(key, exec).first;
            e->launches = 0;
        }
        ECU(cudaGraphLaunch(it->second, e->stream));
        e->launches += 1;
    }
    return ens_errors(e);
}

int genga_ensemble_autotune(genga_ensemble_t *e, int64_t trial_steps, int *threads_out, int *ctas_out) {
    if (!e || trial_steps < 1) return GENGA_EINVAL;
    const int maxn = e->maxn;
    // save the state, time each tile shape on the same start, restore
    const size_t nt = (size_t)e->ntot, ns = (size_t)e->d.n_systems;
    double *save = nullptr;
    ECU(cudaMalloc(&save, sizeof(double) * (9 * nt + 8 * ns)));
    auto copy_state = [&](bool to_save) -> cudaError_t {
        const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
        double *s0 = save, *s1 = save + 3 * nt, *s2 = save + 6 * nt, *s3 = save + 9 * nt;
        cudaError_t r;
        if (to_save) {
            if ((r = cudaMemcpyAsync(s0, e->d.pos, 24 * nt, k, e->stream)) != cudaSuccess) return r;
            if ((r = cudaMemcpyAsync(s1, e->d.vel, 24 * nt, k, e->stream)) != cudaSuccess) return r;
            if ((r = cudaMemcpyAsync(s2, e->d.spin, 24 * nt, k, e->stream)) != cudaSuccess) return r;
            return cudaMemcpyAsync(s3, e->d.star, 64 * ns, k, e->stream);
        }
        if ((r = cudaMemcpyAsync(e->d.pos, s0, 24 * nt, k, e->stream)) != cudaSuccess) return r;
        if ((r = cudaMemcpyAsync(e->d.vel, s1, 24 * nt, k, e->stream)) != cudaSuccess) return r;
        if ((r = cudaMemcpyAsync(e->d.spin, s2, 24 * nt, k, e->stream)) != cudaSuccess) return r;
        return cudaMemcpyAsync(e->d.star, s3, 64 * ns, k, e->stream);
    };
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int bt = e->threads, bc = e->ctas_per_sm;
    const int cand_t[3] = {32, 64, 128};
    const int cand_c[3] = {2, 4, 8};
    cudaError_t r = copy_state(true);
    for (int ti = 0; ti < 3 && r == cudaSuccess; ti++) {
        if (cand_t[ti] < maxn) continue;
        for (int ci = 0; ci < 3 && r == cudaSuccess; ci++) {
            e->threads = cand_t[ti];
            e->ctas_per_sm = cand_c[ci];
            cudaEventRecord(a, e->stream);
            r = launch_ensemble(e, (long long)trial_steps, e->stream);
            cudaEventRecord(b, e->stream);
            if (r == cudaSuccess) r = cudaEventSynchronize(b);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            if (r == cudaSuccess && ms < best) { best = ms; bt = cand_t[ti]; bc = cand_c[ci]; }
            if (r == cudaSuccess) r = copy_state(false);
        }
    }
    cudaStreamSynchronize(e->stream);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(save);
    ECU(r);
    e->threads = bt;
    e->ctas_per_sm = bc;
    if (threads_out) *threads_out = bt;
    if (ctas_out) *ctas_out = bc;
    return ens_errors(e);
}

int genga_ensemble_angmom(genga_ensemble_t *e, double *L_host) {
    if (!e || !L_host) return GENGA_EINVAL;
    double *L = nullptr;
    ECU(cudaMalloc(&L, sizeof(double) * 3 * (size_t)e->d.n_systems));
    EnsArgs A = ens_args(e, 0);
    ensemble_angmom_kernel<<<(unsigned)((e->d.n_systems + 127) / 128), 128, 0, e->stream>>>(A, L);
    cudaError_t r = cudaGetLastError();
    if (r == cudaSuccess)
        r = cudaMemcpyAsync(L_host, L, sizeof(double) * 3 * (size_t)e->d.n_systems, cudaMemcpyDeviceToHost, e->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
    cudaFree(L);
    ECU(r);
    return GENGA_OK;
}

int genga_ensemble_get_stats(genga_ensemble_t *e, genga_stats_t *st) {
    if (!e || !st) return GENGA_EINVAL;
    *st = e->stats;
    return GENGA_OK;
}

// The same calls under the names of the boundary's call list.
int genga_init_ensemble(genga_ensemble_t **out, const genga_params_t *p, const genga_ensemble_desc_t *d,
                        void *stream) {
    return genga_ensemble_create(out, p, d, stream);
}
int genga_step_ensemble(genga_ensemble_t *e, int64_t nsteps) { return genga_ensemble_step(e, nsteps); }

}  // extern "C"
