// adjoint.cu -- reverse-mode derivative of kick-drift-kick steps with frozen
// encounters (the adjoint form around the method of Appendix A).
//
// Forward: normal steps of the original scheme (slevels = 1) that record each
// step's level-0 critical radii and encounter pairs, with checkpoints of the
// state every C steps.  Backward: for each segment (last first) the states at
// the step starts are recomputed from the checkpoint by replaying the steps
// with the recorded rc and pairs, then each step is differentiated in reverse:
//   Kick(dt/2) at x3  -> lx += h (da/dx)^T lv,  lm += h (da/dm)^T lv
//   HC(dt/2)          -> lv_j += (h/m*) m_j sum(lx), lm_j += (h/m*) v_j . sum(lx)
//   FG(dt)            -> (lx, lv) = Phi^T (lx, lv), Phi the 6x6 state-transition
//                        matrix of the Kepler drift (dual numbers, exact)
//   BS(dt) of a group -> the continuous adjoint: the group ODE, its adjoint
//                        lambda' = -J^T lambda and the mass gradient integrated
//                        backwards in time by the same Bulirsch-Stoer scheme
//   HC(dt/2), Kick(dt/2) at x as above.
// There is no derivative through rc (frozen), and the changeover function's
// derivative dK/dr is included in the force derivatives.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace genga {
namespace {

// ------------------------------------------------------------ dual numbers
struct D6 {
    double v;
    double d[6];
};
__device__ __forceinline__ D6 dconst(double a) { D6 r; r.v = a; for (int k = 0; k < 6; k++) r.d[k] = 0.0; return r; }
__device__ __forceinline__ D6 operator+(const D6 &a, const D6 &b) { D6 r; r.v = a.v + b.v; for (int k = 0; k < 6; k++) r.d[k] = a.d[k] + b.d[k]; return r; }
__device__ __forceinline__ D6 operator-(const D6 &a, const D6 &b) { D6 r; r.v = a.v - b.v; for (int k = 0; k < 6; k++) r.d[k] = a.d[k] - b.d[k]; return r; }
__device__ __forceinline__ D6 operator*(const D6 &a, const D6 &b) { D6 r; r.v = a.v * b.v; for (int k = 0; k < 6; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
__device__ __forceinline__ D6 operator*(double s, const D6 &a) { D6 r; r.v = s * a.v; for (int k = 0; k < 6; k++) r.d[k] = s * a.d[k]; return r; }
__device__ __forceinline__ D6 operator/(const D6 &a, const D6 &b) {
    D6 r; r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
    for (int k = 0; k < 6; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
__device__ __forceinline__ D6 dsqrt(const D6 &a) {
    D6 r; r.v = sqrt(a.v);
    const double h = 0.5 / r.v;
    for (int k = 0; k < 6; k++) r.d[k] = a.d[k] * h;
    return r;
}
__device__ __forceinline__ D6 operator-(const D6 &a) { return (-1.0) * a; }

// Stumpff functions on duals (same series and quartering as stumpff()).
__device__ void stumpff_d6(D6 z, D6 &c0, D6 &c1, D6 &c2, D6 &c3) {
    int q = 0;
    while (fabs(z.v) > 0.1 && q < 60) { z = 0.25 * z; q++; }
    const double ic2[10] = {1.0 / 2.0, 1.0 / 24.0, 1.0 / 720.0, 1.0 / 40320.0, 1.0 / 3628800.0,
                            1.0 / 479001600.0, 1.0 / 87178291200.0, 1.0 / 20922789888000.0,
                            1.0 / 6402373705728000.0, 1.0 / 2432902008176640000.0};
    const double ic3[10] = {1.0 / 6.0, 1.0 / 120.0, 1.0 / 5040.0, 1.0 / 362880.0,
                            1.0 / 39916800.0, 1.0 / 6227020800.0, 1.0 / 1307674368000.0,
                            1.0 / 355687428096000.0, 1.0 / 121645100408832000.0,
                            1.0 / 51090942171709440000.0};
    D6 s2 = dconst(0.0), s3 = dconst(0.0);
    for (int m = 9; m >= 0; m--) {
        s2 = dconst(ic2[m]) - z * s2;
        s3 = dconst(ic3[m]) - z * s3;
    }
    D6 C2 = s2, C3 = s3, C0 = dconst(1.0) - z * C2, C1 = dconst(1.0) - z * C3;
    for (int k = 0; k < q; k++) {
        const D6 n3 = 0.25 * (C2 + C0 * C3);
        const D6 n2 = 0.5 * (C1 * C1);
        const D6 n1 = C0 * C1;
        const D6 n0 = 2.0 * (C0 * C0) - dconst(1.0);
        C0 = n0; C1 = n1; C2 = n2; C3 = n3;
    }
    c0 = C0; c1 = C1; c2 = C2; c3 = C3;
}

// ------------------------------------------------------------ drift VJP
// For bodies outside every group: (lx, lv) <- Phi^T (lx, lv) with Phi the
// Jacobian of the Kepler drift at the pre-drift state (x1, v1).  The
// universal variable s is solved in double; one Newton step in dual
// arithmetic from it gives ds/d(x0, v0) by the implicit function theorem.
__global__ void drift_vjp_kernel(int n, const double *x1, const double *v1, const int *label,
                                 double mu, double dt, int max_iter, double *lx, double *lv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (label && label[i] >= 0) return;
    const size_t N = (size_t)n;
    D6 X[3], V[3];
    for (int c = 0; c < 3; c++) {
        X[c] = dconst(x1[c * N + i]); X[c].d[c] = 1.0;
        V[c] = dconst(v1[c * N + i]); V[c].d[3 + c] = 1.0;
    }
    const D6 r0 = dsqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    const D6 v2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const D6 u = X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
    const D6 beta = (2.0 * mu) * (dconst(1.0) / r0) - v2;
    double s;
    kepler_solve_s(r0.v, u.v, beta.v, mu, dt, max_iter, s);
    // one dual Newton step: s_d = s - (t(s) - dt) / r(s)
    D6 sd = dconst(s);
    D6 c0, c1, c2, c3;
    stumpff_d6(beta * sd * sd, c0, c1, c2, c3);
    {
        const D6 G1 = sd * c1, G2 = sd * sd * c2, G3 = sd * sd * sd * c3;
        const D6 t = r0 * G1 + u * G2 + mu * G3;
        const D6 rr = r0 * c0 + u * G1 + mu * G2;
        sd = sd - (t - dconst(dt)) / rr;
    }
    stumpff_d6(beta * sd * sd, c0, c1, c2, c3);
    const D6 G1 = sd * c1, G2 = sd * sd * c2, G3 = sd * sd * sd * c3;
    const D6 r = r0 * c0 + u * G1 + mu * G2;
    const D6 fm1 = -(mu * G2 / r0);
    const D6 g = dconst(dt) - mu * G3;
    const D6 fd = -(mu * G1 / (r * r0));
    const D6 gdm1 = -(mu * G2 / r);
    // outputs x = x0 + fm1 x0 + g v0, v = v0 + fd x0 + gdm1 v0; J[row][col]
    double J[6][6];
    for (int c = 0; c < 3; c++) {
        const D6 xo = X[c] + fm1 * X[c] + g * V[c];
        const D6 vo = V[c] + fd * X[c] + gdm1 * V[c];
        for (int k = 0; k < 6; k++) { J[c][k] = xo.d[k]; J[3 + c][k] = vo.d[k]; }
    }
    double lo[6], li[6];
    for (int c = 0; c < 3; c++) { lo[c] = lx[c * N + i]; lo[3 + c] = lv[c * N + i]; }
    for (int k = 0; k < 6; k++) {
        double acc = 0.0;
        for (int row = 0; row < 6; row++) acc += J[row][k] * lo[row];
        li[k] = acc;
    }
    for (int c = 0; c < 3; c++) { lx[c * N + i] = li[c]; lv[c * N + i] = li[3 + c]; }
}

// ------------------------------------------------------------ kick VJP
// For each body k (FP64):
//   gx_k = G sum_j M_kj (m_k lv_j - m_j lv_k),  M = K (I/r^3 - 3 d d^T/r^5) + K' d d^T / r^4
//   gm_k = -G sum_j K lv_j . d / r^3,            d = x_j - x_k
constexpr int kAdjThreads = 128;
constexpr int kAdjTile = 128;

// Inverse distances from the Newton rsqrt; K and dK/dr only for the pairs whose
// FP32 r^2 is below the conservative bound of rc_ij^2 (K = 1, K' = 0 beyond
// rc_ij), from the changeover function with 1/rc_ij = min(1/rc_k, 1/rc_j).
__global__ void __launch_bounds__(kAdjThreads)
kick_vjp_kernel(int n, const double *pos, const double *mass, const double *irc, const float *thr,
                const double *lv, int chunk, double *part /* [nchunk][4][n] */) {
    __shared__ double sx[kAdjTile], sy[kAdjTile], sz[kAdjTile], sm[kAdjTile], sirc[kAdjTile];
    __shared__ double sl0[kAdjTile], sl1[kAdjTile], sl2[kAdjTile];
    __shared__ float sthr[kAdjTile];
    const size_t N = (size_t)n;
    const int k = blockIdx.x * kAdjThreads + threadIdx.x;
    const bool valid = k < n;
    double xk = 0, yk = 0, zk = 0, mk = 0, irck = 0, l0 = 0, l1 = 0, l2 = 0;
    float thrk = 0.0f;
    if (valid) {
        xk = pos[k]; yk = pos[N + k]; zk = pos[2 * N + k]; mk = mass[k]; irck = irc[k]; thrk = thr[k];
        l0 = lv[k]; l1 = lv[N + k]; l2 = lv[2 * N + k];
    }
    const int jbeg = blockIdx.y * chunk, jend = min(n, jbeg + chunk);
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, gm = 0.0;
    for (int jt = jbeg; jt < jend; jt += kAdjTile) {
        const int cnt = min(kAdjTile, jend - jt);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += kAdjThreads) {
            const int j = jt + q;
            sx[q] = pos[j]; sy[q] = pos[N + j]; sz[q] = pos[2 * N + j]; sm[q] = mass[j];
            sirc[q] = irc[j]; sthr[q] = thr[j];
            sl0[q] = lv[j]; sl1[q] = lv[N + j]; sl2[q] = lv[2 * N + j];
        }
        __syncthreads();
        if (!valid) continue;
        for (int q = 0; q < cnt; q++) {
            if (jt + q == k) continue;
            const double dx = sx[q] - xk, dy = sy[q] - yk, dz = sz[q] - zk;
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double id = rsqrt_newton(r2), id2 = id * id, id3 = id2 * id;
            double K = 1.0, Kp = 0.0;
            if (f32_of_f64_trunc(r2) < fmaxf(thrk, sthr[q]))
                changeover_fast_dr(r2 * id, fmin(irck, sirc[q]), K, Kp);
            // e = m_k lv_j - m_j lv_k
            const double e0 = mk * sl0[q] - sm[q] * l0, e1 = mk * sl1[q] - sm[q] * l1, e2 = mk * sl2[q] - sm[q] * l2;
            const double de = fma(dz, e2, fma(dy, e1, dx * e0));
            const double a = K * id3;
            const double b = (-3.0 * K * id3 + Kp * id2) * id2 * de;   // -3 K de / r^5 + K' de / r^4
            g0 += a * e0 + b * dx; g1 += a * e1 + b * dy; g2 += a * e2 + b * dz;
            gm -= a * fma(sl2[q], dz, fma(sl1[q], dy, sl0[q] * dx));
        }
    }
    if (valid) {
        double *p = part + (size_t)blockIdx.y * 4 * N;
        p[k] = g0; p[N + k] = g1; p[2 * N + k] = g2; p[3 * N + k] = gm;
    }
}

__global__ void kick_vjp_finalize(int n, int nchunk, const double *part, double G, double h,
                                  double *lx, double *lm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const size_t N = (size_t)n;
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < nchunk; q++)
        for (int c = 0; c < 4; c++) g[c] += part[(size_t)q * 4 * N + c * N + k];
    lx[k] += h * G * g[0];
    lx[N + k] += h * G * g[1];
    lx[2 * N + k] += h * G * g[2];
    lm[k] += h * G * g[3];
}

// ------------------------------------------------------------ HC VJP
__global__ void __launch_bounds__(1024) sum3_kernel(int n, const double *a, double *out) {
    __shared__ double sp[3][1024];
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int j = threadIdx.x; j < n; j += 1024) { p0 += a[j]; p1 += a[(size_t)n + j]; p2 += a[2 * (size_t)n + j]; }
    sp[0][threadIdx.x] = p0; sp[1][threadIdx.x] = p1; sp[2][threadIdx.x] = p2;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 3; c++) sp[c][threadIdx.x] += sp[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = sp[threadIdx.x][0];
}

__global__ void hc_vjp_kernel(int n, const double *sigma, const double *vel, const double *mass,
                              double h_over_mstar, double *lv, double *lm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const size_t N = (size_t)n;
    const double s0 = sigma[0], s1 = sigma[1], s2 = sigma[2];
    lv[j] += h_over_mstar * mass[j] * s0;
    lv[N + j] += h_over_mstar * mass[j] * s1;
    lv[2 * N + j] += h_over_mstar * mass[j] * s2;
    lm[j] += h_over_mstar * (vel[j] * s0 + vel[N + j] * s1 + vel[2 * N + j] * s2);
}

// ------------------------------------------------------------ BS adjoint
// Per member: y (6), adjoint lambda (6), mass-gradient integral g (1); in
// reversed time tau = dt - t:
//   dy/dtau = -f(y)
//   dlx/dtau = A^T lv,  dlv/dtau = lx        (J = [[0, I], [A, 0]], A = da/dx)
//   dg_a/dtau = G sum_p W lv_p . (x_a - x_p)/r^3   (da_p/dm_a)
// Error control on y only.  One CTA per group of at most kBlockGroupMax
// members, state in a global scratch (larger groups: bsm.cu).
constexpr int kAD = 13;                      // values per member
constexpr int kABs = 64;                     // threads per CTA

struct AdjBsArgs {
    int n;
    const double *x2, *v2;                   // post-drift state (start of the backward run)
    double *lx, *lv, *lm;                    // in: adjoint at the end of the drift; out: at its start
    const double *mass, *rc;
    const double *irc;                       // 1 / rc (level 0)
    const int *off, *list;
    const int *goff, *member, *slotof;
    const int *blist;                        // group labels of one size bucket, one block each
    double *scr;                             // [kAD * 14][S]
    size_t S;
    double G, mu, dt, tol;
    int max_steps;
    DevCounters *ctr;
};

__device__ __forceinline__ double &AR(const AdjBsArgs &A, int row, int slot) { return A.scr[(size_t)row * A.S + slot]; }

// derivative in reversed time of the augmented state in rows z0..z0+12 into
// f0..f0+12.  Inverse distances from the Newton rsqrt, K and dK/dr from the
// changeover function with 1/rc_ij = min(1/rc_b, 1/rc_p) (no divisions): the
// kernel is bound by the latency of this chain of dependent FP64 instructions.
__device__ void adj_deriv(const AdjBsArgs &A, int z0, int f0, int s) {
    const int b = A.member[s];
    const double x = AR(A, z0, s), y = AR(A, z0 + 1, s), z = AR(A, z0 + 2, s);
    const double lvx = AR(A, z0 + 9, s), lvy = AR(A, z0 + 10, s), lvz = AR(A, z0 + 11, s);
    const double mb = A.mass[b];
    const double r2 = fma(z, z, fma(y, y, x * x));
    const double ir = rsqrt_newton(r2), ir2 = ir * ir, mir3 = A.mu * (ir2 * ir);
    // star: acc = -mu x / r^3; A_star = -mu (I/r^3 - 3 x x^T / r^5) (symmetric)
    double ax = -mir3 * x, ay = -mir3 * y, az = -mir3 * z;
    const double c3 = 3.0 * fma(z, lvz, fma(y, lvy, x * lvx)) * ir2;
    double tx = -mir3 * (lvx - c3 * x);
    double ty = -mir3 * (lvy - c3 * y);
    double tz = -mir3 * (lvz - c3 * z);
    double px = 0.0, py = 0.0, pz = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, gm = 0.0;
    const double ircb = A.irc[b];
    for (int q = A.off[b]; q < A.off[b + 1]; q++) {
        const int p = A.list[q];
        const int sp = A.slotof[p];
        const double dx = AR(A, z0, sp) - x, dy = AR(A, z0 + 1, sp) - y, dz = AR(A, z0 + 2, sp) - z;
        const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double id = rsqrt_newton(d2), id2 = id * id, id3 = id2 * id;
        double K, dK;
        changeover_fast_dr(d2 * id, fmin(ircb, A.irc[p]), K, dK);
        const double W = 1.0 - K;                    // Wp = dW/dr = -dK
        const double mp = A.mass[p];
        const double mw = mp * W * id3;
        px = fma(mw, dx, px); py = fma(mw, dy, py); pz = fma(mw, dz, pz);
        const double qx = AR(A, z0 + 9, sp), qy = AR(A, z0 + 10, sp), qz = AR(A, z0 + 11, sp);
        const double e0 = mb * qx - mp * lvx, e1 = mb * qy - mp * lvy, e2 = mb * qz - mp * lvz;
        const double de = fma(dz, e2, fma(dy, e1, dx * e0));
        const double a = W * id3;
        // -3 W de / d^5 + (dW/dr) de / d^4, dW/dr = -dK
        const double bb = (-3.0 * W * id3 - dK * id2) * id2 * de;
        gx += a * e0 + bb * dx; gy += a * e1 + bb * dy; gz += a * e2 + bb * dz;
        gm -= W * fma(qz, dz, fma(qy, dy, qx * dx)) * id3;
    }
    ax += A.G * px; ay += A.G * py; az += A.G * pz;
    // reversed time
    AR(A, f0 + 0, s) = -AR(A, z0 + 3, s);
    AR(A, f0 + 1, s) = -AR(A, z0 + 4, s);
    AR(A, f0 + 2, s) = -AR(A, z0 + 5, s);
    AR(A, f0 + 3, s) = -ax;
    AR(A, f0 + 4, s) = -ay;
    AR(A, f0 + 5, s) = -az;
    AR(A, f0 + 6, s) = tx + A.G * gx;
    AR(A, f0 + 7, s) = ty + A.G * gy;
    AR(A, f0 + 8, s) = tz + A.G * gz;
    AR(A, f0 + 9, s) = AR(A, z0 + 6, s);
    AR(A, f0 + 10, s) = AR(A, z0 + 7, s);
    AR(A, f0 + 11, s) = AR(A, z0 + 8, s);
    AR(A, f0 + 12, s) = A.G * gm;
}

__global__ void __launch_bounds__(kABs) bs_adjoint_kernel(AdjBsArgs A) {
    enum { Y = 0, F0 = kAD, ZM = 2 * kAD, ZN = 3 * kAD, FZ = 4 * kAD, SC = 5 * kAD, TT = 6 * kAD };
    __shared__ double red[kABs / 32];
    __shared__ int stop;
    __shared__ double st_t, st_H;
    const int g = A.blist[blockIdx.x];
    const int s0 = A.goff[g], s1 = A.goff[g + 1];
    if (s1 - s0 > kBlockGroupMax) return;                // the batched driver's groups
    const size_t N = (size_t)A.n;
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int b = A.member[s];
        for (int c = 0; c < 3; c++) {
            AR(A, Y + c, s) = A.x2[c * N + b];
            AR(A, Y + 3 + c, s) = A.v2[c * N + b];
            AR(A, Y + 6 + c, s) = A.lx[c * N + b];
            AR(A, Y + 9 + c, s) = A.lv[c * N + b];
        }
        AR(A, Y + 12, s) = 0.0;
    }
    if (threadIdx.x == 0) { st_t = 0.0; st_H = A.dt; }
    int attempts = 0;
    bool failed = false;
    __syncthreads();
    while (st_t < A.dt) {
        if (threadIdx.x == 0) stop = attempts >= A.max_steps;
        __syncthreads();
        if (stop) { failed = true; break; }
        attempts++;
        double H = st_H;
        if (H > A.dt - st_t) H = A.dt - st_t;
        for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) adj_deriv(A, Y, F0, s);
        for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
            for (int c = 0; c < kAD; c++) AR(A, SC + c, s) = fabs(AR(A, Y + c, s)) + fabs(H * AR(A, F0 + c, s)) + 1e-300;
        int kconv = -1;
        for (int k = 0; k < 8 && kconv < 0; k++) {
            const int nk = 2 * (k + 1);
            const double h = H / nk;
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                for (int c = 0; c < kAD; c++) {
                    const double y0 = AR(A, Y + c, s);
                    AR(A, ZM + c, s) = y0;
                    AR(A, ZN + c, s) = y0 + h * AR(A, F0 + c, s);
                }
            for (int mm = 1; mm < nk; mm++) {
                __syncthreads();
                for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) adj_deriv(A, ZN, FZ, s);
                __syncthreads();
                for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                    for (int c = 0; c < kAD; c++) {
                        const double tt = AR(A, ZM + c, s) + 2.0 * h * AR(A, FZ + c, s);
                        AR(A, ZM + c, s) = AR(A, ZN + c, s);
                        AR(A, ZN + c, s) = tt;
                    }
            }
            __syncthreads();
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) adj_deriv(A, ZN, FZ, s);
            double err = 0.0;
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                for (int c = 0; c < kAD; c++) {
                    double cur = 0.5 * (AR(A, ZN + c, s) + AR(A, ZM + c, s) + h * AR(A, FZ + c, s));
                    double prev = AR(A, TT + c, s);
                    AR(A, TT + c, s) = cur;
                    for (int j = 1; j <= k; j++) {
                        const double coef = (double)((k - j + 1) * (k - j + 1)) / (double)(j * (2 * k + 2 - j));
                        const double nxt = fma(cur - prev, coef, cur);
                        prev = AR(A, TT + j * kAD + c, s);
                        AR(A, TT + j * kAD + c, s) = nxt;
                        cur = nxt;
                    }
                    if (k >= 1 && c < 6)
                        err = fmax(err, fabs(AR(A, TT + k * kAD + c, s) - AR(A, TT + (k - 1) * kAD + c, s)) / AR(A, SC + c, s));
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = err;
            __syncthreads();
            double e = red[0];
            for (int w = 1; w < kABs / 32; w++) e = fmax(e, red[w]);
            __syncthreads();
            if (k >= 1 && e <= A.tol) kconv = k;
        }
        if (kconv >= 0) {
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                for (int c = 0; c < kAD; c++) AR(A, Y + c, s) = AR(A, TT + kconv * kAD + c, s);
            __syncthreads();
            if (threadIdx.x == 0) { st_t += H; st_H = (kconv < 4) ? 1.5 * H : H; }
        } else {
            __syncthreads();
            if (threadIdx.x == 0) st_H = 0.5 * H;
        }
        __syncthreads();
    }
    __syncthreads();
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int b = A.member[s];
        for (int c = 0; c < 3; c++) {
            A.lx[c * N + b] = AR(A, Y + 6 + c, s);
            A.lv[c * N + b] = AR(A, Y + 9 + c, s);
        }
        A.lm[b] += AR(A, Y + 12, s);
    }
    if (threadIdx.x == 0 && failed) {
        atomicAdd(&A.ctr->bs_fail, 1ull);
        latch_error(A.ctr, kErrBS);
    }
}

// ------------------------------------------------------------ BS adjoint, column-parallel
// The same integration for groups of at most M <= 16 members with the 8
// extrapolation columns of an attempt advanced at once (as bs_cols_kernel does
// for the forward ODE): thread (k, a) takes column k for member a, so an
// attempt costs at most 16 sequential derivative evaluations instead of
// 1 + 2 + 4 + ... + 16.  The arithmetic is the serial kernel's (the same
// derivative with the partners in ascending body order, the same midpoint,
// smoothing and Neville expressions, the same acceptance test); the column of
// an attempt's first converged extrapolation is taken as there.
template <int M>
struct AdjColsShared {
    double zp[6][8 * M];            // per (column, member): x, y, z, lv of the current state
    double y[kAD][M], f0[6][M];     // attempt start (accepted state) and its derivative (y part)
    double zf[3][kAD][M];           // the completing column's z_n, z_{n-1}, f(z_n)
    double hcol[8];
    double m[M], irc[M];
    unsigned pmask[M];
    int rank_of_slot[M];
    int stop;
};

// Derivative (reversed time) of member a's augmented state z in column col;
// the partners' positions and lv from the column's shared copy.
template <int M>
__device__ __forceinline__ void adj_cols_deriv(const AdjBsArgs &A, const AdjColsShared<M> &S, int col, int a,
                                               unsigned pmask, const double (&z)[kAD], double (&f)[kAD]) {
    const double x = z[0], y = z[1], zz = z[2];
    const double lvx = z[9], lvy = z[10], lvz = z[11];
    const double mb = S.m[a];
    const double r2 = fma(zz, zz, fma(y, y, x * x));
    const double ir = rsqrt_newton(r2), ir2 = ir * ir, mir3 = A.mu * (ir2 * ir);
    double ax = -mir3 * x, ay = -mir3 * y, az = -mir3 * zz;
    const double c3 = 3.0 * fma(zz, lvz, fma(y, lvy, x * lvx)) * ir2;
    const double tx = -mir3 * (lvx - c3 * x);
    const double ty = -mir3 * (lvy - c3 * y);
    const double tz = -mir3 * (lvz - c3 * zz);
    double px = 0.0, py = 0.0, pz = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, gm = 0.0;
    const double ircb = S.irc[a];
    unsigned mm = pmask;
    while (mm) {
        const int q = __ffs(mm) - 1;
        mm &= mm - 1;
        const int l = col * M + q;
        const double dx = S.zp[0][l] - x, dy = S.zp[1][l] - y, dz = S.zp[2][l] - zz;
        const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double id = rsqrt_newton(d2), id2 = id * id, id3 = id2 * id;
        double K, dK;
        changeover_fast_dr(d2 * id, fmin(ircb, S.irc[q]), K, dK);
        const double W = 1.0 - K;
        const double mp = S.m[q];
        const double mw = mp * W * id3;
        px = fma(mw, dx, px); py = fma(mw, dy, py); pz = fma(mw, dz, pz);
        const double qx = S.zp[3][l], qy = S.zp[4][l], qz = S.zp[5][l];
        const double e0 = mb * qx - mp * lvx, e1 = mb * qy - mp * lvy, e2 = mb * qz - mp * lvz;
        const double de = fma(dz, e2, fma(dy, e1, dx * e0));
        const double aa = W * id3;
        const double bb = (-3.0 * W * id3 - dK * id2) * id2 * de;
        gx += aa * e0 + bb * dx; gy += aa * e1 + bb * dy; gz += aa * e2 + bb * dz;
        gm -= W * fma(qz, dz, fma(qy, dy, qx * dx)) * id3;
    }
    ax += A.G * px; ay += A.G * py; az += A.G * pz;
    f[0] = -z[3]; f[1] = -z[4]; f[2] = -z[5];
    f[3] = -ax; f[4] = -ay; f[5] = -az;
    f[6] = tx + A.G * gx; f[7] = ty + A.G * gy; f[8] = tz + A.G * gz;
    f[9] = z[6]; f[10] = z[7]; f[11] = z[8];
    f[12] = A.G * gm;
}

// Row k of the Neville table of one component (T in place, cur the column's
// smoothed value), with the serial kernel's expressions; returns T_kk, T_k,k-1.
template <int K>
__device__ __forceinline__ void adj_neville_k(double (&T)[8], double cur, double &diag, double &prevdiag) {
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
    prevdiag = T[K >= 1 ? K - 1 : 0];
}
__device__ __forceinline__ void adj_neville(int k, double (&T)[8], double cur, double &diag, double &prevdiag) {
    switch (k) {
    case 0: adj_neville_k<0>(T, cur, diag, prevdiag); break;
    case 1: adj_neville_k<1>(T, cur, diag, prevdiag); break;
    case 2: adj_neville_k<2>(T, cur, diag, prevdiag); break;
    case 3: adj_neville_k<3>(T, cur, diag, prevdiag); break;
    case 4: adj_neville_k<4>(T, cur, diag, prevdiag); break;
    case 5: adj_neville_k<5>(T, cur, diag, prevdiag); break;
    case 6: adj_neville_k<6>(T, cur, diag, prevdiag); break;
    default: adj_neville_k<7>(T, cur, diag, prevdiag); break;
    }
}

template <int M>
__global__ void __launch_bounds__(8 * M) bs_adj_cols_kernel(AdjBsArgs A) {
    __shared__ AdjColsShared<M> S;
    const int tid = threadIdx.x;
    const int col = tid / M, a = tid % M;
    const int g = A.blist[blockIdx.x];
    const int s0 = A.goff[g], nm = A.goff[g + 1] - s0;
    if (nm > M || (M > 4 && nm <= M / 2)) return;          // not this bucket (never taken)
    const size_t N = (size_t)A.n;
    // member of rank a (ascending body index)
    if (tid < M) {
        const int mine = (a < nm) ? A.member[s0 + a] : 0x7fffffff;
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
    unsigned pmask = 0;
    if (active)
        for (int q = A.off[b]; q < A.off[b + 1]; q++) pmask |= 1u << S.rank_of_slot[A.slotof[A.list[q]] - s0];
    if (col == 0) {
        S.m[a] = active ? A.mass[b] : 0.0;
        S.irc[a] = active ? A.irc[b] : 0.0;
        for (int c = 0; c < 3; c++) {
            S.y[c][a] = active ? A.x2[c * N + b] : 0.0;
            S.y[3 + c][a] = active ? A.v2[c * N + b] : 0.0;
            S.y[6 + c][a] = active ? A.lx[c * N + b] : 0.0;
            S.y[9 + c][a] = active ? A.lv[c * N + b] : 0.0;
        }
        S.y[12][a] = 0.0;
    }
    // the Neville lanes: component c0 = col (and c1 = col + 8 while < kAD) of member a
    const int c0 = col, c1 = col + 8;
    const bool has1 = c1 < kAD;
    double T0[8], T1[8];
    double sc0 = 1.0, sc1 = 1.0, d0 = 0.0, d1 = 0.0;
    const int nk = 2 * (col + 1);
    double t = 0.0, H = A.dt;
    int attempts = 0;
    bool failed = false;
    __syncthreads();
    while (t < A.dt) {
        if (tid == 0) S.stop = attempts >= A.max_steps;
        __syncthreads();
        if (S.stop) { failed = true; break; }
        attempts++;
        if (H > A.dt - t) H = A.dt - t;
        double zm[kAD], zn[kAD], fz[kAD];
        // the attempt's start and its derivative, in every column
#pragma unroll
        for (int c = 0; c < kAD; c++) zm[c] = S.y[c][a];
        S.zp[0][tid] = zm[0]; S.zp[1][tid] = zm[1]; S.zp[2][tid] = zm[2];
        S.zp[3][tid] = zm[9]; S.zp[4][tid] = zm[10]; S.zp[5][tid] = zm[11];
        __syncthreads();
        adj_cols_deriv<M>(A, S, col, a, pmask, zm, fz);
        if (col == 0)
#pragma unroll
            for (int c = 0; c < 6; c++) S.f0[c][a] = fz[c];
        const double h = H / nk;
        if (a == 0) S.hcol[col] = h;
#pragma unroll
        for (int c = 0; c < kAD; c++) zn[c] = zm[c] + h * fz[c];
        int kconv = -1;
        for (int it = 1; it <= 16; it++) {
            __syncthreads();                          // the previous reads of zp are done
            S.zp[0][tid] = zn[0]; S.zp[1][tid] = zn[1]; S.zp[2][tid] = zn[2];
            S.zp[3][tid] = zn[9]; S.zp[4][tid] = zn[10]; S.zp[5][tid] = zn[11];
            __syncthreads();
            adj_cols_deriv<M>(A, S, col, a, pmask, zn, fz);
            if (it < nk) {
#pragma unroll
                for (int c = 0; c < kAD; c++) {
                    const double tt = zm[c] + 2.0 * h * fz[c];
                    zm[c] = zn[c];
                    zn[c] = tt;
                }
            } else if (it == nk) {
#pragma unroll
                for (int c = 0; c < kAD; c++) {
                    S.zf[0][c][a] = zn[c];
                    S.zf[1][c][a] = zm[c];
                    S.zf[2][c][a] = fz[c];
                }
            }
            if (it & 1) continue;
            const int k = it / 2 - 1;                 // column just completed
            __syncthreads();
            bool ok = true;
            if (active) {
                const double hk = S.hcol[k];
                if (k == 0) {
                    if (c0 < 6) sc0 = fabs(S.y[c0][a]) + fabs(H * S.f0[c0][a]) + 1e-300;
                    if (has1 && c1 < 6) sc1 = fabs(S.y[c1][a]) + fabs(H * S.f0[c1][a]) + 1e-300;
                }
                double p0 = 0.0, p1 = 0.0;
                adj_neville(k, T0, 0.5 * (S.zf[0][c0][a] + S.zf[1][c0][a] + hk * S.zf[2][c0][a]), d0, p0);
                if (k >= 1 && c0 < 6) ok = fabs(d0 - p0) / sc0 <= A.tol;
                if (has1) {
                    adj_neville(k, T1, 0.5 * (S.zf[0][c1][a] + S.zf[1][c1][a] + hk * S.zf[2][c1][a]), d1, p1);
                    if (k >= 1 && c1 < 6) ok = ok && fabs(d1 - p1) / sc1 <= A.tol;
                }
            }
            if (k >= 1 && __syncthreads_and(ok)) { kconv = k; break; }
        }
        __syncthreads();                              // every read of S.y is done
        if (kconv >= 0) {
            if (active) {
                S.y[c0][a] = d0;
                if (has1) S.y[c1][a] = d1;
            }
            t += H;
            if (kconv < 4) H *= 1.5;
        } else {
            H *= 0.5;
        }
        __syncthreads();
    }
    if (active && col == 0) {
        for (int c = 0; c < 3; c++) {
            A.lx[c * N + b] = S.y[6 + c][a];
            A.lv[c * N + b] = S.y[9 + c][a];
        }
        A.lm[b] += S.y[12][a];
    }
    if (tid == 0 && failed) {
        atomicAdd(&A.ctr->bs_fail, 1ull);
        latch_error(A.ctr, kErrBS);
    }
}

}  // namespace

// ============================================================== host driver
struct Adjoint {
    int64_t nsteps = 0, every = 0;
    std::vector<int64_t> pair_off;            // host, nsteps + 1
    double *rc_hist = nullptr;                // device, nsteps * n
    uint2 *pair_hist = nullptr;               // device
    int64_t pair_cap = 0;
    double *x0 = nullptr, *v0 = nullptr;      // initial state, 3n each
    double *ckpt = nullptr;                   // device, ncheck * 6n
    double *seg = nullptr;                    // device, every * 6n (step-start states of a segment)
    double *tmp = nullptr;                    // device, 6n (x2, v2)
    double *part = nullptr;                   // kick VJP partials
    int nchunk = 0, chunk = 0;
    double *sigma = nullptr;                  // 3 doubles
    double *bs_scr = nullptr;                 // kAD * 14 rows * n
    double *save_pos = nullptr, *save_vel = nullptr;
};

}  // namespace genga

using namespace genga;

namespace {

#define ACU(expr)                                                        \
    do {                                                                 \
        cudaError_t e__ = (expr);                                        \
        if (e__ != cudaSuccess) {                                        \
            snprintf(s->err, sizeof(s->err), "%s: %s", #expr, cudaGetErrorString(e__)); \
            return e__ == cudaErrorMemoryAllocation ? GENGA_ENOMEM : GENGA_ECUDA; \
        }                                                                \
    } while (0)

Adjoint *adj_of(genga_system *s) {
    if (!s->adj) s->adj = new Adjoint();
    return (Adjoint *)s->adj;
}

int adj_alloc(genga_system *s, int64_t nsteps, int64_t every) {
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    auto fr = [](double *&p) { if (p) cudaFree(p); p = nullptr; };
    fr(a->rc_hist); fr(a->ckpt); fr(a->seg);
    a->nsteps = nsteps;
    a->every = every;
    const int64_t ncheck = (nsteps + every - 1) / every + 1;
    ACU(cudaMalloc(&a->rc_hist, sizeof(double) * n * (size_t)std::max<int64_t>(nsteps, 1)));
    ACU(cudaMalloc(&a->ckpt, sizeof(double) * 6 * n * (size_t)ncheck));
    ACU(cudaMalloc(&a->seg, sizeof(double) * 6 * n * (size_t)every));
    if (!a->x0) {
        ACU(cudaMalloc(&a->x0, sizeof(double) * 3 * n));
        ACU(cudaMalloc(&a->v0, sizeof(double) * 3 * n));
        ACU(cudaMalloc(&a->tmp, sizeof(double) * 6 * n));
        ACU(cudaMalloc(&a->sigma, sizeof(double) * 4));
        ACU(cudaMalloc(&a->bs_scr, sizeof(double) * (size_t)kAD * 14 * n));
        ACU(cudaMalloc(&a->save_pos, sizeof(double) * 3 * n));
        ACU(cudaMalloc(&a->save_vel, sizeof(double) * 3 * n));
        const int iblocks = (int)((n + kAdjThreads - 1) / kAdjThreads);
        int want = (8 * s->num_sms + iblocks - 1) / iblocks;
        const int tiles = (int)((n + kAdjTile - 1) / kAdjTile);
        int tpc = std::max(1, std::min(16, (tiles + want - 1) / std::max(1, want)));
        if ((tiles + tpc - 1) / tpc > kMaxKickChunks) tpc = (tiles + kMaxKickChunks - 1) / kMaxKickChunks;
        a->chunk = tpc * kAdjTile;
        a->nchunk = (int)((n + a->chunk - 1) / a->chunk);
        ACU(cudaMalloc(&a->part, sizeof(double) * 4 * n * (size_t)a->nchunk));
    }
    a->pair_off.assign(1, 0);
    return GENGA_OK;
}

int adj_push_pairs(genga_system *s, const uint2 *dev_pairs, int64_t np, bool from_host) {
    Adjoint *a = adj_of(s);
    const int64_t have = a->pair_off.back();
    if (have + np > a->pair_cap) {
        const int64_t cap = std::max<int64_t>(2 * (have + np), 1 << 16);
        uint2 *nb = nullptr;
        ACU(cudaMalloc(&nb, sizeof(uint2) * (size_t)cap));
        if (a->pair_hist) {
            ACU(cudaMemcpyAsync(nb, a->pair_hist, sizeof(uint2) * (size_t)have, cudaMemcpyDeviceToDevice, s->stream));
            ACU(cudaStreamSynchronize(s->stream));
            cudaFree(a->pair_hist);
        }
        a->pair_hist = nb;
        a->pair_cap = cap;
    }
    if (np > 0)
        ACU(cudaMemcpyAsync(a->pair_hist + have, dev_pairs, sizeof(uint2) * (size_t)np,
                            from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s->stream));
    a->pair_off.push_back(have + np);
    return GENGA_OK;
}

// One step with the recorded rc and pairs of step k (Appendix A, slevels = 1).
int replay_step(genga_system *s, int64_t k) {
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    const double dt = s->p.dt, h = 0.5 * dt;
    ACU(cudaMemcpyAsync(s->rcl[0].rc, a->rc_hist + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(launch_rcrit_derive(s));
    ACU(launch_kick(s, h, false, nullptr));
    ACU(launch_hc(s, h));
    ACU(launch_drift(s, 0, dt, nullptr, (int)n));
    const int64_t np = a->pair_off[(size_t)k + 1] - a->pair_off[(size_t)k];
    s->npairs_host[0] = np;
    if (np > 0) {
        int rc = ensure_pair_capacity(s, 0, np);
        if (rc != GENGA_OK) return rc;
        ACU(cudaMemcpyAsync(s->pairs[0], a->pair_hist + a->pair_off[(size_t)k], sizeof(uint2) * (size_t)np,
                            cudaMemcpyDeviceToDevice, s->stream));
        ACU(build_csr(s, 0, np));
        ACU(build_groups(s, 0, np));
        {
            const int brc = run_bs(s, 0, dt, np);
            if (brc != GENGA_OK) return brc;
        }
    }
    ACU(launch_hc(s, h));
    ACU(launch_kick(s, h, false, nullptr));
    return GENGA_OK;
}

int kick_vjp(genga_system *s, const double *pos, const double *lv, double *lx, double *lm, double h) {
    Adjoint *a = adj_of(s);
    const int n = (int)s->n;
    dim3 grid((n + kAdjThreads - 1) / kAdjThreads, a->nchunk);
    kick_vjp_kernel<<<grid, kAdjThreads, 0, s->stream>>>(n, pos, s->mass, s->rcl[0].irc, s->rcl[0].thr_rc, lv,
                                                         a->chunk, a->part);
    ++s->launches;
    ACU(cudaGetLastError());
    kick_vjp_finalize<<<(n + 255) / 256, 256, 0, s->stream>>>(n, a->nchunk, a->part, s->p.G, h, lx, lm);
    ++s->launches;
    ACU(cudaGetLastError());
    return GENGA_OK;
}

int hc_vjp(genga_system *s, const double *lx, const double *vel, double *lv, double *lm, double h) {
    Adjoint *a = adj_of(s);
    const int n = (int)s->n;
    sum3_kernel<<<1, 1024, 0, s->stream>>>(n, lx, a->sigma);
    ++s->launches;
    ACU(cudaGetLastError());
    hc_vjp_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, a->sigma, vel, s->mass, h / s->p.m_star, lv, lm);
    ++s->launches;
    ACU(cudaGetLastError());
    return GENGA_OK;
}

// Reverse of step k from the step-start state at `start` (6n: x then v).
int step_vjp(genga_system *s, int64_t k, const double *start, double *lx, double *lv, double *lm) {
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    const double dt = s->p.dt, h = 0.5 * dt;
    // recompute the intermediate states of step k
    ACU(cudaMemcpyAsync(s->pos, start, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(s->vel, start + 3 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(s->rcl[0].rc, a->rc_hist + (size_t)k * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(launch_rcrit_derive(s));
    ACU(launch_kick(s, h, false, nullptr));
    ACU(launch_hc(s, h));
    ACU(launch_drift(s, 0, dt, nullptr, (int)n));          // pre_pos/pre_vel[0] = x1, v1
    const int64_t np = a->pair_off[(size_t)k + 1] - a->pair_off[(size_t)k];
    s->npairs_host[0] = np;
    if (np > 0) {
        int rc = ensure_pair_capacity(s, 0, np);
        if (rc != GENGA_OK) return rc;
        ACU(cudaMemcpyAsync(s->pairs[0], a->pair_hist + a->pair_off[(size_t)k], sizeof(uint2) * (size_t)np,
                            cudaMemcpyDeviceToDevice, s->stream));
        ACU(build_csr(s, 0, np));
        ACU(build_groups(s, 0, np));
        {
            const int brc = run_bs(s, 0, dt, np);
            if (brc != GENGA_OK) return brc;
        }
    }
    // (x2, v2)
    ACU(cudaMemcpyAsync(a->tmp, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(a->tmp + 3 * n, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(launch_hc(s, h));                                  // pos = x3, vel = v2
    // reverse
    int rc;
    if ((rc = kick_vjp(s, s->pos, lv, lx, lm, h)) != GENGA_OK) return rc;
    if ((rc = hc_vjp(s, lx, s->vel, lv, lm, h)) != GENGA_OK) return rc;
    drift_vjp_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s->stream>>>((int)n, s->pre_pos[0], s->pre_vel[0],
        np > 0 ? s->label : nullptr, s->p.G * s->p.m_star, dt, s->p.kepler_max_iter, lx, lv);
    ++s->launches;
    ACU(cudaGetLastError());
    if (np > 0) {
        AdjBsArgs B;
        B.n = (int)n; B.x2 = a->tmp; B.v2 = a->tmp + 3 * n;
        B.lx = lx; B.lv = lv; B.lm = lm;
        B.mass = s->mass; B.rc = s->rcl[0].rc; B.irc = s->rcl[0].irc;
        B.off = s->csr[0].off; B.list = s->csr[0].list;
        B.goff = s->goff; B.member = s->member; B.slotof = s->slotof;
        B.scr = a->bs_scr; B.S = n;
        B.G = s->p.G; B.mu = s->p.G * s->p.m_star; B.dt = dt; B.tol = s->p.bs_tol;
        B.max_steps = s->p.bs_max_steps; B.ctr = s->ctr;
        unsigned counts[kBuckets];
        ACU(bucket_groups(s, counts));
        for (int b = 0; b < kBuckets - 1; b++) {
            if (!counts[b]) continue;
            B.blist = s->bucket_list + (size_t)b * s->bucket_stride;
            // groups of up to 16 members: the columns of an attempt at once
            if (b == 0) bs_adj_cols_kernel<4><<<counts[b], 32, 0, s->stream>>>(B);
            else if (b == 1) bs_adj_cols_kernel<8><<<counts[b], 64, 0, s->stream>>>(B);
            else if (b == 2) bs_adj_cols_kernel<16><<<counts[b], 128, 0, s->stream>>>(B);
            else bs_adjoint_kernel<<<counts[b], kABs, 0, s->stream>>>(B);
            ++s->launches;
            ACU(cudaGetLastError());
        }
        if (counts[kBuckets - 1] &&
            (rc = bsm_adjoint_groups(s, a->tmp, a->tmp + 3 * n, lx, lv, lm, dt)) != GENGA_OK)
            return rc;
    }
    if ((rc = hc_vjp(s, lx, s->pre_vel[0], lv, lm, h)) != GENGA_OK) return rc;
    if ((rc = kick_vjp(s, start, lv, lx, lm, h)) != GENGA_OK) return rc;
    return GENGA_OK;
}

int forward_checkpointed(genga_system *s) {
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    ACU(cudaMemcpyAsync(s->pos, a->x0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(s->vel, a->v0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    for (int64_t k = 0; k < a->nsteps; k++) {
        if (k % a->every == 0) {
            double *c = a->ckpt + (size_t)(k / a->every) * 6 * n;
            ACU(cudaMemcpyAsync(c, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
            ACU(cudaMemcpyAsync(c + 3 * n, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
        }
        int rc = replay_step(s, k);
        if (rc != GENGA_OK) return rc;
    }
    return GENGA_OK;
}

}  // namespace

extern "C" {

// Sums (maxima for the largest group and attempt counts) of per-step statistics.
static void accumulate_stats(genga_stats_t &t, const genga_stats_t &x) {
    t.n_candidates += x.n_candidates;
    for (int l = 0; l < 8; l++) t.n_pairs[l] += x.n_pairs[l];
    t.n_groups += x.n_groups;
    t.max_group = std::max(t.max_group, x.max_group);
    t.bs_steps += x.bs_steps;
    t.bs_rejects += x.bs_rejects;
    t.kepler_fail += x.kepler_fail;
    t.bs_fail += x.bs_fail;
    t.kernel_launches += x.kernel_launches;
    t.bs_max_attempts = std::max(t.bs_max_attempts, x.bs_max_attempts);
}

int genga_adjoint_forward(genga_system_t *s, int64_t nsteps, int64_t checkpoint_every) {
    if (!s || nsteps < 1 || checkpoint_every < 1 || s->p.slevels != 1 || s->p.tp_mode != 0) return GENGA_EINVAL;
    int rc = adj_alloc(s, nsteps, checkpoint_every);
    if (rc != GENGA_OK) return rc;
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    ACU(cudaMemcpyAsync(a->x0, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(a->v0, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    genga_stats_t total;
    memset(&total, 0, sizeof(total));
    for (int64_t k = 0; k < nsteps; k++) {
        if (k % checkpoint_every == 0) {
            double *c = a->ckpt + (size_t)(k / checkpoint_every) * 6 * n;
            ACU(cudaMemcpyAsync(c, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
            ACU(cudaMemcpyAsync(c + 3 * n, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
        }
        rc = genga_step(s, 1);
        if (rc != GENGA_OK) return rc;
        accumulate_stats(total, s->stats);
        ACU(cudaMemcpyAsync(a->rc_hist + (size_t)k * n, s->rcl[0].rc, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
        rc = adj_push_pairs(s, s->pairs[0], s->npairs_host[0], false);
        if (rc != GENGA_OK) return rc;
    }
    s->stats = total;
    ACU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

int genga_adjoint_load(genga_system_t *s, int64_t nsteps, int64_t checkpoint_every, const double *rc_hist,
                       const int64_t *pair_offsets, const uint32_t *pairs) {
    if (!s || nsteps < 1 || checkpoint_every < 1 || !rc_hist || !pair_offsets || s->p.slevels != 1 ||
        s->p.tp_mode != 0)
        return GENGA_EINVAL;
    int rc = adj_alloc(s, nsteps, checkpoint_every);
    if (rc != GENGA_OK) return rc;
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    ACU(cudaMemcpyAsync(a->x0, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(a->v0, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(a->rc_hist, rc_hist, sizeof(double) * n * (size_t)nsteps, cudaMemcpyHostToDevice, s->stream));
    for (int64_t k = 0; k < nsteps; k++) {
        const int64_t np = pair_offsets[k + 1] - pair_offsets[k];
        if (np < 0) return GENGA_EINVAL;
        rc = adj_push_pairs(s, (const uint2 *)(pairs + 2 * pair_offsets[k]), np, true);
        if (rc != GENGA_OK) return rc;
    }
    rc = forward_checkpointed(s);
    if (rc != GENGA_OK) return rc;
    ACU(cudaStreamSynchronize(s->stream));
    return genga_sync(s);
}

int genga_adjoint_backward(genga_system_t *s, const double *lam_x, const double *lam_v, double *grad_x0,
                           double *grad_v0, double *grad_m) {
    if (!s || !lam_x || !lam_v || !grad_x0 || !grad_v0 || !grad_m || !s->adj || s->p.tp_mode != 0)
        return GENGA_EINVAL;
    Adjoint *a = adj_of(s);
    if (a->nsteps < 1) return GENGA_EINVAL;
    const size_t n = (size_t)s->n;
    // keep the caller's (final) state
    ACU(cudaMemcpyAsync(a->save_pos, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(a->save_vel, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(grad_x0, lam_x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(grad_v0, lam_v, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemsetAsync(grad_m, 0, sizeof(double) * n, s->stream));
    const int64_t nseg = (a->nsteps + a->every - 1) / a->every;
    for (int64_t seg = nseg - 1; seg >= 0; seg--) {
        const int64_t k0 = seg * a->every, k1 = std::min(a->nsteps, k0 + a->every);
        const double *c = a->ckpt + (size_t)seg * 6 * n;
        ACU(cudaMemcpyAsync(s->pos, c, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
        ACU(cudaMemcpyAsync(s->vel, c + 3 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
        for (int64_t k = k0; k < k1; k++) {
            double *st = a->seg + (size_t)(k - k0) * 6 * n;
            ACU(cudaMemcpyAsync(st, s->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
            ACU(cudaMemcpyAsync(st + 3 * n, s->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
            if (k + 1 < k1) {
                int rc = replay_step(s, k);
                if (rc != GENGA_OK) return rc;
            }
        }
        for (int64_t k = k1 - 1; k >= k0; k--) {
            int rc = step_vjp(s, k, a->seg + (size_t)(k - k0) * 6 * n, grad_x0, grad_v0, grad_m);
            if (rc != GENGA_OK) return rc;
        }
    }
    ACU(cudaMemcpyAsync(s->pos, a->save_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaMemcpyAsync(s->vel, a->save_vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s->stream));
    ACU(cudaStreamSynchronize(s->stream));
    return genga_sync(s);
}

int genga_adjoint_export(genga_system_t *s, double *rc_hist, int64_t *pair_offsets, uint32_t *pairs,
                         int64_t cap, int64_t *n_steps, int64_t *n_pairs) {
    if (!s || !s->adj) return GENGA_EINVAL;
    Adjoint *a = adj_of(s);
    const size_t n = (size_t)s->n;
    const int64_t total = a->pair_off.back();
    if (n_steps) *n_steps = a->nsteps;
    if (n_pairs) *n_pairs = total;
    if (rc_hist)
        ACU(cudaMemcpyAsync(rc_hist, a->rc_hist, sizeof(double) * n * (size_t)a->nsteps, cudaMemcpyDeviceToHost, s->stream));
    if (pair_offsets)
        for (int64_t k = 0; k <= a->nsteps; k++) pair_offsets[k] = a->pair_off[(size_t)k];
    if (pairs && total > 0)
        ACU(cudaMemcpyAsync(pairs, a->pair_hist, sizeof(uint2) * (size_t)std::min(cap, total), cudaMemcpyDeviceToHost, s->stream));
    ACU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

// The same call under the name of the boundary's call list.
int genga_step_backward(genga_system_t *s, const double *lam_x, const double *lam_v, double *grad_x0,
                        double *grad_v0, double *grad_m) {
    return genga_adjoint_backward(s, lam_x, lam_v, grad_x0, grad_v0, grad_m);
}

}  // extern "C"

namespace genga {
void adjoint_free(genga_system *s) {
    if (!s->adj) return;
    Adjoint *a = (Adjoint *)s->adj;
    double *ps[] = {a->rc_hist, a->x0, a->v0, a->ckpt, a->seg, a->tmp, a->part, a->sigma, a->bs_scr,
                    a->save_pos, a->save_vel};
    for (double *p : ps) if (p) cudaFree(p);
    if (a->pair_hist) cudaFree(a->pair_hist);
    delete a;
    s->adj = nullptr;
}
}  // namespace genga
