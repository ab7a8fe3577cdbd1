// particle.cu -- per-body kernels of the hybrid step (Appendix A): Rcrit
// (Eq. rcrit), HC (Eq. Hc), FG (Kepler part of Eq. Ha) with the pre-drift copy,
// the level restore of the higher-level scheme (Sec. 6.3), and the energy /
// angular-momentum report (Eq. H).
//
// These kernels are memory/latency bound (a few hundred bytes per body); they
// use one thread per body, coalesced SoA loads and no shared memory.  FG runs
// its Newton iteration per thread; its Stumpff functions need no
// transcendental calls (series + argument quartering).
#include <algorithm>

#include "common.cuh"

namespace genga {
namespace {

// ---------------------------------------------------------------- Rcrit
// rc_i = max(n1 R_H,i, n2 dt |v_i|), R_H,i = |x_i| (m_i/(3 m_star))^(1/3).
// |x| and |v| use the detection operation order (no contraction) so that the
// thresholds compare bit-for-bit with a plain CPU evaluation.
__device__ __forceinline__ void derive_thresholds(double rc, double f_pc, double *rc2, double *pc2,
                                                  float *thr_rc, double *irc) {
    *irc = __ddiv_rn(1.0, rc);
    const double r2 = __dmul_rn(rc, rc);
    const double t = __dmul_rn(f_pc, rc);
    const double p2 = __dmul_rn(t, t);
    *rc2 = r2;
    if (pc2) *pc2 = p2;
    // conservative FP32 upper bound (rounded up, + 2^-16)
    if (thr_rc) *thr_rc = fmaxf(__double2float_ru(r2) * 1.0000153f, 1.17549435e-38f);
}

__global__ void rcrit_kernel(int n, const double *pos, const double *vel, const double *mass,
                             double m_star, double dt, double n1, double n2, double f_pc,
                             RcritArrays out, const int *bodies, int nb, DevCounters *ctr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int i = bodies ? bodies[k] : k;
    const double x = pos[i], y = pos[(size_t)n + i], z = pos[2 * (size_t)n + i];
    const double vx = vel[i], vy = vel[(size_t)n + i], vz = vel[2 * (size_t)n + i];
    const double r = sqrt(dist2_rn(x, y, z));
    const double vabs = sqrt(dist2_rn(vx, vy, vz));
    if (!(r > 0.0) || !isfinite(r) || !isfinite(vabs)) latch_error(ctr, kErrBadState);
    const double hill = __dmul_rn(r, cbrt(__ddiv_rn(mass[i], __dmul_rn(3.0, m_star))));
    const double a = __dmul_rn(n1, hill);
    const double b = __dmul_rn(__dmul_rn(n2, dt), vabs);
    const double rc = a > b ? a : b;
    out.rc[i] = rc;
    derive_thresholds(rc, f_pc, &out.rc2[i], out.pc2 ? &out.pc2[i] : nullptr,
                      out.thr_rc ? &out.thr_rc[i] : nullptr, &out.irc[i]);
}

__global__ void rcrit_derive_kernel(int n, double f_pc, RcritArrays a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    derive_thresholds(a.rc[i], f_pc, &a.rc2[i], &a.pc2[i], &a.thr_rc[i], &a.irc[i]);
}

// ---------------------------------------------------------------- HC
// P = sum_j m_j v_j in a fixed order (strided per-thread sums, then a fixed
// tree), shift = dt_half P / m_star; then x_i += shift.
constexpr int kHcThreads = 256;

// P = sum_j m_j v_j in a fixed order: each block sums a contiguous range of
// bodies (strided per-thread sums, then a fixed tree), and the last block to
// finish adds the block sums in block order; shift = dt_half P / m_star.  One
// launch over every SM (a single block was bound by one SM's FP64 rate).
__global__ void __launch_bounds__(kHcThreads)
hc_reduce_kernel(int n, const double *vel, const double *mass, double m_star, double dt_half,
                 double *part, DevCounters *ctr) {
    __shared__ double sp[3][kHcThreads];
    __shared__ bool last;
    const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int j0 = (int)blockIdx.x * per, j1 = min(n, j0 + per);
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int j = j0 + (int)threadIdx.x; j < j1; j += kHcThreads) {
        const double mj = mass[j];
        p0 += mj * vel[j];
        p1 += mj * vel[(size_t)n + j];
        p2 += mj * vel[2 * (size_t)n + j];
    }
    sp[0][threadIdx.x] = p0; sp[1][threadIdx.x] = p1; sp[2][threadIdx.x] = p2;
    __syncthreads();
    for (int w = kHcThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sp[0][threadIdx.x] += sp[0][threadIdx.x + w];
            sp[1][threadIdx.x] += sp[1][threadIdx.x + w];
            sp[2][threadIdx.x] += sp[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) part[3 * blockIdx.x + threadIdx.x] = sp[threadIdx.x][0];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctr->hc_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 3) {
        const volatile double *vp = part;
        double sum = 0.0;
        for (unsigned q = 0; q < gridDim.x; q++) sum += vp[3 * q + threadIdx.x];
        ctr->hc_shift[threadIdx.x] = dt_half * sum / m_star;
    }
    if (threadIdx.x == 0) ctr->hc_done = 0;
}

__global__ void hc_apply_kernel(int n, double *pos, const DevCounters *ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pos[i] += ctr->hc_shift[0];
    pos[(size_t)n + i] += ctr->hc_shift[1];
    pos[2 * (size_t)n + i] += ctr->hc_shift[2];
}

// ---------------------------------------------------------------- FG
// kepler_drift() and stumpff() live in common.cuh (shared with the ensemble).

__global__ void drift_kernel(int n, double *pos, double *vel, double *pre_pos, double *pre_vel,
                             double mu, double dt, int max_iter, const int *bodies, int nb,
                             DevCounters *ctr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int i = bodies ? bodies[k] : k;
    const size_t N = (size_t)n;
    double x = pos[i], y = pos[N + i], z = pos[2 * N + i];
    double vx = vel[i], vy = vel[N + i], vz = vel[2 * N + i];
    if (pre_pos) {
        pre_pos[i] = x; pre_pos[N + i] = y; pre_pos[2 * N + i] = z;
        pre_vel[i] = vx; pre_vel[N + i] = vy; pre_vel[2 * N + i] = vz;
    }
    if (!kepler_drift(x, y, z, vx, vy, vz, mu, dt, max_iter)) {
        latch_error(ctr, kErrKepler);
        atomicAdd(&ctr->kepler_fail, 1ull);
    }
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) && isfinite(vz)))
        latch_error(ctr, kErrBadState);
    pos[i] = x; pos[N + i] = y; pos[2 * N + i] = z;
    vel[i] = vx; vel[N + i] = vy; vel[2 * N + i] = vz;
}

__global__ void restore_kernel(int n, double *pos, double *vel, const double *pre_pos,
                               const double *pre_vel, const int *bodies, int nb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int i = bodies[k];
    const size_t N = (size_t)n;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        pos[c * N + i] = pre_pos[c * N + i];
        vel[c * N + i] = pre_vel[c * N + i];
    }
}

// ---------------------------------------------------------------- energy
// Per body: kinetic, star potential, half of the pair potential (all j != i),
// angular momentum and momentum; then a fixed-order compensated reduction.
constexpr int kEnThreads = 128;
constexpr int kEnTile = 256;

__global__ void __launch_bounds__(kEnThreads)
energy_terms_kernel(int n, int nm, const double *pos, const double *vel, const double *mass, double G,
                    double m_star, double *terms /* [8][n] */) {
    __shared__ double sx[kEnTile], sy[kEnTile], sz[kEnTile], sm[kEnTile];
    const int i = blockIdx.x * kEnThreads + threadIdx.x;
    const size_t N = (size_t)n;
    const bool valid = i < n;
    double xi = 0, yi = 0, zi = 0;
    if (valid) { xi = pos[i]; yi = pos[N + i]; zi = pos[2 * N + i]; }
    double S = 0.0, C = 0.0;
    const int jlim = i >= nm ? nm : n;     // a test particle has no pair term with another
    for (int jt = 0; jt < n; jt += kEnTile) {
        const int cnt = min(kEnTile, n - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kEnThreads) {
            sx[k] = pos[jt + k]; sy[k] = pos[N + jt + k]; sz[k] = pos[2 * N + jt + k]; sm[k] = mass[jt + k];
        }
        __syncthreads();
        double part = 0.0;
        for (int k = 0; k < cnt; k++) {
            if (jt + k == i || jt + k >= jlim) continue;
            const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
            part += sm[k] / sqrt(dx * dx + dy * dy + dz * dz);
        }
        double t, e;
        two_sum(S, part, t, e); S = t; C += e;
    }
    if (!valid) return;
    const double m = mass[i];
    const double vx = vel[i], vy = vel[N + i], vz = vel[2 * N + i];
    const double r = sqrt(xi * xi + yi * yi + zi * zi);
    terms[0 * N + i] = 0.5 * m * (vx * vx + vy * vy + vz * vz);
    terms[1 * N + i] = -G * m_star * m / r;
    terms[2 * N + i] = -0.5 * G * m * (S + C);
    terms[3 * N + i] = m * (yi * vz - zi * vy);
    terms[4 * N + i] = m * (zi * vx - xi * vz);
    terms[5 * N + i] = m * (xi * vy - yi * vx);
    terms[6 * N + i] = m * vx;
    terms[7 * N + i] = m * vy;
    terms[8 * N + i] = m * vz;
}

// One block per row: compensated fixed-order sum of terms[row][0..n).
__global__ void row_sum_kernel(int n, const double *terms, int rows, double *out) {
    __shared__ double ss[256], sc[256];
    const int row = blockIdx.x;
    const double *t = terms + (size_t)row * n;
    double S = 0.0, C = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        double a, e;
        two_sum(S, t[i], a, e); S = a; C += e;
    }
    ss[threadIdx.x] = S; sc[threadIdx.x] = C;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S2 = 0.0, C2 = 0.0;
        for (int k = 0; k < 256; k++) {
            double a, e;
            two_sum(S2, ss[k], a, e); S2 = a; C2 += e + sc[k];
        }
        out[row] = S2 + C2;
    }
}

// E = (kinetic + star + pairs) + |P|^2 / (2 m_star); L as summed.
__global__ void energy_combine_kernel(double m_star, double *sums) {
    const double P2 = sums[6] * sums[6] + sums[7] * sums[7] + sums[8] * sums[8];
    sums[9] = ((sums[0] + sums[1]) + sums[2]) + P2 / (2.0 * m_star);
}

}  // namespace

cudaError_t launch_rcrit(genga_system *s, int level, double dt, const int *bodies, int nb) {
    if (nb <= 0) return cudaSuccess;
    RcritArrays out = s->rcl[level];
    if (level > 0) { out.pc2 = nullptr; out.thr_rc = nullptr; }
    rcrit_kernel<<<(nb + 255) / 256, 256, 0, s->stream>>>((int)s->n, s->pos, s->vel, s->mass,
        s->p.m_star, dt, s->p.n1, s->p.n2, s->p.f_pc, out, bodies, nb, s->ctr); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_rcrit_derive(genga_system *s) {
    const int n = (int)s->n;
    rcrit_derive_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->p.f_pc, s->rcl[0]); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_hc(genga_system *s, double dt_half) {
    const int n = (int)s->n;
    const int nblk = std::max(1, std::min(s->num_sms, (n + kHcThreads - 1) / kHcThreads));
    hc_reduce_kernel<<<nblk, kHcThreads, 0, s->stream>>>(n, s->vel, s->mass, s->p.m_star, dt_half, s->red,
                                                        s->ctr); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    hc_apply_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->pos, s->ctr); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_drift(genga_system *s, int level, double dt, const int *bodies, int nb) {
    if (nb <= 0) return cudaSuccess;
    drift_kernel<<<(nb + 127) / 128, 128, 0, s->stream>>>((int)s->n, s->pos, s->vel,
        s->pre_pos[level], s->pre_vel[level], s->p.G * s->p.m_star, dt, s->p.kepler_max_iter,
        bodies, nb, s->ctr); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_restore(genga_system *s, int from_level, const int *bodies, int nb) {
    if (nb <= 0) return cudaSuccess;
    restore_kernel<<<(nb + 255) / 256, 256, 0, s->stream>>>((int)s->n, s->pos, s->vel,
        s->pre_pos[from_level], s->pre_vel[from_level], bodies, nb); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_energy(genga_system *s, double *E_host, double *L_host) {
    const int n = (int)s->n;
    double *terms = s->red;            // 9 rows of n, then 10 sums
    energy_terms_kernel<<<(n + kEnThreads - 1) / kEnThreads, kEnThreads, 0, s->stream>>>(
        n, tp_bound(s), s->pos, s->vel, s->mass, s->p.G, s->p.m_star, terms); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    double *sums = terms + 9 * (size_t)n;
    row_sum_kernel<<<9, 256, 0, s->stream>>>(n, terms, 9, sums); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    energy_combine_kernel<<<1, 1, 0, s->stream>>>(s->p.m_star, sums); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    double h[10];
    GENGA_CUDA_TRY(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    GENGA_CUDA_TRY(cudaStreamSynchronize(s->stream));
    *E_host = h[9];
    L_host[0] = h[3]; L_host[1] = h[4]; L_host[2] = h[5];
    return cudaSuccess;
}

}  // namespace genga
