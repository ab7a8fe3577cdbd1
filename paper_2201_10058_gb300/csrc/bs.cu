// bs.cu -- Bulirsch-Stoer integration of close-encounter groups (Sec. 4.1,
// Appendix A "Bulirsch-Stoer(dt)") and the level kick KickS of the
// higher-level changeover scheme (Sec. 4.3, Appendix A).
//
// BS: one CTA per group, members strided over the CTA's threads.  Each member
// integrates
//     dx/dt = v,   dv/dt = -mu x/|x|^3 + G sum_{partners j} m_j W_ij (x_j - x)/r^3,
//     W_ij = prod_{k=0..level} (1 - K(r_ij; rc_k,ij)),
// with partners taken from the ascending partner list of the level's
// encounter pairs (the BS-A partner-list scheme of Sec. 4.1; the sum order is
// fixed, so results do not depend on member layout).  Modified midpoint with
// n = 2, 4, ..., 16 and polynomial extrapolation in h^2 (Neville, in place);
// error = max over members and components of |T_kk - T_k,k-1| / scale with
// scale = |y| + |H dy/dt| + 1e-300; accept at the first column k >= 1 with
// error <= tol, grow H by 1.5 if k < 4, otherwise halve H.  The step control is
// evaluated identically by every thread after a CTA-wide max reduction.
// State lives in a global scratch (84 doubles per member slot, component-major,
// L2-resident), so the kernel has no group-size limit.
#include "common.cuh"

namespace genga {
namespace {

constexpr int kBsThreads = 64;
constexpr int kBsCols = 8;

struct BsArgs {
    int n;
    const double *pre_pos, *pre_vel;
    double *pos, *vel;
    const double *mass;
    const double *rc[kMaxLevels];
    int nlev;
    const int *off, *list;
    const int *glist, *goff, *member, *slotof;
    double *scr;     // [84][S]
    size_t S;
    double G, mu, dt, tol;
    int max_steps;
    unsigned long long time_limit_ns;
    DevCounters *ctr;
};

// scratch rows
enum { kY = 0, kF0 = 6, kZM = 12, kZN = 18, kFZ = 24, kSC = 30, kT = 36 };  // T: 48 rows

__device__ __forceinline__ double &R(const BsArgs &A, int row, int slot) {
    return A.scr[(size_t)row * A.S + slot];
}

// derivative of member slot s from the state rows z0..z0+5 into rows f0..f0+5
__device__ void bs_deriv(const BsArgs &A, int z0, int f0, int s) {
    const int b = A.member[s];
    const double x = R(A, z0 + 0, s), y = R(A, z0 + 1, s), z = R(A, z0 + 2, s);
    const double r2 = x * x + y * y + z * z;
    const double sst = -A.mu / (r2 * sqrt(r2));
    double px = 0.0, py = 0.0, pz = 0.0;
    for (int q = A.off[b]; q < A.off[b + 1]; q++) {
        const int p = A.list[q];
        const int sp = A.slotof[p];
        const double dx = R(A, z0 + 0, sp) - x, dy = R(A, z0 + 1, sp) - y, dz = R(A, z0 + 2, sp) - z;
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double d = sqrt(d2);
        double W = 1.0;
        for (int l = 0; l < A.nlev; l++) W *= 1.0 - changeover(d, fmax(A.rc[l][b], A.rc[l][p]));
        const double c = A.mass[p] * W / (d2 * d);
        px += c * dx; py += c * dy; pz += c * dz;
    }
    R(A, f0 + 0, s) = R(A, z0 + 3, s);
    R(A, f0 + 1, s) = R(A, z0 + 4, s);
    R(A, f0 + 2, s) = R(A, z0 + 5, s);
    R(A, f0 + 3, s) = sst * x + A.G * px;
    R(A, f0 + 4, s) = sst * y + A.G * py;
    R(A, f0 + 5, s) = sst * z + A.G * pz;
}

__device__ double block_max(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double m = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) m = fmax(m, red[k]);
    __syncthreads();
    return m;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kBsThreads)
bs_kernel(BsArgs A) {
    __shared__ double red[kBsThreads / 32];
    __shared__ int stop;
    if (blockIdx.x >= A.ctr->ngroups) return;
    const unsigned long long t_start = global_ns();
    const int g = A.glist[blockIdx.x];
    const int s0 = A.goff[g], s1 = A.goff[g + 1];
    const size_t N = (size_t)A.n;

    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int b = A.member[s];
        for (int c = 0; c < 3; c++) {
            R(A, kY + c, s) = A.pre_pos[c * N + b];
            R(A, kY + 3 + c, s) = A.pre_vel[c * N + b];
        }
    }
    double t = 0.0, H = A.dt;
    int attempts = 0;
    long long acc = 0, rej = 0;
    bool failed = false;
    while (t < A.dt) {
        // attempt limit and a wall-clock limit, decided by one thread for the CTA
        if (threadIdx.x == 0)
            stop = (attempts >= A.max_steps) || (global_ns() - t_start > A.time_limit_ns);
        __syncthreads();
        if (stop) { failed = true; break; }
        attempts++;
        if (H > A.dt - t) H = A.dt - t;
        for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) bs_deriv(A, kY, kF0, s);
        for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
            for (int c = 0; c < 6; c++)
                R(A, kSC + c, s) = fabs(R(A, kY + c, s)) + fabs(H * R(A, kF0 + c, s)) + 1e-300;
        bool accepted = false;
        int kconv = 0;
        for (int k = 0; k < kBsCols; k++) {
            const int nk = 2 * (k + 1);
            const double h = H / nk;
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                for (int c = 0; c < 6; c++) {
                    const double y0 = R(A, kY + c, s);
                    R(A, kZM + c, s) = y0;
                    R(A, kZN + c, s) = y0 + h * R(A, kF0 + c, s);
                }
            for (int m = 1; m < nk; m++) {
                __syncthreads();
                for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) bs_deriv(A, kZN, kFZ, s);
                __syncthreads();
                for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                    for (int c = 0; c < 6; c++) {
                        const double tt = R(A, kZM + c, s) + 2.0 * h * R(A, kFZ + c, s);
                        R(A, kZM + c, s) = R(A, kZN + c, s);
                        R(A, kZN + c, s) = tt;
                    }
            }
            __syncthreads();
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) bs_deriv(A, kZN, kFZ, s);
            double err = 0.0;
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                for (int c = 0; c < 6; c++) {
                    const double cur0 = 0.5 * (R(A, kZN + c, s) + R(A, kZM + c, s) + h * R(A, kFZ + c, s));
                    double prev = R(A, kT + 0 * 6 + c, s);
                    double cur = cur0;
                    R(A, kT + 0 * 6 + c, s) = cur;
                    for (int j = 1; j <= k; j++) {
                        const double ratio = (double)nk / (double)(2 * (k - j + 1));
                        const double nxt = cur + (cur - prev) / (ratio * ratio - 1.0);
                        prev = R(A, kT + j * 6 + c, s);
                        R(A, kT + j * 6 + c, s) = nxt;
                        cur = nxt;
                    }
                    if (k >= 1) {
                        const double e = fabs(R(A, kT + k * 6 + c, s) - R(A, kT + (k - 1) * 6 + c, s)) / R(A, kSC + c, s);
                        err = fmax(err, e);
                    }
                }
            err = block_max(err, red);
            if (k >= 1 && err <= A.tol) { accepted = true; kconv = k; break; }
        }
        if (accepted) {
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
                for (int c = 0; c < 6; c++) R(A, kY + c, s) = R(A, kT + kconv * 6 + c, s);
            t += H;
            acc++;
            if (kconv < 4) H *= 1.5;
        } else {
            rej++;
            H *= 0.5;
        }
    }
    __syncthreads();
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int b = A.member[s];
        for (int c = 0; c < 3; c++) {
            A.pos[c * N + b] = R(A, kY + c, s);
            A.vel[c * N + b] = R(A, kY + 3 + c, s);
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd(&A.ctr->bs_steps, (unsigned long long)acc);
        atomicAdd(&A.ctr->bs_rejects, (unsigned long long)rej);
        if (failed) {
            atomicAdd(&A.ctr->bs_fail, 1ull);
            latch_error(A.ctr, kErrBS);
        }
    }
}

// KickS at level l >= 1 over the partner lists of the level-(l-1) pairs:
//   v_b += dt_half G sum_p m_p prod_{k<l}(1 - K_k) K_l (x_p - x_b)/r^3.
struct KickPairsArgs {
    int n, nb, level;
    const int *bodies;
    const int *off, *list;
    const double *pos;
    double *vel;
    const double *mass;
    const double *rc[kMaxLevels];
    double G, dt_half;
};

__global__ void kick_pairs_kernel(KickPairsArgs A) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.nb) return;
    const int b = A.bodies[k];
    const size_t N = (size_t)A.n;
    const double x = A.pos[b], y = A.pos[N + b], z = A.pos[2 * N + b];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int q = A.off[b]; q < A.off[b + 1]; q++) {
        const int p = A.list[q];
        const double dx = A.pos[p] - x, dy = A.pos[N + p] - y, dz = A.pos[2 * N + p] - z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double r = sqrt(r2);
        double W = 1.0;
        for (int l = 0; l < A.level; l++) W *= 1.0 - changeover(r, fmax(A.rc[l][b], A.rc[l][p]));
        W *= changeover(r, fmax(A.rc[A.level][b], A.rc[A.level][p]));
        const double f = A.mass[p] * W / (r2 * r);
        sx += f * dx; sy += f * dy; sz += f * dz;
    }
    A.vel[b] += A.dt_half * (A.G * sx);
    A.vel[N + b] += A.dt_half * (A.G * sy);
    A.vel[2 * N + b] += A.dt_half * (A.G * sz);
}

}  // namespace

cudaError_t launch_bs(genga_system *s, int level, double dt_l, int64_t max_groups) {
    if (max_groups <= 0) return cudaSuccess;
    BsArgs A;
    A.n = (int)s->n;
    A.pre_pos = s->pre_pos[level];
    A.pre_vel = s->pre_vel[level];
    A.pos = s->pos; A.vel = s->vel; A.mass = s->mass;
    for (int l = 0; l < kMaxLevels; l++) A.rc[l] = s->rcl[l].rc;
    A.nlev = level + 1;
    A.off = s->csr[level].off; A.list = s->csr[level].list;
    A.glist = s->glist; A.goff = s->goff; A.member = s->member; A.slotof = s->slotof;
    A.scr = s->bs_scratch; A.S = (size_t)s->n;
    A.G = s->p.G; A.mu = s->p.G * s->p.m_star; A.dt = dt_l; A.tol = s->p.bs_tol;
    A.max_steps = s->p.bs_max_steps;
    A.time_limit_ns = 10000000000ull;   // 10 s per group call
    A.ctr = s->ctr;
    bs_kernel<<<(unsigned)max_groups, kBsThreads, 0, s->stream>>>(A); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_kick_pairs(genga_system *s, int level, double dt_half, int nb) {
    if (nb <= 0) return cudaSuccess;
    KickPairsArgs A;
    A.n = (int)s->n; A.nb = nb; A.level = level;
    A.bodies = s->bodies[level];
    A.off = s->csr[level - 1].off; A.list = s->csr[level - 1].list;
    A.pos = s->pos; A.vel = s->vel; A.mass = s->mass;
    for (int l = 0; l < kMaxLevels; l++) A.rc[l] = s->rcl[l].rc;
    A.G = s->p.G; A.dt_half = dt_half;
    kick_pairs_kernel<<<(nb + 127) / 128, 128, 0, s->stream>>>(A); ++s->launches;
    return cudaGetLastError();
}

}  // namespace genga
