// bsm.cu -- Bulirsch-Stoer for close-encounter groups of more than
// kBlockGroupMax members, spread over the whole GPU (the role of the paper's
// BS-M, Sec. 4.1), with every such group of the current grouping advanced
// together.
//
// One round is one attempt of every still-running group, at its own step H:
//   start      derivative at the attempt's start, error scale, first
//              midpoint sub-step of all 8 extrapolation columns;
//   sub-step   launch `it` (1..16) moves every column whose n_k = 2(k+1)
//              still has sub-steps left, over all (column, member) pairs
//              (one thread each; ping-pong state buffers, so partner reads
//              never race with writes);
//   Neville    per (component, member): the extrapolation table, its
//              diagonal, and each column's error folded into the group's 8
//              error words (atomic max on the bits of non-negative doubles);
//   decide     one thread per group: first column k >= 1 under tolerance
//              -> accept (grow H by 1.5 if k < 4), else halve H; attempt
//              and time bookkeeping; done / failed status;
//   accept     members of accepting groups take the accepted column.
// The step control never leaves the device.  The host enqueues a batch of
// rounds and then reads the groups' status words once; rounds enqueued after
// a group finished return at once for it.  A group fails after bs_max_steps
// attempts, so at most bs_max_steps rounds run.  Scheme and acceptance rule
// are those of the in-block kernels (modified midpoint n = 2..16, Neville in
// h^2, error scale |y| + |H dy/dt| + 1e-300).
//
// The ODE is a template policy: the group's forward ODE (6 values per member)
// or the adjoint's augmented backward ODE (13 values per member).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace genga {
namespace {

constexpr int kMThreads = 64;

// Batch of groups: compact member index m in [0, M) over the groups.
struct BsmArgs {
    int n;                         // bodies in the system
    int M;                         // members over all batched groups
    int ng;                        // batched groups
    const int *mbody;              // [M] body of compact member m
    const int *mgroup;             // [M] batched group of m
    const double *irc;             // [nlev][M] 1/rc of compact member m per level
    const int *gbase;              // [ng] first compact index of the group
    const int *gslot0;             // [ng] first global slot of the group
    const int *slotof;             // body -> global slot
    const int *off, *list;         // partner CSR (global ids, ascending per row)
    const double *mass;
    int nlev;
    double G, mu, dt, tol;
    int max_steps;
    // per-group step control (device)
    double *gt, *gH;
    int *gstat;                    // 0 running, 1 done, 2 failed
    int *gkconv;                   // accepted column of the last round, -1 none
    long long *gatt, *gacc, *grej;
    unsigned long long *gerr;      // [ng][8]
};

// Partners of a member belong to its group (groups are connected components
// of the same pair graph), so their compact index follows from the slot.
__device__ __forceinline__ int partner_index(const BsmArgs &A, int g, int p) {
    return A.gbase[g] + (A.slotof[p] - A.gslot0[g]);
}

__device__ __forceinline__ double step_of(const BsmArgs &A, int g) {
    const double H = A.gH[g];
    const double left = A.dt - A.gt[g];
    return H > left ? left : H;
}

// Forward group ODE: y = (x, v); a = -mu x/r^3 + G sum_p m_p W (x_p - x)/r^3,
// W = prod_{levels} (1 - K); partners in ascending order (fixed sum order).
struct FwdOde {
    static constexpr int D = 6;
    static constexpr int NERR = 6;
    __device__ static void deriv(const BsmArgs &A, const double *Z, size_t ld, int m, int g, double *f) {
        const int b = A.mbody[m];
        const double x = Z[0 * ld + m], y = Z[1 * ld + m], z = Z[2 * ld + m];
        const double r2 = fma(z, z, fma(y, y, x * x));
        const double ys = rsqrt_newton(r2);
        const double sst = -A.mu * (ys * ys * ys);
        double px = 0.0, py = 0.0, pz = 0.0;
        for (int q = A.off[b]; q < A.off[b + 1]; q++) {
            const int p = A.list[q];
            const int sp = partner_index(A, g, p);
            const double dx = Z[0 * ld + sp] - x, dy = Z[1 * ld + sp] - y, dz = Z[2 * ld + sp] - z;
            const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double yv = rsqrt_newton(d2);
            const double d = d2 * yv;
            double W = 1.0;
            for (int l = 0; l < A.nlev; l++)
                W *= 1.0 - changeover_fast(d, fmin(A.irc[(size_t)l * A.M + m], A.irc[(size_t)l * A.M + sp]));
            const double c = A.mass[p] * W * (yv * yv * yv);
            px = fma(c, dx, px); py = fma(c, dy, py); pz = fma(c, dz, pz);
        }
        f[0] = Z[3 * ld + m]; f[1] = Z[4 * ld + m]; f[2] = Z[5 * ld + m];
        f[3] = fma(sst, x, A.G * px); f[4] = fma(sst, y, A.G * py); f[5] = fma(sst, z, A.G * pz);
    }
};

// Adjoint augmented ODE in reversed time (level 0): y (6), lambda (6), the
// mass-gradient integral (1); with A = da/dx:
//   dy/dtau = -f(y),  dlx/dtau = A^T lv,  dlv/dtau = lx,
//   dg_a/dtau = G sum_p W lv_p . (x_a - x_p)/r^3   (da_p/dm_a).
struct AdjOde {
    static constexpr int D = 13;
    static constexpr int NERR = 6;
    __device__ static void deriv(const BsmArgs &A, const double *Z, size_t ld, int m, int g, double *f) {
        const int b = A.mbody[m];
        const double x = Z[0 * ld + m], y = Z[1 * ld + m], z = Z[2 * ld + m];
        const double lvx = Z[9 * ld + m], lvy = Z[10 * ld + m], lvz = Z[11 * ld + m];
        const double mb = A.mass[b];
        const double r2 = fma(z, z, fma(y, y, x * x));
        const double ys = rsqrt_newton(r2);
        const double ir2 = ys * ys, ir3 = ir2 * ys;
        double ax = -A.mu * x * ir3, ay = -A.mu * y * ir3, az = -A.mu * z * ir3;
        const double xl = x * lvx + y * lvy + z * lvz;
        const double tx = -A.mu * ir3 * (lvx - 3.0 * x * xl * ir2);
        const double ty = -A.mu * ir3 * (lvy - 3.0 * y * xl * ir2);
        const double tz = -A.mu * ir3 * (lvz - 3.0 * z * xl * ir2);
        double px = 0.0, py = 0.0, pz = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, gm = 0.0;
        for (int q = A.off[b]; q < A.off[b + 1]; q++) {
            const int p = A.list[q];
            const int sp = partner_index(A, g, p);
            const double dx = Z[0 * ld + sp] - x, dy = Z[1 * ld + sp] - y, dz = Z[2 * ld + sp] - z;
            const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double yv = rsqrt_newton(d2);
            const double d = d2 * yv, id2 = yv * yv, id3 = id2 * yv;
            double K, dK;
            changeover_fast_dr(d, fmin(A.irc[m], A.irc[sp]), K, dK);
            const double W = 1.0 - K;
            const double Wp = -dK;
            const double mp = A.mass[p];
            const double cw = mp * W * id3;
            px = fma(cw, dx, px); py = fma(cw, dy, py); pz = fma(cw, dz, pz);
            const double qx = Z[9 * ld + sp], qy = Z[10 * ld + sp], qz = Z[11 * ld + sp];
            const double e0 = mb * qx - mp * lvx, e1 = mb * qy - mp * lvy, e2 = mb * qz - mp * lvz;
            const double de = dx * e0 + dy * e1 + dz * e2;
            const double aa = W * id3;
            const double bb = de * id2 * (Wp * id2 - 3.0 * W * id3);
            gx += aa * e0 + bb * dx; gy += aa * e1 + bb * dy; gz += aa * e2 + bb * dz;
            gm -= W * (qx * dx + qy * dy + qz * dz) * id3;
        }
        ax += A.G * px; ay += A.G * py; az += A.G * pz;
        f[0] = -Z[3 * ld + m]; f[1] = -Z[4 * ld + m]; f[2] = -Z[5 * ld + m];
        f[3] = -ax; f[4] = -ay; f[5] = -az;
        f[6] = tx + A.G * gx; f[7] = ty + A.G * gy; f[8] = tz + A.G * gz;
        f[9] = Z[6 * ld + m]; f[10] = Z[7 * ld + m]; f[11] = Z[8 * ld + m];
        f[12] = A.G * gm;
    }
};

// Buffers, component-major over the M compact members ([..][D][M]):
//   Y, F0, SC           attempt start, its derivative, error scale
//   ZM[8], ZA[8], ZB[8] per column: previous midpoint state, two buffers of the current
//   OUT[8], DIAG[8]     column results and the Neville diagonal T_kk
template <class Ode>
__global__ void __launch_bounds__(kMThreads)
bsm_start_kernel(BsmArgs A, const double *Y, double *F0, double *SC, double *ZM, double *ZA) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.M) return;
    const int g = A.mgroup[m];
    if (A.gstat[g] != 0) return;
    constexpr int D = Ode::D;
    const size_t ld = (size_t)A.M, blk = (size_t)D * ld;
    const double H = step_of(A, g);
    double f[D];
    Ode::deriv(A, Y, ld, m, g, f);
    for (int c = 0; c < D; c++) {
        const double y = Y[c * ld + m];
        F0[c * ld + m] = f[c];
        SC[c * ld + m] = fabs(y) + fabs(H * f[c]) + 1e-300;
        for (int k = 0; k < 8; k++) {
            const double h = H / (2 * (k + 1));
            ZM[k * blk + c * ld + m] = y;
            ZA[k * blk + c * ld + m] = y + h * f[c];
        }
    }
}

// Sub-step `it` for all (column, member): reads Zcur, writes Znext or OUT.
template <class Ode>
__global__ void __launch_bounds__(kMThreads)
bsm_substep_kernel(BsmArgs A, const double *Zcur, double *Znext, double *ZM, double *OUT, int it) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8LL * A.M) return;
    const int k = (int)(t / A.M), m = (int)(t % A.M);
    const int nk = 2 * (k + 1);
    if (it > nk) return;
    const int g = A.mgroup[m];
    if (A.gstat[g] != 0) return;
    constexpr int D = Ode::D;
    const size_t ld = (size_t)A.M, blk = (size_t)D * ld;
    const double h = step_of(A, g) / nk;
    const double *Z = Zcur + k * blk;
    double f[D];
    Ode::deriv(A, Z, ld, m, g, f);
    if (it < nk) {
        for (int c = 0; c < D; c++) {
            const double tt = ZM[k * blk + c * ld + m] + 2.0 * h * f[c];
            ZM[k * blk + c * ld + m] = Z[c * ld + m];
            Znext[k * blk + c * ld + m] = tt;
        }
    } else {
        for (int c = 0; c < D; c++)
            OUT[k * blk + c * ld + m] = 0.5 * (Z[c * ld + m] + ZM[k * blk + c * ld + m] + h * f[c]);
    }
}

// Neville per (component, member); column errors of the first NERR
// components folded into the group's error words.
template <class Ode>
__global__ void __launch_bounds__(kMThreads)
bsm_neville_kernel(BsmArgs A, const double *OUT, const double *SC, double *DIAG) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int D = Ode::D;
    const size_t ld = (size_t)A.M, blk = (size_t)D * ld;
    double e[8];
    for (int k = 0; k < 8; k++) e[k] = 0.0;
    int g = -1;
    if (t < (long long)D * A.M) {
        const int c = (int)(t / A.M), m = (int)(t % A.M);
        g = A.mgroup[m];
        if (A.gstat[g] == 0) {
            double T[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < 8; k++) {
                double cur = OUT[k * blk + c * ld + m];
                double prev = T[0];
                T[0] = cur;
                for (int j = 1; j <= k; j++) {
                    const double coef = (double)((k - j + 1) * (k - j + 1)) / (double)(j * (2 * k + 2 - j));
                    const double nxt = fma(cur - prev, coef, cur);
                    prev = T[j];
                    T[j] = nxt;
                    cur = nxt;
                }
                DIAG[k * blk + c * ld + m] = T[k];
                if (k >= 1 && c < Ode::NERR) e[k] = fabs(T[k] - T[k - 1]) / SC[c * ld + m];
            }
        } else {
            g = -1;
        }
    }
    // one atomic per warp when all its threads belong to one running group
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

// Step control, one thread per group (the in-block kernels' rule).
__global__ void bsm_decide_kernel(BsmArgs A) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= A.ng) return;
    A.gkconv[g] = -1;
    if (A.gstat[g] != 0) return;
    double H = step_of(A, g);
    int kconv = -1;
    for (int k = 1; k < 8 && kconv < 0; k++) {
        const double e = __longlong_as_double((long long)A.gerr[(size_t)g * 8 + k]);
        if (e <= A.tol) kconv = k;
    }
    for (int k = 0; k < 8; k++) A.gerr[(size_t)g * 8 + k] = 0ull;
    A.gatt[g] += 1;
    if (kconv >= 0) {
        A.gt[g] += H;
        A.gacc[g] += 1;
        if (kconv < 4) H *= 1.5;
    } else {
        A.grej[g] += 1;
        H *= 0.5;
    }
    A.gH[g] = H;
    A.gkconv[g] = kconv;
    if (!(A.gt[g] < A.dt)) A.gstat[g] = 1;
    else if (A.gatt[g] >= A.max_steps) A.gstat[g] = 2;
}

template <class Ode>
__global__ void __launch_bounds__(kMThreads)
bsm_accept_kernel(BsmArgs A, const double *DIAG, double *Y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int D = Ode::D;
    const size_t blk = (size_t)D * A.M;
    if (t >= (long long)D * A.M) return;
    const int m = (int)(t % A.M);
    const int k = A.gkconv[A.mgroup[m]];
    if (k >= 0) Y[t] = DIAG[k * blk + t];
}

// ---------------------------------------------------------------- set-up
struct RcPtrs {
    const double *p[kMaxLevels];
};

__global__ void bsm_members_kernel(int ng, const int *gbase, const int *gslot0, const int *member,
                                   int M, int *mbody, int *mgroup, RcPtrs rc, int nlev, double *irc) {
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
    for (int l = 0; l < nlev; l++) irc[(size_t)l * M + m] = 1.0 / rc.p[l][b];
}

__global__ void bsm_init_groups_kernel(BsmArgs A) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= A.ng) return;
    A.gt[g] = 0.0;
    A.gH[g] = A.dt;
    A.gstat[g] = 0;
    A.gkconv[g] = -1;
    A.gatt[g] = 0;
    A.gacc[g] = 0;
    A.grej[g] = 0;
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

// Device and pinned host buffers of the batch, grown on demand, kept by the system.
struct BsmBuffers {
    void *raw = nullptr;
    size_t bytes = 0;
    int *host_stat = nullptr;
    size_t host_cap = 0;
};

void *bsm_reserve(genga_system *s, size_t bytes, int ng) {
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
    if (b->host_cap < (size_t)ng) {
        if (b->host_stat) cudaFreeHost(b->host_stat);
        b->host_stat = nullptr;
        b->host_cap = 0;
        if (cudaMallocHost(&b->host_stat, sizeof(int) * (size_t)ng) != cudaSuccess) return nullptr;
        b->host_cap = (size_t)ng;
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
    if ((int)c.max_group <= kBlockGroupMax || c.ngroups == 0) return 0;
    std::vector<int> glist(c.ngroups), goff((size_t)s->n + 1);
    if (cudaMemcpyAsync(glist.data(), s->glist, sizeof(int) * c.ngroups, cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(goff.data(), s->goff, sizeof(int) * goff.size(), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return -1;
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
    std::vector<int> gbase(ng), gslot0(ng);
    int M = 0;
    for (int g = 0; g < ng; g++) {
        gbase[g] = M;
        gslot0[g] = groups[g].x;
        M += groups[g].y;
    }
    const size_t blk = (size_t)D * M;
    const size_t bytes = aligned(sizeof(double) * blk) * 3 + aligned(sizeof(double) * 8 * blk) * 5 +
                         aligned(sizeof(double) * (size_t)(level + 1) * M) +
                         aligned(sizeof(int) * M) * 2 + aligned(sizeof(int) * ng) * 4 +
                         aligned(sizeof(double) * ng) * 2 + aligned(sizeof(long long) * ng) * 3 +
                         aligned(sizeof(unsigned long long) * 8 * (size_t)ng);
    char *p = static_cast<char *>(bsm_reserve(s, bytes, ng));
    if (!p) return GENGA_ENOMEM;
    int *host_stat = static_cast<BsmBuffers *>(s->bsm)->host_stat;
    double *Y = carve<double>(p, blk), *F0 = carve<double>(p, blk), *SC = carve<double>(p, blk);
    double *ZM = carve<double>(p, 8 * blk), *ZA = carve<double>(p, 8 * blk), *ZB = carve<double>(p, 8 * blk);
    double *OUT = carve<double>(p, 8 * blk), *DIAG = carve<double>(p, 8 * blk);
    double *irc = carve<double>(p, (size_t)(level + 1) * M);
    int *mbody = carve<int>(p, M), *mgroup = carve<int>(p, M);
    int *d_gbase = carve<int>(p, ng), *d_gslot0 = carve<int>(p, ng);
    BsmArgs A;
    A.gstat = carve<int>(p, ng);
    A.gkconv = carve<int>(p, ng);
    A.gt = carve<double>(p, ng);
    A.gH = carve<double>(p, ng);
    A.gatt = carve<long long>(p, ng);
    A.gacc = carve<long long>(p, ng);
    A.grej = carve<long long>(p, ng);
    A.gerr = carve<unsigned long long>(p, 8 * (size_t)ng);
    A.n = (int)s->n; A.M = M; A.ng = ng;
    A.mbody = mbody; A.mgroup = mgroup; A.irc = irc; A.gbase = d_gbase; A.gslot0 = d_gslot0;
    A.slotof = s->slotof;
    A.off = s->csr[level].off; A.list = s->csr[level].list;
    A.mass = s->mass;
    A.nlev = level + 1;
    A.G = s->p.G; A.mu = s->p.G * s->p.m_star; A.dt = dt; A.tol = s->p.bs_tol;
    A.max_steps = s->p.bs_max_steps;

    cudaStream_t st = s->stream;
    if (cudaMemcpyAsync(d_gbase, gbase.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_gslot0, gslot0.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GENGA_ECUDA;
    const unsigned gm = (unsigned)((M + kMThreads - 1) / kMThreads);
    const unsigned g8 = (unsigned)((8LL * M + kMThreads - 1) / kMThreads);
    const unsigned gD = (unsigned)(((long long)D * M + kMThreads - 1) / kMThreads);
    const unsigned gg = (unsigned)((ng + 127) / 128);
    RcPtrs rcp;
    for (int l = 0; l < kMaxLevels; l++) rcp.p[l] = s->rcl[l].rc;
    bsm_members_kernel<<<gm, kMThreads, 0, st>>>(ng, d_gbase, d_gslot0, s->member, M, mbody, mgroup, rcp,
                                                 level + 1, irc);
    bsm_init_groups_kernel<<<gg, 128, 0, st>>>(A);
    gather(st, A, Y);
    s->launches += 3;
    if (cudaGetLastError() != cudaSuccess) return GENGA_ECUDA;

    // rounds in batches (4, 8, ..., 64) between reads of the status words;
    // the host copies go through pinned memory and the synchronisation
    long long rounds = 0;
    int batch = 4;
    bool running = true;
    while (running) {
        for (int r = 0; r < batch; r++) {
            bsm_start_kernel<Ode><<<gm, kMThreads, 0, st>>>(A, Y, F0, SC, ZM, ZA);
            double *cur = ZA, *nxt = ZB;
            for (int it = 1; it <= 16; it++) {
                bsm_substep_kernel<Ode><<<g8, kMThreads, 0, st>>>(A, cur, nxt, ZM, OUT, it);
                std::swap(cur, nxt);
            }
            bsm_neville_kernel<Ode><<<gD, kMThreads, 0, st>>>(A, OUT, SC, DIAG);
            bsm_decide_kernel<<<gg, 128, 0, st>>>(A);
            bsm_accept_kernel<Ode><<<gD, kMThreads, 0, st>>>(A, DIAG, Y);
            s->launches += 20;
        }
        rounds += batch;
        if (cudaGetLastError() != cudaSuccess) return GENGA_ECUDA;
        if (cudaMemcpyAsync(host_stat, A.gstat, sizeof(int) * ng, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return GENGA_ECUDA;
        running = false;
        for (int g = 0; g < ng; g++) running = running || host_stat[g] == 0;
        // each round is one attempt of every running group, and a group stops
        // after bs_max_steps attempts: more rounds than that cannot happen
        if (running && rounds > (long long)A.max_steps) return GENGA_ENONCONV;
        batch = std::min(batch * 2, 64);
    }
    scatter(st, A, Y);
    bsm_stats_kernel<<<1, 1, 0, st>>>(A, s->ctr, count_steps ? 1 : 0);
    s->launches += 2;
    return cudaGetLastError() == cudaSuccess ? GENGA_OK : GENGA_ECUDA;
}

}  // namespace

void bsm_release(genga_system *s) {
    BsmBuffers *b = static_cast<BsmBuffers *>(s->bsm);
    if (!b) return;
    if (b->raw) cudaFree(b->raw);
    if (b->host_stat) cudaFreeHost(b->host_stat);
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
    return bsm_run<FwdOde>(
        s, level, dt_l, groups, true,
        [&](cudaStream_t st, const BsmArgs &A, double *Y) {
            bsm_gather_fwd<<<(A.M + 127) / 128, 128, 0, st>>>(n, A.M, A.mbody, pre_pos, pre_vel, Y);
        },
        [&](cudaStream_t st, const BsmArgs &A, const double *Y) {
            bsm_scatter_fwd<<<(A.M + 127) / 128, 128, 0, st>>>(n, A.M, A.mbody, Y, pos, vel);
        });
}

// Bulirsch-Stoer of every group of the current grouping at `level`: the
// in-block kernels for groups of up to kBlockGroupMax members and the
// batched grid-wide driver for the larger ones, concurrently.
int run_bs(genga_system *s, int level, double dt_l, int64_t np) {
    if (np <= 0) return GENGA_OK;
    if (launch_bs(s, level, dt_l, std::min<int64_t>(np, s->n / 2 + 1)) != cudaSuccess) {
        join_bs(s);
        return GENGA_ECUDA;
    }
    // the batched groups run on the system stream while the side streams
    // integrate the small groups (disjoint members)
    const int rc = bsm_forward_groups(s, level, dt_l);
    if (join_bs(s) != cudaSuccess) return GENGA_ECUDA;
    return rc;
}

// Adjoint BS (backward, augmented) of every group larger than kBlockGroupMax.
int bsm_adjoint_groups(genga_system *s, const double *x2, const double *v2, double *lx, double *lv,
                       double *lm, double dt) {
    std::vector<int2> groups;
    if (batched_groups(s, groups) != 0) return GENGA_ECUDA;
    if (groups.empty()) return GENGA_OK;
    const int n = (int)s->n;
    return bsm_run<AdjOde>(
        s, 0, dt, groups, false,
        [&](cudaStream_t st, const BsmArgs &A, double *Y) {
            bsm_gather_adj<<<(A.M + 127) / 128, 128, 0, st>>>(n, A.M, A.mbody, x2, v2, lx, lv, Y);
        },
        [&](cudaStream_t st, const BsmArgs &A, const double *Y) {
            bsm_scatter_adj<<<(A.M + 127) / 128, 128, 0, st>>>(n, A.M, A.mbody, Y, lx, lv, lm);
        });
}

}  // namespace genga
