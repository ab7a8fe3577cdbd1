// collide.cu -- collisions (Sec. 7.1-7.2) on the host side: switching them
// on, the merger log, the alive flags, and taking merged-away bodies out.
// The mergers themselves happen inside the Bulirsch-Stoer kernels (bs.cu for
// groups of up to 32 members, bsm.cu for larger ones) through merge_bodies
// (common.cuh); each writes one record to a device log.  Records carry the
// Bulirsch-Stoer call, the group label and the merger's sequence number in its
// group, so the host restores the order of the integration -- calls in time
// order, groups by ascending label, each group's mergers in time order -- and
// sums the collision energy in that order, whatever order the concurrent
// groups wrote their records in.
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace genga {

CollArgs coll_args(const genga_system *s) {
    CollArgs c;
    memset(&c, 0, sizeof(c));
    if (!s->coll_on) return c;
    c.on = 1;
    c.tol = s->coll_tol;
    c.mass = const_cast<double *>(s->mass);
    c.radius = s->radius;
    c.spin = s->spin;
    c.alive = s->alive;
    c.log = s->mlog;
    c.log_cap = (unsigned long long)s->mlog_cap;
    c.call = s->bs_call;
    c.G = s->p.G;
    c.n = s->n;
    return c;
}

namespace {

int cfail(genga_system *s, int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->err, sizeof(s->err), fmt, ap);
    va_end(ap);
    return code;
}

#define CCU(expr)                                                                          \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return cfail(s, e__ == cudaErrorMemoryAllocation ? GENGA_ENOMEM : GENGA_ECUDA, \
                         "%s: %s", #expr, cudaGetErrorString(e__));                        \
    } while (0)

__global__ void alive_flags_kernel(int n, const unsigned char *alive, int *flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = alive[i] ? 1 : 0;
}

// dst[c * n_new + slot[i]] = src[c * n_old + i] for the alive bodies i.
__global__ void compact_gather_kernel(int n_old, int n_new, int ncomp, const int *slot,
                                      const unsigned char *alive, const double *src, double *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_old || !alive[i]) return;
    for (int c = 0; c < ncomp; c++) dst[(size_t)c * n_new + slot[i]] = src[(size_t)c * n_old + i];
}

__global__ void compact_index_kernel(int n_old, const int *slot, const unsigned char *alive, int *old_index) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_old && alive[i]) old_index[slot[i]] = i;
}

}  // namespace
}  // namespace genga

using namespace genga;

extern "C" {

int genga_set_collisions(genga_system_t *s, double *mass, double *radius, double *spin, double precision) {
    if (!s) return GENGA_EINVAL;
    if (mass != s->mass) return cfail(s, GENGA_EINVAL, "mass must be the system's mass array");
    if (!radius || !spin) return cfail(s, GENGA_EINVAL, "radius and spin are required");
    if (!(precision >= 0.0)) return cfail(s, GENGA_EINVAL, "collision precision must be >= 0");
    const size_t n = (size_t)s->n;
    CCU(cudaStreamSynchronize(s->stream));
    if (!s->alive) CCU(cudaMalloc((void **)&s->alive, n));
    if (!s->mlog) {
        s->mlog_cap = std::max<int64_t>(4096, s->n);
        CCU(cudaMalloc((void **)&s->mlog, sizeof(double) * kMergeRec * (size_t)s->mlog_cap));
    }
    CCU(cudaMemset(s->alive, 1, n));
    CCU(cudaMemset(&s->ctr->merge_count, 0, sizeof(unsigned long long)));
    s->radius = radius;
    s->spin = spin;
    s->coll_tol = precision;
    s->coll_on = true;
    s->bs_call = 0;
    return GENGA_OK;
}

int genga_get_mergers(genga_system_t *s, double *log, int64_t cap, int64_t *n, double *dU) {
    if (!s) return GENGA_EINVAL;
    if (n) *n = 0;
    if (dU) *dU = 0.0;
    if (!s->coll_on) return GENGA_OK;
    unsigned long long cnt = 0;
    CCU(cudaMemcpyAsync(&cnt, &s->ctr->merge_count, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream));
    CCU(cudaStreamSynchronize(s->stream));
    const int64_t k = (int64_t)std::min<unsigned long long>(cnt, (unsigned long long)s->mlog_cap);
    if (n) *n = k;
    if (log && cap < k) return cfail(s, GENGA_ECAPACITY, "merger log: %lld records", (long long)k);
    std::vector<double> h((size_t)k * kMergeRec);
    if (k) CCU(cudaMemcpy(h.data(), s->mlog, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> order((size_t)k);
    for (int64_t q = 0; q < k; q++) order[(size_t)q] = q;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const double *x = &h[(size_t)a * kMergeRec], *y = &h[(size_t)b * kMergeRec];
        for (int c = 0; c < 3; c++)     // call, group label, sequence in the group
            if (x[c] != y[c]) return x[c] < y[c];
        return false;
    });
    double sum = 0.0;
    for (int64_t q = 0; q < k; q++) {
        const double *e = &h[(size_t)order[(size_t)q] * kMergeRec];
        if (log)
            for (int c = 0; c < 6; c++) log[(size_t)q * 6 + c] = e[3 + c];
        sum += e[8];
    }
    if (dU) *dU = sum;
    if (!log) return GENGA_OK;            // a size query keeps the log
    CCU(cudaMemsetAsync(&s->ctr->merge_count, 0, sizeof(unsigned long long), s->stream));
    CCU(cudaStreamSynchronize(s->stream));
    if (cnt > (unsigned long long)s->mlog_cap)
        return cfail(s, GENGA_ECAPACITY, "merger log overflowed: %llu mergers, %lld kept", cnt,
                     (long long)s->mlog_cap);
    return GENGA_OK;
}

int genga_get_alive(genga_system_t *s, uint8_t *alive) {
    if (!s || !alive) return GENGA_EINVAL;
    if (!s->coll_on) {
        memset(alive, 1, (size_t)s->n);
        return GENGA_OK;
    }
    CCU(cudaMemcpyAsync(alive, s->alive, (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    CCU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

int genga_remove_merged(genga_system_t *s, int64_t *n_new_out, int64_t *old_index) {
    if (!s || !s->coll_on) return GENGA_EINVAL;
    const int n_old = (int)s->n;
    const unsigned grid = (unsigned)((n_old + 255) / 256);
    int *slot = s->gfill;                 // n + 1 ints: exclusive scan of the alive flags
    alive_flags_kernel<<<grid, 256, 0, s->stream>>>(n_old, s->alive, s->flags);
    CCU(cudaGetLastError());
    CCU(exclusive_scan(s, s->flags, slot, n_old));
    int n_new = 0, nm_keep = 0;
    CCU(cudaMemcpyAsync(&n_new, slot + n_old, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    const int64_t nm = s->p.tp_mode == 2 ? std::min<int64_t>(std::max<int64_t>(s->p.n_massive, 0), n_old) : 0;
    if (s->p.tp_mode == 2)
        CCU(cudaMemcpyAsync(&nm_keep, slot + nm, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CCU(cudaStreamSynchronize(s->stream));
    if (n_new_out) *n_new_out = n_new;
    if (n_new == n_old) return GENGA_OK;
    if (n_new < 1) return cfail(s, GENGA_EINVAL, "no alive body left");
    double *tmp = nullptr;
    CCU(cudaMalloc((void **)&tmp, sizeof(double) * 3 * (size_t)n_new));
    struct Arr { double *p; int ncomp; };
    const Arr arrs[] = {{s->pos, 3}, {s->vel, 3}, {const_cast<double *>(s->mass), 1}, {s->radius, 1},
                        {s->spin, 3}};
    for (const Arr &a : arrs) {
        compact_gather_kernel<<<grid, 256, 0, s->stream>>>(n_old, n_new, a.ncomp, slot, s->alive, a.p, tmp);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(a.p, tmp, sizeof(double) * a.ncomp * (size_t)n_new, cudaMemcpyDeviceToDevice,
                                s->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cfail(s, GENGA_ECUDA, "compaction: %s", cudaGetErrorString(e));
        }
    }
    if (old_index) {
        int *idx = s->member;             // n + 1 ints, rewritten by the next grouping
        compact_index_kernel<<<grid, 256, 0, s->stream>>>(n_old, slot, s->alive, idx);
        std::vector<int> h((size_t)n_new);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data(), idx, sizeof(int) * (size_t)n_new, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cfail(s, GENGA_ECUDA, "compaction index: %s", cudaGetErrorString(e));
        }
        for (int q = 0; q < n_new; q++) old_index[q] = h[(size_t)q];
    }
    CCU(cudaStreamSynchronize(s->stream));
    cudaFree(tmp);
    // the system now holds n_new bodies; arrays sized for more stay in use
    s->n = n_new;
    if (s->p.tp_mode == 2) s->p.n_massive = nm_keep;
    CCU(cudaMemsetAsync(s->alive, 1, (size_t)n_new, s->stream));
    s->kick_chunk = 0;                    // kick geometry and buffers redone for the new count
    s->ksym_n = -1;
    CCU(kick_reserve(s));
    for (int l = 0; l < kMaxLevels; l++) s->npairs_host[l] = 0;
    s->label_level = -1;
    adjoint_free(s);                      // a recording refers to the old indices
    CCU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

}  // extern "C"
