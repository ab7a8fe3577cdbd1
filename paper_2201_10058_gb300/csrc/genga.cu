// genga.cu -- host side of the C ABI declared in include/genga.h: the system
// object, its device scratch, and the driver of one step of Appendix A
//   Rcrit(dt); Kick(dt/2) + pre-check; HC(dt/2); FG(dt);
//   detection; grouping + Bulirsch-Stoer(dt)   (or SEnc for slevels > 1);
//   HC(dt/2); Kick(dt/2)
// with the SEnc recursion of Appendix A for the higher-level changeover
// scheme (Sec. 6.3).  Every arithmetic step runs in the kernels of kick.cu,
// particle.cu, encounter.cu and bs.cu; the host only orders launches, reads
// pair counts to size the next launch, and grows capacities on overflow.
#include <algorithm>
#include <cstdarg>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

using namespace genga;

namespace {

int fail(genga_system *s, int code, const char *fmt, ...) {
    if (s) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->err, sizeof(s->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CU(expr)                                                                        \
    do {                                                                                \
        cudaError_t e__ = (expr);                                                       \
        if (e__ != cudaSuccess)                                                         \
            return fail(s, e__ == cudaErrorMemoryAllocation ? GENGA_ENOMEM : GENGA_ECUDA, \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, __LINE__); \
    } while (0)

#define TRY(expr)                    \
    do {                             \
        int r__ = (expr);            \
        if (r__ != GENGA_OK) return r__; \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// ---------------------------------------------------------------- phase timing
// From this point of the stream on, device time counts for `phase`.
int mark(genga_system *s, int phase) {
    if (!s->timing) return GENGA_OK;
    if (s->nmarks == s->mark_ev.size()) {
        cudaEvent_t e = nullptr;
        CU(cudaEventCreate(&e));
        s->mark_ev.push_back(e);
        s->mark_phase.push_back(-1);
    }
    CU(cudaEventRecord(s->mark_ev[s->nmarks], s->stream));
    s->mark_phase[s->nmarks] = phase;
    s->nmarks++;
    return GENGA_OK;
}

// Adds the intervals between the recorded marks to the phase sums (waits for
// the last mark); the last mark closes the step.
int fold_marks(genga_system *s) {
    if (!s->timing || s->nmarks == 0) return GENGA_OK;
    CU(cudaEventSynchronize(s->mark_ev[s->nmarks - 1]));
    for (size_t k = 0; k + 1 < s->nmarks; k++) {
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, s->mark_ev[k], s->mark_ev[k + 1]));
        const int ph = s->mark_phase[k];
        if (ph >= 0 && ph < GENGA_NPHASES) s->phase_ms[ph] += (double)ms;
    }
    s->nmarks = 0;
    s->timed_steps++;
    return GENGA_OK;
}

void free_marks(genga_system *s) {
    for (cudaEvent_t e : s->mark_ev) cudaEventDestroy(e);
    s->mark_ev.clear();
    s->mark_phase.clear();
    s->nmarks = 0;
}

int levels_of(const genga_params_t &p) {
    return std::min(std::max(p.slevels, 1), kMaxLevels);
}

int check_params(genga_system *s, const genga_params_t *p) {
    if (!p) return fail(s, GENGA_EINVAL, "params is NULL");
    if (!(p->m_star > 0) || !(p->G > 0)) return fail(s, GENGA_EINVAL, "G and m_star must be > 0");
    if (p->slevels < 1 || p->slevels > kMaxLevels)
        return fail(s, GENGA_EINVAL, "slevels must be in [1, %d]", kMaxLevels);
    if (p->slevels > 1 && p->substeps < 1) return fail(s, GENGA_EINVAL, "substeps must be >= 1");
    if (p->precision != GENGA_FP64 && p->precision != GENGA_MIXED)
        return fail(s, GENGA_EINVAL, "precision must be GENGA_FP64 or GENGA_MIXED");
    if (p->kepler_max_iter < 1 || p->bs_max_steps < 1)
        return fail(s, GENGA_EINVAL, "iteration limits must be >= 1");
    if (!(p->bs_tol > 0)) return fail(s, GENGA_EINVAL, "bs_tol must be > 0");
    if (p->tp_mode != 0 && p->tp_mode != 2)
        return fail(s, GENGA_EINVAL, "tp_mode must be 0 or 2 (mode 1: mode 2 with massless test particles)");
    if (p->tp_mode == 2 && p->n_massive < 0) return fail(s, GENGA_EINVAL, "n_massive must be >= 0");
    return GENGA_OK;
}

int alloc_pairs(genga_system *s, int level, int64_t cap) {
    // partner-list entries (2 per pair) and their directions 2 k + d are ints
    if (cap > (int64_t)0x3fffffff)
        return fail(s, GENGA_ECAPACITY, "level %d: %lld encounter pairs exceed the 2^30 limit", level,
                    (long long)cap);
    dfree(s->pairs[level]);
    dfree(s->csr[level].list);
    dfree(s->csr[level].lpair);
    dfree(s->csr[level].ent);
    dfree(s->csr[level].term);
    CU(dalloc(&s->pairs[level], (size_t)cap));
    CU(dalloc(&s->csr[level].list, 2 * (size_t)cap));
    CU(dalloc(&s->csr[level].lpair, 2 * (size_t)cap));
    CU(dalloc(&s->csr[level].ent, 2 * (size_t)cap));
    CU(dalloc(&s->csr[level].term, 8 * (size_t)cap));
    s->pair_cap[level] = cap;
    s->csr[level].cap = cap;
    return GENGA_OK;
}

// Every per-level array of level l; what already exists is kept (a level
// dropped by genga_set_params and taken up again reuses its arrays).
int alloc_level(genga_system *s, int l) {
    const size_t n = (size_t)s->n;
    if (!s->rcl[l].rc) {
        CU(dalloc(&s->rcl[l].rc, n));
        CU(cudaMemset(s->rcl[l].rc, 0, sizeof(double) * n));
    }
    if (!s->rcl[l].rc2) {
        CU(dalloc(&s->rcl[l].rc2, n));
        CU(cudaMemset(s->rcl[l].rc2, 0, sizeof(double) * n));
    }
    if (!s->rcl[l].irc) {
        CU(dalloc(&s->rcl[l].irc, n));
        CU(cudaMemset(s->rcl[l].irc, 0, sizeof(double) * n));
    }
    if (!s->pre_pos[l]) CU(dalloc(&s->pre_pos[l], 3 * n));
    if (!s->pre_vel[l]) CU(dalloc(&s->pre_vel[l], 3 * n));
    if (!s->csr[l].deg) CU(dalloc(&s->csr[l].deg, n + 1));
    if (!s->csr[l].off) CU(dalloc(&s->csr[l].off, n + 1));
    if (!s->csr[l].fill) CU(dalloc(&s->csr[l].fill, n + 1));
    if (!s->bodies[l]) CU(dalloc(&s->bodies[l], n));
    if (!s->pairs[l]) {
        const int64_t pc = s->p.pair_capacity > 0 ? s->p.pair_capacity : std::max<int64_t>(1 << 16, 4 * (int64_t)n);
        TRY(alloc_pairs(s, l, pc));
    }
    return GENGA_OK;
}

int alloc_all(genga_system *s) {
    const size_t n = (size_t)s->n;
    CU(dalloc(&s->ctr, 1));
    CU(cudaMemset(s->ctr, 0, sizeof(DevCounters)));
    for (int l = 0; l < levels_of(s->p); l++) TRY(alloc_level(s, l));
    CU(dalloc(&s->rcl[0].pc2, n));
    CU(dalloc(&s->rcl[0].thr_rc, n));
    for (int k = 0; k < 4; k++) {
        CU(cudaStreamCreateWithFlags(&s->side[k], cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&s->ev_join[k], cudaEventDisableTiming));
    }
    CU(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&s->ev_counts, cudaEventDisableTiming));
    CU(cudaMallocHost((void **)&s->bucket_host, sizeof(unsigned) * kBuckets));
    CU(cudaMallocHost((void **)&s->np_host, sizeof(unsigned long long) * kMaxLevels));
    for (int l = 0; l < kMaxLevels; l++) s->np_host[l] = 0;
    s->kick_chunk = 0;
    CU(kick_reserve(s));
    s->cand_cap = s->p.cand_capacity > 0 ? s->p.cand_capacity : std::max<int64_t>(1 << 20, 64 * (int64_t)n);
    CU(dalloc(&s->cand, (size_t)s->cand_cap));
    CU(dalloc(&s->flags, n + 1));
    CU(dalloc(&s->parent, n));
    CU(dalloc(&s->label, n));
    CU(dalloc(&s->gsize, n + 1));
    CU(dalloc(&s->goff, n + 1));
    CU(dalloc(&s->gfill, n + 1));
    CU(dalloc(&s->glist, n + 1));
    CU(dalloc(&s->member, n + 1));
    CU(dalloc(&s->slotof, n));
    s->bucket_stride = (int)(n / 2 + 1);
    CU(dalloc(&s->bucket_list, (size_t)kBuckets * s->bucket_stride));
    CU(dalloc(&s->red, 9 * n + 16));
    s->scr.scan_blocks_cap = (int)((n + 1 + 4095) / 4096) + 2;
    CU(dalloc(&s->scr.scan_blocks, (size_t)s->scr.scan_blocks_cap));
    return GENGA_OK;
}

void free_all(genga_system *s) {
    dfree(s->ctr);
    for (int l = 0; l < kMaxLevels; l++) {
        dfree(s->rcl[l].rc); dfree(s->rcl[l].rc2); dfree(s->rcl[l].pc2); dfree(s->rcl[l].irc);
        dfree(s->rcl[l].thr_rc);
        dfree(s->pre_pos[l]); dfree(s->pre_vel[l]);
        dfree(s->pairs[l]);
        dfree(s->csr[l].deg); dfree(s->csr[l].off); dfree(s->csr[l].fill); dfree(s->csr[l].list);
        dfree(s->csr[l].lpair); dfree(s->csr[l].ent); dfree(s->csr[l].term);
        dfree(s->bodies[l]);
    }
    dfree(s->kick_part); dfree(s->ksym_list); dfree(s->ksym_ctr); dfree(s->ksym_irc); dfree(s->ksym_mhl); dfree(s->ksym_thrpc); dfree(s->ksym_pcf); dfree(s->ksym_ircf);
    s->kick_part_cap = 0; s->ksym_list_cap = 0; s->ksym_body_cap = 0; s->ksym_n = -1;
    dfree(s->cand); dfree(s->flags); dfree(s->parent); dfree(s->label);
    dfree(s->gsize); dfree(s->goff); dfree(s->gfill); dfree(s->glist); dfree(s->member);
    dfree(s->slotof); dfree(s->bucket_list); bsm_release(s); dfree(s->red); dfree(s->scr.scan_blocks);
    dfree(s->alive); dfree(s->mlog);
    for (int k = 0; k < 4; k++) {
        if (s->side[k]) cudaStreamDestroy(s->side[k]);
        if (s->ev_join[k]) cudaEventDestroy(s->ev_join[k]);
        s->side[k] = nullptr; s->ev_join[k] = nullptr;
    }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    s->ev_fork = nullptr;
    if (s->ev_counts) cudaEventDestroy(s->ev_counts);
    s->ev_counts = nullptr;
    if (s->bucket_host) cudaFreeHost(s->bucket_host);
    s->bucket_host = nullptr;
    if (s->np_host) cudaFreeHost(s->np_host);
    s->np_host = nullptr;
    free_marks(s);
}

template <typename T>
int read_dev(genga_system *s, T *host, const T *dev) {
    CU(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    ++s->host_syncs;
    return GENGA_OK;
}

int device_errors(genga_system *s) {
    unsigned err = 0;
    TRY(read_dev(s, &err, &s->ctr->err));
    if (!err) return GENGA_OK;
    CU(cudaMemsetAsync(&s->ctr->err, 0, sizeof(unsigned), s->stream));
    if (err & kErrBadState) return fail(s, GENGA_EBADSTATE, "non-finite state or body at the origin");
    if (err & kErrKepler) return fail(s, GENGA_ENONCONV, "Kepler solve hit kepler_max_iter");
    if (err & kErrTimeout)
        return fail(s, GENGA_ETIMEOUT, "Bulirsch-Stoer: a group call exceeded its time limit of %.3g s",
                    1e-9 * (double)s->bs_group_limit_ns);
    if (err & kErrBS) return fail(s, GENGA_ENONCONV, "Bulirsch-Stoer hit bs_max_steps");
    if (err & kErrUnionFind) return fail(s, GENGA_ETIMEOUT, "grouping retry limit reached");
    if (err & kErrMergeLog)
        return fail(s, GENGA_ECAPACITY, "merger log full (%lld records): read it with genga_get_mergers",
                    (long long)s->mlog_cap);
    return fail(s, GENGA_ECAPACITY, "capacity exceeded (error word 0x%x)", err);
}

// Stops a step before the encounter phase when the state is already bad.
int early_errors(genga_system *s) {
    unsigned err = 0;
    TRY(read_dev(s, &err, &s->ctr->err));
    if (err & (kErrBadState | kErrKepler)) return device_errors(s);
    return GENGA_OK;
}

// ---------------------------------------------------------------- step pieces
int kick(genga_system *s, double dt_half, bool precheck, double *acc_out) {
    CU(launch_kick(s, dt_half, precheck, acc_out));
    return GENGA_OK;
}

// Candidate count after a pre-check kick; regrows and recomputes on overflow
// (the positions must still be those of the pre-check).
int settle_candidates(genga_system *s, int64_t *ncand) {
    unsigned long long c = 0;
    TRY(read_dev(s, &c, &s->ctr->cand_count));
    if ((int64_t)c > s->cand_cap) {
        dfree(s->cand);
        s->cand_cap = (int64_t)(c + c / 2 + 1024);
        CU(dalloc(&s->cand, (size_t)s->cand_cap));
        CU(launch_precheck_only(s));
        TRY(read_dev(s, &c, &s->ctr->cand_count));
        if ((int64_t)c > s->cand_cap) return fail(s, GENGA_ECAPACITY, "candidate list overflow");
    }
    *ncand = (int64_t)c;
    return GENGA_OK;
}

// Detection at `level` over `in`; regrows the level list on overflow.
int detect(genga_system *s, const uint2 *in, int64_t nin, int level, int64_t *np) {
    unsigned long long c = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        CU(launch_detect(s, in, nin, level, s->pairs[level], s->pair_cap[level], &s->ctr->pair_count[level]));
        TRY(read_dev(s, &c, &s->ctr->pair_count[level]));
        if ((int64_t)c <= s->pair_cap[level]) break;
        TRY(alloc_pairs(s, level, (int64_t)(c + c / 2 + 1024)));
    }
    if ((int64_t)c > s->pair_cap[level]) return fail(s, GENGA_ECAPACITY, "pair list overflow");
    *np = (int64_t)c;
    s->npairs_host[level] = *np;
    if (s->pair_log) {
        std::vector<uint2> h((size_t)c);
        if (c) {
            CU(cudaMemcpyAsync(h.data(), s->pairs[level], sizeof(uint2) * (size_t)c, cudaMemcpyDeviceToHost,
                               s->stream));
            CU(cudaStreamSynchronize(s->stream));
        }
        std::sort(h.begin(), h.end(), [](const uint2 &a, const uint2 &b) {
            return a.x < b.x || (a.x == b.x && a.y < b.y);
        });
        if (s->log_off.empty()) s->log_off.push_back(0);
        s->log_level.push_back(level);
        for (const uint2 &q : h) { s->log_pairs.push_back(q.x); s->log_pairs.push_back(q.y); }
        s->log_off.push_back((int64_t)(s->log_pairs.size() / 2));
    }
    return GENGA_OK;
}

// Detection at `level` over `in` with the pair count left on the device: the
// level's list is first made as large as the input (the pairs found are a
// subset of it), so it cannot overflow and the host need not read the count.
int detect_dev(genga_system *s, const uint2 *in, int64_t nin, int level) {
    if (s->pair_cap[level] < nin) TRY(alloc_pairs(s, level, nin + nin / 2 + 1024));
    CU(launch_detect(s, in, nin, level, s->pairs[level], s->pair_cap[level], &s->ctr->pair_count[level]));
    s->npairs_host[level] = -1;          // the count is on the device only
    // a copy for the host, read once a later wait has passed it (it picks
    // the next partner-list sort; nothing else depends on it)
    CU(cudaMemcpyAsync(&s->np_host[level], &s->ctr->pair_count[level], sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s->stream));
    return GENGA_OK;
}

int bs_groups(genga_system *s, int level, int64_t np, double dt_l) {
    TRY(mark(s, GENGA_PH_GROUPING));
    CU(build_groups(s, level, np));
    return run_bs(s, level, dt_l, np);
}

int senc(genga_system *s, int level, double dt_l) {
    const int L = levels_of(s->p);
    int nb = 0;
    TRY(mark(s, GENGA_PH_LEVELSETUP));
    CU(build_bodies(s, level - 1, level, &nb));
    CU(launch_restore(s, level - 1, s->bodies[level], nb));
    for (int sub = 0; sub < s->p.substeps; sub++) {
        TRY(mark(s, GENGA_PH_RCRITS));
        CU(launch_rcrit(s, level, dt_l, s->bodies[level], nb));
        TRY(mark(s, GENGA_PH_KICKS));
        CU(launch_kick_pairs(s, level, 0.5 * dt_l, nb));
        TRY(mark(s, GENGA_PH_FGS));
        CU(launch_drift(s, level, dt_l, s->bodies[level], nb));
        int64_t np = 0;
        TRY(mark(s, GENGA_PH_DETECTS));
        if (level == L - 1 && !s->pair_log) {
            // the deepest level: detection, partner lists, groups and BS take
            // the pair count from the device (grids sized by the input count),
            // so the host queues the sub-step without waiting for the GPU
            const int64_t bound = s->npairs_host[level - 1];
            const unsigned long long *npd = &s->ctr->pair_count[level];
            // the previous sub-step's count (its copy was passed by the wait
            // in that sub-step's run_bs_dev)
            const int64_t hint = (int64_t)s->np_host[level];
            TRY(detect_dev(s, s->pairs[level - 1], bound, level));
            TRY(mark(s, GENGA_PH_CSRS));
            CU(build_csr(s, level, bound, npd, &s->ctr->pair_total[level], hint));
            TRY(mark(s, GENGA_PH_GROUPING));
            CU(build_groups(s, level, bound, npd));
            TRY(run_bs_dev(s, level, dt_l));
        } else {
            TRY(detect(s, s->pairs[level - 1], s->npairs_host[level - 1], level, &np));
            s->stats.n_pairs[level] += np;
            if (np > 0) {
                TRY(mark(s, GENGA_PH_CSRS));
                CU(build_csr(s, level, np));
                if (level < L - 1) TRY(senc(s, level + 1, dt_l / s->p.substeps));
                else TRY(bs_groups(s, level, np, dt_l));
            }
        }
        TRY(mark(s, GENGA_PH_KICKS));
        CU(launch_kick_pairs(s, level, 0.5 * dt_l, nb));
    }
    return GENGA_OK;
}

int one_step(genga_system *s) {
    const double dt = s->p.dt;
    const int n = (int)s->n;
    const int L = levels_of(s->p);
    TRY(mark(s, GENGA_PH_RCRIT));
    CU(launch_rcrit(s, 0, dt, nullptr, n));
    TRY(mark(s, GENGA_PH_KICK1));
    TRY(kick(s, 0.5 * dt, true, nullptr));
    // the candidate count before HC and the drift move the bodies: a list
    // that overflowed is recomputed from the positions the pre-check saw
    int64_t ncand = 0;
    TRY(mark(s, GENGA_PH_CANDCOUNT));
    TRY(settle_candidates(s, &ncand));
    TRY(mark(s, GENGA_PH_HC_DRIFT));
    CU(launch_hc(s, 0.5 * dt));
    CU(launch_drift(s, 0, dt, nullptr, n));
    s->stats.n_candidates += ncand;
    TRY(early_errors(s));
    s->npairs_host[0] = 0;
    if (ncand > 0) {
        int64_t np = 0;
        TRY(mark(s, GENGA_PH_DETECT0));
        TRY(detect(s, s->cand, ncand, 0, &np));
        s->stats.n_pairs[0] += np;
        if (np > 0) {
            TRY(mark(s, GENGA_PH_CSR0));
            CU(build_csr(s, 0, np));
            if (L > 1) TRY(senc(s, 1, dt / s->p.substeps));
            else TRY(bs_groups(s, 0, np, dt));
        }
    }
    TRY(mark(s, GENGA_PH_HC2));
    CU(launch_hc(s, 0.5 * dt));
    TRY(mark(s, GENGA_PH_KICK2));
    TRY(kick(s, 0.5 * dt, false, nullptr));
    TRY(mark(s, -1));
    return fold_marks(s);
}

int collect_stats(genga_system *s) {
    DevCounters c;
    CU(cudaMemcpyAsync(&c, s->ctr, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    s->stats.n_groups = (int64_t)c.groups_total;
    s->stats.max_group = (int64_t)c.max_group_total;
    s->stats.bs_steps = (int64_t)c.bs_steps;
    s->stats.bs_max_attempts = (int64_t)c.bs_max_attempts;
    s->stats.bs_rejects = (int64_t)c.bs_rejects;
    s->stats.bs_fail = (int64_t)c.bs_fail;
    s->stats.kepler_fail = (int64_t)c.kepler_fail;
    for (int l = 0; l < kMaxLevels; l++) s->stats.n_pairs[l] += (int64_t)c.pair_total[l];
    s->stats.kernel_launches = s->launches;
    s->stats.host_syncs = s->host_syncs;
    return GENGA_OK;
}

int reset_stats(genga_system *s) {
    memset(&s->stats, 0, sizeof(s->stats));
    s->launches = 0;
    s->host_syncs = 0;
    // kepler_fail .. bs_max_attempts and pair_total (contiguous)
    CU(cudaMemsetAsync(&s->ctr->kepler_fail, 0, (7 + kMaxLevels) * sizeof(unsigned long long), s->stream));
    return GENGA_OK;
}

int copy_pairs_sorted(genga_system *s, const uint2 *dev, int64_t count, uint32_t *ij, int64_t cap,
                      int64_t *n_out) {
    if (n_out) *n_out = count;
    if (!ij || count == 0) return GENGA_OK;
    std::vector<uint2> h((size_t)count);
    CU(cudaMemcpyAsync(h.data(), dev, sizeof(uint2) * (size_t)count, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    std::sort(h.begin(), h.end(), [](const uint2 &a, const uint2 &b) {
        return a.x < b.x || (a.x == b.x && a.y < b.y);
    });
    const int64_t m = std::min(cap, count);
    for (int64_t k = 0; k < m; k++) { ij[2 * k] = h[k].x; ij[2 * k + 1] = h[k].y; }
    return GENGA_OK;
}

}  // namespace

namespace genga {
int phase_mark(genga_system *s, int phase) { return mark(s, phase); }

int ensure_pair_capacity(genga_system *s, int level, int64_t np) {
    if (np <= s->pair_cap[level]) return GENGA_OK;
    return alloc_pairs(s, level, np + np / 2 + 1024);
}
}  // namespace genga

// ============================================================== public ABI
extern "C" {

void genga_default_params(genga_params_t *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->G = 0.01720209895 * 0.01720209895;
    p->m_star = 1.0;
    p->dt = 6.0875;
    p->n1 = 3.0;
    p->n2 = 0.4;
    p->f_pc = 4.0;
    p->bs_tol = 1e-13;
    p->slevels = 1;
    p->substeps = 1;
    p->precision = GENGA_FP64;
    p->kepler_max_iter = 50;
    p->bs_max_steps = 100000;
}

int genga_create(genga_system_t **out, const genga_params_t *p, int64_t n, double *pos, double *vel,
                 const double *mass, void *stream) {
    if (!out) return GENGA_EINVAL;
    *out = nullptr;
    if (n < 1 || n > (int64_t)1 << 30 || !pos || !vel || !mass) return GENGA_EINVAL;
    genga_system *s = new (std::nothrow) genga_system();
    if (!s) return GENGA_ENOMEM;
    int rc = check_params(s, p);
    if (rc != GENGA_OK) { delete s; return rc; }
    s->p = *p;
    s->n = n;
    s->pos = pos; s->vel = vel; s->mass = mass;
    s->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        delete s;
        return GENGA_ECUDA;
    }
    rc = alloc_all(s);
    if (rc != GENGA_OK) { free_all(s); delete s; return rc; }
    *out = s;
    return GENGA_OK;
}

int genga_init_system(genga_system_t **out, const genga_params_t *p, int64_t n, double *pos, double *vel,
                      const double *mass, void *stream) {
    return genga_create(out, p, n, pos, vel, mass, stream);
}

void genga_destroy(genga_system_t *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    adjoint_free(s);
    free_all(s);
    delete s;
}

const char *genga_last_error(const genga_system_t *s) { return s ? s->err : "null system"; }

int genga_set_params(genga_system_t *s, const genga_params_t *p) {
    if (!s) return GENGA_EINVAL;
    TRY(check_params(s, p));
    for (int l = 0; l < levels_of(*p); l++) TRY(alloc_level(s, l));   // levels not yet held
    s->p = *p;
    return GENGA_OK;
}

int genga_sync(genga_system_t *s) {
    if (!s) return GENGA_EINVAL;
    CU(cudaStreamSynchronize(s->stream));
    return device_errors(s);
}

int genga_rcrit(genga_system_t *s, double dt) {
    if (!s) return GENGA_EINVAL;
    CU(launch_rcrit(s, 0, dt, nullptr, (int)s->n));
    return GENGA_OK;
}

int genga_set_rcrit(genga_system_t *s, const double *rc_host) {
    if (!s || !rc_host) return GENGA_EINVAL;
    CU(cudaMemcpyAsync(s->rcl[0].rc, rc_host, sizeof(double) * (size_t)s->n, cudaMemcpyHostToDevice, s->stream));
    CU(launch_rcrit_derive(s));
    CU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

int genga_kick(genga_system_t *s, double dt_half, int precheck, double *acc_out) {
    if (!s) return GENGA_EINVAL;
    TRY(kick(s, dt_half, precheck != 0, acc_out));
    if (precheck) {
        int64_t nc = 0;
        TRY(settle_candidates(s, &nc));
        s->stats.n_candidates = nc;
    }
    return GENGA_OK;
}

int genga_hc(genga_system_t *s, double dt_half) {
    if (!s) return GENGA_EINVAL;
    CU(launch_hc(s, dt_half));
    return GENGA_OK;
}

int genga_drift(genga_system_t *s, double dt) {
    if (!s) return GENGA_EINVAL;
    CU(launch_drift(s, 0, dt, nullptr, (int)s->n));
    return GENGA_OK;
}

int genga_build_encounters(genga_system_t *s, int64_t *n_pairs, int64_t *n_groups, int64_t *max_group) {
    if (!s) return GENGA_EINVAL;
    int64_t nc = 0, np = 0;
    TRY(read_dev(s, (unsigned long long *)&nc, &s->ctr->cand_count));
    TRY(detect(s, s->cand, nc, 0, &np));
    CU(build_csr(s, 0, np));
    CU(build_groups(s, 0, np));
    DevCounters c;
    CU(cudaMemcpyAsync(&c, s->ctr, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    if (n_pairs) *n_pairs = np;
    if (n_groups) *n_groups = c.ngroups;
    if (max_group) *max_group = c.max_group;
    s->stats.n_pairs[0] = np;
    s->stats.n_groups = c.ngroups;
    s->stats.max_group = c.max_group;
    return device_errors(s);
}

int genga_bs(genga_system_t *s, double dt) {
    if (!s) return GENGA_EINVAL;
    TRY(reset_stats(s));
    const int64_t np = s->npairs_host[0];
    if (np > 0) {
        if (s->label_level != 0) CU(build_groups(s, 0, np));
        TRY(run_bs(s, 0, dt, np));
    }
    TRY(collect_stats(s));
    return device_errors(s);
}

int genga_step(genga_system_t *s, int64_t nsteps) {
    if (!s || nsteps < 0) return GENGA_EINVAL;
    TRY(reset_stats(s));
    for (int64_t k = 0; k < nsteps; k++) {
        TRY(one_step(s));
    }
    TRY(collect_stats(s));
    return device_errors(s);
}

int genga_tune_levels(genga_system_t *s, const int32_t *slevels, const int32_t *substeps, int32_t ncand,
                      int64_t trial_steps, int32_t *best_out, double *ms_out) {
    if (!s || !slevels || !substeps || ncand < 1 || trial_steps < 1) return GENGA_EINVAL;
    const genga_params_t p0 = s->p;
    for (int c = 0; c < ncand; c++) {
        genga_params_t q = p0;
        q.slevels = slevels[c];
        q.substeps = substeps[c];
        TRY(check_params(s, &q));
    }
    const size_t n3 = 3 * (size_t)s->n;
    double *save = nullptr;
    CU(dalloc(&save, 2 * n3));
    const genga_stats_t st0 = s->stats;
    const long long l0 = s->launches;
    auto copy_state = [&](bool to_save) -> cudaError_t {
        const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
        const size_t b = sizeof(double) * n3;
        const cudaError_t r = to_save ? cudaMemcpyAsync(save, s->pos, b, k, s->stream)
                                      : cudaMemcpyAsync(s->pos, save, b, k, s->stream);
        if (r != cudaSuccess) return r;
        return to_save ? cudaMemcpyAsync(save + n3, s->vel, b, k, s->stream)
                       : cudaMemcpyAsync(s->vel, save + n3, b, k, s->stream);
    };
    cudaEvent_t a = nullptr, b = nullptr;
    const bool saved = copy_state(true) == cudaSuccess;
    int rc = (saved && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
                 ? GENGA_OK : fail(s, GENGA_ECUDA, "tune: set-up failed");
    int best = 0;
    double best_ms = 0.0;
    for (int c = 0; c < ncand && rc == GENGA_OK; c++) {
        genga_params_t q = p0;
        q.slevels = slevels[c];
        q.substeps = substeps[c];
        rc = genga_set_params(s, &q);
        if (rc == GENGA_OK) rc = one_step(s);                  // untimed: lists grow here
        if (rc == GENGA_OK) rc = device_errors(s);
        if (rc == GENGA_OK && copy_state(false) != cudaSuccess) rc = fail(s, GENGA_ECUDA, "tune: restore");
        if (rc == GENGA_OK && cudaEventRecord(a, s->stream) != cudaSuccess) rc = fail(s, GENGA_ECUDA, "tune: event");
        for (int64_t k = 0; k < trial_steps && rc == GENGA_OK; k++) rc = one_step(s);
        float ms = 0.0f;
        if (rc == GENGA_OK && (cudaEventRecord(b, s->stream) != cudaSuccess ||
                               cudaEventSynchronize(b) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
            rc = fail(s, GENGA_ECUDA, "tune: timing");
        if (rc == GENGA_OK) rc = device_errors(s);
        if (rc == GENGA_OK && copy_state(false) != cudaSuccess) rc = fail(s, GENGA_ECUDA, "tune: restore");
        if (rc != GENGA_OK) break;
        const double per_step = (double)ms / (double)trial_steps;
        if (ms_out) ms_out[c] = per_step;
        if (c == 0 || per_step < best_ms) { best_ms = per_step; best = c; }
    }
    // the state of before the call and the chosen (or, after an error, the previous) setting
    if (saved) copy_state(false);
    cudaStreamSynchronize(s->stream);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    dfree(save);
    genga_params_t q = p0;
    if (rc == GENGA_OK) {
        q.slevels = slevels[best];
        q.substeps = substeps[best];
    }
    const int rs = genga_set_params(s, &q);
    s->stats = st0;
    s->launches = l0;
    if (rc != GENGA_OK) return rc;
    if (rs != GENGA_OK) return rs;
    if (best_out) *best_out = best;
    return GENGA_OK;
}

int genga_step_host(genga_system_t *s, double *pos_host, double *vel_host, int64_t nsteps) {
    if (!s || !pos_host || !vel_host) return GENGA_EINVAL;
    const size_t bytes = sizeof(double) * 3 * (size_t)s->n;
    CU(cudaMemcpyAsync(s->pos, pos_host, bytes, cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemcpyAsync(s->vel, vel_host, bytes, cudaMemcpyHostToDevice, s->stream));
    TRY(genga_step(s, nsteps));
    CU(cudaMemcpyAsync(pos_host, s->pos, bytes, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaMemcpyAsync(vel_host, s->vel, bytes, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

int genga_energy(genga_system_t *s, double *E, double *L) {
    if (!s || !E || !L) return GENGA_EINVAL;
    CU(launch_energy(s, E, L));
    return device_errors(s);
}

int genga_get_candidates(genga_system_t *s, uint32_t *ij, int64_t cap, int64_t *n) {
    if (!s) return GENGA_EINVAL;
    unsigned long long c = 0;
    TRY(read_dev(s, &c, &s->ctr->cand_count));
    const int64_t cnt = std::min<int64_t>((int64_t)c, s->cand_cap);
    return copy_pairs_sorted(s, s->cand, cnt, ij, cap, n);
}

int genga_get_pairs(genga_system_t *s, int level, uint32_t *ij, int64_t cap, int64_t *n) {
    if (!s || level < 0 || level >= levels_of(s->p)) return GENGA_EINVAL;
    int64_t cnt = s->npairs_host[level];
    if (cnt < 0) {                       // left on the device by the last detection
        unsigned long long c = 0;
        TRY(read_dev(s, &c, &s->ctr->pair_count[level]));
        cnt = std::min<int64_t>((int64_t)c, s->pair_cap[level]);
    }
    return copy_pairs_sorted(s, s->pairs[level], cnt, ij, cap, n);
}

int genga_get_groups(genga_system_t *s, int64_t *label) {
    if (!s || !label) return GENGA_EINVAL;
    std::vector<int> h((size_t)s->n);
    CU(cudaMemcpyAsync(h.data(), s->label, sizeof(int) * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < s->n; i++) label[i] = h[(size_t)i];
    return GENGA_OK;
}

int genga_get_rcrit(genga_system_t *s, int level, double *rc_host) {
    if (!s || !rc_host || level < 0 || level >= levels_of(s->p)) return GENGA_EINVAL;
    CU(cudaMemcpyAsync(rc_host, s->rcl[level].rc, sizeof(double) * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

int genga_set_predrift(genga_system_t *s, const double *pos_host, const double *vel_host) {
    if (!s || !pos_host || !vel_host) return GENGA_EINVAL;
    const size_t bytes = sizeof(double) * 3 * (size_t)s->n;
    CU(cudaMemcpyAsync(s->pre_pos[0], pos_host, bytes, cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemcpyAsync(s->pre_vel[0], vel_host, bytes, cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return GENGA_OK;
}

int genga_get_stats(genga_system_t *s, genga_stats_t *st) {
    if (!s || !st) return GENGA_EINVAL;
    *st = s->stats;
    return GENGA_OK;
}

int genga_set_wait_limits(genga_system_t *s, double bs_group_seconds, double barrier_seconds,
                          int32_t barrier_absent_blocks) {
    if (!s || barrier_absent_blocks < 0 || !(bs_group_seconds < 1e9) || !(barrier_seconds < 1e9))
        return GENGA_EINVAL;
    s->bs_group_limit_ns = bs_group_seconds < 0 ? 10000000000ull
                                                : (unsigned long long)(bs_group_seconds * 1e9);
    s->barrier_limit_ns = barrier_seconds < 0 ? 2000000000ull
                                              : (unsigned long long)(barrier_seconds * 1e9);
    s->barrier_absent = (unsigned)barrier_absent_blocks;
    return GENGA_OK;
}

int genga_set_pair_log(genga_system_t *s, int enable) {
    if (!s) return GENGA_EINVAL;
    s->pair_log = enable != 0;
    s->log_level.clear();
    s->log_off.clear();
    s->log_pairs.clear();
    return GENGA_OK;
}

int genga_get_pair_log(genga_system_t *s, int32_t *level, int64_t *off, uint32_t *ij, int64_t max_events,
                       int64_t max_pairs, int64_t *n_events, int64_t *n_pairs) {
    if (!s) return GENGA_EINVAL;
    const int64_t ne = (int64_t)s->log_level.size();
    const int64_t np = (int64_t)(s->log_pairs.size() / 2);
    if (n_events) *n_events = ne;
    if (n_pairs) *n_pairs = np;
    if (level && off) {
        if (max_events < ne) return fail(s, GENGA_ECAPACITY, "pair log: %lld events", (long long)ne);
        for (int64_t k = 0; k < ne; k++) level[k] = s->log_level[(size_t)k];
        for (int64_t k = 0; k <= ne; k++) off[k] = ne ? s->log_off[(size_t)k] : 0;
    }
    if (ij) {
        if (max_pairs < np) return fail(s, GENGA_ECAPACITY, "pair log: %lld pairs", (long long)np);
        std::copy(s->log_pairs.begin(), s->log_pairs.end(), ij);
    }
    return GENGA_OK;
}

int genga_set_timing(genga_system_t *s, int enable) {
    if (!s) return GENGA_EINVAL;
    CU(cudaStreamSynchronize(s->stream));
    s->timing = enable != 0;
    s->nmarks = 0;
    s->timed_steps = 0;
    for (double &v : s->phase_ms) v = 0.0;
    return GENGA_OK;
}

int genga_get_phase_ms(genga_system_t *s, double *ms, int64_t *nsteps) {
    if (!s || !ms) return GENGA_EINVAL;
    for (int k = 0; k < GENGA_NPHASES; k++) ms[k] = s->phase_ms[k];
    if (nsteps) *nsteps = s->timed_steps;
    return GENGA_OK;
}

const char *genga_phase_name(int phase) {
    static const char *const names[GENGA_NPHASES] = {
        "rcrit", "kick1", "cand_count", "hc_drift", "detect0", "csr0", "level_setup", "rcritS",
        "kickS", "fgS", "detectS", "csrS", "grouping", "buckets", "bs_small", "bs_large", "hc2",
        "kick2"};
    return (phase >= 0 && phase < GENGA_NPHASES) ? names[phase] : nullptr;
}

}  // extern "C"
