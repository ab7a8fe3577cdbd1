// kick.cu -- all-pairs changeover kick of Eq. Hb (Appendix A "Kick(dt/2)"):
//   a_i = G sum_{j != i} m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3
// and the close-encounter pre-check (Appendix A) as a separate FP32 pass.
//
// GB300 design.  The kick is bound by the FP64 pipe (1.68 FP64 instructions per
// clock per SM on GB300, measured, 1/74 of FP32), so the kernel minimises FP64 instructions per
// pair and keeps everything else on the FP32, MUFU and integer pipes:
//   * j bodies are staged in shared memory in tiles of 256 (x, y, z, m and the
//     per-body thresholds); every thread owns one target i;
//   * the grid is (i-tiles x j-chunks) so that thousands of equal blocks
//     balance across the 152 SMs; each block writes compensated partial sums
//     for its chunk, folded in a fixed order by kick_finalize (deterministic);
//   * the rare pairs inside rc_ij are found by an FP32 test on r^2 against a
//     conservative threshold; only those evaluate the changeover function;
//   * the pre-check runs over the pairs i < j on the FP32 pipe alone
//     (precheck_kernel below), so the FP64-bound kick carries none of it;
//   * MIXED: FP64 displacement; r^2 formed as an unevaluated sum of two floats
//     from an exact integer split of the displacement (no FP64 work); FP32
//     rsqrt seed y0; one Newton correction from the residual e = 1 - r^2 y0^2
//     (its leading part 1 - u y0 by an FP32 FMA on the exact float product
//     u y0, rounded once: the float a double residual would be rounded to;
//     the tails in FP32); r^-3 = y0^3 (1 + 1.5 e + 1.875 e^2) = m y0^3 + corr
//     in float-float; FP64 accumulation of (m y0^3) dx, the corrections
//     corr dx (< 2^-19 of each term) summed in float-float per tile and added
//     to the FP64 sums once per tile; per-tile sums folded with TwoSum:
//     6 FP64 instructions per pair (3 subtractions, 3 accumulations).
//     FP64: CUDA's double rsqrt, 17 FP64 instructions per pair (counted).
#include "common.cuh"

namespace genga {
namespace {

constexpr int kKickThreads = 128;
// Resident blocks per SM the register allocation must allow (128 threads
// each), chosen by measurement at N = 65,540: mixed 5 (at most 96
// registers), FP64 7 (72).
constexpr int kick_min_blocks(bool mixed) {
    return mixed ? 5 : 7;
}
constexpr int kTile = 256;

struct KickArgs {
    const double *x, *y, *z, *m;
    const double *rc, *rc2, *pc2;
    const float *thr_rc;        // FP32 upper bound of rc^2
    int n;
    int nm;                     // bodies i >= nm are test particles (nm = n: none)
    int chunk;
    double *part;               // [nchunk][6][n]
    uint2 *cand;
    unsigned long long *cand_count;
    unsigned long long cand_cap;
};

// FP32 value of a positive double, mantissa truncated (never above the input);
// 0 for inputs below 2^-126 (including 0).
__device__ __forceinline__ float r2_to_float_trunc(double r2) {
    unsigned hi = (unsigned)__double2hiint(r2);
    unsigned lo = (unsigned)__double2loint(r2);
    unsigned fb = (hi >= 0x38100000u) ? (((hi - 0x38000000u) << 3) | (lo >> 29)) : 0u;
    return __uint_as_float(fb);
}

// 1 / rc: the Newton reciprocal for every rc the FP32 seed can take, an exact
// division for smaller ones, infinite for rc = 0 (so that min(1/rc_i, 1/rc_j) is
// 1 / max(rc_i, rc_j) for any pair).
__device__ __forceinline__ double inv_rc(double rc) {
    if (rc > 1e-30) return rcp_newton(rc);
    return rc > 0.0 ? 1.0 / rc : __longlong_as_double(0x7ff0000000000000ll);
}

// TP: semi-active test particles (Sec. 8.1): a test particle i takes only the
// sources j < nm; the block that holds the boundary masks the test-particle
// pairs, the blocks past it shorten their source range.
template <bool MIXED, bool TP>
__global__ void __launch_bounds__(kKickThreads, kick_min_blocks(MIXED))
kick_kernel(KickArgs A)
{
    __shared__ double sx[kTile], sy[kTile], sz[kTile], sm[kTile];
    __shared__ double sirc[kTile];            // 1 / rc_j
    __shared__ float sthr[kTile], smh[kTile], sml[kTile];

    const int n = A.n;
    const int i = blockIdx.x * kKickThreads + threadIdx.x;
    const bool valid = i < n;

    double xi = 1e15, yi = 1e15, zi = 1e15;
    double irci = 0.0;                        // 1 / rc_i (infinite for rc_i = 0)
    float thri = 0.0f;
    if (valid) {
        xi = A.x[i]; yi = A.y[i]; zi = A.z[i];
        thri = A.thr_rc[i];
        irci = inv_rc(A.rc[i]);
    }

    const int jbeg = blockIdx.y * A.chunk;
    int jend = min(n, jbeg + A.chunk);
    const int i0 = blockIdx.x * kKickThreads;
    const bool straddle = TP && i0 < A.nm && i0 + kKickThreads > A.nm;
    if (TP && i0 >= A.nm) jend = min(jend, A.nm);

    double S0 = 0.0, S1 = 0.0, S2 = 0.0;   // compensated chunk totals
    double C0 = 0.0, C1 = 0.0, C2 = 0.0;

    for (int jt = jbeg; jt < jend; jt += kTile) {
        const int cnt = min(kTile, jend - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kKickThreads) {
            const int j = jt + k;
            sx[k] = A.x[j]; sy[k] = A.y[j]; sz[k] = A.z[j]; sm[k] = A.m[j];
            sthr[k] = A.thr_rc[j];
            sirc[k] = inv_rc(A.rc[j]);
            if (MIXED) {     // mass as an unevaluated sum of two floats
                const float mh = __double2float_rn(A.m[j]);
                smh[k] = mh;
                sml[k] = __double2float_rn(A.m[j] - (double)mh);
            }
        }
        __syncthreads();

        double ax = 0.0, ay = 0.0, az = 0.0;
        // MIXED: the small correction terms corr * dx (|corr| < 2^-19 m r^-3) of
        // this tile, summed in float-float (TwoSum) and folded into the FP64
        // sums once per tile
        float cxh = 0.0f, cxl = 0.0f, cyh = 0.0f, cyl = 0.0f, czh = 0.0f, czl = 0.0f;
#pragma unroll 4
        for (int k = 0; k < cnt; k++) {
            const int j = jt + k;
            const double dx = sx[k] - xi;
            const double dy = sy[k] - yi;
            const double dz = sz[k] - zi;
            // r^2: FP64 (FP64 form) or Rh + Rl, two floats (MIXED: float-float
            // square sum of the split displacement, relative error ~2^-46).
            // r2f, used only against thresholds with 2^-16 margins, is a
            // float within 2^-23 of r^2.
            double r2 = 0.0;
            float Rh = 0.0f, Rl = 0.0f, hx = 0.0f, hy = 0.0f, hz = 0.0f;
            float r2f;
            if (MIXED) {
                float lx, ly, lz;
                split_f64(dx, hx, lx);
                split_f64(dy, hy, ly);
                split_f64(dz, hz, lz);
                const float px = hx * hx, py = hy * hy, pz = hz * hz;
                const float pxe = fmaf(hx, hx, -px), pye = fmaf(hy, hy, -py), pze = fmaf(hz, hz, -pz);
                const float s1 = px + py, b1 = s1 - px;
                const float e1 = (px - (s1 - b1)) + (py - b1);
                const float s2 = s1 + pz, b2 = s2 - s1;
                const float e2 = (s1 - (s2 - b2)) + (pz - b2);
                const float cross = 2.0f * fmaf(hx, lx, fmaf(hy, ly, hz * lz));
                const float tail = ((e1 + e2) + (pxe + pye + pze)) + cross;
                Rh = s2 + tail;
                Rl = tail - (Rh - s2);
                r2f = Rh;
            } else {
                r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                r2f = r2_to_float_trunc(r2);
            }
            double mk = sm[k];
            float mh = 0.0f, ml = 0.0f;
            if (MIXED) { mh = smh[k]; ml = sml[k]; }
            if (TP && straddle && i >= A.nm && j >= A.nm) {   // two test particles
                mk = 0.0; mh = 0.0f; ml = 0.0f;
            }
            // Changeover band (rare): K < 1 needs r < rc_ij.  K is flat (zero slope) at
            // r = rc, so the branch may follow the FP32 bound and K uses the r^2 above.
            // The branch runs on few lanes of a warp while the FP64 pipe charges the
            // whole warp, so it keeps to short FP64 forms: r from the Newton rsqrt,
            // K with 1/rc_ij = min(1/rc_i, 1/rc_j) staged beforehand (no division).
            if (r2f < fmaxf(thri, sthr[k])) {
                if (j == i) {
                    mk = 0.0; r2 = 1.0; r2f = 1.0f;          // self term: zero, finite
                    Rh = 1.0f; Rl = 0.0f;
                    mh = 0.0f; ml = 0.0f;
                } else {
                    const double r2d = MIXED ? fma(dz, dz, fma(dy, dy, dx * dx)) : r2;
                    mk = mk * changeover_fast(r2d * rsqrt_newton(r2d), fmin(irci, sirc[k]));
                    if (MIXED) {
                        mh = __double2float_rn(mk);
                        ml = __double2float_rn(mk - (double)mh);
                    }
                }
            }
            {
                double s;
                if (MIXED) {
                    // FP32 seed y0 ~ r^-1; Newton residual e = 1 - r^2 y0^2 with
                    // r^2 = Rh + Rl and Rh y0 = u + ue (exact float product): 1 - u y0
                    // by one FP32 FMA (the product u y0 is exact inside the FMA, so the
                    // result is 1 - u y0 rounded once to a float, error < 2^-46), the
                    // tails ue y0 + Rl y0^2 (~2^-24) in FP32.
                    // r^-3 = y0^3 (1 - e)^(-3/2) = y0^3 (1 + 1.5 e + 1.875 e^2 + O(e^3)),
                    // |e| < 2^-20.  m y0^3 is formed exactly enough (~2^-46) as a sum of
                    // two floats, the correction in FP32, and the parts meet in one FP64 add.
                    const float y0f = rsqrtf(Rh);
                    const float u = Rh * y0f, ue = fmaf(Rh, y0f, -u);   // Rh y0 = u + ue exactly
                    const float e1 = fmaf(-u, y0f, 1.0f);
                    const float p = y0f * y0f, pe = fmaf(y0f, y0f, -p);
                    const float q = p * y0f;
                    float qe = fmaf(p, y0f, -q);
                    qe = fmaf(pe, y0f, qe);
                    const float ch = q * mh;
                    float ce = fmaf(q, mh, -ch);
                    ce = fmaf(q, ml, ce);
                    ce = fmaf(qe, mh, ce);
                    const float ef = e1 - fmaf(ue, y0f, Rl * p);
                    const float corr = fmaf(ch, fmaf(1.875f * ef, ef, 1.5f * ef), ce);
                    s = f64_of_f32_any(ch);
                    float_two_sum_acc(cxh, cxl, corr * hx);
                    float_two_sum_acc(cyh, cyl, corr * hy);
                    float_two_sum_acc(czh, czl, corr * hz);
                } else {
                    const double yv = rsqrt(r2);
                    s = (mk * yv) * (yv * yv);
                }
                ax = fma(s, dx, ax);
                ay = fma(s, dy, ay);
                az = fma(s, dz, az);
            }
        }
        if (MIXED) {
            ax += f64_of_f32_any(cxh) + f64_of_f32_any(cxl);
            ay += f64_of_f32_any(cyh) + f64_of_f32_any(cyl);
            az += f64_of_f32_any(czh) + f64_of_f32_any(czl);
        }
        {
            double t, e;
            two_sum(S0, ax, t, e); S0 = t; C0 += e;
            two_sum(S1, ay, t, e); S1 = t; C1 += e;
            two_sum(S2, az, t, e); S2 = t; C2 += e;
        }
    }
    if (valid) {
        double *p = A.part + (size_t)blockIdx.y * 6 * n;
        p[0 * (size_t)n + i] = S0;
        p[1 * (size_t)n + i] = S1;
        p[2 * (size_t)n + i] = S2;
        p[3 * (size_t)n + i] = C0;
        p[4 * (size_t)n + i] = C1;
        p[5 * (size_t)n + i] = C2;
    }
}

// Close-encounter pre-check over the pairs i < j: candidates are the pairs
// with r_ij^2 < (f_pc rc_ij)^2, the exact FP64 test in the defining operation
// order (dist2_rn, no contraction).  Most pairs are decided in FP32 from float
// copies of the positions (round to nearest, |x_f - x| <= 2^-24 |x| per
// component): the float distance r_f differs from r by at most
//   m_ij = sqrt(3) 2^-23 (max|x_i| + max|x_j|)   plus relative rounding,
// so r_f^2 >= ((1 + 2^-20) P + m_ij)^2 (1 + 2^-20) is surely outside and
// r_f^2 < ((1 - 2^-20) P - m_ij)^2 (1 - 2^-20) surely inside (P = f_pc rc_ij
// in FP32); only the band between takes the exact test.  Candidates collect
// in a per-warp shared-memory buffer and go to the global list in batches.
constexpr int kPcThreads = 128;
constexpr int kPcI = 4;                         // targets i per thread
constexpr int kPcTile = 512;

constexpr int kPcWarpBuf = 256;                  // per-warp candidate buffer (shared memory)

// Appends the warp's pending candidates to the global list: one atomic per
// flush reserves the space (a single global counter serialises on its L2
// slice, so it is touched about once per hundred candidates).
__device__ __forceinline__ void precheck_flush(const KickArgs &A, const uint2 *buf, unsigned &cnt,
                                               unsigned lane) {
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0 && cnt) base = atomicAdd(A.cand_count, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (unsigned t = lane; t < cnt; t += 32) {
        const unsigned long long idx = base + t;
        if (idx < A.cand_cap) A.cand[idx] = buf[t];
    }
    __syncwarp();
    cnt = 0;
}

__global__ void __launch_bounds__(kPcThreads)
precheck_kernel(KickArgs A, double f_pc)
{
    __shared__ float4 sj[kPcTile];                   // x, y, z, P = f_pc rc (floats)
    __shared__ float sM[kPcTile];
    __shared__ uint2 wbuf[kPcThreads / 32][kPcWarpBuf];
    const int n = A.n;
    const int i0 = blockIdx.x * (kPcThreads * kPcI);
    if (i0 >= A.nm) return;                              // only test-particle rows: no pairs
    const int jbeg = max(blockIdx.y * A.chunk, i0 + 1);
    const int jend = min(n, blockIdx.y * A.chunk + A.chunk);
    if (jbeg >= jend) return;                            // block below the diagonal
    const unsigned lane = threadIdx.x & 31u;
    uint2 *buf = wbuf[threadIdx.x >> 5];
    unsigned pend = 0;                                   // candidates in buf (warp-uniform)
    constexpr float kM = 1.7320509f * 1.1920929e-07f;    // sqrt(3) 2^-23
    constexpr float kUp = 1.0f + 9.5367432e-07f, kDn = 1.0f - 9.5367432e-07f;   // 1 +- 2^-20
    float xf[kPcI], yf[kPcI], zf[kPcI], Pi[kPcI], Mi[kPcI];
    int ii[kPcI];
#pragma unroll
    for (int r = 0; r < kPcI; r++) {
        const int i = i0 + r * kPcThreads + threadIdx.x;
        ii[r] = i;
        xf[r] = yf[r] = zf[r] = 3.0e38f; Pi[r] = 0.0f; Mi[r] = 0.0f;
        if (i < n && i < A.nm) {        // a test-particle row pairs only with j > i: none
            xf[r] = f32_of_f64_rn(A.x[i]); yf[r] = f32_of_f64_rn(A.y[i]); zf[r] = f32_of_f64_rn(A.z[i]);
            Pi[r] = (float)f_pc * f32_of_f64_rn(A.rc[i]);
            Mi[r] = kM * fmaxf(fabsf(xf[r]), fmaxf(fabsf(yf[r]), fabsf(zf[r])));
        }
    }
    for (int jt = jbeg; jt < jend; jt += kPcTile) {
        const int cnt = min(kPcTile, jend - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kPcThreads) {
            const int j = jt + k;
            const float x = f32_of_f64_rn(A.x[j]), y = f32_of_f64_rn(A.y[j]), z = f32_of_f64_rn(A.z[j]);
            sj[k] = make_float4(x, y, z, (float)f_pc * f32_of_f64_rn(A.rc[j]));
            sM[k] = kM * fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
        }
        __syncthreads();
        for (int k = 0; k < cnt; k++) {
            const int j = jt + k;
            const float4 q = sj[k];
            const float Mj = sM[k];
            bool maybe[kPcI];
            bool any = false;
#pragma unroll
            for (int r = 0; r < kPcI; r++) {
                const float dx = q.x - xf[r], dy = q.y - yf[r], dz = q.z - zf[r];
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float to = fmaf(fmaxf(Pi[r], q.w), kUp, Mi[r] + Mj);
                maybe[r] = (j > ii[r]) && (r2 < to * to * kUp);
                any |= maybe[r];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
#pragma unroll
            for (int r = 0; r < kPcI; r++) {
                bool emit = false;
                if (maybe[r]) {
                    const float dx = q.x - xf[r], dy = q.y - yf[r], dz = q.z - zf[r];
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    const float ti = fmaf(fmaxf(Pi[r], q.w), kDn, -(Mi[r] + Mj));
                    if (ti > 0.0f && r2 < ti * ti * kDn) {
                        emit = true;
                    } else {
                        const int i = ii[r];
                        emit = dist2_rn(A.x[j] - A.x[i], A.y[j] - A.y[i], A.z[j] - A.z[i]) <
                               fmax(A.pc2[i], A.pc2[j]);
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, emit);
                if (emit) buf[pend + __popc(ball & ((1u << lane) - 1u))] = make_uint2((unsigned)ii[r], (unsigned)j);
                pend += __popc(ball);
            }
            if (pend > kPcWarpBuf - 32 * kPcI) precheck_flush(A, buf, pend, lane);
        }
    }
    precheck_flush(A, buf, pend, lane);
}

// Folds the chunk partials in chunk order (TwoSum), scales by G and applies the
// kick v += dt_half a; optionally stores a.
__global__ void kick_finalize(const double *part, int nchunk, int n, double G, double dt_half,
                              double *vel, double *acc_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double S = 0.0, C = 0.0;
        for (int q = 0; q < nchunk; q++) {
            const double *p = part + (size_t)q * 6 * n;
            double t, e;
            two_sum(S, p[(size_t)c * n + i], t, e);
            S = t;
            C += e + p[(size_t)(3 + c) * n + i];
        }
        const double a = G * (S + C);
        if (acc_out) acc_out[(size_t)c * n + i] = a;
        if (dt_half != 0.0) vel[(size_t)c * n + i] += dt_half * a;
    }
}

void kick_geometry(int n, int num_sms, int *chunk, int *nchunk) {
    // (i-tiles x j-chunks) grid
    const int iblocks = (n + kKickThreads - 1) / kKickThreads;
    const int max_chunks = (n + kTile - 1) / kTile;
    // aim for at least 8 blocks per SM, each at least one tile and at most 16
    int want = (8 * num_sms + iblocks - 1) / iblocks;
    int tiles_per_chunk = (max_chunks + want - 1) / (want > 0 ? want : 1);
    if (tiles_per_chunk > 16) tiles_per_chunk = 16;
    if (tiles_per_chunk < 1) tiles_per_chunk = 1;
    if ((max_chunks + tiles_per_chunk - 1) / tiles_per_chunk > kMaxKickChunks)
        tiles_per_chunk = (max_chunks + kMaxKickChunks - 1) / kMaxKickChunks;
    *chunk = tiles_per_chunk * kTile;
    *nchunk = (n + *chunk - 1) / *chunk;
}

}  // namespace

static KickArgs make_args(genga_system *s, bool precheck) {
    KickArgs A;
    const int64_t n = s->n;
    A.x = s->pos; A.y = s->pos + n; A.z = s->pos + 2 * n; A.m = s->mass;
    A.rc = s->rcl[0].rc; A.rc2 = s->rcl[0].rc2; A.pc2 = s->rcl[0].pc2;
    A.thr_rc = s->rcl[0].thr_rc;
    A.n = (int)n;
    A.nm = tp_bound(s);
    A.chunk = s->kick_chunk;
    A.part = s->kick_part;
    A.cand = s->cand;
    A.cand_count = &s->ctr->cand_count;
    A.cand_cap = (unsigned long long)s->cand_cap;
    return A;
}

cudaError_t launch_kick(genga_system *s, double dt_half, bool precheck, double *acc_out) {
    const int n = (int)s->n;
    if (!s->kick_part) return cudaErrorInvalidValue;
    if (s->kick_chunk == 0) kick_geometry(n, s->num_sms, &s->kick_chunk, &s->kick_nchunk);
    KickArgs A = make_args(s, false);
    dim3 grid((n + kKickThreads - 1) / kKickThreads, s->kick_nchunk);
    if (precheck) GENGA_CUDA_TRY(launch_precheck_only(s));
    const bool mixed = s->p.precision == GENGA_MIXED;
    if (A.nm < n) {
        if (mixed) kick_kernel<true, true><<<grid, kKickThreads, 0, s->stream>>>(A);
        else kick_kernel<false, true><<<grid, kKickThreads, 0, s->stream>>>(A);
    } else {
        if (mixed) kick_kernel<true, false><<<grid, kKickThreads, 0, s->stream>>>(A);
        else kick_kernel<false, false><<<grid, kKickThreads, 0, s->stream>>>(A);
    }
    ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    kick_finalize<<<(n + 255) / 256, 256, 0, s->stream>>>(s->kick_part, s->kick_nchunk, n, s->p.G,
                                                          dt_half, s->vel, acc_out); ++s->launches;
    return cudaGetLastError();
}

cudaError_t launch_precheck_only(genga_system *s) {
    const int n = (int)s->n;
    if (!s->kick_part) return cudaErrorInvalidValue;
    if (s->kick_chunk == 0) kick_geometry(n, s->num_sms, &s->kick_chunk, &s->kick_nchunk);
    KickArgs A = make_args(s, true);
    // (i-tile x j-chunk) grid like the kick; blocks wholly below the diagonal return at once
    dim3 grid((n + kPcThreads * kPcI - 1) / (kPcThreads * kPcI), s->kick_nchunk);
    GENGA_CUDA_TRY(cudaMemsetAsync(&s->ctr->cand_count, 0, sizeof(unsigned long long), s->stream));
    precheck_kernel<<<grid, kPcThreads, 0, s->stream>>>(A, s->p.f_pc); ++s->launches;
    return cudaGetLastError();
}

// Launches the kick (no pre-check) on caller-provided arrays, with the number of
// j-chunks capped at max_nchunk; used by the allocation-free entry point.
cudaError_t launch_kick_raw(const KickRaw &k, int num_sms, int max_nchunk, cudaStream_t stream) {
    int chunk, nchunk;
    kick_geometry(k.n, num_sms, &chunk, &nchunk);
    if (nchunk > max_nchunk) {
        const int tiles = (k.n + kTile - 1) / kTile;
        const int tiles_per_chunk = (tiles + max_nchunk - 1) / max_nchunk;
        chunk = tiles_per_chunk * kTile;
        nchunk = (k.n + chunk - 1) / chunk;
    }
    KickArgs A;
    A.x = k.pos; A.y = k.pos + k.n; A.z = k.pos + 2 * (size_t)k.n; A.m = k.mass;
    A.rc = k.rc; A.rc2 = k.rc2; A.pc2 = nullptr; A.thr_rc = k.thr;
    A.n = k.n; A.nm = k.n; A.chunk = chunk; A.part = k.part;
    A.cand = nullptr; A.cand_count = nullptr; A.cand_cap = 0;
    dim3 grid((k.n + kKickThreads - 1) / kKickThreads, nchunk);
    if (k.mixed) kick_kernel<true, false><<<grid, kKickThreads, 0, stream>>>(A);
    else kick_kernel<false, false><<<grid, kKickThreads, 0, stream>>>(A);
    GENGA_CUDA_TRY(cudaGetLastError());
    kick_finalize<<<(k.n + 255) / 256, 256, 0, stream>>>(k.part, nchunk, k.n, k.G, k.dt_half, k.vel, k.acc_out);
    return cudaGetLastError();
}

int kick_nchunk_for(int n, int num_sms) {
    int c, nc;
    kick_geometry(n, num_sms, &c, &nc);
    return nc;
}

}  // namespace genga
