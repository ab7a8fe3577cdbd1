// kick.cu -- all-pairs changeover kick of Eq. Hb (Appendix A "Kick(dt/2)"):
//   a_i = G sum_{j != i} m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3
// and the close-encounter pre-check (Appendix A).
//
// GB300 design.  The kick is bound by the FP64 pipe (1.68 FP64 instructions per
// clock per SM on GB300, measured, 1/74 of FP32), so the kernels minimise FP64
// instructions per interaction and keep everything else on the FP32, MUFU and
// integer pipes.  Two layouts:
//   * symmetric (kick_sym_kernel, below): each unordered pair once, its force to
//     both bodies (Newton's third law) -- 9 FP64 instructions per pair in the
//     mixed form, 4.5 per interaction; the pre-check rides along on the FP32
//     pipe.  Used where it is predicted faster (N of ~8k and more);
//   * tiled (kick_kernel): every ordered pair, one target per thread against
//     source tiles in shared memory, an (i-tile x j-chunk) grid of equal blocks;
//     for small N, test particles and the allocation-free entry point, with the
//     pre-check as its own FP32 pass over i < j (precheck_kernel).
// Both write compensated partial sums folded in a fixed order by kick_finalize
// (deterministic).  The rare pairs inside rc_ij are found by an FP32 test on
// r^2 against a conservative threshold; only those evaluate the changeover
// function.
//
// MIXED: FP64 displacement; r^2 formed as an unevaluated sum of two floats from
// an exact integer split of the displacement (no FP64 work); FP32 rsqrt seed
// y0; one Newton correction from the residual e = 1 - r^2 y0^2 (its leading
// part 1 - u y0 by an FP32 FMA on the exact float product u y0, rounded once:
// the float a double residual would be rounded to; the tails in FP32);
// r^-3 = y0^3 (1 + 1.5 e + 1.875 e^2) = m y0^3 + corr in float-float; FP64
// accumulation of (m y0^3) dx, the corrections corr dx (< 2^-19 of each term)
// summed in float-float and added to the FP64 sums with the partials; 6 FP64
// instructions per ordered pair in the tiled layout (3 subtractions, 3
// accumulations).  FP64: CUDA's double rsqrt in the tiled layout (17 FP64
// instructions per pair, counted), the Newton rsqrt of common.cuh in the
// symmetric one (21 per unordered pair).
#include <algorithm>
#include <queue>
#include <utility>
#include <vector>

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
    __shared__ float2 sircf[MIXED ? kTile : 1]; // MIXED: 1 / rc_j as two floats
    __shared__ float sthr[kTile], smh[kTile], sml[kTile];

    const int n = A.n;
    const int i = blockIdx.x * kKickThreads + threadIdx.x;
    const bool valid = i < n;

    double xi = 1e15, yi = 1e15, zi = 1e15;
    double irci = 0.0;                        // 1 / rc_i (infinite for rc_i = 0)
    float thri = 0.0f;
    float2 ircfi = make_float2(0.0f, 0.0f);
    if (valid) {
        xi = A.x[i]; yi = A.y[i]; zi = A.z[i];
        thri = A.thr_rc[i];
        irci = inv_rc(A.rc[i]);
        if (MIXED) ircfi = ff_of_irc(irci);
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
            if (MIXED) sircf[k] = ff_of_irc(sirc[k]);
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
            // whole warp: the FP64 form takes r from the Newton rsqrt and
            // 1/rc_ij = min(1/rc_i, 1/rc_j) staged beforehand (no division); MIXED
            // evaluates K in float-float on the FP32 pipe (below).
            const bool band = r2f < fmaxf(thri, sthr[k]);
            if (band && j == i) {
                mk = 0.0; r2 = 1.0; r2f = 1.0f;              // self term: zero, finite
                Rh = 1.0f; Rl = 0.0f;
                mh = 0.0f; ml = 0.0f;
            }
            if (!MIXED && band && j != i)
                mk = mk * changeover_fast(r2 * rsqrt_newton(r2), fmin(irci, sirc[k]));
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
                    const float ef = e1 - fmaf(ue, y0f, Rl * p);
                    if (band && j != i) {      // K in float-float, the mass scaled by it
                        const float2 cj = sircf[k];
                        const bool ci = ircfi.x < cj.x || (ircfi.x == cj.x && ircfi.y <= cj.y);
                        float Kh, Kl;
                        changeover_ff(u, ue, Rl, y0f, ef, ci ? ircfi.x : cj.x, ci ? ircfi.y : cj.y, Kh, Kl);
                        ff_mul(mh, ml, Kh, Kl);
                    }
                    const float ch = q * mh;
                    float ce = fmaf(q, mh, -ch);
                    ce = fmaf(q, ml, ce);
                    ce = fmaf(qe, mh, ce);
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

// ---------------------------------------------------------------------------
// Symmetric kick: each unordered pair {i, j} is evaluated once and its force
// goes to both bodies with opposite signs (Newton's third law): the terms
// m_j K r^-3 (x_j - x_i) of a_i and -m_i K r^-3 (x_j - x_i) of a_j share the
// displacement, r^-3 and K.  FP64 instructions per unordered pair: MIXED 9
// (3 subtractions, 3 + 3 accumulations), FP64 form 21 (the Newton rsqrt of
// common.cuh instead of CUDA's double rsqrt) -- per ordered pair 4.5 and 10.5
// against 6 and ~17 of kick_kernel.
//
// Work decomposition.  Bodies in tiles of 128 (one per thread of a 4-warp
// block), tiles in super-ranges of P tiles.  A work item is a super-tile pair
// (X, Y), X <= Y: the rows a of X (the i-tile, one body per thread, sums in
// registers) against the tiles b of Y (b >= a when X == Y).  In a tile pair,
// warp w holds i-subtile w (32 bodies, one per lane) and meets the j-subtiles
// q = (w + s) mod 4 in four phases s.  In a phase, lane L at step t pairs its
// i with body (L + t) mod 32 of subtile q, whose running sums ride along the
// lanes (one shuffle per step: every j is handled by one lane at a time); at
// the end of the phase the lanes add them to the item's j sums in shared
// memory -- one warp per subtile per phase, so without conflicts and in a fixed
// order.  A diagonal subtile (q = w, a = b) takes the steps 1..16, step 16 on
// lanes 0..15 only: every pair inside it once, no self pair.
//
// Partial sums.  Every body gets one compensated partial per super-range
// (nS = ceil(nT / P)): item (X, Y) writes its row sums to slot Y of the X
// bodies and its j sums to slot X of the Y bodies; a diagonal item (X, X)
// writes both, added, to slot X as each row completes.  Every (slot, body) is
// written exactly once, and kick_finalize folds the slots in slot order, so
// the result is deterministic.
//
// Dispatch.  One persistent block per resident block slot takes items from a
// counter in the host's order (largest first, the diagonal items last); the
// host picks P for each N by list-scheduling the items over the resident
// blocks, with the finalize's cost counted.
constexpr int kSymT = 128;
constexpr int kSymMaxP = 6;

struct SymArgs {
    const double *x, *y, *z, *m;
    const double *irc;          // 1 / rc per body (inv_rc)
    const float2 *ircf;         // MIXED: the same as two floats
    const float *thr;           // FP32 upper bound of rc^2
    const float2 *mhl;          // MIXED: mass as an unevaluated sum of two floats
    int n, nT, P, nItems;
    int nm;                     // TP: bodies i >= nm are test particles (no pair of two)
    const int2 *items;          // (X, Y) super-tile pairs, X <= Y, in dispatch order
    unsigned *ctr;              // dispatch counter, zero at launch
    double *part;               // [nS][6][n]
    // fused pre-check (PC): candidates i < j with r^2 < max(pc2_i, pc2_j)
    const double *pc2;          // (f_pc rc)^2
    const float *thr_pc;        // FP32 upper bound of pc2 (2^-16 margin)
    const float2 *pcf;          // pc2 as an unevaluated sum of two floats
    uint2 *cand;
    unsigned long long *cand_count;
    unsigned long long cand_cap;
};

// Resident blocks per SM the register allocation must allow (128 threads each):
// 6 (80 registers) for the mixed form and the FP64 form with the pre-check,
// without spills; the FP64 form without it needs only 72.  (The mixed form
// also fits 72 registers, 7 blocks, but ran no faster.)
constexpr int sym_min_blocks(bool mixed, bool pc) {
    return mixed ? 6 : (pc ? 6 : 4);
}

// Dynamic shared memory: the staged j tile (x, y, z, m, 1/rc; thr, mh, ml),
// then the item's j sums (x, y, z; MIXED: float-float corrections).
constexpr size_t sym_smem(bool mixed, int P) {
    return (size_t)kSymT * (5 * sizeof(double) + 3 * sizeof(float)) +
           (size_t)P * kSymT * (3 * sizeof(double) + (mixed ? 6 * sizeof(float) : 0));
}

// Far-away stand-in position of the k-th padding body of the last tile:
// distinct for distinct k (no zero separation), massless.
__device__ __forceinline__ double pad_pos(int k) { return 1.0e15 + 1.0e13 * (double)k; }

__global__ void kick_pack_kernel(const double *m, const double *rc, const double *pc2, int n, double *irc,
                                 float2 *ircf, float2 *mhl, float *thr_pc, float2 *pcf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ir = inv_rc(rc[i]);
    irc[i] = ir;
    ircf[i] = ff_of_irc(ir);
    // rounded up, then 2^-16 more: any float r^2 within 2^-23 of an r^2 below
    // pc2 is below it
    thr_pc[i] = fmaxf(__double2float_ru(pc2[i]) * 1.0000153f, 1.17549435e-38f);
    const float ph = __double2float_rn(pc2[i]);
    pcf[i] = make_float2(ph, __double2float_rn(pc2[i] - (double)ph));
    const float mh = __double2float_rn(m[i]);
    mhl[i] = make_float2(mh, __double2float_rn(m[i] - (double)mh));
}

constexpr int kSymPcBuf = 128;                 // per-warp candidate buffer (shared memory)

// Appends a warp's buffered candidates to the global list (one atomic per flush).
__device__ __forceinline__ void sym_pc_flush(const SymArgs &A, const uint2 *buf, int &cnt, int lane) {
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0 && cnt) base = atomicAdd(A.cand_count, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int t = lane; t < cnt; t += 32) {
        const unsigned long long idx = base + (unsigned long long)t;
        if (idx < A.cand_cap) A.cand[idx] = buf[t];
    }
    __syncwarp();
    cnt = 0;
}

// One pair's pre-check inside the kick (warp-uniform call).  Lanes with
// `maybe` decide r^2 < max(pc2_i, pc2_j) from the kick's float r^2 (Rh + Rl,
// within rel of r^2) against that pc2 as two floats (pc2 = h + l; rounding to
// nearest is monotone, so the larger pair of floats is the larger pc2): outside
// a band of width `band` around it the sign of (Rh - h) + (Rl - l) decides, on
// the FP32 pipe; inside it (never met in practice) the exact FP64 test of
// precheck_kernel does.  The warp appends its candidates (i < j) to its
// buffer, flushed when it could overflow on the next step.
__device__ __forceinline__ void sym_precheck(const SymArgs &A, uint2 *buf, int &pend, int lane, bool maybe,
                                             int i, int j, double dx, double dy, double dz, float Rh, float Rl,
                                             float2 pci, float2 pcj, float band) {
    if (!__any_sync(0xffffffffu, maybe)) return;
    bool emit = false;
    if (maybe && i < A.n && j < A.n) {
        const float2 P = (pci.x > pcj.x || (pci.x == pcj.x && pci.y >= pcj.y)) ? pci : pcj;
        const float D = (Rh - P.x) + (Rl - P.y);
        const float w = band * P.x;
        if (D < -w) emit = true;
        else if (D > w) emit = false;
        else emit = dist2_rn(dx, dy, dz) < fmax(A.pc2[i], A.pc2[j]);
    }
    const unsigned ball = __ballot_sync(0xffffffffu, emit);
    if (emit) buf[pend + __popc(ball & ((1u << lane) - 1u))] = make_uint2((unsigned)min(i, j), (unsigned)max(i, j));
    pend += __popc(ball);
    if (pend > kSymPcBuf - 32) sym_pc_flush(A, buf, pend, lane);
}

// PC: the close-encounter pre-check of Appendix A fused into the kick: a pair
// whose float r^2 (within 2^-23 of r^2) is below max(thr_pc_i, thr_pc_j) takes
// the exact FP64 test of precheck_kernel (dist2_rn, no contraction) -- the same
// candidates, found on the FP32/INT pipes the FP64-bound kick leaves idle.
template <bool MIXED, bool PC, bool TP>
__global__ void __launch_bounds__(kSymT, sym_min_blocks(MIXED, PC))
kick_sym_kernel(SymArgs A)
{
    extern __shared__ __align__(16) unsigned char sym_sh[];
    double *sx = reinterpret_cast<double *>(sym_sh);
    double *sy = sx + kSymT, *sz = sy + kSymT, *sm = sz + kSymT, *sirc = sm + kSymT;
    float2 *sircf = reinterpret_cast<float2 *>(sirc);     // MIXED: 1/rc as two floats
    float *sthr = reinterpret_cast<float *>(sirc + kSymT);
    float *smh = sthr + kSymT, *sml = smh + kSymT;
    const int PT = A.P * kSymT;
    double *jax = reinterpret_cast<double *>(sml + kSymT);
    double *jay = jax + PT, *jaz = jay + PT;
    float *jc = reinterpret_cast<float *>(jaz + PT);      // [6][PT]: x hi, x lo, y hi, y lo, z hi, z lo
    __shared__ int s_item;
    __shared__ float sthp[PC ? kSymT : 1];                // thr_pc of the j tile
    __shared__ float2 spcf[PC ? kSymT : 1];               // pc2 of the j tile as two floats
    __shared__ uint2 pcb[PC ? kSymT / 32 : 1][PC ? kSymPcBuf : 1];
    int pend = 0;                                         // candidates in this warp's buffer

    const int n = A.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();                      // the previous item's shared sums are written out
        if (threadIdx.x == 0) s_item = (int)atomicAdd(A.ctr, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= A.nItems) break;
        const int2 XY = A.items[it];
        const int a0 = XY.x * A.P, a1 = min(A.nT, a0 + A.P);
        const int b0 = XY.y * A.P, b1 = min(A.nT, b0 + A.P);
        const bool diag = XY.x == XY.y;
        const int nj = (b1 - b0) * kSymT;
        for (int e = threadIdx.x; e < nj; e += kSymT) {
            jax[e] = 0.0; jay[e] = 0.0; jaz[e] = 0.0;
            if (MIXED)
#pragma unroll
                for (int c = 0; c < 6; c++) jc[c * PT + e] = 0.0f;
        }
        for (int a = a0; a < a1; a++) {
            const int i = a * kSymT + threadIdx.x;
            const bool valid = i < n;
            double xi, yi, zi, mi = 0.0, irci = 0.0;
            float thri = 0.0f, mhi = 0.0f, mli = 0.0f, thpi = 0.0f;
            float2 pcfi = make_float2(0.0f, 0.0f);
            float2 ircfi = make_float2(0.0f, 0.0f);
            if (valid) {
                xi = A.x[i]; yi = A.y[i]; zi = A.z[i]; mi = A.m[i];
                thri = A.thr[i];
                if (MIXED) ircfi = A.ircf[i];
                else irci = A.irc[i];
                if (PC) { thpi = A.thr_pc[i]; pcfi = A.pcf[i]; }
                if (MIXED) { const float2 q = A.mhl[i]; mhi = q.x; mli = q.y; }
            } else {
                xi = yi = zi = pad_pos(threadIdx.x);
            }
            double ax = 0.0, ay = 0.0, az = 0.0;
            float cxh = 0.0f, cxl = 0.0f, cyh = 0.0f, cyl = 0.0f, czh = 0.0f, czl = 0.0f;

            for (int b = diag ? a : b0; b < b1; b++) {
                __syncthreads();              // the tile buffer is free
                {
                    const int k = threadIdx.x, j = b * kSymT + k;
                    if (j < n) {
                        sx[k] = A.x[j]; sy[k] = A.y[j]; sz[k] = A.z[j]; sm[k] = A.m[j];
                        if (MIXED) sircf[k] = A.ircf[j];
                        else sirc[k] = A.irc[j];
                        sthr[k] = A.thr[j];
                        if (MIXED) { const float2 q = A.mhl[j]; smh[k] = q.x; sml[k] = q.y; }
                        if (PC) { sthp[k] = A.thr_pc[j]; spcf[k] = A.pcf[j]; }
                    } else {
                        sx[k] = sy[k] = sz[k] = pad_pos(k); sm[k] = 0.0;
                        if (MIXED) sircf[k] = make_float2(0.0f, 0.0f);
                        else sirc[k] = 0.0;
                        sthr[k] = 0.0f; smh[k] = 0.0f; sml[k] = 0.0f;
                        if (PC) { sthp[k] = 0.0f; spcf[k] = make_float2(0.0f, 0.0f); }
                    }
                }
                __syncthreads();
                const bool same = a == b;
                for (int s = 0; s < 4; s++) {
                    const int q = (w + s) & 3;
                    if (!same || q >= w) {
                        const bool dsub = same && q == w;
                        const int t0 = dsub ? 1 : 0, t1 = dsub ? 17 : 32;
                        const int qb = q * 32;
                        // running sums of the j body this lane holds: (lane + t) mod 32 at step t
                        double jx = 0.0, jy = 0.0, jz = 0.0;
                        float jxh = 0.0f, jxl = 0.0f, jyh = 0.0f, jyl = 0.0f, jzh = 0.0f, jzl = 0.0f;
#pragma unroll 4
                        for (int t = t0; t < t1; t++) {
                            const int k = qb + ((lane + t) & 31);
                            // no contribution and no candidate: the pair lane - 16 takes in
                            // a diagonal subtile's step 16; TP, a pair of two test particles
                            const bool half = (dsub && t == 16 && lane >= 16) ||
                                              (TP && i >= A.nm && b * kSymT + k >= A.nm);
                            const double dx = sx[k] - xi;
                            const double dy = sy[k] - yi;
                            const double dz = sz[k] - zi;
                            if (MIXED) {
                                float hx, hy, hz, lx, ly, lz;
                                split_f64(dx, hx, lx);
                                split_f64(dy, hy, ly);
                                split_f64(dz, hz, lz);
                                const float px = hx * hx, py = hy * hy, pz = hz * hz;
                                const float pxe = fmaf(hx, hx, -px), pye = fmaf(hy, hy, -py), pze = fmaf(hz, hz, -pz);
                                const float s1 = px + py, bb1 = s1 - px;
                                const float e1 = (px - (s1 - bb1)) + (py - bb1);
                                const float s2 = s1 + pz, bb2 = s2 - s1;
                                const float e2 = (s1 - (s2 - bb2)) + (pz - bb2);
                                const float cross = 2.0f * fmaf(hx, lx, fmaf(hy, ly, hz * lz));
                                const float tail = ((e1 + e2) + (pxe + pye + pze)) + cross;
                                const float Rh = s2 + tail;
                                const float Rl = tail - (Rh - s2);
                                if (PC) sym_precheck(A, pcb[w], pend, lane, !half && Rh < fmaxf(thpi, sthp[k]), i,
                                                     b * kSymT + k, dx, dy, dz, Rh, Rl, pcfi, spcf[k],
                                                     9.094947e-13f);          // 2^-40

                                // r^-3 = y0^3 (1 + 1.5 e + 1.875 e^2) as in kick_kernel; the
                                // mass-free parts are shared by the two sides
                                const float y0f = rsqrtf(Rh);
                                const float u = Rh * y0f, ue = fmaf(Rh, y0f, -u);
                                const float r1 = fmaf(-u, y0f, 1.0f);
                                const float p = y0f * y0f, pe = fmaf(y0f, y0f, -p);
                                const float qq = p * y0f;
                                float qe = fmaf(p, y0f, -qq);
                                qe = fmaf(pe, y0f, qe);
                                const float ef = r1 - fmaf(ue, y0f, Rl * p);
                                float mhj = smh[k], mlj = sml[k], mhI = mhi, mlI = mli;
                                // changeover band (rare): K in float-float from r = r^2 r^-1,
                                // 1/rc_ij = min(1/rc_i, 1/rc_j) (as float pairs: rounding is
                                // monotone), both masses scaled by K -- no FP64 work
                                if (Rh < fmaxf(thri, sthr[k])) {
                                    const float2 cj = sircf[k];
                                    const bool ci = ircfi.x < cj.x || (ircfi.x == cj.x && ircfi.y <= cj.y);
                                    float Kh, Kl;
                                    changeover_ff(u, ue, Rl, y0f, ef, ci ? ircfi.x : cj.x, ci ? ircfi.y : cj.y, Kh, Kl);
                                    ff_mul(mhj, mlj, Kh, Kl);
                                    ff_mul(mhI, mlI, Kh, Kl);
                                }
                                if (half) { mhj = 0.0f; mlj = 0.0f; mhI = 0.0f; mlI = 0.0f; }
                                const float poly = fmaf(1.875f * ef, ef, 1.5f * ef);
                                // i side: m_j r^-3 dx
                                {
                                    const float ch = qq * mhj;
                                    float ce = fmaf(qq, mhj, -ch);
                                    ce = fmaf(qq, mlj, ce);
                                    ce = fmaf(qe, mhj, ce);
                                    const float corr = fmaf(ch, poly, ce);
                                    const double sj = f64_of_f32_any(ch);
                                    ax = fma(sj, dx, ax);
                                    ay = fma(sj, dy, ay);
                                    az = fma(sj, dz, az);
                                    float_two_sum_acc(cxh, cxl, corr * hx);
                                    float_two_sum_acc(cyh, cyl, corr * hy);
                                    float_two_sum_acc(czh, czl, corr * hz);
                                }
                                // j side: -m_i r^-3 dx
                                {
                                    const float ch = qq * mhI;
                                    float ce = fmaf(qq, mhI, -ch);
                                    ce = fmaf(qq, mlI, ce);
                                    ce = fmaf(qe, mhI, ce);
                                    const float corr = fmaf(ch, poly, ce);
                                    const double si = f64_of_f32_any(ch);
                                    jx = fma(-si, dx, jx);
                                    jy = fma(-si, dy, jy);
                                    jz = fma(-si, dz, jz);
                                    float_two_sum_acc(jxh, jxl, -(corr * hx));
                                    float_two_sum_acc(jyh, jyl, -(corr * hy));
                                    float_two_sum_acc(jzh, jzl, -(corr * hz));
                                }
                            } else {
                                const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                                const float r2f = r2_to_float_trunc(r2);
                                if (PC) sym_precheck(A, pcb[w], pend, lane, !half && r2f < fmaxf(thpi, sthp[k]), i,
                                                     b * kSymT + k, dx, dy, dz, r2f, 0.0f, pcfi, spcf[k],
                                                     9.536743e-07f);          // 2^-20

                                const double yv = rsqrt_newton(r2);
                                double y3 = (yv * yv) * yv;
                                if (r2f < fmaxf(thri, sthr[k]))
                                    y3 *= changeover_fast(r2 * yv, fmin(irci, sirc[k]));
                                const double sj = half ? 0.0 : sm[k] * y3;
                                const double si = half ? 0.0 : mi * y3;
                                ax = fma(sj, dx, ax);
                                ay = fma(sj, dy, ay);
                                az = fma(sj, dz, az);
                                jx = fma(-si, dx, jx);
                                jy = fma(-si, dy, jy);
                                jz = fma(-si, dz, jz);
                            }
                            // pass the j sums on: lane L takes over lane L + 1's body
                            const int src = (lane + 1) & 31;
                            jx = __shfl_sync(0xffffffffu, jx, src);
                            jy = __shfl_sync(0xffffffffu, jy, src);
                            jz = __shfl_sync(0xffffffffu, jz, src);
                            if (MIXED) {
                                jxh = __shfl_sync(0xffffffffu, jxh, src);
                                jxl = __shfl_sync(0xffffffffu, jxl, src);
                                jyh = __shfl_sync(0xffffffffu, jyh, src);
                                jyl = __shfl_sync(0xffffffffu, jyl, src);
                                jzh = __shfl_sync(0xffffffffu, jzh, src);
                                jzl = __shfl_sync(0xffffffffu, jzl, src);
                            }
                        }
                        // after the last step's hand-over the lane holds body (lane + t1) mod 32
                        const int e = (b - b0) * kSymT + qb + ((lane + t1) & 31);
                        jax[e] += jx;
                        jay[e] += jy;
                        jaz[e] += jz;
                        if (MIXED) {
                            float_two_sum_acc(jc[0 * PT + e], jc[1 * PT + e], jxh);
                            jc[1 * PT + e] += jxl;
                            float_two_sum_acc(jc[2 * PT + e], jc[3 * PT + e], jyh);
                            jc[3 * PT + e] += jyl;
                            float_two_sum_acc(jc[4 * PT + e], jc[5 * PT + e], jzh);
                            jc[5 * PT + e] += jzl;
                        }
                    }
                    __syncthreads();          // subtile sums handed to the next warp
                }
            }
            // row a done: its sums over the tiles of Y (slot Y), or, in a
            // diagonal item, with the j sums of tile a, now complete (slot X)
            if (valid) {
                double S[3] = {ax, ay, az};
                double C[3] = {0.0, 0.0, 0.0};
                if (MIXED) {
                    C[0] = f64_of_f32_any(cxh) + f64_of_f32_any(cxl);
                    C[1] = f64_of_f32_any(cyh) + f64_of_f32_any(cyl);
                    C[2] = f64_of_f32_any(czh) + f64_of_f32_any(czl);
                }
                if (diag) {
                    const int e = (a - b0) * kSymT + threadIdx.x;
                    const double J[3] = {jax[e], jay[e], jaz[e]};
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        double t, err;
                        two_sum(S[c], J[c], t, err);
                        S[c] = t;
                        C[c] += err;
                        if (MIXED) C[c] += f64_of_f32_any(jc[(2 * c) * PT + e]) + f64_of_f32_any(jc[(2 * c + 1) * PT + e]);
                    }
                }
                double *pp = A.part + (size_t)(diag ? XY.x : XY.y) * 6 * n;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    pp[(size_t)c * n + i] = S[c];
                    pp[(size_t)(3 + c) * n + i] = C[c];
                }
            }
        }
        if (!diag) {                          // j sums of the Y tiles: slot X
            double *pp = A.part + (size_t)XY.x * 6 * n;
            for (int e = threadIdx.x; e < nj; e += kSymT) {
                const int j = b0 * kSymT + e;
                if (j >= n) continue;
                const double J[3] = {jax[e], jay[e], jaz[e]};
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    pp[(size_t)c * n + j] = J[c];
                    pp[(size_t)(3 + c) * n + j] =
                        MIXED ? f64_of_f32_any(jc[(2 * c) * PT + e]) + f64_of_f32_any(jc[(2 * c + 1) * PT + e]) : 0.0;
                }
            }
        }
    }
    if (PC) sym_pc_flush(A, pcb[w], pend, lane);
}

// Folds the chunk partials in chunk order (TwoSum), scales by G and applies the
// kick v += dt_half a; optionally stores a.
__global__ void kick_finalize(const double *part, int nchunk, int tp_first, int tp_slots, int n, double G,
                              double dt_half, double *vel, double *acc_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // symmetric kick with test particles: the bodies of the test-particle
    // super-ranges have partials only from the ranges holding large bodies
    if (i >= tp_first) nchunk = tp_slots;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double S = 0.0, C = 0.0;
        for (int q = 0; q < nchunk; q++) {
            const double *p = part + (size_t)q * 6 * n;
            double t, e;
            two_sum_ordered(S, p[(size_t)c * n + i], t, e);
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

// Symmetric-kick geometry for the system's N and precision: the super-range P
// (0: the symmetric kick is not used), chosen by list-scheduling the items,
// largest first, over the resident blocks and adding the finalize's cost.
namespace {

struct SymPlan {
    int P = 0, nS = 0, blocks = 0;
    int R = 0;                     // super-ranges holding large bodies (TP); nS otherwise
    std::vector<int2> items;
};

double sym_item_cost(int nT, int P, int X, int Y) {
    const int px = std::min(P, nT - X * P), py = std::min(P, nT - Y * P);
    return X == Y ? 0.5 * px * px : (double)px * py;
}

// Items in dispatch order and the predicted makespan (tile-pair units per
// block), each item also costing `ovh` units of fixed work (its tile loads,
// partial-sum writes and dispatch).  Only rows X < Xmax: with test particles,
// a super-range made only of test particles has no pair left with a later one.
double sym_schedule(int nT, int P, int slots, int Xmax, double ovh, std::vector<int2> *order) {
    const int nS = (nT + P - 1) / P;
    std::vector<std::pair<double, int2>> it;
    it.reserve((size_t)nS * (nS + 1) / 2);
    for (int X = 0; X < std::min(nS, Xmax); X++)
        for (int Y = X; Y < nS; Y++) it.push_back({sym_item_cost(nT, P, X, Y), make_int2(X, Y)});
    std::stable_sort(it.begin(), it.end(), [](const std::pair<double, int2> &u, const std::pair<double, int2> &v) {
        return u.first > v.first;
    });
    std::priority_queue<double, std::vector<double>, std::greater<double>> h;
    for (int k = 0; k < slots; k++) h.push(0.0);
    double ms = 0.0;
    for (const auto &e : it) {
        const double t = h.top() + e.first + ovh;
        h.pop();
        h.push(t);
        ms = std::max(ms, t);
    }
    if (order) {
        order->clear();
        for (const auto &e : it) order->push_back(e.second);
    }
    return ms;
}

template <bool MIXED>
SymPlan sym_plan(int n, int nm, int num_sms, int layout, int req_P) {
    SymPlan best;
    const int nT = (n + kSymT - 1) / kSymT;
    // FP64 instructions per unordered pair (symmetric) and per ordered pair
    // (kick_kernel), and per partial slot per body in kick_finalize (15 in its
    // loop; 17 fits the measured fold, which also streams the slots from DRAM)
    const double c_sym = MIXED ? 9.2 : 21.5, c_old = MIXED ? 6.1 : 17.1, c_fin = 17.0;
    // fixed work per item, in FP64-instruction equivalents of one block,
    // fitted to the mixed kick's measured times over P at N = 65,536 and
    // 65,540; the FP64 form's measured times follow the model without it
    const double ovh = MIXED ? 7500.0 / (c_sym * kSymT * kSymT) : 0.0;
    // predicted time in FP64 instructions per SM: kick_kernel at 95 % balance;
    // the symmetric kick's makespan (tile pairs per block, each block at 1/nb
    // of its SM) plus the finalize's slots
    if (layout == GENGA_KICK_TILED) return best;
    // tiled: the large bodies' rows meet every source, the test particles' rows the large ones
    const double t_old = c_old * (2.0 * n * nm - (double)nm * nm) / (0.95 * num_sms);
    double t_best = layout == GENGA_KICK_SYMMETRIC ? 1e300 : t_old;
    for (int P = req_P > 0 ? req_P : 1; P <= (req_P > 0 ? req_P : kSymMaxP); P++) {
        const int nS = (nT + P - 1) / P;
        if ((double)nS * 6.0 * n * sizeof(double) > 16.0 * (1ull << 30)) continue;   // partial sums
        if ((double)nS * (nS + 1) / 2 > 4.0e6) continue;                                // host schedule
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kick_sym_kernel<MIXED, false, false>, kSymT,
                                                          sym_smem(MIXED, P)) != cudaSuccess || nb < 1)
            continue;
        const int slots = nb * num_sms;
        const int R = (nm + P * kSymT - 1) / (P * kSymT);
        const double ms = sym_schedule(nT, P, slots, R, ovh, nullptr);
        const double t = c_sym * (double)kSymT * kSymT * ms * nb + c_fin * (double)nS * n / num_sms;
        if (t < t_best) {
            t_best = t;
            best.P = P; best.nS = nS; best.blocks = slots; best.R = R;
        }
    }
    if (best.P) sym_schedule(nT, best.P, best.blocks, best.R, ovh, &best.items);
    return best;
}

}  // namespace

// Chooses the kick geometry for the current N and precision and makes sure the
// partial-sum and symmetric-kick buffers are large enough.
cudaError_t kick_reserve(genga_system *s) {
    const int n = (int)s->n;
    if (s->kick_chunk == 0) kick_geometry(n, s->num_sms, &s->kick_chunk, &s->kick_nchunk);
    const int prec = s->p.precision;
    const int nm = tp_bound(s);
    if (s->ksym_n != s->n || s->ksym_prec != prec || s->ksym_nm != nm) {
        SymPlan plan = prec == GENGA_MIXED ? sym_plan<true>(n, nm, s->num_sms, s->ksym_layout, s->ksym_req_P)
                                           : sym_plan<false>(n, nm, s->num_sms, s->ksym_layout, s->ksym_req_P);
        s->ksym_P = plan.P;
        s->ksym_nS = plan.nS;
        s->ksym_blocks = plan.blocks;
        s->ksym_items = (int)plan.items.size();
        s->ksym_R = plan.R;
        if (plan.P) {
            if ((size_t)s->ksym_items > s->ksym_list_cap) {
                if (s->ksym_list) cudaFree(s->ksym_list);
                s->ksym_list = nullptr;
                s->ksym_list_cap = 0;
                GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_list, sizeof(int2) * plan.items.size()));
                s->ksym_list_cap = plan.items.size();
            }
            if (!plan.items.empty())
                GENGA_CUDA_TRY(cudaMemcpy(s->ksym_list, plan.items.data(), sizeof(int2) * plan.items.size(),
                                          cudaMemcpyHostToDevice));
            if (!s->ksym_ctr) GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_ctr, sizeof(unsigned)));
            if ((size_t)n > s->ksym_body_cap) {
                if (s->ksym_irc) cudaFree(s->ksym_irc);
                if (s->ksym_mhl) cudaFree(s->ksym_mhl);
                if (s->ksym_thrpc) cudaFree(s->ksym_thrpc);
                if (s->ksym_pcf) cudaFree(s->ksym_pcf);
                if (s->ksym_ircf) cudaFree(s->ksym_ircf);
                s->ksym_irc = nullptr; s->ksym_mhl = nullptr; s->ksym_thrpc = nullptr; s->ksym_pcf = nullptr;
                s->ksym_ircf = nullptr;
                s->ksym_body_cap = 0;
                GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_irc, sizeof(double) * (size_t)n));
                GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_mhl, sizeof(float2) * (size_t)n));
                GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_thrpc, sizeof(float) * (size_t)n));
                GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_pcf, sizeof(float2) * (size_t)n));
                GENGA_CUDA_TRY(cudaMalloc((void **)&s->ksym_ircf, sizeof(float2) * (size_t)n));
                s->ksym_body_cap = (size_t)n;
            }
        }
        s->ksym_n = s->n;
        s->ksym_prec = prec;
        s->ksym_nm = nm;
    }
    const size_t need = (size_t)std::max(s->kick_nchunk, s->ksym_nS) * 6 * (size_t)n;
    if (need > s->kick_part_cap) {
        if (s->kick_part) cudaFree(s->kick_part);
        s->kick_part = nullptr;
        s->kick_part_cap = 0;
        GENGA_CUDA_TRY(cudaMalloc((void **)&s->kick_part, sizeof(double) * need));
        s->kick_part_cap = need;
    }
    return cudaSuccess;
}

cudaError_t launch_kick(genga_system *s, double dt_half, bool precheck, double *acc_out) {
    const int n = (int)s->n;
    GENGA_CUDA_TRY(kick_reserve(s));
    KickArgs A = make_args(s, false);
    const bool mixed = s->p.precision == GENGA_MIXED;
    int nparts = s->kick_nchunk;
    int tp_first = n, tp_slots = 0;               // bodies from tp_first fold tp_slots partials
    if (s->ksym_P > 0) {
        // symmetric layout; the pre-check, if asked for, rides along
        kick_pack_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(s->mass, s->rcl[0].rc, s->rcl[0].pc2, n,
                                                               s->ksym_irc, s->ksym_ircf, s->ksym_mhl,
                                                               s->ksym_thrpc, s->ksym_pcf);
        ++s->launches;
        GENGA_CUDA_TRY(cudaMemsetAsync(s->ksym_ctr, 0, sizeof(unsigned), s->stream));
        if (precheck)
            GENGA_CUDA_TRY(cudaMemsetAsync(&s->ctr->cand_count, 0, sizeof(unsigned long long), s->stream));
        SymArgs S;
        S.x = A.x; S.y = A.y; S.z = A.z; S.m = A.m;
        S.irc = s->ksym_irc; S.ircf = s->ksym_ircf; S.thr = A.thr_rc; S.mhl = s->ksym_mhl;
        S.n = n; S.nT = (n + kSymT - 1) / kSymT; S.P = s->ksym_P; S.nItems = s->ksym_items;
        S.nm = A.nm;
        S.items = s->ksym_list; S.ctr = s->ksym_ctr; S.part = s->kick_part;
        S.pc2 = s->rcl[0].pc2; S.thr_pc = s->ksym_thrpc; S.pcf = s->ksym_pcf;
        S.cand = s->cand; S.cand_count = &s->ctr->cand_count; S.cand_cap = (unsigned long long)s->cand_cap;
        const size_t smem = sym_smem(mixed, s->ksym_P);
        const unsigned nb = (unsigned)s->ksym_blocks;
        const bool tp = A.nm < n;
#define GENGA_SYM_LAUNCH(M, PCK, TPK) kick_sym_kernel<M, PCK, TPK><<<nb, kSymT, smem, s->stream>>>(S)
        if (mixed) {
            if (tp) { if (precheck) GENGA_SYM_LAUNCH(true, true, true); else GENGA_SYM_LAUNCH(true, false, true); }
            else { if (precheck) GENGA_SYM_LAUNCH(true, true, false); else GENGA_SYM_LAUNCH(true, false, false); }
        } else {
            if (tp) { if (precheck) GENGA_SYM_LAUNCH(false, true, true); else GENGA_SYM_LAUNCH(false, false, true); }
            else { if (precheck) GENGA_SYM_LAUNCH(false, true, false); else GENGA_SYM_LAUNCH(false, false, false); }
        }
#undef GENGA_SYM_LAUNCH
        if (tp) {
            tp_first = (int)std::min<int64_t>((int64_t)s->ksym_R * s->ksym_P * kSymT, n);
            tp_slots = s->ksym_R;
        }
        nparts = s->ksym_nS;
    } else {
        if (precheck) GENGA_CUDA_TRY(launch_precheck_only(s));
        dim3 grid((n + kKickThreads - 1) / kKickThreads, s->kick_nchunk);
        if (A.nm < n) {
            if (mixed) kick_kernel<true, true><<<grid, kKickThreads, 0, s->stream>>>(A);
            else kick_kernel<false, true><<<grid, kKickThreads, 0, s->stream>>>(A);
        } else {
            if (mixed) kick_kernel<true, false><<<grid, kKickThreads, 0, s->stream>>>(A);
            else kick_kernel<false, false><<<grid, kKickThreads, 0, s->stream>>>(A);
        }
    }
    ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    kick_finalize<<<(n + 255) / 256, 256, 0, s->stream>>>(s->kick_part, nparts, tp_first, tp_slots, n, s->p.G,
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
    kick_finalize<<<(k.n + 255) / 256, 256, 0, stream>>>(k.part, nchunk, k.n, 0, k.n, k.G, k.dt_half, k.vel,
                                                         k.acc_out);
    return cudaGetLastError();
}

int kick_nchunk_for(int n, int num_sms) {
    int c, nc;
    kick_geometry(n, num_sms, &c, &nc);
    return nc;
}

}  // namespace genga

using namespace genga;

extern "C" int genga_set_kick_layout(genga_system_t *s, int32_t layout, int32_t P) {
    if (!s || layout < GENGA_KICK_AUTO || layout > GENGA_KICK_SYMMETRIC || P < 0 || P > kSymMaxP)
        return GENGA_EINVAL;
    s->ksym_layout = layout;
    s->ksym_req_P = P;
    s->ksym_n = -1;                       // geometry redone by the next kick
    return GENGA_OK;
}

extern "C" int genga_get_kick_layout(genga_system_t *s, int32_t *layout, int32_t *P, int32_t *slots,
                                     int32_t *blocks) {
    if (!s) return GENGA_EINVAL;
    if (kick_reserve(s) != cudaSuccess) return GENGA_ECUDA;
    const bool sym = s->ksym_P > 0;
    if (layout) *layout = sym ? GENGA_KICK_SYMMETRIC : GENGA_KICK_TILED;
    if (P) *P = sym ? s->ksym_P : 0;
    if (slots) *slots = sym ? s->ksym_nS : s->kick_nchunk;
    if (blocks)
        *blocks = sym ? s->ksym_blocks
                      : (int32_t)(((s->n + kKickThreads - 1) / kKickThreads) * (int64_t)s->kick_nchunk);
    return GENGA_OK;
}

