// encounter.cu -- close-encounter detection, pair compaction and grouping
// (Appendix A "close-encounter detection", "grouping", "groupS"; Sec. 2).
//
//  * detect: one thread per candidate pair; a pair is an encounter when its
//    squared distance before or after the drift is below rc_ij^2 (exact FP64,
//    fixed operation order); survivors are appended with one atomic per warp
//    (ballot + popc prefix).
//  * CSR: partner lists of a pair list in both directions (degree count,
//    exclusive scan, atomic fill, per-row insertion sort -> ascending lists,
//    so every later sum over partners runs in a fixed order: Serial Grouping,
//    Appendix B).
//  * level bodies (groupS): bodies with at least one partner, compacted in
//    ascending order by a scan over flags.
//  * grouping: union-find with atomicCAS hooking of the larger root under the
//    smaller one, so every component's root is its smallest member whatever
//    the order of the races; then group sizes, a scan for offsets and member
//    slots.
#include "common.cuh"

namespace genga {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

// ---------------------------------------------------------------- scan
// Exclusive scan of int32 in blocks of kScanBlock, then a scan of block sums,
// then the block offsets are added.  out has len+1 entries (out[len] = total).
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;   // inclusive
    }
    __syncthreads();
    const int before = (warp > 0) ? warp_sums[warp - 1] : 0;
    total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------- detection
// Encounter <=> r_ij^2 < max(rc_i^2, rc_j^2) before (pre-drift state) or after
// the drift, the exact FP64 test in the defining operation order (dist2_rn).
// Most candidates are decided in FP32 from float copies of the positions
// (round to nearest): the float distance differs from r by at most
// m_ij = sqrt(3) 2^-23 (max|x_i| + max|x_j|) plus relative rounding, so
// r_f >= R (1 + 2^-20) + m_ij is surely outside and r_f < R (1 - 2^-20) - m_ij
// surely inside (R = rc_ij in FP32, squared comparisons with a further
// 1 +- 2^-20); only the band between takes the exact test.  Encounters are
// compacted with a block-wide scan and one global atomic per block.
__device__ __forceinline__ int detect_state(const double *p, size_t N, int i, int j, float Rf) {
    constexpr float kM = 1.7320509f * 1.1920929e-07f;    // sqrt(3) 2^-23
    constexpr float kUp = 1.0f + 9.5367432e-07f, kDn = 1.0f - 9.5367432e-07f;
    const float xi = f32_of_f64_rn(p[i]), yi = f32_of_f64_rn(p[N + i]), zi = f32_of_f64_rn(p[2 * N + i]);
    const float xj = f32_of_f64_rn(p[j]), yj = f32_of_f64_rn(p[N + j]), zj = f32_of_f64_rn(p[2 * N + j]);
    const float m = kM * (fmaxf(fabsf(xi), fmaxf(fabsf(yi), fabsf(zi))) +
                          fmaxf(fabsf(xj), fmaxf(fabsf(yj), fabsf(zj))));
    const float dx = xj - xi, dy = yj - yi, dz = zj - zi;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float to = fmaf(Rf, kUp, m);
    if (r2 >= to * to * kUp) return 0;                   // surely outside
    const float ti = fmaf(Rf, kDn, -m);
    if (ti > 0.0f && r2 < ti * ti * kDn) return 1;       // surely inside
    return 2;                                            // exact test
}

__global__ void detect_kernel(const uint2 *in, const unsigned long long *nin_dev, long long nin_host,
                              int n, const double *pre, const double *post, const double *rc2,
                              uint2 *out, unsigned long long cap, unsigned long long *count) {
    __shared__ int warp_sums[32];
    __shared__ unsigned long long base;
    const long long nin = nin_dev ? (long long)*nin_dev : nin_host;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool enc = false;
    uint2 pr = make_uint2(0, 0);
    if (k < nin) {
        pr = in[k];
        const int i = (int)pr.x, j = (int)pr.y;
        const size_t N = (size_t)n;
        const double lim = fmax(rc2[i], rc2[j]);
        const float Rf = sqrtf(f32_of_f64_rn(lim));
        const int s0 = detect_state(pre, N, i, j, Rf);
        const int s1 = s0 == 1 ? 1 : detect_state(post, N, i, j, Rf);
        enc = s0 == 1 || s1 == 1;
        if (!enc && s0 == 2)
            enc = dist2_rn(pre[j] - pre[i], pre[N + j] - pre[N + i], pre[2 * N + j] - pre[2 * N + i]) < lim;
        if (!enc && s1 == 2)
            enc = dist2_rn(post[j] - post[i], post[N + j] - post[N + i], post[2 * N + j] - post[2 * N + i]) < lim;
    }
    int total = 0;
    const int pos = block_exclusive_scan(enc ? 1 : 0, warp_sums, total);
    if (total == 0) return;                               // uniform across the block
    if (threadIdx.x == 0) base = atomicAdd(count, (unsigned long long)total);
    __syncthreads();
    if (enc) {
        const unsigned long long idx = base + (unsigned long long)pos;
        if (idx < cap) out[idx] = pr;
    }
}

__global__ void __launch_bounds__(kScanThreads)
scan_blocks_kernel(const int *in, int *out, long long len, int *block_sums) {
    __shared__ int ws[32];
    const long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int local = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
        v[q] = (base + q < len) ? in[base + q] : 0;
        local += v[q];
    }
    int total;
    int ex = block_exclusive_scan(local, ws, total);
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
        if (base + q < len) out[base + q] = ex;
        ex += v[q];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_sums_kernel(int *block_sums, int nblocks, int *total_out) {
    __shared__ int ws[32];
    int running = 0;
    for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int b = b0 + threadIdx.x;
        const int v = (b < nblocks) ? block_sums[b] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, ws, tot);
        if (b < nblocks) block_sums[b] = running + ex;
        running += tot;
    }
    if (threadIdx.x == 0) *total_out = running;
}

__global__ void scan_add_kernel(int *out, long long len, const int *block_sums) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < len) out[k] += block_sums[k / kScanBlock];
}

// ---------------------------------------------------------------- CSR
// Pairs in a list: np, or the count the detection left on the device (npd,
// at most np, the bound the grid was sized for) when the host has not read it.
__device__ __forceinline__ long long pairs_in(long long np, const unsigned long long *npd) {
    return npd ? min(np, (long long)*npd) : np;
}

// The pair kernels stride over the list, so that a grid sized for a bound
// (the count on the device) stays small.
__global__ void csr_degree_kernel(const uint2 *pairs, long long np, const unsigned long long *npd, int *deg,
                                  unsigned long long *total) {
    const long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    np = pairs_in(np, npd);
    if (total && k0 == 0) *total += (unsigned long long)np;
    for (long long k = k0; k < np; k += stride) {
        const uint2 p = pairs[k];
        atomicAdd(&deg[p.x], 1);
        atomicAdd(&deg[p.y], 1);
    }
}

__global__ void csr_fill_kernel(const uint2 *pairs, long long np, const unsigned long long *npd, const int *off,
                                int *fill, int *list, int *lpair) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    np = pairs_in(np, npd);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride) {
        const uint2 p = pairs[k];
        const int a = off[p.x] + atomicAdd(&fill[p.x], 1);
        list[a] = (int)p.y;
        lpair[a] = (int)(2 * k);
        const int b = off[p.y] + atomicAdd(&fill[p.y], 1);
        list[b] = (int)p.x;
        lpair[b] = (int)(2 * k + 1);
    }
}

// Sorts every row by partner index, carrying the pair index along.  Sparse
// lists (most rows empty or short, as at the higher levels): one thread per
// row, insertion sort.  Dense lists: one warp per row; a row of up to kSortMax
// entries is held in registers (lane k takes entries k, k + 32, ...), each
// entry's rank is the number of smaller keys in the row (the partners of a row
// are distinct, so the ranks are a permutation and the result is the sorted
// row), and the entries are written to their ranks; longer rows take the
// insertion sort on one lane.  Both give the same sorted rows, and both record
// where each pair direction 2 k + d ended up (ent), so that per-pair results can
// be written straight to their entries and read row by row.
__global__ void csr_sort_rows_kernel(int n, const int *off, int *list, int *lpair, int *ent) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int s = off[b], e = off[b + 1];
    for (int u = s + 1; u < e; u++) {
        const int key = list[u], kp = lpair[u];
        int w = u - 1;
        while (w >= s && list[w] > key) { list[w + 1] = list[w]; lpair[w + 1] = lpair[w]; w--; }
        list[w + 1] = key;
        lpair[w + 1] = kp;
    }
    for (int u = s; u < e; u++) ent[lpair[u]] = u;
}

constexpr int kSortPer = 8;
constexpr int kSortMax = 32 * kSortPer;

__global__ void csr_sort_warp_kernel(int n, const int *off, int *list, int *lpair, int *ent) {
    const int b = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= n) return;                                   // whole warps leave together
    const int s = off[b], e = off[b + 1], L = e - s;
    if (L == 0) return;
    if (L == 1) {
        if (lane == 0) ent[lpair[s]] = s;
        return;
    }
    if (L > kSortMax) {
        if (lane == 0)
            for (int u = s + 1; u < e; u++) {
                const int key = list[u], kp = lpair[u];
                int w = u - 1;
                while (w >= s && list[w] > key) { list[w + 1] = list[w]; lpair[w + 1] = lpair[w]; w--; }
                list[w + 1] = key;
                lpair[w + 1] = kp;
            }
        __syncwarp();
        for (int u = s + lane; u < e; u += 32) ent[lpair[u]] = u;
        return;
    }
    int key[kSortPer], kp[kSortPer], rank[kSortPer];
#pragma unroll
    for (int c = 0; c < kSortPer; c++) {
        const int u = c * 32 + lane;
        key[c] = u < L ? list[s + u] : 0x7fffffff;
        kp[c] = u < L ? lpair[s + u] : 0;
        rank[c] = 0;
    }
#pragma unroll
    for (int c2 = 0; c2 < kSortPer; c2++) {
        if (c2 * 32 >= L) break;                          // warp-uniform
        for (int k = 0; k < 32; k++) {
            const int other = __shfl_sync(0xffffffffu, key[c2], k);
#pragma unroll
            for (int c = 0; c < kSortPer; c++) rank[c] += other < key[c] ? 1 : 0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < kSortPer; c++) {
        const int u = c * 32 + lane;
        if (u < L) {
            list[s + rank[c]] = key[c];
            lpair[s + rank[c]] = kp[c];
            ent[kp[c]] = s + rank[c];
        }
    }
}

__global__ void flag_nonzero_kernel(int n, const int *deg, int *flags) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) flags[b] = deg[b] > 0 ? 1 : 0;
}

__global__ void compact_kernel(int n, const int *flags, const int *pos, int *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n && flags[b]) out[pos[b]] = b;
}

// ---------------------------------------------------------------- grouping
__device__ __forceinline__ int uf_find(const int *parent, int a) {
    // parent pointers only ever decrease, so the chain is finite
    int p = __ldcg(parent + a);
    while (p != a) { a = p; p = __ldcg(parent + a); }
    return a;
}

__global__ void uf_init_kernel(int n, int *parent) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) parent[b] = b;
}

// Joins the sets of one pair's bodies (bounded retries); false if it gave up.
__device__ bool uf_hook_pair(int *parent, uint2 p) {
    for (int it = 0; it < (1 << 20); it++) {
        const int ru = uf_find(parent, (int)p.x);
        const int rv = uf_find(parent, (int)p.y);
        if (ru == rv) return true;
        const int lo = min(ru, rv), hi = max(ru, rv);
        if (atomicCAS(&parent[hi], hi, lo) == hi) return true;
    }
    return false;
}

__global__ void uf_hook_kernel(const uint2 *pairs, long long np, const unsigned long long *npd, int *parent,
                               DevCounters *ctr) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    np = pairs_in(np, npd);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += stride)
        if (!uf_hook_pair(parent, pairs[k])) latch_error(ctr, kErrUnionFind);
}

__global__ void uf_label_kernel(int n, const int *parent, const int *deg, int *label, int *gsize) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    if (deg[b] > 0) {
        const int r = uf_find(parent, b);
        label[b] = r;
        atomicAdd(&gsize[r], 1);
    } else {
        label[b] = -1;
    }
}

__global__ void group_members_kernel(int n, const int *label, const int *goff, int *gfill,
                                     int *member, int *slotof, DevCounters *ctr) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int g = label[b];
    if (g < 0) return;
    const int slot = goff[g] + atomicAdd(&gfill[g], 1);
    member[slot] = b;
    slotof[b] = slot;
    if (g == b) {
        const unsigned sz = (unsigned)(goff[g + 1] - goff[g]);
        atomicAdd(&ctr->ngroups, 1u);
        atomicMax(&ctr->max_group, sz);
        atomicAdd(&ctr->groups_total, 1ull);
        atomicMax(&ctr->max_group_total, (unsigned long long)sz);
    }
}

}  // namespace

cudaError_t exclusive_scan(genga_system *s, const int *in, int *out, int64_t len) {
    const int nblocks = (int)((len + kScanBlock - 1) / kScanBlock);
    if (nblocks > s->scr.scan_blocks_cap) return cudaErrorInvalidValue;
    if (len > 0) {
        scan_blocks_kernel<<<nblocks, kScanThreads, 0, s->stream>>>(in, out, len, s->scr.scan_blocks); ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
    }
    scan_sums_kernel<<<1, kScanThreads, 0, s->stream>>>(s->scr.scan_blocks, nblocks, out + len); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    if (len > 0) {
        scan_add_kernel<<<(unsigned)((len + 255) / 256), 256, 0, s->stream>>>(out, len, s->scr.scan_blocks); ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

cudaError_t launch_detect(genga_system *s, const uint2 *in, int64_t nin, int level, uint2 *out,
                          int64_t cap, unsigned long long *count) {
    GENGA_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s->stream));
    if (nin <= 0) return cudaSuccess;
    detect_kernel<<<(unsigned)((nin + 255) / 256), 256, 0, s->stream>>>(in, nullptr, nin, (int)s->n,
        s->pre_pos[level], s->pos, s->rcl[level].rc2, out, (unsigned long long)cap, count); ++s->launches;
    return cudaGetLastError();
}

// Blocks of 256 for a pair kernel over np pairs (a bound when the count is on
// the device: then at most a few per SM, the kernels striding).
static unsigned pair_grid(const genga_system *s, int64_t np, const unsigned long long *npd) {
    const long long g = (np + 255) / 256;
    return (unsigned)(npd ? std::min<long long>(g, 4LL * s->num_sms) : g);
}

cudaError_t build_csr(genga_system *s, int level, int64_t np, const unsigned long long *npd,
                      unsigned long long *total, int64_t np_hint) {
    const int n = (int)s->n;
    Csr &c = s->csr[level];
    GENGA_CUDA_TRY(cudaMemsetAsync(c.deg, 0, sizeof(int) * (n + 1), s->stream));
    GENGA_CUDA_TRY(cudaMemsetAsync(c.fill, 0, sizeof(int) * n, s->stream));
    if (np > 0) {
        csr_degree_kernel<<<pair_grid(s, np, npd), 256, 0, s->stream>>>(s->pairs[level], np, npd, c.deg,
                                                                         total); ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
    }
    GENGA_CUDA_TRY(exclusive_scan(s, c.deg, c.off, n));
    if (np > 0) {
        csr_fill_kernel<<<pair_grid(s, np, npd), 256, 0, s->stream>>>(s->pairs[level], np, npd, c.off, c.fill,
                                                                       c.list, c.lpair); ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
        // dense: a warp per row (with the count on the device, judged by a
        // recent count of the same level; both sorts give the same rows)
        if (2 * (npd ? np_hint : np) >= n)
            csr_sort_warp_kernel<<<(unsigned)(((long long)n * 32 + 255) / 256), 256, 0, s->stream>>>(
                n, c.off, c.list, c.lpair, c.ent);
        else
            csr_sort_rows_kernel<<<(n + 127) / 128, 128, 0, s->stream>>>(n, c.off, c.list, c.lpair, c.ent);
        ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

// Bodies with a partner in the pair list of `level_pairs`, ascending, into
// s->bodies[out_level]; the count is returned through a synchronising copy.
cudaError_t build_bodies(genga_system *s, int level_pairs, int out_level, int *nb_host) {
    const int n = (int)s->n;
    int *pos = s->gfill;   // temporary n+1 ints
    flag_nonzero_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->csr[level_pairs].deg, s->flags); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    GENGA_CUDA_TRY(exclusive_scan(s, s->flags, pos, n));
    compact_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->flags, pos, s->bodies[out_level]); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    GENGA_CUDA_TRY(cudaMemcpyAsync(nb_host, pos + n, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    ++s->host_syncs;
    return cudaStreamSynchronize(s->stream);
}

// Connected components of the pair list of `level` (its CSR must be built).
__global__ void bucket_groups_kernel(const DevCounters *ctr, const int *glist, const int *goff, int stride,
                                     int *blist, unsigned *bcount) {
    const unsigned ng = ctr->ngroups;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < ng; q += gridDim.x * blockDim.x) {
        const int g = glist[q];
        const int sz = goff[g + 1] - goff[g];
        const int b = sz <= 4 ? 0 : sz <= 8 ? 1 : sz <= 16 ? 2 : sz <= kBlockGroupMax ? 3 : 4;
        const unsigned k = atomicAdd(&bcount[b], 1u);
        blist[(size_t)b * stride + k] = g;
    }
}

static_assert(offsetof(DevCounters, bucket_next) == offsetof(DevCounters, bucket_count) + 8 * sizeof(unsigned) &&
                  offsetof(DevCounters, pad3) == offsetof(DevCounters, bucket_next) + kBuckets * sizeof(unsigned),
              "bucket counts and claim counters must be contiguous");

cudaError_t bucket_groups_async(genga_system *s) {
    // the counts and the BS kernels' claim counters
    GENGA_CUDA_TRY(cudaMemsetAsync(s->ctr->bucket_count, 0, 16 * sizeof(unsigned), s->stream));
    bucket_groups_kernel<<<2 * s->num_sms, 256, 0, s->stream>>>(s->ctr, s->glist, s->goff, s->bucket_stride,
                                                               s->bucket_list, s->ctr->bucket_count);
    ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    GENGA_CUDA_TRY(cudaMemcpyAsync(s->bucket_host, s->ctr->bucket_count, sizeof(unsigned) * kBuckets,
                                   cudaMemcpyDeviceToHost, s->stream));
    return cudaEventRecord(s->ev_counts, s->stream);
}

cudaError_t bucket_groups(genga_system *s, unsigned counts[kBuckets]) {
    GENGA_CUDA_TRY(bucket_groups_async(s));
    GENGA_CUDA_TRY(cudaEventSynchronize(s->ev_counts));
    ++s->host_syncs;
    for (int q = 0; q < kBuckets; q++) counts[q] = s->bucket_host[q];
    return cudaSuccess;
}

cudaError_t build_groups(genga_system *s, int level, int64_t np, const unsigned long long *npd) {
    const int n = (int)s->n;
    GENGA_CUDA_TRY(cudaMemsetAsync(s->gsize, 0, sizeof(int) * (n + 1), s->stream));
    GENGA_CUDA_TRY(cudaMemsetAsync(s->gfill, 0, sizeof(int) * (n + 1), s->stream));
    GENGA_CUDA_TRY(cudaMemsetAsync(&s->ctr->ngroups, 0, 2 * sizeof(unsigned), s->stream));
    uf_init_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->parent); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    if (np > 0) {
        uf_hook_kernel<<<pair_grid(s, np, npd), 256, 0, s->stream>>>(s->pairs[level], np, npd, s->parent,
                                                                      s->ctr); ++s->launches;
        GENGA_CUDA_TRY(cudaGetLastError());
    }
    uf_label_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->parent, s->csr[level].deg, s->label, s->gsize); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    GENGA_CUDA_TRY(exclusive_scan(s, s->gsize, s->goff, n));
    // group list: labels with a non-empty group, ascending
    flag_nonzero_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->gsize, s->flags); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    int *pos = s->member;   // temporary, rewritten below
    GENGA_CUDA_TRY(exclusive_scan(s, s->flags, pos, n));
    compact_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->flags, pos, s->glist); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    group_members_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(n, s->label, s->goff, s->gfill,
                                                                 s->member, s->slotof, s->ctr); ++s->launches;
    GENGA_CUDA_TRY(cudaGetLastError());
    s->label_level = level;
    return cudaSuccess;
}

}  // namespace genga
