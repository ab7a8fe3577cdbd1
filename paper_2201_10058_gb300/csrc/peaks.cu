// peaks.cu -- issue-rate probe of the arithmetic pipes that bound the kernels
// of this library: FP64 fused multiply-add, add and multiply (the all-pairs
// kick, the Kepler drift and Bulirsch-Stoer are FP64-pipe bound on GB300),
// FP32 fused multiply-add and the MUFU reciprocal square root (the mixed
// kick's seed).
//
// One block of 1024 threads per SM; every thread runs 8 independent chains of
// the probed instruction (inline PTX, so none is folded away), and the block's
// thread 0 reads the SM cycle counter before and after, between barriers.  The
// host adds the work of the blocks that ran on each SM and divides by that SM's
// cycle span: thread-level operations per clock per SM, independent of the
// clock frequency.  A second probe (fp64_chain_kernel) times a chain of
// dependent FP64 FMAs in one warp, and in one thread, alone on the device: the
// cost of an instruction on the critical path of a latency-bound kernel.
#include <vector>

#include "common.cuh"

namespace genga {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;

struct ProbeRec {
    long long start, end;
    unsigned smid;
    unsigned pad;
};

__device__ __forceinline__ unsigned sm_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) pipe_probe_kernel(int iters, double seed, ProbeRec *rec,
                                                                  double *sink) {
    double d[kChains];
    float f[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) {
        d[k] = seed + 1e-3 * (threadIdx.x + k);
        f[k] = (float)d[k];
    }
    const double db = 0.999999, dc = 1e-7;
    const float fb = 0.999999f, fc = 1e-7f;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) {
            if (KIND == 0) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[k]) : "d"(db), "d"(dc));
            if (KIND == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d[k]) : "d"(dc));
            if (KIND == 2) asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(d[k]) : "d"(db));
            if (KIND == 3) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(fb), "f"(fc));
            if (KIND == 4) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[k]));
        }
    }
    __syncthreads();
    long long t1 = clock64();
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) acc += d[k] + (double)f[k];
    if (acc == 12345.678) sink[threadIdx.x] = acc;     // keeps the chains live
    if (threadIdx.x == 0) {
        rec[blockIdx.x].start = t0;
        rec[blockIdx.x].end = t1;
        rec[blockIdx.x].smid = sm_id();
    }
}

template <int KIND>
cudaError_t probe(int sms, int iters, double *rate, std::vector<ProbeRec> &h, ProbeRec *drec, double *sink) {
    pipe_probe_kernel<KIND><<<sms, kProbeThreads>>>(iters, 1.0, drec, sink);
    GENGA_CUDA_TRY(cudaGetLastError());
    GENGA_CUDA_TRY(cudaMemcpy(h.data(), drec, sizeof(ProbeRec) * h.size(), cudaMemcpyDeviceToHost));
    // per SM: all its blocks' operations over the span from the first start
    // to the last end on that SM
    std::vector<long long> lo(4096, -1), hi(4096, -1);
    std::vector<double> ops(4096, 0.0);
    for (const ProbeRec &r : h) {
        const unsigned m = r.smid & 4095u;
        if (lo[m] < 0 || r.start < lo[m]) lo[m] = r.start;
        if (hi[m] < 0 || r.end > hi[m]) hi[m] = r.end;
        ops[m] += (double)kProbeThreads * kChains * iters;
    }
    double sum = 0.0;
    int cnt = 0;
    for (int m = 0; m < 4096; m++)
        if (lo[m] >= 0 && hi[m] > lo[m]) { sum += ops[m] / (double)(hi[m] - lo[m]); cnt++; }
    *rate = cnt ? sum / cnt : 0.0;
    return cudaSuccess;
}

// Latency of a chain of dependent FP64 FMAs in a warp that is alone on its SM
// (one block of `threads` threads): SM cycles per instruction of the chain.
__global__ void fp64_chain_kernel(int iters, double seed, long long *cycles, double *sink) {
    double d = seed + 1e-3 * threadIdx.x;
    const double b = 0.999999, c = 1e-7;
    __syncwarp();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 16; k++) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d) : "d"(b), "d"(c));
    }
    const long long t1 = clock64();
    if (d == 12345.678) sink[threadIdx.x] = d;
    if (threadIdx.x == 0) *cycles = t1 - t0;
}

}  // namespace
}  // namespace genga

using namespace genga;

extern "C" int genga_measure_fp64_latency(double *warp_cycles, double *lane_cycles) {
    long long *dc = nullptr;
    double *sink = nullptr;
    if (cudaMalloc(&dc, sizeof(long long)) != cudaSuccess) return GENGA_ENOMEM;
    if (cudaMalloc(&sink, sizeof(double) * 32) != cudaSuccess) {
        cudaFree(dc);
        return GENGA_ENOMEM;
    }
    const int iters = 4096;
    double r[2] = {0.0, 0.0};
    cudaError_t e = cudaSuccess;
    const int threads[2] = {32, 1};
    for (int q = 0; q < 2 && e == cudaSuccess; q++) {
        long long cyc = 0;
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {       // the first launch warms up
            fp64_chain_kernel<<<1, threads[q]>>>(iters, 1.0, dc, sink);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(&cyc, dc, sizeof(cyc), cudaMemcpyDeviceToHost);
        }
        r[q] = (double)cyc / (16.0 * iters);
    }
    cudaFree(dc);
    cudaFree(sink);
    if (e != cudaSuccess) return GENGA_ECUDA;
    if (warp_cycles) *warp_cycles = r[0];
    if (lane_cycles) *lane_cycles = r[1];
    return GENGA_OK;
}

extern "C" int genga_measure_pipe_rates(double *dfma, double *dadd, double *dmul, double *ffma,
                                        double *mufu_rsqrt) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return GENGA_ECUDA;
    ProbeRec *drec = nullptr;
    double *sink = nullptr;
    if (cudaMalloc(&drec, sizeof(ProbeRec) * sms) != cudaSuccess) return GENGA_ENOMEM;
    if (cudaMalloc(&sink, sizeof(double) * kProbeThreads) != cudaSuccess) {
        cudaFree(drec);
        return GENGA_ENOMEM;
    }
    std::vector<ProbeRec> h((size_t)sms);
    double r[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    // warm-up launch, then the measured ones (each a few ms)
    if (e == cudaSuccess) e = probe<0>(sms, 256, &r[0], h, drec, sink);
    if (e == cudaSuccess) e = probe<0>(sms, 4096, &r[0], h, drec, sink);
    if (e == cudaSuccess) e = probe<1>(sms, 4096, &r[1], h, drec, sink);
    if (e == cudaSuccess) e = probe<2>(sms, 4096, &r[2], h, drec, sink);
    if (e == cudaSuccess) e = probe<3>(sms, 65536, &r[3], h, drec, sink);
    if (e == cudaSuccess) e = probe<4>(sms, 16384, &r[4], h, drec, sink);
    cudaFree(drec);
    cudaFree(sink);
    if (e != cudaSuccess) return GENGA_ECUDA;
    if (dfma) *dfma = r[0];
    if (dadd) *dadd = r[1];
    if (dmul) *dmul = r[2];
    if (ffma) *ffma = r[3];
    if (mufu_rsqrt) *mufu_rsqrt = r[4];
    return GENGA_OK;
}
