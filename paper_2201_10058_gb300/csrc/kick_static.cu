// kick_static.cu -- the changeover kick for callers that cannot allocate
// device memory.
//
// Who needs it: code that must not call cudaMalloc -- for example a caller
// whose framework's caching allocator already holds the device's free memory
// (a cudaMalloc would fail or fragment its pool), or a caller on a latency-
// critical loop where cudaMalloc/cudaFree would stall every stream of the
// device.  genga_create allocates per-system scratch; this entry point instead
// keeps its scratch in one file-scope device array of fixed size that lives as
// long as the library is loaded (every GPU that loads the library holds it).
//
// Scratch layout (doubles): rc^2 [n], FP32 thresholds [n floats], then the
// kick's per-chunk partial sums [nchunk][6][n], nchunk reduced as needed to fit.
#include <mutex>

#include "common.cuh"

namespace genga {
namespace {

constexpr size_t kStaticDoubles = size_t(1) << 21;   // 16 MiB
static __device__ __align__(256) double g_kick_static_scratch[kStaticDoubles];

std::mutex g_setup_mutex;
double *g_scratch_addr[256] = {};   // device address of the array, per device ordinal

__global__ void static_thresholds_kernel(int n, const double *rc, double *rc2, float *thr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r2 = __dmul_rn(rc[i], rc[i]);
    rc2[i] = r2;
    thr[i] = fmaxf(__double2float_ru(r2) * 1.0000153f, 1.17549435e-38f);
}

}  // namespace
}  // namespace genga

using namespace genga;

extern "C" int genga_kick_static(int64_t n, const double *pos, const double *mass, const double *rc,
                                 double G, double dt_half, int precision, double *vel,
                                 double *acc_out, void *stream) {
    if (n < 1 || !pos || !mass || !rc || (!vel && dt_half != 0.0)) return GENGA_EINVAL;
    if (precision != GENGA_FP64 && precision != GENGA_MIXED) return GENGA_EINVAL;
    if (n > GENGA_KICK_STATIC_MAX_N) return GENGA_ECAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return GENGA_ECUDA;
    double *base = nullptr;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_kick_static_scratch) != cudaSuccess || !p) return GENGA_ECUDA;
            g_scratch_addr[dev] = (double *)p;
        }
        base = g_scratch_addr[dev];
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GENGA_ECUDA;
    const size_t N = (size_t)n;
    double *rc2 = base;
    float *thr = (float *)(base + N);
    const size_t part_off = ((N + (N + 1) / 2) + 31) / 32 * 32;   // 256-byte aligned
    double *part = base + part_off;
    const size_t room = kStaticDoubles - part_off;
    const int max_nchunk = (int)(room / (6 * N));
    if (max_nchunk < 1) return GENGA_ECAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    static_thresholds_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>((int)n, rc, rc2, thr);
    if (cudaGetLastError() != cudaSuccess) return GENGA_ECUDA;
    KickRaw k;
    k.pos = pos; k.mass = mass; k.rc = rc; k.rc2 = rc2; k.thr = thr; k.part = part;
    k.n = (int)n; k.G = G; k.dt_half = dt_half; k.vel = vel; k.acc_out = acc_out;
    k.mixed = precision == GENGA_MIXED;
    if (launch_kick_raw(k, sms, max_nchunk, st) != cudaSuccess) return GENGA_ECUDA;
    return GENGA_OK;
}
