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
#include <cuda.h>
#include <mutex>

#include "common.cuh"

namespace genga {
namespace {

constexpr size_t kStaticDoubles = size_t(1) << 21;   // 16 MiB
static __device__ __align__(256) double g_kick_static_scratch[kStaticDoubles];

std::mutex g_setup_mutex;
// device address of the array per device ordinal, with the id of the context
// it was looked up in: cudaDeviceReset destroys the device's primary context,
// the next call creates a new one (new id) and the library's device code is
// loaded again, possibly at another address -- so a changed id means set-up
// again
struct ScratchAddr {
    double *addr;
    unsigned long long ctx;
};
ScratchAddr g_scratch[256] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the current context (driver entry points looked up through the
// runtime, so the library does not link the driver library); 0 when unknown.
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

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
        // set-up once per device (and again after a device reset), with that
        // device current
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        const unsigned long long id = current_ctx_id();
        if (!g_scratch[dev].addr || id == 0 || id != g_scratch[dev].ctx) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_kick_static_scratch) != cudaSuccess || !p) return GENGA_ECUDA;
            g_scratch[dev].addr = (double *)p;
            g_scratch[dev].ctx = current_ctx_id();   // the look-up made the context current
        }
        base = g_scratch[dev].addr;
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
