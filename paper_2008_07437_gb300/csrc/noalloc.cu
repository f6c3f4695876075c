// geo_loglik_noalloc: the Eq. 1 evaluation of geo_loglik for small problems,
// for callers that cannot allocate device memory.
//
// Who cannot allocate, and why: a caller whose device memory is entirely
// owned by another allocator (for example a host application or framework
// that reserved the GPU's memory pool up front, so a cudaMalloc from this
// library would fail or fragment that pool), and a caller on a
// latency-critical path that cannot afford cudaMalloc / cudaFree, which can
// synchronise the device and fail at unpredictable times.  Such callers pass
// only their inputs and outputs; every intermediate lives in one fixed-size
// array in device global memory, declared below, that the library owns.
//
// Scratch: one file-scope __device__ array of GEO_NOALLOC_SCRATCH_DOUBLES
// doubles (about 34 MB), present on every GPU that loads the library until
// the process exits.  It holds the matrix (order N = p*n <= GEO_NOALLOC_MAX_N,
// leading dimension round_up(N + 1, 32), the extra row carrying Z / L^-1 Z),
// the locations in SoA form (caller's order), the K_nu tables of theta and
// the status words.  In host code the array's name is
// only a host-side stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached;
// that look-up happens during the first call on each device, which should
// therefore come before any stream capture.  Every call shares the array and
// it keeps the last call's contents: the status words are cleared at the start
// of each call, everything else is overwritten before it is read.  Calls whose
// work overlaps on the GPU (other streams, other host threads) race on the
// array and must be serialised by the caller.  The cached address belongs to
// the device's primary context as it was at the look-up: calling again after
// cudaDeviceReset on that device is not supported.
//
// The entry point reuses the kernels of geo_loglik unchanged, in the caller's
// location order (no Morton reordering: the ordering needs a host buffer, and
// Eq. 1 does not depend on the order).
#include <mutex>

#include "geo_internal.cuh"

namespace {

constexpr long long kLdMax = ((GEO_NOALLOC_MAX_N + 1 + 31) / 32) * 32;
constexpr long long kMatDoubles = kLdMax * GEO_NOALLOC_MAX_N;
constexpr long long kLocDoubles = 2LL * GEO_NOALLOC_MAX_N;
constexpr long long kTabDoubles = GEO_TAB_DOUBLES;
constexpr long long kStatusDoubles = (sizeof(DevStatus) + sizeof(double) - 1) / sizeof(double);
constexpr long long kScratchDoubles = kMatDoubles + kLocDoubles + kTabDoubles + kStatusDoubles;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// The call has no context that could switch devices: every buffer must be
// device (or managed) memory of the current device.  A pointer of another GPU
// or plain host memory is refused before anything is enqueued.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

static_assert(kScratchDoubles == GEO_NOALLOC_SCRATCH_DOUBLES, "scratch size in geo.h out of date");

extern "C" int geo_loglik_noalloc(const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                                  int nb, double *out_dev, int *info_dev, void *stream) {
    if (n <= 0 || !locs_dev || !z_dev || !out_dev || !theta) return GEO_EINVAL;
    if (theta->p < 1 || theta->p > GEO_PMAX) return GEO_EINVAL;
    if ((long long)theta->p * n > GEO_NOALLOC_MAX_N) return GEO_ESCRATCH;
    if (nb < 64) return GEO_EINVAL;
    CovParams cp;
    std::string err;
    if (theta_to_params(theta, &cp, &err) != GEO_OK) return GEO_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GEO_ECUDA;
    }
    if (!on_device(locs_dev, dev) || !on_device(z_dev, dev) || !on_device(out_dev, dev) ||
        (info_dev && !on_device(info_dev, dev)))
        return GEO_EINVAL;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return GEO_ECUDA;
    }
    const int N = theta->p * n;
    const long long ld = ((long long)(N + 1) + 31) / 32 * 32;
    double *A = scratch;
    double *lx = scratch + kMatDoubles;
    double *ly = lx + n;
    double *tab = scratch + kMatDoubles + kLocDoubles;
    DevStatus *st = (DevStatus *)(scratch + kMatDoubles + kLocDoubles + kTabDoubles);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s)) ||
        (e = launch_gather_locs(locs_dev, nullptr, n, lx, ly, s)) ||
        (e = launch_gather_vec(z_dev, nullptr, n, theta->p, A + N, ld, s)) ||
        (e = launch_cheb_build(cp, tab, s)) ||
        (e = launch_covgen_sym(cp, lx, ly, n, A, ld, s)) ||
        (e = chol64_factor(A, ld, N, N + 1, nb, st, s)) ||
        (e = launch_loglik_reduce(A, ld, N, A + N, ld, st, (DevResults *)out_dev, s))) {
        return GEO_ECUDA;
    }
    if (info_dev) {
        e = cudaMemcpyAsync(info_dev, &st->info, sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return GEO_ECUDA;
    }
    return GEO_OK;
}
