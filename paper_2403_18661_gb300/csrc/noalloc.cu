// Allocation-free Welch PSD entry point (afg_psd_estimate_noalloc).
//
// For callers that must not call cudaMalloc (see the header for who and
// why): the periodogram scratch the Welch kernels need lives in a file-scope
// __device__ array of fixed size that every GPU loading this library holds
// until the process exits, as does the transforms' twiddle table.  No call
// here allocates or frees device memory.
//
// Host code must not use the array's name as a device address (on the host
// it is a stand-in symbol); the address is looked up once per device with
// cudaGetSymbolAddress in setup() and passed to the kernels.
#include <mutex>

#include "afg_internal.cuh"

namespace {

constexpr int kMaxPeriodograms = AFG_NOALLOC_MAX_PERIODOGRAMS;
constexpr int kMaxDevices = 64;

// periodogram scratch: [n_det][n_seg][NBIN] doubles, n_det * n_seg <= kMaxPeriodograms (4.2 MB)
static __device__ __align__(256) double g_noalloc_periodograms[kMaxPeriodograms * NBIN];

struct DeviceState {
    bool ready = false;
    double *scratch = nullptr;
};

DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: resolve the array's device
// address, fill the FP32 twiddle table if no context has, and opt the
// periodogram kernel into its shared memory (all synchronous, so this must
// not run under stream capture).
int setup(int dev, DeviceState **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &s = g_dev[dev];
    if (!s.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_periodograms) != cudaSuccess) return AFG_ERR_CUDA;
        s.scratch = static_cast<double *>(p);
        if (prepare_psd_kernels() != cudaSuccess) return AFG_ERR_CUDA;
        s.ready = true;
    }
    *out = &s;
    return AFG_OK;
}

}  // namespace

extern "C" int afg_psd_estimate_noalloc(const float *x, int64_t n, int32_t n_det, int64_t n_psd, int64_t psd_step,
                                        int64_t psd_span, int32_t fs, int32_t hop, double *psd, void *stream) {
    if (!x || !psd || fs < 1) return AFG_ERR_ARG;
    int64_t n_seg = 0;
    if (!psd_request_ok(n, n_det, n_psd, psd_step, psd_span, hop, &n_seg)) return AFG_ERR_ARG;
    if (n_seg > kMaxPeriodograms / n_det) return AFG_ERR_BUDGET;  // n_det * n_seg > the scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AFG_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DeviceState *s = nullptr;
    int rc = setup(dev, &s);
    if (rc != AFG_OK) return rc;
    // every periodogram the mean reads is written earlier in the same call,
    // so the scratch needs no clearing between calls
    if (launch_psd_on(x, n, n_det, n_psd, psd_step, psd_span, hop, fs, s->scratch, psd, st) !=
        cudaSuccess)
        return AFG_ERR_CUDA;
    return AFG_OK;
}
