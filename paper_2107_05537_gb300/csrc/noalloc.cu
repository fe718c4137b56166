// pmlsh_project_noalloc: the query projection of pmlsh_project without any
// device allocation.
//
// Who needs it: callers that cannot let a library call cudaMalloc, e.g. a
// process whose device memory is owned by its own caching allocator (a
// library cudaMalloc could fail or fragment that reservation), or a
// latency-critical serving loop where cudaMalloc's implicit device-wide
// synchronisation would stall work on other streams.
//
// The staging buffer (the query rows padded to the index's row length) lives
// in the file-scope device array below instead of the index's scratch
// buffers.  Every GPU that loads the library holds this array until the
// process exits.
#include <mutex>

#include "pmlsh_impl.h"

// 4,194,304 floats = 16 MiB: nq * (d rounded up to a multiple of 32) must not
// exceed this.
#define PM_NOALLOC_FLOATS (1u << 22)

static __device__ __align__(256) float g_noalloc_rows[PM_NOALLOC_FLOATS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float *g_rows_addr[kMaxDevices] = {};

// Device address of g_noalloc_rows on the current device.  Host code cannot
// use the symbol itself (on the host it names a stand-in, not device memory),
// so the address is looked up once per device, with that device current.
pmlsh_status rows_address(float **out)
{
    int dev = 0;
    PM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        pm_set_error("device ordinal %d beyond the supported %d", dev, kMaxDevices);
        return PMLSH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_rows_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_rows);
        if (e != cudaSuccess || !p) {
            pm_set_error("cudaGetSymbolAddress(g_noalloc_rows) failed: %s", cudaGetErrorString(e));
            return PMLSH_ECUDA;
        }
        g_rows_addr[dev] = (float *)p;
    }
    *out = g_rows_addr[dev];
    return PMLSH_OK;
}
}  // namespace

extern "C" pmlsh_status pmlsh_project_noalloc(const pmlsh_index *ix, const float *Q, int64_t nq,
                                              double *out64, float *out32, void *stream)
{
    if (!ix) {
        pm_set_error("index is NULL");
        return PMLSH_EINVAL;
    }
    if (nq < 0) {
        pm_set_error("nq must be >= 0");
        return PMLSH_EINVAL;
    }
    if (nq == 0) return PMLSH_OK;
    if (!Q || (!out64 && !out32)) {
        pm_set_error("NULL argument");
        return PMLSH_EINVAL;
    }
    if ((uint64_t)nq * (uint64_t)ix->ld > PM_NOALLOC_FLOATS) {
        pm_set_error("nq * padded d = %lld exceeds the no-allocation limit of %u floats "
                     "(at d = %d at most %lld rows per call)",
                     (long long)(nq * ix->ld), PM_NOALLOC_FLOATS, ix->d,
                     (long long)(PM_NOALLOC_FLOATS / (unsigned)ix->ld));
        return PMLSH_EINVAL;
    }
    if ((out64 && !pm_is_device_ptr(out64)) || (out32 && !pm_is_device_ptr(out32))) {
        pm_set_error("outputs must be device memory (no staging buffer can be allocated)");
        return PMLSH_EINVAL;
    }
    float *rows = nullptr;
    PM_TRY(rows_address(&rows));
    cudaStream_t st = (cudaStream_t)stream;
    const int d = ix->d, ld = ix->ld;
    // Every call shares the array, which keeps the previous call's contents:
    // clear the rows this call uses (the padding columns must read as zero),
    // then copy Q in.  Calls that overlap on the GPU race on the array.
    PM_CUDA(cudaMemsetAsync(rows, 0, (size_t)nq * ld * sizeof(float), st));
    PM_CUDA(cudaMemcpy2DAsync(rows, ld * sizeof(float), Q, d * sizeof(float), d * sizeof(float), nq,
                              pm_is_device_ptr(Q) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    pm_launch_project64_noprof(rows, nq, ld, d, ix->m, ix->A32, out64, out32, st, ix->m);
    PM_CUDA(cudaGetLastError());
    return PMLSH_OK;
}
