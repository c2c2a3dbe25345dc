// bf_noalloc.cu -- bf_errnorm_noalloc: the accuracy report of bf_errnorm for
// callers that cannot allocate device memory.
//
// Who needs it: a per-TTI real-time loop (one slot every 0.5 ms) must not call
// cudaMalloc or cudaFree, which can synchronise the whole device and take an
// unbounded time; neither can code running where another allocator owns all of
// the process's device memory, or code that has no plan at hand. This entry
// point needs no plan and allocates nothing: its scratch (the per-block
// partial sums and the two totals) is a file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "bf.h"
#include "bf_plan.h"
#include "bf_prep.h"

namespace {

constexpr int MAX_DEVICES = 64;

// Scratch shared by every call: 2 doubles per block, then the 2 totals.
static __device__ __align__(256) double g_errnorm_scratch[2 * BF_ERRNORM_NOALLOC_MAX_BLOCKS + 2];

// Per-device SM count for the grid (an attribute of the device ordinal, which
// no reset or context change alters).
int g_sms[MAX_DEVICES];
std::mutex g_mu;

}  // namespace

extern "C" bf_status bf_errnorm_noalloc(const void *R_dev, const void *Rref_dev, int64_t n_blocks,
                                        double *total_host, void *stream) {
    if (!total_host) return bf_fail(nullptr, BF_EINVAL, "total_host is NULL");
    if (n_blocks < 0 || n_blocks > BF_ERRNORM_NOALLOC_MAX_BLOCKS)
        return bf_fail(nullptr, BF_EINVAL, "n_blocks = %lld is outside [0, %d], the size of the fixed scratch",
                       (long long)n_blocks, BF_ERRNORM_NOALLOC_MAX_BLOCKS);
    if (n_blocks > 0 && (!R_dev || !Rref_dev)) return bf_fail(nullptr, BF_EINVAL, "NULL R_dev or Rref_dev");
    if (((uintptr_t)R_dev & 15u) || ((uintptr_t)Rref_dev & 15u))
        return bf_fail(nullptr, BF_EINVAL, "R_dev and Rref_dev must be 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return bf_fail(nullptr, BF_ECUDA, "device ordinal %d out of range", dev);
    // The array's device address, looked up on every call for the current
    // device and context (in host code the symbol is only a host-side stand-in):
    // a cached address would outlive a cudaDeviceReset or belong to another
    // context. The first lookup on a device may load the library's device code,
    // so make the first call before any stream capture.
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_errnorm_scratch);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_sms[dev] == 0) {
            e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) {
                g_sms[dev] = 0;
                return bf_fail(nullptr, BF_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
            }
        }
        sms = g_sms[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Nothing needs clearing: the kernels write every per-block pair they later
    // read, and the totals, before anything reads them.
    double *per_block = static_cast<double *>(p);
    double *total = per_block + 2 * BF_ERRNORM_NOALLOC_MAX_BLOCKS;
    e = bfi::launch_errnorm((const float2 *)R_dev, (const double2 *)Rref_dev, n_blocks, per_block, total,
                            sms * 8, s);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "error-norm launch: %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(total_host, total, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bf_fail(nullptr, BF_ECUDA, "copying the totals: %s", cudaGetErrorString(e));
    return BF_OK;
}
