// pa_static.cu -- pa_copy_numbers_static: the copy numbers of one resampling step computed
// without any caller-provided workspace.
//
// Why it exists: pa_resample needs a workspace buffer from the caller.  Some callers have no
// way to provide one: code that may only touch the arrays it was handed (a plugin running
// inside another program's memory pool, or a process that fixes its device memory at start-up
// and forbids any later cudaMalloc so that memory use never changes while it runs).  This
// entry point serves them: the caller passes only the parents' energy levels (input) and the
// copy-number array (output); the level histogram, the per-level tables and the block sums
// live in one file-scope device array of fixed size, g_static_scratch below.
//
// The array is part of the library image, so every GPU that loads the library holds its
// kStaticScratchBytes until the process exits.  Host code cannot use the array's name as a
// device address (on the host it is only a stand-in symbol); every call looks up its device
// address with cudaGetSymbolAddress on the current device (a lookup, not an allocation), so an
// address never outlives the context it came from (e.g. across cudaDeviceReset).  The first
// call on a device may load the library's code onto it, so that first call should come before
// any stream capture.  The stream passed must belong to the current device.
// All calls share the one array: each call clears the state and histogram it relies on, and
// two calls whose kernels overlap on the GPU (e.g. on two streams) race on it.
//
// The kernels are the library's own level-table, copy-number and prefix-sum kernels; only the
// location of their scratch differs.  Nothing here allocates device memory.
#include <cmath>

#include "pa_common.cuh"
#include "pa_kernels.h"

namespace pa {
namespace {

constexpr int kStaticMaxL = 128;
constexpr int kStaticMaxLevels = kStaticMaxL * kStaticMaxL + 1;
constexpr long long kStaticMaxParents = 1LL << 22;
constexpr long long kStaticMaxBlocks = kStaticMaxParents / kCountBlockItems;

constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffState = 0;
constexpr size_t kOffHist = a256(kOffState + sizeof(DevState));
constexpr size_t kOffFl = a256(kOffHist + (size_t)kStaticMaxLevels * 4);
constexpr size_t kOffThr = a256(kOffFl + (size_t)kStaticMaxLevels * 4);
constexpr size_t kOffTau = a256(kOffThr + (size_t)kStaticMaxLevels * 4);
constexpr size_t kOffW = a256(kOffTau + (size_t)kStaticMaxLevels * 8);
constexpr size_t kOffBlock = a256(kOffW + (size_t)kStaticMaxLevels * 8);
constexpr size_t kStaticScratchBytes = a256(kOffBlock + (size_t)kStaticMaxBlocks * 8);  // 493,056 bytes

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch in the current device's context.  Looked up on every
// call: after a cudaDeviceReset the array lives in a new context, possibly at another address.
cudaError_t scratch_for_current_device(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    *out = p;
    return cudaSuccess;
}

// True if `s` is a stream of the current device (the legacy and per-thread default streams
// always are).
bool stream_on_current_device(cudaStream_t s)
{
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return true;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return false;
    return sdev == dev;
}

// Level histogram of the caller's parents; a level outside [0, N] is reported, not used.
__global__ void k_static_levels(const int *level, long long R, int N, int *hist, DevState *st)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < R;
         j += (long long)gridDim.x * blockDim.x) {
        const int k = level[j];
        if (k < 0 || k > N) set_error(st, PA_ERR_INVALID_ARG);
        else atomicAdd(&hist[k], 1);
    }
}

bool static_supported_L(int L) { return L >= 4 && L <= 128 && (L % 2) == 0; }

}  // namespace
}  // namespace pa

extern "C" pa_status pa_copy_numbers_static(int L, long long R_target, long long R_prev, const int *level_dev,
                                            double beta_prev, double beta_new, unsigned int step,
                                            unsigned long long seed, int kind, int *counts_dev,
                                            double *lnQ_out, long long *R_new_out, void *stream)
{
    using namespace pa;
    if (!static_supported_L(L) || R_target < 1 || R_target > 2147483647LL || R_prev < 1 || !level_dev ||
        !counts_dev || !lnQ_out || !R_new_out || (kind != PA_RESAMPLE_NEAREST && kind != PA_RESAMPLE_POISSON) ||
        !std::isfinite(beta_prev) || !std::isfinite(beta_new) || beta_new < beta_prev)
        return PA_ERR_INVALID_ARG;
    if (R_prev > kStaticMaxParents) return PA_ERR_TOO_LARGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!stream_on_current_device(s)) return PA_ERR_INVALID_ARG;
    void *base = nullptr;
    if (scratch_for_current_device(&base) != cudaSuccess) return PA_ERR_CUDA;
    unsigned char *b = static_cast<unsigned char *>(base);
    DevState *st = reinterpret_cast<DevState *>(b + kOffState);
    int *hist = reinterpret_cast<int *>(b + kOffHist);
    const int N = L * L;

    // clears the state block and the histogram, and sets R_{i-1} = R_prev
    cudaError_t e = launch_setup(st, R_prev, hist, N, PA_UPDATE_METROPOLIS, s);
    if (e != cudaSuccess) return PA_ERR_CUDA;
    const unsigned int blocks = (unsigned int)((R_prev + 255) / 256 < 4096 ? (R_prev + 255) / 256 : 4096);
    k_static_levels<<<blocks, 256, 0, s>>>(level_dev, R_prev, N, hist, st);
    if (cudaGetLastError() != cudaSuccess) return PA_ERR_CUDA;

    ResampleArgs a{};
    a.L = L;
    a.kind = kind;
    a.R_target = R_target;
    a.capacity = 2147483647LL;
    a.beta_prev = beta_prev;
    a.beta_new = beta_new;
    a.step = step;
    a.k0 = (unsigned int)(seed & 0xffffffffu);
    a.k1 = (unsigned int)(seed >> 32);
    a.st = st;
    a.hist = hist;
    a.fl = reinterpret_cast<int *>(b + kOffFl);
    a.thr = reinterpret_cast<unsigned int *>(b + kOffThr);
    a.tau = reinterpret_cast<double *>(b + kOffTau);
    a.w = reinterpret_cast<double *>(b + kOffW);
    a.counts = counts_dev;
    a.blocksum = reinterpret_cast<long long *>(b + kOffBlock);
    a.nblk = (R_prev + kCountBlockItems - 1) / kCountBlockItems;
    a.level_src = level_dev;
    if (launch_copy_numbers(a, s) != cudaSuccess) return PA_ERR_CUDA;

    DevState host{};
    if (cudaMemcpyAsync(&host, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PA_ERR_CUDA;
    if (host.error) return (pa_status)host.error;
    *lnQ_out = host.lnQ;
    *R_new_out = host.R_cur;
    return PA_OK;
}
