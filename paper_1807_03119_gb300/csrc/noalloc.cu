// lnf_entropy_noalloc: the image entropy of a volume without any allocation.
//
// Who needs this: code that must not call cudaMalloc / cudaFree at the point
// where it measures entropy -- for example a render or acquisition loop that
// cannot afford the device-wide synchronisation those calls can cause, code
// running while another component holds all of the GPU's free memory in its
// own pool, or a plugin that has no lnf_ctx (creating one allocates scratch).
// Such callers pass their own input and output buffers; the only scratch is
// the file-scope device array below, which exists once per GPU that loads the
// library and lives until the process exits.
//
// Set-up: the first call on each device, with that device current, looks up
// the array's device address with cudaGetSymbolAddress (host code cannot use
// the array's name as a device address) and caches it, and makes CUDA load
// all four kernels of this file (cudaFuncGetAttributes on each).  With lazy
// module loading, CUDA's default, a kernel is otherwise loaded -- which can
// allocate device memory -- the first time it is launched, so a later first
// call with the other dtype could still load code.  Make that first call
// before any stream capture.  The cached address does not survive a
// cudaDeviceReset of that device (the process would need to restart).
//
// A CUDA error left pending by the caller's earlier work is reported as
// LNF_ECUDA before anything is enqueued and is left in place (not cleared), so
// that it is not mistaken for a failure of this call's own launches.
//
// Every call reuses the same array and zeroes it first; two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and both results are then undefined.  Order such calls on one stream.
#include "lnf.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

typedef unsigned int u32;
typedef unsigned long long u64;

constexpr int kNoAllocBins = 65536;          // one counter per 16-bit grey level
constexpr int kShBins = 8192;                 // per-CTA shared sub-histogram (values below this)
constexpr int kThreads = 512;
constexpr int kMaxDevices = 64;

// 256 KiB of counters: the whole scratch of this entry point.
static __device__ __align__(256) u32 g_noalloc_hist[kNoAllocBins];

std::mutex g_mu;
u32 *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

__global__ void k_clear(u32 *h)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNoAllocBins; i += gridDim.x * blockDim.x)
        h[i] = 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_count(const T *vol, u64 n, u32 *h)
{
    __shared__ u32 sh[kShBins];
    for (int i = threadIdx.x; i < kShBins; i += blockDim.x)
        sh[i] = 0;
    __syncthreads();
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const u32 v = vol[i];
        if (v < (u32)kShBins)
            atomicAdd(&sh[v], 1u);
        else
            atomicAdd(&h[v], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kShBins; i += blockDim.x)
        if (sh[i])
            atomicAdd(&h[i], sh[i]);
}

__global__ void __launch_bounds__(1024) k_reduce(const u32 *h, int levels, u64 n, double *H)
{
    __shared__ double sd[1024];
    double acc = 0.0;
    const double N = (double)n;
    for (int v = threadIdx.x; v < levels; v += blockDim.x)
        if (h[v]) {
            const double p = (double)h[v] / N;
            acc += -p * log2(p);
        }
    sd[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            sd[threadIdx.x] += sd[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *H = sd[0];
}

}  // namespace

extern "C" lnf_status lnf_entropy_noalloc(const void *vol, const int64_t dims[3], int dtype, double *d_entropy,
                                          void *stream)
{
    if (!vol || !dims || !d_entropy || (dtype != LNF_U8 && dtype != LNF_U16))
        return LNF_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1)
            return LNF_EINVAL;
    // the counters are 32-bit: at most 2^32 - 1 voxels
    const unsigned __int128 n128 = (unsigned __int128)dims[0] * dims[1] * dims[2];
    if (n128 > 0xFFFFFFFFull)
        return LNF_EINVAL;
    const u64 n = (u64)n128;
    // an error pending from earlier work is the caller's: report it, leave it set
    if (cudaPeekAtLastError() != cudaSuccess)
        return LNF_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return LNF_ECUDA;
    u32 *h = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_hist) != cudaSuccess || !p)
                return LNF_ECUDA;
            int s = 0;
            if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s < 1)
                s = 1;
            // load every kernel now, so that no later call loads code
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, k_clear) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, k_count<uint8_t>) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, k_count<uint16_t>) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, k_reduce) != cudaSuccess)
                return LNF_ECUDA;
            g_sms[dev] = s;
            g_addr[dev] = static_cast<u32 *>(p);
        }
        h = g_addr[dev];
        sms = g_sms[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_clear<<<64, 256, 0, st>>>(h);
    u64 want = (n + kThreads * 16ull - 1) / (kThreads * 16ull);
    const int grid = (int)(want < (u64)(4 * sms) ? (want ? want : 1) : 4 * sms);
    if (dtype == LNF_U8)
        k_count<uint8_t><<<grid, kThreads, 0, st>>>(static_cast<const uint8_t *>(vol), n, h);
    else
        k_count<uint16_t><<<grid, kThreads, 0, st>>>(static_cast<const uint16_t *>(vol), n, h);
    k_reduce<<<1, 1024, 0, st>>>(h, dtype == LNF_U8 ? 256 : kNoAllocBins, n, d_entropy);
    return cudaGetLastError() == cudaSuccess ? LNF_OK : LNF_ECUDA;
}
