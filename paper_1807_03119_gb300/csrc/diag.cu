// Failure-detection self-test: a wait that can never complete must give up
// after its limit, record the failure in a device status word and return,
// leaving the context usable.  The probe waits on a shared-memory mbarrier
// that expects one arrival nobody makes, through the same bounded wait
// (mbar_wait_bounded) that every filter kernel uses on its TMA barriers; no
// trap, no assert, no bad address, no unbounded loop.
#include "lnf_ctx.h"

#include <chrono>

namespace {

__global__ void k_wait_probe(u32 *status, u64 limit_ns)
{
    using namespace lnfdev;
    __shared__ __align__(8) u64 bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival completes the phase; none comes
        fence_mbar_init();
        mbar_wait_bounded(&bar, 0u, status, limit_ns);
    }
}

}  // namespace

extern "C" lnf_status lnf_selftest_wait(lnf_ctx *ctx, double limit_ms, double *elapsed_ms)
{
    LNF_RANGE("lnf_selftest_wait");
    if (!ctx)
        return LNF_EINVAL;
    if (!(limit_ms > 0.0) || limit_ms > 2000.0)
        return lnf_fail(ctx, LNF_EINVAL, "limit %g ms not in (0, 2000]", limit_ms);
    u32 *status = ctx->d_counter + 15;   // the self-test's own status word
    cudaStream_t st = ctx->stream;
    if (cudaMemsetAsync(status, 0, sizeof(u32), st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "self-test: status reset failed");
    const auto t0 = std::chrono::steady_clock::now();
    k_wait_probe<<<1, 32, 0, st>>>(status, (u64)(limit_ms * 1e6));
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "self-test: launch failed");
    u32 h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "self-test: synchronisation failed");
    if (elapsed_ms)
        *elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (h & LNF_DERR_TIMEOUT)
        return lnf_fail(ctx, LNF_ETIMEOUT, "self-test: the bounded wait gave up as designed");
    return LNF_OK;
}
