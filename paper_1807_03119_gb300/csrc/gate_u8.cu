// The gate-first kernels (gate.cuh) for 8-bit volumes: one translation unit per
// dtype, so that the two compile in parallel.
#include "gate.cuh"

lnf_status lnf_gate_launch_u8(lnf_ctx *ctx, const FilterJob &j, void *const outs[5], u64 *const hists[5],
                              cudaStream_t st, int *handled, bool eloc, u32 *counter)
{
    return gatek::gate_dispatch_t<uint8_t>(ctx, j, outs, hists, st, handled, eloc, counter);
}
