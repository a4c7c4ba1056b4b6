// The box kernels of fast2.cuh: mean (Eq. 4) and entropy filter (Eq. 7).
#include "fast2.cuh"

lnf_status lnf_fast2_box(lnf_ctx *ctx, const FilterJob &job, cudaStream_t stream, u32 *counter, int *handled)
{
    const bool u8 = job.dtype == LNF_U8;
    if (job.filter == LNF_MEAN)
        return u8 ? by_radius<uint8_t, LNF_MEAN>(ctx, job, stream, counter, handled)
                  : by_radius<uint16_t, LNF_MEAN>(ctx, job, stream, counter, handled);
    return u8 ? by_radius<uint8_t, LNF_ENTROPY>(ctx, job, stream, counter, handled)
              : by_radius<uint16_t, LNF_ENTROPY>(ctx, job, stream, counter, handled);
}
