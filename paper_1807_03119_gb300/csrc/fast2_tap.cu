// The tap kernels of fast2.cuh: sigma (Eq. 5) and Okada (Eq. 6); and the
// dispatch of the four comparison filters to the specialised kernels.
#include "fast2.cuh"

// Route mean / sigma / entropy / Okada jobs on TMA-able volumes (whole or a
// region of interest) at radius 1..4 (sigma 1..2) to the specialised kernels.
lnf_status lnf_fast2_dispatch(lnf_ctx *ctx, const FilterJob &job, const CUtensorMap *tmap, cudaStream_t stream,
                              int *handled, u32 *counter)
{
    *handled = 0;
    if (!tmap || job.filter == LNF_OURS || !lnf_fast_covers(job.filter, job.radius, job.offset))
        return LNF_OK;
    const bool u8 = job.dtype == LNF_U8;
    switch (job.filter) {
    case LNF_MEAN:
    case LNF_ENTROPY: return lnf_fast2_box(ctx, job, stream, counter, handled);
    case LNF_SIGMA: return u8 ? by_radius<uint8_t, LNF_SIGMA>(ctx, job, stream, counter, handled)
                              : by_radius<uint16_t, LNF_SIGMA>(ctx, job, stream, counter, handled);
    case LNF_OKADA: return u8 ? by_radius<uint8_t, LNF_OKADA>(ctx, job, stream, counter, handled)
                              : by_radius<uint16_t, LNF_OKADA>(ctx, job, stream, counter, handled);
    default: return LNF_OK;
    }
}
