// The gate-first kernels (gate.cuh) for 16-bit volumes, and the entry points the
// rest of the library calls.
#include "gate.cuh"

lnf_status lnf_gate_launch_u8(lnf_ctx *ctx, const FilterJob &j, void *const outs[5], u64 *const hists[5],
                              cudaStream_t st, int *handled, bool eloc, u32 *counter);

bool lnf_gate_covers(const FilterJob &j, int filter)
{
    const bool whole = !(j.ox || j.oy || j.oz || j.bx != j.nx || j.by != j.ny || j.bz != j.nz);
    // the entropy filter with local probabilities at r = 1..2 (the generic kernel,
    // launched beside it with the job marked gated, does the work when many pass)
    if (filter == LNF_ENTROPY_LOCAL)
        return whole && !j.aniso && j.radius >= 1 && j.radius <= 2;
    // the five filters only where a ring kernel with the matching early return
    // exists (it does the work when many voxels pass)
    return whole && !j.aniso && filter >= LNF_MEAN && filter <= LNF_OURS && j.radius >= 1 && j.radius <= 4 &&
           lnf_fast_covers(filter, j.radius, j.offset);
}

lnf_status lnf_gate_launch(lnf_ctx *ctx, const FilterJob &j, void *const outs[5], u64 *const hists[5],
                           cudaStream_t st, int *handled, u32 *counter)
{
    *handled = 0;
    for (int f = 0; f < 5; ++f)
        if (outs[f] && !lnf_gate_covers(j, f))
            return lnf_fail(ctx, LNF_EINVAL, "gate-first kernel: filter %d not covered", f);
    // the kernels read the caller's dense volume (not a row-padded copy of it)
    FilterJob jd = j;
    if (j.orig) {
        jd.in = j.orig;
        jd.pitch = j.nx;
    }
    if (j.dtype == LNF_U8)
        return lnf_gate_launch_u8(ctx, jd, outs, hists, st, handled, false, counter);
    return gatek::gate_dispatch_t<uint16_t>(ctx, jd, outs, hists, st, handled, false, counter);
}

lnf_status lnf_gate_launch_eloc(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, int *handled)
{
    *handled = 0;
    if (!lnf_gate_covers(j, LNF_ENTROPY_LOCAL))
        return lnf_fail(ctx, LNF_EINVAL, "gate-first kernel: local entropy job not covered");
    void *outs[5] = {nullptr, nullptr, j.out, nullptr, nullptr};
    u64 *hists[5] = {nullptr, nullptr, j.out_hist, nullptr, nullptr};
    FilterJob jd = j;
    if (j.orig) {
        jd.in = j.orig;
        jd.pitch = j.nx;
    }
    if (j.dtype == LNF_U8)
        return lnf_gate_launch_u8(ctx, jd, outs, hists, st, handled, true, nullptr);
    return gatek::gate_dispatch_t<uint16_t>(ctx, jd, outs, hists, st, handled, true);
}
