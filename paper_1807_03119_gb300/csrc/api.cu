// Host side of liblnf: the C ABI of include/lnf.h (plain, multi-filter, ROI,
// entropy and batched entry points).  The serving loop lives in serve.cu.
//
// Every step of the filter path runs on the device: statistics (stats.cu),
// parameter derivation (stats.cu, one CTA), filters (filter.cu, fast.cu) and
// the entropy reduction.  The host only validates arguments, encodes TMA
// descriptors, packs job descriptors into kernel parameters and enqueues.
#include "lnf_ctx.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

// ------------------------------------------------------------------ errors

lnf_status lnf_fail(lnf_ctx *ctx, lnf_status s, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> g(ctx->err_mu);
        ctx->err = buf;
    }
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return lnf_fail(ctx, LNF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));             \
    } while (0)

// ------------------------------------------------------------------ validation

lnf_status lnf_check_volume(lnf_ctx *ctx, const void *p, const int64_t dims[3], int dtype)
{
    if (!p)
        return lnf_fail(ctx, LNF_EINVAL, "null volume pointer");
    if (!dims)
        return lnf_fail(ctx, LNF_EINVAL, "null dims");
    if (dtype != LNF_U8 && dtype != LNF_U16)
        return lnf_fail(ctx, LNF_EINVAL, "dtype must be LNF_U8 or LNF_U16 (got %d)", dtype);
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1 || dims[i] > (1ll << 30))
            return lnf_fail(ctx, LNF_EINVAL, "dims[%d] = %lld out of range [1, 2^30]", i, (long long)dims[i]);
    const unsigned __int128 n = (unsigned __int128)dims[0] * dims[1] * dims[2];
    if (n >= ((unsigned __int128)1 << 32))
        return lnf_fail(ctx, LNF_EINVAL, "volume has %llu voxels; the limit is 2^32 - 1",
                        (unsigned long long)n);
    return LNF_OK;
}

bool lnf_fault_parse(const char *spec, FaultPlan &plan)
{
    static const char *const names[FAULT_NSITES] = {"scratch", "resident", "output", "stage", "launch"};
    if (!spec)
        return true;
    const char *p = spec;
    while (*p) {
        const char *end = p;
        while (*end && *end != ',')
            ++end;
        const char *at = p;
        while (at < end && *at != '@')
            ++at;
        int site = -1;
        for (int i = 0; i < FAULT_NSITES; ++i)
            if ((size_t)(at - p) == std::strlen(names[i]) && std::strncmp(p, names[i], at - p) == 0)
                site = i;
        if (site < 0 && at > p)
            return false;
        int64_t n = -1;
        if (at < end) {
            n = 0;
            for (const char *c = at + 1; c < end; ++c) {
                if (*c < '0' || *c > '9' || n > (1ll << 40))
                    return false;
                n = n * 10 + (*c - '0');
            }
            if (n < 1)
                return false;
        }
        if (site >= 0)
            plan.nth[site] = n;
        p = *end ? end + 1 : end;
    }
    return true;
}

static lnf_status check_filter(lnf_ctx *ctx, int filter_id, int radius)
{
    if (filter_id < LNF_MEAN || filter_id > LNF_ENTROPY_LOCAL)
        return lnf_fail(ctx, LNF_EINVAL, "filter_id %d not in 0..8", filter_id);
    if (radius < 0 || radius > LNF_MAX_RADIUS)
        return lnf_fail(ctx, LNF_EINVAL, "radius %d not in 0..%d", radius, LNF_MAX_RADIUS);
    return LNF_OK;
}

static bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

static size_t esize(int dtype) { return dtype == LNF_U8 ? 1 : 2; }

static u64 nvox(const int64_t d[3]) { return (u64)d[0] * (u64)d[1] * (u64)d[2]; }

// ------------------------------------------------------------------ config

extern "C" void lnf_config_default(lnf_config *cfg)
{
    if (!cfg)
        return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->stream = nullptr;
    cfg->hbm_budget_bytes = 40ull << 30;
    cfg->max_inflight = 64;
    cfg->threshold_mode = LNF_THRESH_OTSU;
    cfg->threshold_value = 0;
    cfg->sigma_k = 2;
    cfg->okada_td = LNF_TD_AUTO;
    cfg->entropy_te_q = LNF_TE_AUTO;
    cfg->cluster_offset = 1;
    cfg->autotune = 0;
    cfg->entropy_local_te_q = LNF_TE_AUTO;
}

ParamCfg lnf_param_cfg(const lnf_ctx *ctx)
{
    const lnf_config &c = ctx->cfg;
    ParamCfg p;
    std::memset(&p, 0, sizeof p);
    p.threshold_mode = c.threshold_mode;
    p.threshold_value = c.threshold_value;
    p.sigma_k = c.sigma_k;
    p.okada_td = c.okada_td;
    p.entropy_te = c.entropy_te_q;
    p.entropy_local_te = c.entropy_local_te_q;
    p.lt = ctx->d_lt;
    return p;
}

static lnf_status alloc_scratch(lnf_ctx *ctx, VolScratch &vs)
{
    if (lnf_fault(ctx, FAULT_SCRATCH))
        return lnf_fail(ctx, LNF_ENOMEM, "injected fault: scratch allocation failed");
    CK(cudaMalloc(&vs.hist, sizeof(u64) * LNF_LEVELS_U16));
    CK(cudaMalloc(&vs.st, sizeof(DevStats)));
    CK(cudaMalloc(&vs.prm, sizeof(DevParams)));
    CK(cudaMalloc(&vs.lut, sizeof(u32) * LNF_LEVELS_U16));
    CK(cudaMalloc(&vs.pscr, lnf_param_scratch_bytes()));
    CK(cudaMemset(vs.prm, 0, sizeof(DevParams)));
    CK(cudaMemset(vs.pscr, 0, lnf_param_scratch_bytes()));
    return LNF_OK;
}

static void free_scratch(VolScratch &vs)
{
    cudaFree(vs.hist);
    cudaFree(vs.st);
    cudaFree(vs.prm);
    cudaFree(vs.lut);
    cudaFree(vs.pscr);
    vs = VolScratch{};
}

lnf_status lnf_scratch_pool(lnf_ctx *ctx, size_t n)
{
    while (ctx->pool.size() < n) {
        VolScratch vs{};
        lnf_status s = alloc_scratch(ctx, vs);
        if (s != LNF_OK) {
            free_scratch(vs);
            return s;
        }
        ctx->pool.push_back(vs);
    }
    return LNF_OK;
}

static void prof_clear(lnf_ctx *ctx);

extern "C" lnf_status lnf_create(const lnf_config *cfg_in, lnf_ctx **out)
{
    LNF_RANGE("lnf_create");
    if (!out)
        return LNF_EINVAL;
    *out = nullptr;
    lnf_config cfg;
    if (cfg_in)
        cfg = *cfg_in;
    else
        lnf_config_default(&cfg);
    if (cfg.threshold_mode < 0 || cfg.threshold_mode > 2 || cfg.sigma_k < 0 || cfg.sigma_k > 255 ||
        cfg.cluster_offset < 0 || cfg.cluster_offset > 8 || cfg.okada_td < LNF_TD_AUTO ||
        cfg.entropy_te_q < LNF_TE_AUTO || cfg.entropy_local_te_q < LNF_TE_AUTO)
        return LNF_EINVAL;
    if (cfg.hbm_budget_bytes == 0)
        cfg.hbm_budget_bytes = 40ull << 30;
    if (cfg.max_inflight <= 0)
        cfg.max_inflight = 64;
    FaultPlan plan;
    if (!lnf_fault_parse(getenv("LNF_FAULT"), plan))
        return LNF_EINVAL;
    lnf_ctx *ctx = new (std::nothrow) lnf_ctx();
    if (!ctx)
        return LNF_ENOMEM;
    ctx->cfg = cfg;
    for (int i = 0; i < FAULT_NSITES; ++i)
        ctx->fault.nth[i] = plan.nth[i];
    ctx->stream = static_cast<cudaStream_t>(cfg.stream);
    lnf_status s = LNF_OK;
    do {
        if (cudaGetDevice(&ctx->device) != cudaSuccess) {
            s = LNF_ECUDA;
            break;
        }
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (ctx->num_sms < 1)
            ctx->num_sms = 1;
        if ((s = alloc_scratch(ctx, ctx->vs)) != LNF_OK)
            break;
        if (cudaMalloc(&ctx->out_hist, sizeof(u64) * LNF_LEVELS_U16 * LNF_MAX_PACK) != cudaSuccess ||
            cudaMalloc(&ctx->d_H, sizeof(double) * (LNF_MAX_PACK + 1)) != cudaSuccess ||
            cudaMalloc(&ctx->d_err, sizeof(u32)) != cudaSuccess ||
            cudaMalloc(&ctx->d_counter, sizeof(u32) * 16) != cudaSuccess ||
            cudaMalloc(&ctx->d_ent_part, sizeof(double) * LNF_ENT_SPLIT * LNF_MAX_ENT) != cudaSuccess ||
            cudaMalloc(&ctx->d_ent_done, sizeof(u32) * LNF_MAX_ENT) != cudaSuccess ||
            cudaMalloc(&ctx->d_range, sizeof(u32) * 4) != cudaSuccess) {
            s = LNF_ENOMEM;
            break;
        }
        if ((s = lnf_lt_upload(ctx)) != LNF_OK)
            break;
        cudaMemset(ctx->d_err, 0, sizeof(u32));
        cudaMemset(ctx->d_counter, 0, sizeof(u32) * 16);
        cudaMemset(ctx->d_ent_done, 0, sizeof(u32) * LNF_MAX_ENT);
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            ctx->encode = reinterpret_cast<PFN_encodeTiled>(fn);
        // test hooks: force the plain-load path / the generic kernel / the ring
        // kernels alone (no gate-first kernels)
        const char *ev = getenv("LNF_FORCE_PLAIN");
        ctx->no_tma = ev && ev[0] == '1';
        ev = getenv("LNF_FORCE_GENERIC");
        ctx->no_fast = ev && ev[0] == '1';
        ev = getenv("LNF_NO_GATE");
        ctx->no_gate = ev && ev[0] == '1';
        // test hook: the plane-ring kernels' work-item z length (planes per item)
        ev = getenv("LNF_FAST_ZLEN");
        if (ev && atoi(ev) >= 1 && atoi(ev) <= 1024)
            ctx->fast_zlen = atoi(ev);

        if (cudaDeviceSynchronize() != cudaSuccess)
            s = LNF_ECUDA;
    } while (0);
    if (s != LNF_OK) {
        lnf_destroy(ctx);
        return s;
    }
    *out = ctx;
    return LNF_OK;
}

extern "C" void lnf_destroy(lnf_ctx *ctx)
{
    if (!ctx)
        return;
    lnf_serve_shutdown(ctx);
    cudaStreamSynchronize(ctx->stream);
    lnf_batch_cache_clear(ctx);
    lnf_batch_streams_free(ctx);
    free_scratch(ctx->vs);
    for (auto &vs : ctx->pool)
        free_scratch(vs);
    prof_clear(ctx);
    for (cudaEvent_t e : ctx->prof_free)
        cudaEventDestroy(e);
    cudaFree(ctx->out_hist);
    cudaFree(ctx->d_H);
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_counter);
    cudaFree(ctx->pitched);
    cudaFree(ctx->f32_lv);
    cudaFree(ctx->d_range);
    cudaFree(ctx->d_lt);
    for (cudaEvent_t e : ctx->filter_done)
        cudaEventDestroy(e);
    if (ctx->copy_stream)
        cudaStreamDestroy(ctx->copy_stream);
    cudaFree(ctx->d_ent_part);
    cudaFree(ctx->d_ent_done);
    cudaFree(ctx->st_in);
    for (void *p : ctx->st_out)
        cudaFree(p);
    delete ctx;
}

extern "C" lnf_status lnf_set_stream(lnf_ctx *ctx, void *stream)
{
    if (!ctx)
        return LNF_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->cfg.stream = stream;
    return LNF_OK;
}

extern "C" const char *lnf_last_error(lnf_ctx *ctx)
{
    if (!ctx)
        return "null context";
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->err_copy = ctx->err;
    return ctx->err_copy.c_str();
}

extern "C" const char *lnf_version(void) { return "lnf 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ profiling

static cudaEvent_t prof_event(lnf_ctx *ctx)
{
    if (!ctx->prof_free.empty()) {
        cudaEvent_t e = ctx->prof_free.back();
        ctx->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int lnf_prof_begin(lnf_ctx *ctx, cudaStream_t st)
{
    if (!ctx->prof)
        return -1;
    lnf_ctx::ProfRec r;
    r.a = prof_event(ctx);
    r.b = prof_event(ctx);
    cudaEventRecord(r.a, st);
    ctx->prof_recs.push_back(r);
    return (int)ctx->prof_recs.size() - 1;
}

void lnf_prof_end(lnf_ctx *ctx, int rec, const char *name, cudaStream_t st, int count)
{
    ctx->prof_launches += count;
    if (rec < 0)
        return;
    ctx->prof_recs[rec].name = name;
    cudaEventRecord(ctx->prof_recs[rec].b, st);
}

static void prof_clear(lnf_ctx *ctx)
{
    for (auto &r : ctx->prof_recs) {
        ctx->prof_free.push_back(r.a);
        ctx->prof_free.push_back(r.b);
    }
    ctx->prof_recs.clear();
    ctx->prof_launches = 0;
}

extern "C" lnf_status lnf_profile_enable(lnf_ctx *ctx, int on)
{
    if (!ctx)
        return LNF_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    prof_clear(ctx);
    ctx->prof = on != 0;
    return LNF_OK;
}

extern "C" lnf_status lnf_profile_read(lnf_ctx *ctx, lnf_kernel_time *out, int max, int *n, int64_t *launches)
{
    if (!ctx || (max > 0 && !out))
        return LNF_EINVAL;
    for (auto &r : ctx->prof_recs)
        CK(cudaEventSynchronize(r.b));
    std::vector<lnf_kernel_time> kinds;
    for (auto &r : ctx->prof_recs) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        auto it = std::find_if(kinds.begin(), kinds.end(),
                               [&](const lnf_kernel_time &k) { return r.name == k.name; });
        if (it == kinds.end()) {
            lnf_kernel_time k;
            std::memset(&k, 0, sizeof k);
            std::snprintf(k.name, sizeof k.name, "%s", r.name.c_str());
            kinds.push_back(k);
            it = kinds.end() - 1;
        }
        it->launches += 1;
        it->total_ms += ms;
    }
    for (int i = 0; i < (int)kinds.size() && i < max; ++i)
        out[i] = kinds[i];
    if (n)
        *n = (int)kinds.size();
    if (launches)
        *launches = ctx->prof_launches;
    return LNF_OK;
}

static const char *filter_name(int f)
{
    static const char *names[] = {"filter:mean", "filter:sigma", "filter:entropy", "filter:okada",
                                  "filter:ours", "filter:ours_cross", "filter:ours_cube", "filter:sigma_local",
                                  "filter:entropy_local"};
    return f >= 0 && f <= 8 ? names[f] : "filter:?";
}

// ------------------------------------------------------------------ device steps

lnf_status lnf_analyze(lnf_ctx *ctx, const void *in, const int64_t dims[3], int dtype, VolScratch &vs,
                       cudaStream_t stream)
{
    const u32 levels = dtype == LNF_U8 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
    const u64 n = nvox(dims);
    int rec = lnf_prof_begin(ctx, stream);
    CK(lnf_launch_stats_init(vs.hist, levels, vs.st, n, stream));
    lnf_prof_end(ctx, rec, "stats_init", stream, 1);
    rec = lnf_prof_begin(ctx, stream);
    CK(lnf_launch_stats(in, n, dtype, vs.hist, ctx->num_sms, stream));
    lnf_prof_end(ctx, rec, "stats", stream, 1);
    rec = lnf_prof_begin(ctx, stream);
    CK(lnf_launch_params(vs.hist, vs.st, lnf_param_cfg(ctx), vs.prm, vs.lut, vs.pscr, dtype, stream));
    lnf_prof_end(ctx, rec, "params", stream, 1);
    return LNF_OK;
}

// Fill job `idx` of the pack; encodes a TMA map when the volume allows it.
lnf_status lnf_make_job(lnf_ctx *ctx, FilterPack &pk, int idx, int filter, int radius, const void *in, void *out,
                        const int64_t dims[3], int dtype, const int64_t *roi_o, const int64_t *roi_d,
                        const VolScratch &vs, u64 *out_hist, int64_t pitch, const int *rad3, const int *off3)
{
    FilterJob &j = pk.jobs[idx];
    std::memset(&j, 0, sizeof j);
    int offset = ctx->cfg.cluster_offset;
    for (int a = 0; a < 3; ++a) {
        j.rad[a] = rad3 ? rad3[a] : radius;
        j.off[a] = off3 ? off3[a] : offset;
    }
    if (rad3 || off3) {
        // the halo (and the TMA box) cover the largest reach of any axis
        j.aniso = 1;
        radius = std::max(j.rad[0], std::max(j.rad[1], j.rad[2]));
        offset = std::max(j.off[0], std::max(j.off[1], j.off[2]));
    }
    j.in = in;
    j.out = out;
    j.nx = (int)dims[0];
    j.ny = (int)dims[1];
    j.nz = (int)dims[2];
    j.pitch = pitch > 0 ? (int)pitch : j.nx;
    if (roi_d && roi_d[0] > 0) {
        j.ox = (int)roi_o[0];
        j.oy = (int)roi_o[1];
        j.oz = (int)roi_o[2];
        j.bx = (int)roi_d[0];
        j.by = (int)roi_d[1];
        j.bz = (int)roi_d[2];
    } else {
        j.bx = j.nx;
        j.by = j.ny;
        j.bz = j.nz;
    }
    j.dtype = dtype;
    j.filter = filter;
    j.radius = radius;
    j.offset = offset;
    j.prm = vs.prm;
    j.lut = vs.lut;
    j.out_hist = out_hist;
    j.tmap_idx = -1;
    lnf_filter_decompose(j, ctx->zchunk);
    const size_t es = esize(dtype);
    if (ctx->encode && !ctx->no_tma && (reinterpret_cast<uintptr_t>(in) & 15) == 0 && ((size_t)j.pitch * es) % 16 == 0) {
        unsigned bw = 0, bh = 0;
        lnf_filter_box(filter, radius, offset, dtype, &bw, &bh);
        if (bw <= 256 && bh <= 256) {
            cuuint64_t gdim[3] = {(cuuint64_t)dims[0], (cuuint64_t)dims[1], (cuuint64_t)dims[2]};
            cuuint64_t gstr[2] = {(cuuint64_t)((size_t)j.pitch * es), (cuuint64_t)((size_t)j.pitch * dims[1] * es)};
            cuuint32_t box[3] = {bw, bh, 1};
            cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = ctx->encode(&pk.tmaps[idx], dtype == LNF_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                                     : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                                     3, const_cast<void *>(in), gdim, gstr, box, estr,
                                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r == CUDA_SUCCESS)
                j.tmap_idx = idx;
        }
    }
    return LNF_OK;
}

// Encode a 3D TMA map of the volume with box {box_w, box_h, 1}; false when the
// volume does not meet TMA's alignment rules or encoding fails.
bool lnf_encode_box(lnf_ctx *ctx, const void *in, int nx, int ny, int nz, int pitch, int dtype, unsigned box_w,
                    unsigned box_h, CUtensorMap *map)
{
    const size_t es = esize(dtype);
    if (!ctx->encode || ctx->no_tma || (reinterpret_cast<uintptr_t>(in) & 15) != 0 ||
        ((size_t)pitch * es) % 16 != 0 || pitch < nx || box_w > 256 || box_h > 256 || (box_w * es) % 16 != 0)
        return false;
    cuuint64_t gdim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t gstr[2] = {(cuuint64_t)((size_t)pitch * es), (cuuint64_t)((size_t)pitch * ny * es)};
    cuuint32_t box[3] = {box_w, box_h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return ctx->encode(map, dtype == LNF_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                       const_cast<void *>(in), gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Assign item ranges and launch the generic kernel over the pack.
lnf_status lnf_run_pack(lnf_ctx *ctx, FilterPack &pk, int persistent, cudaStream_t stream)
{
    return lnf_run_pack_counter(ctx, pk, persistent, stream, ctx->d_counter);
}

lnf_status lnf_run_pack_counter(lnf_ctx *ctx, FilterPack &pk, int persistent, cudaStream_t stream, u32 *counter)
{
    int items = 0;
    size_t smem = 0;
    for (int i = 0; i < pk.n_jobs; ++i) {
        pk.jobs[i].item_begin = items;
        items += lnf_filter_items(pk.jobs[i]);
        smem = std::max(smem, lnf_filter_smem_bytes(pk.jobs[i].filter, pk.jobs[i].radius, pk.jobs[i].offset,
                                                    pk.jobs[i].dtype));
    }
    pk.total_items = items;
    if (items == 0)
        return LNF_OK;
    const int occ = lnf_filter_occupancy(smem);
    int grid = std::min(items, ctx->num_sms * occ);
    if (persistent)
        CK(cudaMemsetAsync(counter, 0, sizeof(u32), stream));
    CK(lnf_filter_run(pk, smem, grid, persistent, counter, ctx->d_err, stream));
    return LNF_OK;
}

size_t lnf_pitched_row(const void *in, const int64_t dims[3], int dtype)
{
    const size_t row = (size_t)dims[0] * esize(dtype);
    if ((reinterpret_cast<uintptr_t>(in) & 15) == 0 && row % 16 == 0)
        return 0;
    return (row + 15) / 16 * 16;
}

// A whole-volume input that TMA cannot address (an unaligned base or a row
// length that is not a multiple of 16 bytes) is copied once into the
// context's staging buffer with padded rows, so that the specialised kernels
// can read it; *src / *pitch name what the filter launches read.
static lnf_status stage_input(lnf_ctx *ctx, const void *in, const int64_t dims[3], int dtype, cudaStream_t st,
                              const void **src, int64_t *pitch)
{
    *src = in;
    *pitch = 0;
    const size_t prow = lnf_pitched_row(in, dims, dtype);
    if (prow == 0 || !ctx->encode || ctx->no_tma || ctx->no_fast)
        return LNF_OK;
    const size_t need = prow * dims[1] * dims[2];
    if (ctx->pitched_cap < need) {
        cudaFree(ctx->pitched);   // waits for the work that still reads it
        ctx->pitched = nullptr;
        ctx->pitched_cap = 0;
        if (lnf_fault(ctx, FAULT_STAGE) || cudaMalloc(&ctx->pitched, need) != cudaSuccess) {
            ctx->pitched = nullptr;
            cudaGetLastError();
            return LNF_OK;   // no room for the copy: the generic kernel reads the input itself
        }
        ctx->pitched_cap = need;
    }
    lnf_status s = lnf_copy_pitched(ctx, ctx->pitched, prow, in, dims, dtype, st);
    if (s != LNF_OK)
        return s;
    *src = ctx->pitched;
    *pitch = (int64_t)(prow / esize(dtype));
    return LNF_OK;
}

// Run one filter job on an analysed volume, through the fastest kernel that covers it.
lnf_status lnf_run_one(lnf_ctx *ctx, int filter, int radius, const void *in, void *out, const int64_t dims[3],
                       int dtype, const int64_t *roi_o, const int64_t *roi_d, const VolScratch &vs,
                       u64 *out_hist, cudaStream_t stream, int64_t pitch, const int *rad3, const int *off3,
                       const void *orig)
{
    FilterPack &pk = ctx->pack;
    pk.n_jobs = 1;
    lnf_status s = lnf_make_job(ctx, pk, 0, filter, radius, in, out, dims, dtype, roi_o, roi_d, vs, out_hist,
                                pitch, rad3, off3);
    if (s != LNF_OK)
        return s;
    if (lnf_fault(ctx, FAULT_LAUNCH))
        return lnf_fail(ctx, LNF_ECUDA, "injected fault: filter launch failed");
    LNF_RANGE(filter_name(filter));
    const int rec = lnf_prof_begin(ctx, stream);
    int sparse = 0;
    if (!ctx->no_fast) {
        int handled = 0;
        pk.jobs[0].orig = orig;
        if (lnf_sparse_covers(filter, radius) && !ctx->no_gate && pk.jobs[0].tmap_idx >= 0 && !pk.jobs[0].aniso) {
            // the tap kernel takes the job while few voxels pass the gate (it
            // evaluates the listed voxels alone); the generic kernel below does
            // it otherwise
            if ((s = lnf_fast2_dispatch(ctx, pk.jobs[0], &pk.tmaps[pk.jobs[0].tmap_idx], stream, &sparse, nullptr,
                                        2)) != LNF_OK) {
                lnf_prof_end(ctx, rec, filter_name(filter), stream, 1);
                return s;
            }
            pk.jobs[0].gated = sparse ? 1 : 0;
        }
        if (filter == LNF_ENTROPY_LOCAL && !ctx->no_gate && lnf_gate_covers(pk.jobs[0], filter)) {
            // the gate-first kernel takes the volume while few voxels pass; the
            // generic kernel below does it otherwise
            int gh = 0;
            if ((s = lnf_gate_launch_eloc(ctx, pk.jobs[0], stream, &gh)) != LNF_OK) {
                lnf_prof_end(ctx, rec, filter_name(filter), stream, 1);
                return s;
            }
            pk.jobs[0].gated = gh;
        }
        s = lnf_fast_dispatch(ctx, pk.jobs[0], pk.jobs[0].tmap_idx >= 0 ? &pk.tmaps[0] : nullptr, stream, &handled,
                              nullptr, 1);
        if (s != LNF_OK || handled) {
            lnf_prof_end(ctx, rec, filter_name(filter), stream, handled ? handled : 1);
            return s;
        }
    }
    s = lnf_run_pack(ctx, pk, 0, stream);
    lnf_prof_end(ctx, rec, filter_name(filter), stream, 1 + sparse);
    return s;
}

// ------------------------------------------------------------------ entry points

extern "C" lnf_status lnf_filter_volume(lnf_ctx *ctx, int filter_id, int radius, const void *in, void *out,
                                        const int64_t dims[3], int dtype)
{
    LNF_RANGE("lnf_filter_volume");
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if ((s = check_filter(ctx, filter_id, radius)) != LNF_OK)
        return s;
    if ((s = lnf_check_volume(ctx, in, dims, dtype)) != LNF_OK)
        return s;
    if (!out)
        return lnf_fail(ctx, LNF_EINVAL, "null output pointer");
    const size_t bytes = nvox(dims) * esize(dtype);
    if (overlaps(in, bytes, out, bytes))
        return lnf_fail(ctx, LNF_EINVAL, "input and output overlap");
    if ((s = lnf_analyze(ctx, in, dims, dtype, ctx->vs, ctx->stream)) != LNF_OK)
        return s;
    const void *src = in;
    int64_t pitch = 0;
    if ((lnf_fast_covers(filter_id, radius, ctx->cfg.cluster_offset) || lnf_sparse_covers(filter_id, radius)) &&
        (s = stage_input(ctx, in, dims, dtype, ctx->stream, &src, &pitch)) != LNF_OK)
        return s;
    return lnf_run_one(ctx, filter_id, radius, src, out, dims, dtype, nullptr, nullptr, ctx->vs, nullptr,
                       ctx->stream, pitch, nullptr, nullptr, in);
}

extern "C" lnf_status lnf_filter_roi(lnf_ctx *ctx, int filter_id, int radius, const void *in,
                                     const int64_t dims[3], int dtype, const int64_t roi_origin[3],
                                     const int64_t roi_dims[3], void *out)
{
    LNF_RANGE("lnf_filter_roi");
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if ((s = check_filter(ctx, filter_id, radius)) != LNF_OK)
        return s;
    if ((s = lnf_check_volume(ctx, in, dims, dtype)) != LNF_OK)
        return s;
    if (!out || !roi_origin || !roi_dims)
        return lnf_fail(ctx, LNF_EINVAL, "null ROI argument");
    for (int i = 0; i < 3; ++i)
        if (roi_dims[i] < 1 || roi_origin[i] < 0 || roi_origin[i] + roi_dims[i] > dims[i])
            return lnf_fail(ctx, LNF_EINVAL, "ROI axis %d [%lld, +%lld) outside the volume", i,
                            (long long)roi_origin[i], (long long)roi_dims[i]);
    const size_t es = esize(dtype);
    if (overlaps(in, nvox(dims) * es, out, nvox(roi_dims) * es))
        return lnf_fail(ctx, LNF_EINVAL, "input and output overlap");
    if ((s = lnf_analyze(ctx, in, dims, dtype, ctx->vs, ctx->stream)) != LNF_OK)
        return s;
    return lnf_run_one(ctx, filter_id, radius, in, out, dims, dtype, roi_origin, roi_dims, ctx->vs, nullptr,
                       ctx->stream);
}

extern "C" lnf_status lnf_filter_volume_aniso(lnf_ctx *ctx, int filter_id, const int radius[3],
                                              const int offset[3], const void *in, void *out,
                                              const int64_t dims[3], int dtype)
{
    LNF_RANGE("lnf_filter_volume_aniso");
    if (!ctx)
        return LNF_EINVAL;
    if (!radius)
        return lnf_fail(ctx, LNF_EINVAL, "null radius array");
    int rad[3], off[3];
    for (int a = 0; a < 3; ++a) {
        rad[a] = radius[a];
        off[a] = offset ? offset[a] : ctx->cfg.cluster_offset;
        if (rad[a] < 0 || rad[a] > LNF_MAX_RADIUS)
            return lnf_fail(ctx, LNF_EINVAL, "radius[%d] = %d not in 0..%d", a, rad[a], LNF_MAX_RADIUS);
        if (off[a] < 0 || off[a] > 8)
            return lnf_fail(ctx, LNF_EINVAL, "offset[%d] = %d not in 0..8", a, off[a]);
    }
    const bool iso = rad[0] == rad[1] && rad[1] == rad[2] && off[0] == ctx->cfg.cluster_offset &&
                     off[1] == off[0] && off[2] == off[0];
    if (iso)
        return lnf_filter_volume(ctx, filter_id, rad[0], in, out, dims, dtype);
    lnf_status s;
    if ((s = check_filter(ctx, filter_id, rad[0])) != LNF_OK)
        return s;
    if ((s = lnf_check_volume(ctx, in, dims, dtype)) != LNF_OK)
        return s;
    if (!out)
        return lnf_fail(ctx, LNF_EINVAL, "null output pointer");
    const size_t bytes = nvox(dims) * esize(dtype);
    if (overlaps(in, bytes, out, bytes))
        return lnf_fail(ctx, LNF_EINVAL, "input and output overlap");
    if ((s = lnf_analyze(ctx, in, dims, dtype, ctx->vs, ctx->stream)) != LNF_OK)
        return s;
    const int rmax = std::max(rad[0], std::max(rad[1], rad[2]));
    return lnf_run_one(ctx, filter_id, rmax, in, out, dims, dtype, nullptr, nullptr, ctx->vs, nullptr,
                       ctx->stream, 0, rad, off);
}

extern "C" lnf_status lnf_spacing_radii(double extent, const double spacing[3], int radius[3])
{
    if (!spacing || !radius || !(extent >= 0.0) || !std::isfinite(extent))
        return LNF_EINVAL;
    int out[3];
    for (int a = 0; a < 3; ++a) {
        const double s = spacing[a];
        if (!(s > 0.0) || !std::isfinite(s))
            return LNF_EINVAL;
        const double q = std::floor(extent / s + 0.5);
        if (!(q <= (double)LNF_MAX_RADIUS))
            return LNF_EINVAL;
        out[a] = (int)q;
    }
    for (int a = 0; a < 3; ++a)
        radius[a] = out[a];
    return LNF_OK;
}

// lnf_filter_multi, recording `after[i]` on the context stream once filter i
// has been enqueued (when `after` is not null) and listing in `order` the filter
// indices in the order their events were recorded (when `order` is not null)
static lnf_status multi_impl(lnf_ctx *ctx, int radius, const void *in, const int64_t dims[3], int dtype, int n,
                             const int *filter_ids, void *const *outs, double *d_entropy, cudaEvent_t *after,
                             int *order = nullptr);

extern "C" lnf_status lnf_filter_multi(lnf_ctx *ctx, int radius, const void *in, const int64_t dims[3], int dtype,
                                       int n, const int *filter_ids, void *const *outs, double *d_entropy)
{
    LNF_RANGE("lnf_filter_multi");
    return multi_impl(ctx, radius, in, dims, dtype, n, filter_ids, outs, d_entropy, nullptr);
}

static lnf_status multi_impl(lnf_ctx *ctx, int radius, const void *in, const int64_t dims[3], int dtype, int n,
                             const int *filter_ids, void *const *outs, double *d_entropy, cudaEvent_t *after,
                             int *order)
{
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if ((s = lnf_check_volume(ctx, in, dims, dtype)) != LNF_OK)
        return s;
    if (n < 0 || n > LNF_MAX_PACK || (n > 0 && (!filter_ids || !outs)))
        return lnf_fail(ctx, LNF_EINVAL, "n = %d filters (1..%d) with non-null ids and outputs", n, LNF_MAX_PACK);
    const size_t bytes = nvox(dims) * esize(dtype);
    for (int i = 0; i < n; ++i) {
        if ((s = check_filter(ctx, filter_ids[i], radius)) != LNF_OK)
            return s;
        if (!outs[i] || overlaps(in, bytes, outs[i], bytes))
            return lnf_fail(ctx, LNF_EINVAL, "output %d is null or overlaps the input", i);
        // (one launch may write several outputs at once: they must be distinct)
        for (int k = 0; k < i; ++k)
            if (overlaps(outs[k], bytes, outs[i], bytes))
                return lnf_fail(ctx, LNF_EINVAL, "outputs %d and %d overlap", k, i);
    }
    cudaStream_t st = ctx->stream;
    if ((s = lnf_analyze(ctx, in, dims, dtype, ctx->vs, st)) != LNF_OK)
        return s;
    const u32 levels = dtype == LNF_U8 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
    if (d_entropy && n > 0) {
        const int rec = lnf_prof_begin(ctx, st);
        CK(lnf_launch_zero(ctx->out_hist, (u64)LNF_LEVELS_U16 * n, st));
        lnf_prof_end(ctx, rec, "zero_hist", st, 1);
    }
    // one padded copy serves every filter a specialised kernel covers
    bool any_fast = false;
    for (int i = 0; i < n; ++i)
        any_fast = any_fast || lnf_fast_covers(filter_ids[i], radius, ctx->cfg.cluster_offset) ||
                   lnf_sparse_covers(filter_ids[i], radius);
    const void *src = in;
    int64_t pitch = 0;
    if (any_fast && (s = stage_input(ctx, in, dims, dtype, st, &src, &pitch)) != LNF_OK)
        return s;
    // The filters of this call the gate-first kernel covers, each asked for once,
    // in one launch (one read of the volume, one write per output) while few
    // voxels pass the gate (decided on the device; their ring kernels, launched
    // after it, return at once then).
    int slot5[5] = {-1, -1, -1, -1, -1};
    bool once = true;
    for (int i = 0; i < n; ++i)
        if (filter_ids[i] >= LNF_MEAN && filter_ids[i] <= LNF_OURS) {
            once = once && slot5[filter_ids[i]] < 0;
            slot5[filter_ids[i]] = i;
        }
    ctx->gate_mask = 0;
    if (once && !ctx->no_gate && !ctx->no_fast && n > 0) {
        FilterPack &pk = ctx->pack;
        pk.n_jobs = 1;
        if ((s = lnf_make_job(ctx, pk, 0, filter_ids[0], radius, src, outs[0], dims, dtype, nullptr, nullptr,
                              ctx->vs, nullptr, pitch)) != LNF_OK)
            return s;
        pk.jobs[0].orig = in;
        void *o5[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        u64 *h5[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        int mask = 0;
        for (int f = 0; f < 5; ++f)
            if (slot5[f] >= 0 && lnf_gate_covers(pk.jobs[0], f)) {
                o5[f] = outs[slot5[f]];
                h5[f] = d_entropy ? ctx->out_hist + (size_t)slot5[f] * LNF_LEVELS_U16 : nullptr;
                mask |= 1 << f;
            }
        if (mask) {
            int handled = 0;
            const int rec = lnf_prof_begin(ctx, st);
            s = lnf_gate_launch(ctx, pk.jobs[0], o5, h5, st, &handled);
            lnf_prof_end(ctx, rec, "filter:gate", st, 2);   // the scan and the evaluation
            if (s != LNF_OK)
                return s;
            ctx->gate_mask = handled ? mask : 0;
        }
    }
    int done = 0;
    for (int i = 0; i < n; ++i) {
        u64 *oh = d_entropy ? ctx->out_hist + (size_t)i * LNF_LEVELS_U16 : nullptr;
        const bool f = lnf_fast_covers(filter_ids[i], radius, ctx->cfg.cluster_offset) ||
                       lnf_sparse_covers(filter_ids[i], radius);
        s = lnf_run_one(ctx, filter_ids[i], radius, f ? src : in, outs[i], dims, dtype, nullptr, nullptr, ctx->vs,
                        oh, st, f ? pitch : 0, nullptr, nullptr, in);
        if (s == LNF_OK && after && cudaEventRecord(after[i], st) != cudaSuccess)
            s = lnf_fail(ctx, LNF_ECUDA, "event record failed");
        if (s != LNF_OK) {
            ctx->gate_mask = 0;
            return s;
        }
        if (order)
            order[done++] = i;
    }
    ctx->gate_mask = 0;
    if (d_entropy) {
        CK(cudaMemcpyAsync(d_entropy, &ctx->vs.prm->H_in, sizeof(double), cudaMemcpyDeviceToDevice, st));
        EntropyPack ep;
        std::memset(&ep, 0, sizeof ep);
        ep.count = n;
        for (int i = 0; i < n; ++i) {
            ep.hist[i] = ctx->out_hist + (size_t)i * LNF_LEVELS_U16;
            ep.n[i] = nvox(dims);
            ep.H[i] = d_entropy + 1 + i;
            ep.levels[i] = levels;
        }
        const int rec = lnf_prof_begin(ctx, st);
        CK(lnf_launch_entropy_pack(ep, ctx->d_ent_part, ctx->d_ent_done, st));
        lnf_prof_end(ctx, rec, "entropy", st, 1);
    }
    return LNF_OK;
}

static lnf_status ensure_stage(lnf_ctx *ctx, void **p, size_t *cap, size_t bytes)
{
    if (*cap >= bytes)
        return LNF_OK;
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    CK(cudaMalloc(p, bytes));
    *cap = bytes;
    return LNF_OK;
}

extern "C" lnf_status lnf_filter_multi_host(lnf_ctx *ctx, int radius, const void *in, const int64_t dims[3],
                                            int dtype, int n, const int *filter_ids, void *const *outs,
                                            double *entropy)
{
    LNF_RANGE("lnf_filter_multi_host");
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if ((s = lnf_check_volume(ctx, in, dims, dtype)) != LNF_OK)
        return s;
    if (n < 0 || n > LNF_MAX_PACK || (n > 0 && (!filter_ids || !outs)))
        return lnf_fail(ctx, LNF_EINVAL, "bad filter list");
    for (int i = 0; i < n; ++i)
        if (!outs[i])
            return lnf_fail(ctx, LNF_EINVAL, "null host output %d", i);
    const size_t bytes = nvox(dims) * esize(dtype);
    if ((s = ensure_stage(ctx, &ctx->st_in, &ctx->st_in_cap, bytes)) != LNF_OK)
        return s;
    if (ctx->st_out.size() < (size_t)n) {
        ctx->st_out.resize(n, nullptr);
        ctx->st_out_cap.resize(n, 0);
    }
    for (int i = 0; i < n; ++i)
        if ((s = ensure_stage(ctx, &ctx->st_out[i], &ctx->st_out_cap[i], bytes)) != LNF_OK)
            return s;
    // each output goes back on a copy stream as soon as its filter is done, so
    // the copies overlap the filters that follow
    if (!ctx->copy_stream)
        CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    while ((int)ctx->filter_done.size() < n) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->filter_done.push_back(e);
    }
    cudaStream_t st = ctx->stream, cs = ctx->copy_stream;
    CK(cudaMemcpyAsync(ctx->st_in, in, bytes, cudaMemcpyHostToDevice, st));
    int order[LNF_MAX_PACK];
    if ((s = multi_impl(ctx, radius, ctx->st_in, dims, dtype, n, filter_ids, ctx->st_out.data(), ctx->d_H,
                        ctx->filter_done.data(), order)) != LNF_OK) {
        cudaStreamSynchronize(st);
        return s;
    }
    // in the order the outputs become ready (the fused pass finishes four at once, after
    // the filters that run before it)
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        CK(cudaStreamWaitEvent(cs, ctx->filter_done[i], 0));
        CK(cudaMemcpyAsync(outs[i], ctx->st_out[i], bytes, cudaMemcpyDeviceToHost, cs));
    }
    double hbuf[LNF_MAX_PACK + 1];
    CK(cudaMemcpyAsync(hbuf, ctx->d_H, sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaStreamSynchronize(cs));
    if (entropy)
        std::memcpy(entropy, hbuf, sizeof(double) * (n + 1));
    return LNF_OK;
}

extern "C" lnf_status lnf_render(lnf_ctx *ctx, int filter_id, int radius, const void *in, const int64_t dims[3],
                                 int dtype, int view, uint8_t *image, int32_t *depth, uint32_t *value)
{
    LNF_RANGE("lnf_render");
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if ((s = check_filter(ctx, filter_id, radius)) != LNF_OK)
        return s;
    if ((s = lnf_check_volume(ctx, in, dims, dtype)) != LNF_OK)
        return s;
    if (view < 0 || view > 5)
        return lnf_fail(ctx, LNF_EINVAL, "view %d not in 0..5", view);
    if (!image)
        return lnf_fail(ctx, LNF_EINVAL, "null image");
    if ((s = lnf_analyze(ctx, in, dims, dtype, ctx->vs, ctx->stream)) != LNF_OK)
        return s;
    const int rec = lnf_prof_begin(ctx, ctx->stream);
    CK(lnf_launch_render(in, dims, dims[0], dtype, view, filter_id, radius, ctx->cfg.cluster_offset, ctx->vs.prm,
                         ctx->vs.lut, image, depth, reinterpret_cast<u32 *>(value), ctx->stream));
    lnf_prof_end(ctx, rec, "render", ctx->stream, 1);
    return LNF_OK;
}

extern "C" lnf_status lnf_entropy(lnf_ctx *ctx, const void *vol, const int64_t dims[3], int dtype, double *H)
{
    LNF_RANGE("lnf_entropy");
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if ((s = lnf_check_volume(ctx, vol, dims, dtype)) != LNF_OK)
        return s;
    if (!H)
        return lnf_fail(ctx, LNF_EINVAL, "null H");
    cudaStream_t st = ctx->stream;
    const u32 levels = dtype == LNF_U8 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
    const u64 n = nvox(dims);
    CK(lnf_launch_stats_init(ctx->vs.hist, levels, ctx->vs.st, n, st));
    CK(lnf_launch_stats(vol, n, dtype, ctx->vs.hist, ctx->num_sms, st));
    CK(lnf_launch_entropy(ctx->vs.hist, levels, n, ctx->d_H, st));
    CK(cudaMemcpyAsync(H, ctx->d_H, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return LNF_OK;
}

extern "C" lnf_status lnf_get_params(lnf_ctx *ctx, lnf_params *out, uint32_t *weights)
{
    if (!ctx || !out)
        return LNF_EINVAL;
    DevParams p;
    CK(cudaMemcpyAsync(&p, ctx->vs.prm, sizeof p, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!p.valid)
        return lnf_fail(ctx, LNF_EINVAL, "no volume has been analysed on this context yet");
    if (weights) {
        CK(cudaMemcpyAsync(weights, ctx->vs.lut, sizeof(u32) * p.levels, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    out->n_voxels = p.N;
    out->sum = p.S;
    out->sum_sq = p.Q;
    out->min_value = p.minv;
    out->max_value = p.maxv;
    out->threshold = p.T;
    out->sigma_band = p.delta;
    out->okada_td = p.td;
    out->weight_sum = p.hw_sum;
    out->input_entropy = p.H_in;
    u32 err = 0;
    if (cudaMemcpy(&err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost) == cudaSuccess && err) {
        if (err & LNF_DERR_BADJOB)
            return lnf_fail(ctx, LNF_ECUDA, "a debug bounds check failed (code %u)", err);
        return lnf_fail(ctx, LNF_ETIMEOUT, "a bounded device wait gave up (code %u)", err);
    }
    return LNF_OK;
}

extern "C" int lnf_debug_checks(void)
{
#ifdef LNF_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

extern "C" lnf_status lnf_debug_poll(lnf_ctx *ctx)
{
    if (!ctx)
        return LNF_EINVAL;
#ifdef LNF_DEBUG_CHECKS
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "debug poll: stream synchronisation failed");
    u32 err = 0;
    if (cudaMemcpy(&err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "debug poll: error word unreadable");
    if (err & LNF_DERR_BADJOB) {
        const u32 keep = err & ~LNF_DERR_BADJOB;
        cudaMemcpy(ctx->d_err, &keep, sizeof keep, cudaMemcpyHostToDevice);
        return lnf_fail(ctx, LNF_ECUDA, "a debug bounds check failed");
    }
#endif
    return LNF_OK;
}

extern "C" lnf_status lnf_filter_volume_f32(lnf_ctx *ctx, int filter_id, const int radius[3], const int offset[3],
                                           const float *in, float *out, const int64_t dims[3])
{
    LNF_RANGE("lnf_filter_volume_f32");
    if (!ctx)
        return LNF_EINVAL;
    lnf_status s;
    if (!radius)
        return lnf_fail(ctx, LNF_EINVAL, "null radius array");
    if ((s = check_filter(ctx, filter_id, 0)) != LNF_OK)
        return s;
    if ((s = lnf_check_volume(ctx, in, dims, LNF_U16)) != LNF_OK)
        return s;
    if (!out)
        return lnf_fail(ctx, LNF_EINVAL, "null output pointer");
    const u64 n = nvox(dims);
    if (overlaps(in, n * 4, out, n * 4))
        return lnf_fail(ctx, LNF_EINVAL, "input and output overlap");
    cudaStream_t st = ctx->stream;
    // the range, checked on the host: every value finite, the span finite
    int rec = lnf_prof_begin(ctx, st);
    CK(lnf_launch_f32_range(in, n, ctx->d_range, ctx->num_sms, st));
    lnf_prof_end(ctx, rec, "f32_range", st, 2);
    u32 rg[4];
    CK(cudaMemcpyAsync(rg, ctx->d_range, sizeof rg, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (rg[2] != 0)
        return lnf_fail(ctx, LNF_EINVAL, "the volume holds %u non-finite values", rg[2]);
    auto unkey = [](u32 k) {
        const u32 b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
        float f;
        std::memcpy(&f, &b, sizeof f);
        return f;
    };
    const float lo = unkey(rg[0]), hi = unkey(rg[1]);
    const float span = hi - lo;
    if (!std::isfinite(span))
        return lnf_fail(ctx, LNF_EINVAL, "the volume's range [%g, %g] is wider than float32 can hold", lo, hi);
    if ((s = ensure_stage(ctx, &ctx->f32_lv, &ctx->f32_lv_cap, (size_t)n * 4)) != LNF_OK)
        return s;
    uint16_t *lv_in = static_cast<uint16_t *>(ctx->f32_lv), *lv_out = lv_in + n;
    rec = lnf_prof_begin(ctx, st);
    CK(lnf_launch_f32_quantize(in, n, ctx->d_range, lv_in, ctx->num_sms, st));
    lnf_prof_end(ctx, rec, "f32_quantize", st, 1);
    if ((s = lnf_filter_volume_aniso(ctx, filter_id, radius, offset, lv_in, lv_out, dims, LNF_U16)) != LNF_OK)
        return s;
    rec = lnf_prof_begin(ctx, st);
    CK(lnf_launch_f32_dequantize(lv_out, n, ctx->d_range, out, ctx->num_sms, st));
    lnf_prof_end(ctx, rec, "f32_dequantize", st, 1);
    return LNF_OK;
}
