// Batched delivery: many volumes / ROIs / filters / radii behind one batched
// statistics launch and one batched parameter launch; jobs a specialised kernel
// covers run as its launches (a whole volume of the paper's filter also gets
// the gate-first kernel, which takes the job on the device while few voxels
// pass the gate; inputs TMA cannot address first get one padded copy per
// volume), all other jobs share ONE persistent launch of the generic kernel
// over their flattened tile list.  The specialised launches form one chain per
// input volume (its padded copy, then its jobs in order), and the chains run
// side by side on LNF_BATCH_CHAINS streams forked from the caller's stream
// after the parameter launch and joined back before the generic launch: a
// volume of a few million voxels gives a persistent grid only one or two work
// items per CTA, and one chain's tail is the next chain's start.  Each job has
// its own work counters.  The whole sequence is captured once into a CUDA graph
// and replayed for the same batch.
//
// The autotuner (lnf_config.autotune) times the candidates on the first batch
// it sees: for each class of specialised jobs (dtype, filter, radius), the z
// length of a work item of the plane-ring kernels (planes per item: the halo
// planes re-read per item against the balance of the persistent grid), timed on
// that class's jobs alone; then, when the batch has generic jobs, the generic
// kernel's z chunk.  The choices are kept per context (lnf_get_tuning).  The
// tile shape and threads per tile of the specialised kernels are compile-time
// (set by their register and shared-memory budgets), so they are not tuned.
#include "lnf_ctx.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return lnf_fail(ctx, LNF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));             \
    } while (0)

static void free_stage(std::vector<void *> &stage)
{
    for (void *p : stage)
        if (p)
            cudaFree(p);   // waits for the work that still reads it
    stage.clear();
}

struct BatchEntry {
    std::vector<lnf_job> key;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> stage;   // padded copies of the distinct inputs (owned; null: none needed)
    ~BatchEntry()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        if (graph)
            cudaGraphDestroy(graph);
        free_stage(stage);
    }
};

static void destroy_entry(BatchEntry *b) { delete b; }

void lnf_batch_cache_clear(lnf_ctx *ctx)
{
    for (BatchEntry *b : ctx->batches)
        destroy_entry(b);
    ctx->batches.clear();
}

// the distinct input volumes of a batch, in order of first use
static std::vector<const void *> distinct_inputs(const lnf_job *jobs, int n, std::vector<int> &vol_of)
{
    std::vector<const void *> vols;
    vol_of.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        auto it = std::find(vols.begin(), vols.end(), jobs[i].in);
        if (it == vols.end()) {
            vol_of[i] = (int)vols.size();
            vols.push_back(jobs[i].in);
        } else {
            vol_of[i] = (int)(it - vols.begin());
        }
    }
    return vols;
}

static bool whole_volume(const lnf_job &j)
{
    return j.roi_dims[0] <= 0;
}

// Allocate (outside any capture) a padded copy for each distinct input that
// TMA cannot address and that a whole-volume job of a specialised kernel reads.
static lnf_status alloc_stage(lnf_ctx *ctx, const lnf_job *jobs, int n, std::vector<void *> &stage)
{
    std::vector<int> vol_of;
    const std::vector<const void *> vols = distinct_inputs(jobs, n, vol_of);
    stage.assign(vols.size(), nullptr);
    if (!ctx->encode || ctx->no_tma || ctx->no_fast)
        return LNF_OK;
    for (int i = 0; i < n; ++i) {
        const lnf_job &j = jobs[i];
        const int v = vol_of[i];
        if (stage[v] || !whole_volume(j) || !lnf_fast_covers(j.filter_id, j.radius, ctx->cfg.cluster_offset))
            continue;
        const size_t prow = lnf_pitched_row(j.in, j.dims, j.dtype);
        if (prow == 0)
            continue;
        if (lnf_fault(ctx, FAULT_STAGE) || cudaMalloc(&stage[v], prow * j.dims[1] * j.dims[2]) != cudaSuccess) {
            stage[v] = nullptr;   // no room: the generic kernel reads the input itself
            cudaGetLastError();
        }
    }
    return LNF_OK;
}

// The batch streams, their fork / join events and the per-job work counters,
// made once per context outside any capture; if any of them cannot be made the
// batch runs as one chain on the context's stream.
static void batch_streams(lnf_ctx *ctx)
{
    if (ctx->bfork)
        return;
    bool ok = cudaMalloc(&ctx->d_bcounter, sizeof(u32) * 2 * LNF_MAX_PACK) == cudaSuccess;
    for (int k = 0; ok && k < LNF_BATCH_STREAMS; ++k)
        ok = cudaStreamCreateWithFlags(&ctx->bstream[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->bjoin[k], cudaEventDisableTiming) == cudaSuccess;
    cudaEvent_t fork = nullptr;
    ok = ok && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        ctx->bfork = fork;
        ctx->bchains = LNF_BATCH_CHAINS;
        // test hook: the number of chains side by side (1..LNF_BATCH_STREAMS)
        if (const char *e = std::getenv("LNF_BATCH_CHAINS"))
            ctx->bchains = std::max(1, std::min(LNF_BATCH_STREAMS, std::atoi(e)));
        return;
    }
    cudaGetLastError();
    lnf_batch_streams_free(ctx);
}

void lnf_batch_streams_free(lnf_ctx *ctx)
{
    for (int k = 0; k < LNF_BATCH_STREAMS; ++k) {
        if (ctx->bstream[k])
            cudaStreamDestroy(ctx->bstream[k]);
        if (ctx->bjoin[k])
            cudaEventDestroy(ctx->bjoin[k]);
        ctx->bstream[k] = nullptr;
        ctx->bjoin[k] = nullptr;
    }
    if (ctx->bfork)
        cudaEventDestroy(ctx->bfork);
    ctx->bfork = nullptr;
    ctx->bchains = 0;
    cudaFree(ctx->d_bcounter);
    ctx->d_bcounter = nullptr;
}

static bool same_jobs(const std::vector<lnf_job> &a, const lnf_job *b, int n)
{
    return (int)a.size() == n && std::memcmp(a.data(), b, sizeof(lnf_job) * n) == 0;
}

static lnf_status check_job(lnf_ctx *ctx, const lnf_job &j, int i)
{
    lnf_status s = lnf_check_volume(ctx, j.in, j.dims, j.dtype);
    if (s != LNF_OK)
        return s;
    if (j.filter_id < LNF_MEAN || j.filter_id > LNF_ENTROPY_LOCAL || j.radius < 0 || j.radius > LNF_MAX_RADIUS)
        return lnf_fail(ctx, LNF_EINVAL, "job %d: filter %d / radius %d out of range", i, j.filter_id, j.radius);
    if (!j.out)
        return lnf_fail(ctx, LNF_EINVAL, "job %d: null output", i);
    if (j.roi_dims[0] > 0 || j.roi_dims[1] > 0 || j.roi_dims[2] > 0)
        for (int a = 0; a < 3; ++a)
            if (j.roi_dims[a] < 1 || j.roi_origin[a] < 0 || j.roi_origin[a] + j.roi_dims[a] > j.dims[a])
                return lnf_fail(ctx, LNF_EINVAL, "job %d: ROI outside the volume", i);
    const size_t es = j.dtype == LNF_U8 ? 1 : 2;
    const size_t nin = (size_t)j.dims[0] * j.dims[1] * j.dims[2] * es;
    const size_t nout = j.roi_dims[0] > 0 ? (size_t)j.roi_dims[0] * j.roi_dims[1] * j.roi_dims[2] * es : nin;
    const char *pi = static_cast<const char *>(j.in), *po = static_cast<const char *>(j.out);
    if (pi < po + nout && po < pi + nin)
        return lnf_fail(ctx, LNF_EINVAL, "job %d: input and output overlap", i);
    return LNF_OK;
}

// Enqueue the whole batch (<= LNF_MAX_PACK jobs) on `st`: stats, params,
// histogram zeroing, the padded copies named by `stage` (one per distinct
// input, null: none), the specialised launches, the persistent generic launch
// over the remaining jobs and the entropies.
// the autotuner's job class: dtype, filter, radius
static int job_class(const lnf_job &j) { return (j.dtype * 16 + j.filter_id) * 16 + j.radius; }

// z length of a specialised work item for job j: the tuned one of its class, the
// override `zlen` (> 0, used while tuning), else 0 (the kernel's automatic choice)
static int zlen_for(const lnf_ctx *ctx, const lnf_job &j, int zlen)
{
    if (zlen > 0)
        return zlen;
    auto it = ctx->tuned_zlen.find(job_class(j));
    return it != ctx->tuned_zlen.end() ? it->second : 0;   // 0: the kernel's automatic choice
}

lnf_status lnf_enqueue_batch(lnf_ctx *ctx, const lnf_job *jobs, int n, int zchunk, int zlen, cudaStream_t st,
                             std::vector<VolScratch> *scratch_out, const std::vector<void *> *stage)
{
    // distinct input volumes share one statistics pass
    std::vector<int> vol_of;
    const std::vector<const void *> vols = distinct_inputs(jobs, n, vol_of);
    lnf_status s = lnf_scratch_pool(ctx, vols.size());
    if (s != LNF_OK)
        return s;
    StatsPack sp;
    std::memset(&sp, 0, sizeof sp);
    sp.n_jobs = (int)vols.size();
    for (size_t v = 0; v < vols.size(); ++v) {
        int first = (int)(std::find(vol_of.begin(), vol_of.end(), (int)v) - vol_of.begin());
        const lnf_job &j = jobs[first];
        StatsJob &sj = sp.jobs[v];
        sj.vol = j.in;
        sj.n = (u64)j.dims[0] * j.dims[1] * j.dims[2];
        sj.dtype = j.dtype;
        sj.hist = ctx->pool[v].hist;
        sj.st = ctx->pool[v].st;
        sj.prm = ctx->pool[v].prm;
        sj.lut = ctx->pool[v].lut;
        sj.pscr = ctx->pool[v].pscr;
    }
    const int per = std::max(1, (2 * ctx->num_sms + sp.n_jobs - 1) / sp.n_jobs);
    CK(lnf_launch_stats_init_batched(sp, st));
    CK(lnf_launch_stats_batched(sp, per, st));
    CK(lnf_launch_params_batched(sp, lnf_param_cfg(ctx), st));

    // the job chains: one per input volume, side by side on the batch streams
    // (volume v on stream v % bchains) when the context has them, each
    // job with its own work counters; else one chain on `st`
    const bool fork = ctx->bfork != nullptr && n > 1;
    auto chain = [&](int v) { return fork ? ctx->bstream[v % ctx->bchains] : st; };
    if (fork) {
        CK(cudaEventRecord(ctx->bfork, st));
        for (int k = 0; k < ctx->bchains; ++k)
            CK(cudaStreamWaitEvent(ctx->bstream[k], ctx->bfork, 0));
    }

    // padded copies of the inputs TMA cannot address, at the head of their chains;
    // the copy of a volume whose only job is a whole volume of the paper's filter
    // goes between that job's gate-first and ring kernels instead, where it is
    // skipped on the device while the gate-first kernel takes the volume
    std::vector<int> jobs_of(vols.size(), 0);
    for (int i = 0; i < n; ++i)
        ++jobs_of[vol_of[i]];
    std::vector<int64_t> pitch(vols.size(), 0);
    std::vector<char> deferred(vols.size(), 0);
    for (size_t v = 0; stage && v < vols.size(); ++v) {
        if (!(*stage)[v])
            continue;
        int first = (int)(std::find(vol_of.begin(), vol_of.end(), (int)v) - vol_of.begin());
        const lnf_job &j = jobs[first];
        const size_t prow = lnf_pitched_row(j.in, j.dims, j.dtype);
        pitch[v] = (int64_t)(prow / (j.dtype == LNF_U8 ? 1 : 2));
        if (jobs_of[v] == 1 && j.filter_id == LNF_OURS && whole_volume(j)) {
            deferred[v] = 1;
            continue;
        }
        if ((s = lnf_copy_pitched(ctx, (*stage)[v], prow, j.in, j.dims, j.dtype, chain((int)v))) != LNF_OK)
            return s;
    }

    FilterPack &pk = ctx->pack;
    std::memset(&pk, 0, sizeof(int) * 16);
    int g = 0;   // jobs left to the generic kernel
    EntropyPack ep;
    std::memset(&ep, 0, sizeof ep);
    const int zsave = ctx->zchunk, lsave = ctx->fast_zlen;
    ctx->zchunk = zchunk;
    for (int i = 0; i < n; ++i) {
        const lnf_job &j = jobs[i];
        const int v = vol_of[i];
        const cudaStream_t sk = chain(v);
        u64 *oh = nullptr;
        const u32 levels = j.dtype == LNF_U8 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
        if (j.d_entropy) {
            oh = ctx->out_hist + (size_t)i * LNF_LEVELS_U16;
            CK(lnf_launch_zero(oh, levels, sk));
            const int k = ep.count++;
            ep.hist[k] = oh;
            ep.levels[k] = levels;
            ep.n[k] = j.roi_dims[0] > 0 ? (u64)j.roi_dims[0] * j.roi_dims[1] * j.roi_dims[2]
                                        : (u64)j.dims[0] * j.dims[1] * j.dims[2];
            ep.H[k] = j.d_entropy;
        }
        const bool fast = !ctx->no_fast && lnf_fast_covers(j.filter_id, j.radius, ctx->cfg.cluster_offset);
        const bool staged = fast && stage && (*stage)[v];
        s = lnf_make_job(ctx, pk, g, j.filter_id, j.radius, staged ? (*stage)[v] : j.in, j.out, j.dims, j.dtype,
                         j.roi_origin, j.roi_dims, ctx->pool[v], oh, staged ? pitch[v] : 0);
        int handled = 0;
        PitchedCopy pc{deferred[v] ? (*stage)[v] : nullptr, (size_t)pitch[v] * (j.dtype == LNF_U8 ? 1 : 2), j.in,
                       j.dims, j.dtype, ctx->pool[v].prm, false};
        if (s == LNF_OK && fast) {
            FilterJob &fj = pk.jobs[g];
            // the gate-first kernel reads the caller's dense volume, not a padded copy
            fj.orig = j.in;
            ctx->fast_zlen = zlen_for(ctx, j, zlen);
            s = lnf_fast_dispatch(ctx, fj, fj.tmap_idx >= 0 ? &pk.tmaps[fj.tmap_idx] : nullptr, sk, &handled,
                                  fork ? ctx->d_bcounter + 2 * i : nullptr, 1,
                                  fork ? ctx->d_bcounter + 2 * i + 1 : nullptr, deferred[v] ? &pc : nullptr);
        }
        // a deferred copy the dispatch did not enqueue (no specialised launch):
        // the generic kernel may read it
        if (s == LNF_OK && deferred[v] && !pc.done)
            s = lnf_copy_pitched(ctx, pc.dst, pc.prow, pc.src, pc.dims, pc.dtype, sk);
        if (s != LNF_OK) {
            ctx->zchunk = zsave;
            ctx->fast_zlen = lsave;
            return s;
        }
        if (!handled)
            ++g;
    }
    ctx->zchunk = zsave;
    ctx->fast_zlen = lsave;
    // the chains join before the generic launch (its jobs may read padded copies)
    // and the entropies (every job's output histogram)
    if (fork)
        for (int k = 0; k < ctx->bchains; ++k) {
            CK(cudaEventRecord(ctx->bjoin[k], ctx->bstream[k]));
            CK(cudaStreamWaitEvent(st, ctx->bjoin[k], 0));
        }
    pk.n_jobs = g;
    if (g > 0 && (s = lnf_run_pack(ctx, pk, 1, st)) != LNF_OK)
        return s;
    CK(lnf_launch_entropy_pack(ep, ctx->d_ent_part, ctx->d_ent_done, st));
    if (scratch_out) {
        scratch_out->clear();
        for (int i = 0; i < n; ++i)
            scratch_out->push_back(ctx->pool[vol_of[i]]);
    }
    return LNF_OK;
}

// time one enqueue of the batch with zchunk `zc` and specialised z length `zl`
// (0: the tuned / default one), best of three (events on the context stream)
static float time_batch(lnf_ctx *ctx, const lnf_job *jobs, int n, int zc, int zl, const std::vector<void *> *stage)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a, ctx->stream);
        if (lnf_enqueue_batch(ctx, jobs, n, zc, zl, ctx->stream, nullptr, stage) != LNF_OK) {
            best = 1e30f;
            break;
        }
        cudaEventRecord(b, ctx->stream);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// The autotuner: per class of specialised jobs not tuned yet, the work items' z
// length by timing the class's jobs alone; then, once per context and when the
// batch has jobs the specialised kernels do not cover, the generic z chunk.
static void autotune(lnf_ctx *ctx, const lnf_job *jobs, int n, const std::vector<void *> &stage)
{
    std::map<int, std::vector<int>> classes;   // class -> indices of its specialised jobs
    bool generic = false;
    for (int i = 0; i < n; ++i) {
        if (!ctx->no_fast && lnf_fast_covers(jobs[i].filter_id, jobs[i].radius, ctx->cfg.cluster_offset))
            classes[job_class(jobs[i])].push_back(i);
        else
            generic = true;
    }
    std::vector<int> vol_of;
    distinct_inputs(jobs, n, vol_of);
    for (auto &c : classes) {
        if (ctx->tuned_zlen.count(c.first))
            continue;
        std::vector<lnf_job> sub;
        std::vector<void *> sub_stage;   // padded copies, in the class's own order of first use
        std::vector<int> seen;
        for (int i : c.second) {
            sub.push_back(jobs[i]);
            const int v = vol_of[i];
            if (std::find(seen.begin(), seen.end(), v) == seen.end()) {
                seen.push_back(v);
                sub_stage.push_back(v < (int)stage.size() ? stage[v] : nullptr);
            }
        }
        int best = 16;
        float best_ms = 1e30f;
        std::vector<float> times;
        for (int zl : {4, 8, 16, 32}) {
            const float ms = time_batch(ctx, sub.data(), (int)sub.size(), ctx->zchunk, zl, &sub_stage);
            times.push_back(ms);
            if (ms < best_ms) {
                best_ms = ms;
                best = zl;
            }
        }
        ctx->tuned_zlen[c.first] = best;
        ctx->tuned_zlen_ms[c.first] = times;
    }
    if (generic && ctx->tuned_zchunk == 0) {
        int best_zc = 64;
        float best_ms = 1e30f;
        for (int zc : {16, 32, 64, 128}) {
            const float ms = time_batch(ctx, jobs, n, zc, 0, &stage);
            if (ms < best_ms) {
                best_ms = ms;
                best_zc = zc;
            }
        }
        ctx->tuned_zchunk = best_zc;
    }
}

extern "C" lnf_status lnf_get_tuning(lnf_ctx *ctx, int32_t *classes, int32_t *zlen, float *ms, int cap, int *n,
                                     int32_t *generic_zchunk)
{
    if (!ctx || !n || cap < 0 || (cap > 0 && (!classes || !zlen)))
        return LNF_EINVAL;
    int k = 0;
    for (const auto &c : ctx->tuned_zlen) {
        if (k < cap) {
            classes[k] = c.first;
            zlen[k] = c.second;
            if (ms) {
                const std::vector<float> &t = ctx->tuned_zlen_ms[c.first];
                for (int q = 0; q < 4; ++q)
                    ms[4 * k + q] = q < (int)t.size() ? t[q] : 0.0f;
            }
        }
        ++k;
    }
    *n = k;
    if (generic_zchunk)
        *generic_zchunk = ctx->tuned_zchunk;
    return LNF_OK;
}

extern "C" lnf_status lnf_filter_batch(lnf_ctx *ctx, const lnf_job *jobs, int n_jobs)
{
    LNF_RANGE("lnf_filter_batch");
    if (!ctx)
        return LNF_EINVAL;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs))
        return lnf_fail(ctx, LNF_EINVAL, "bad job list");
    if (n_jobs == 0)
        return LNF_OK;
    for (int i = 0; i < n_jobs; ++i) {
        lnf_status s = check_job(ctx, jobs[i], i);
        if (s != LNF_OK)
            return s;
    }
    if (n_jobs > LNF_MAX_PACK) {   // several packs, in order
        for (int i = 0; i < n_jobs; i += LNF_MAX_PACK) {
            lnf_status s = lnf_filter_batch(ctx, jobs + i, std::min(LNF_MAX_PACK, n_jobs - i));
            if (s != LNF_OK)
                return s;
        }
        return LNF_OK;
    }
    for (auto &b : ctx->batches)
        if (b->stream == ctx->stream && same_jobs(b->key, jobs, n_jobs)) {
            CK(cudaGraphLaunch(b->exec, ctx->stream));
            return LNF_OK;
        }
    std::unique_ptr<BatchEntry> e(new BatchEntry());
    // every allocation happens before the capture (none is allowed inside it):
    // one scratch per distinct input, the padded copies
    std::vector<int> vol_of;
    lnf_status ss = lnf_scratch_pool(ctx, distinct_inputs(jobs, n_jobs, vol_of).size());
    if (ss != LNF_OK)
        return ss;
    if ((ss = alloc_stage(ctx, jobs, n_jobs, e->stage)) != LNF_OK)
        return ss;
    batch_streams(ctx);
    if (ctx->cfg.autotune)
        autotune(ctx, jobs, n_jobs, e->stage);
    const int zc = ctx->tuned_zchunk ? ctx->tuned_zchunk : 64;
    e->key.assign(jobs, jobs + n_jobs);
    e->stream = ctx->stream;
    // capture needs a non-default stream
    cudaStream_t cap = ctx->stream;
    bool own = false;
    if (cap == nullptr) {
        CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        own = true;
    }
    CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    lnf_status s = lnf_enqueue_batch(ctx, jobs, n_jobs, zc, 0, cap, nullptr, &e->stage);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cap, &g);
    if (s != LNF_OK || ce != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        if (own)
            cudaStreamDestroy(cap);
        return s != LNF_OK ? s : lnf_fail(ctx, LNF_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    }
    e->graph = g;
    cudaError_t ie = cudaGraphInstantiate(&e->exec, g, 0);
    if (own)
        cudaStreamDestroy(cap);
    if (ie != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    CK(cudaGraphLaunch(e->exec, ctx->stream));
    if (ctx->batches.size() >= 16) {
        destroy_entry(ctx->batches.front());
        ctx->batches.erase(ctx->batches.begin());
    }
    ctx->batches.push_back(e.release());
    return LNF_OK;
}
