// Serving loop: continuous batching of filter requests on resident volumes.
//
// Volumes are registered once (copied into library memory charged to the HBM
// budget, statistics and parameters computed once on the device).  lnf_submit
// queues a request and returns a ticket.  A scheduler thread admits queued
// requests in arrival order while in-flight slots and budget allow, groups
// what it admitted into a "wave" and enqueues the wave on the next of several
// streams: one filter launch per request, each sized for its own filter,
// radius and region (the specialised kernel where it covers the request, else
// the generic one), then one entropy launch for the whole wave.  Waves overlap
// on the device while later requests keep arriving; the scheduler never waits
// for a running wave before admitting more.  A host function enqueued
// after each wave stamps its finish time and wakes the scheduler, which
// retires the wave's requests and frees their memory.  No device code waits
// on the host or on another kernel.
#include "lnf_ctx.h"

#include <algorithm>
#include <chrono>
#include <cstring>

namespace {

constexpr int kStreams = 4;

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Resident {
    void *d_vol = nullptr;
    int64_t dims[3] = {0, 0, 0};
    int64_t pitch = 0;              // row stride in elements: rows padded to 16 bytes (TMA's rule)
    int dtype = 0;
    size_t bytes = 0;
    VolScratch vs;
    int refs = 0;                   // queued or in-flight requests
};

struct Wave;

struct Req {
    uint64_t ticket = 0;
    lnf_request r{};
    int status = LNF_EPENDING;
    bool admitted = false;
    double t_admit = 0, t_start = 0, t_finish = 0;
    double entropy = 0;
    void *d_out = nullptr;
    size_t out_bytes = 0;
    size_t charge = 0;              // bytes charged to the budget while held
    int slot = -1;                  // pinned entropy slot
    Wave *wave = nullptr;
};

struct Wave {
    std::vector<Req *> reqs;
    int stream_idx = 0;
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    double t_done = 0;
    bool done = false;
    Server *srv = nullptr;
};

}  // namespace

struct Server {
    lnf_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv;         // scheduler wake-up
    std::condition_variable done_cv;    // request completion
    std::map<int, Resident> vols;
    int next_vol = 1;
    std::map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1;
    std::deque<Req *> queue;
    std::vector<Wave *> waves;
    size_t used = 0;                    // resident volumes + held outputs
    int inflight = 0;
    bool stop = false;
    std::thread thr;
    cudaStream_t streams[kStreams] = {};
    int next_stream = 0;
    u64 *hists = nullptr;               // max_inflight output histograms (65536 bins)
    double *d_H = nullptr;              // max_inflight entropies (device)
    double *h_H = nullptr;              // pinned mirror
    double *ent_part = nullptr;         // entropy reduction partials, one block per stream
    u32 *ent_done = nullptr;            // entropy reduction tickets, one block per stream
    std::vector<int> free_slots;
    FilterPack pack;                    // the scheduler's own parameter pack
    std::string last_err;
};

namespace {

void CUDART_CB wave_done_cb(void *p)
{
    Wave *w = static_cast<Wave *>(p);
    const double t = now_s();
    Server *s = w->srv;
    {
        std::lock_guard<std::mutex> g(s->mu);
        w->t_done = t;
        w->done = true;
    }
    s->cv.notify_all();
}

size_t req_voxels(const lnf_request &r, const Resident &v)
{
    if (r.roi_dims[0] > 0)
        return (size_t)r.roi_dims[0] * r.roi_dims[1] * r.roi_dims[2];
    return (size_t)v.dims[0] * v.dims[1] * v.dims[2];
}

// retire finished waves (lock held)
void retire(Server *s)
{
    for (size_t i = 0; i < s->waves.size();) {
        Wave *w = s->waves[i];
        if (!w->done) {
            ++i;
            continue;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, w->ev_start, w->ev_done);
        for (Req *q : w->reqs) {
            q->t_finish = w->t_done;
            q->t_start = w->t_done - ms / 1e3;
            q->status = LNF_OK;
            if (q->r.want_entropy && q->slot >= 0)
                q->entropy = s->h_H[q->slot];
            if (q->slot >= 0)
                s->free_slots.push_back(q->slot);
            q->slot = -1;
            if (q->r.out_host && q->d_out) {   // result already copied to the host
                cudaFreeAsync(q->d_out, s->streams[w->stream_idx]);
                q->d_out = nullptr;
                s->used -= q->charge;
                q->charge = 0;
            }
            s->vols[q->r.vol_id].refs -= 1;
            q->wave = nullptr;
            s->inflight -= 1;
        }
        cudaEventDestroy(w->ev_start);
        cudaEventDestroy(w->ev_done);
        delete w;
        s->waves.erase(s->waves.begin() + i);
    }
}

// take admissible requests off the queue (lock held)
std::vector<Req *> admit(Server *s)
{
    std::vector<Req *> out;
    const lnf_config &cfg = s->ctx->cfg;
    while (!s->queue.empty() && (int)out.size() < LNF_MAX_PACK && s->inflight < cfg.max_inflight &&
           !s->free_slots.empty()) {
        Req *q = s->queue.front();
        const Resident &v = s->vols[q->r.vol_id];
        const size_t need = q->out_bytes;
        if (s->used + need > cfg.hbm_budget_bytes)
            break;   // first-come first-served: wait for memory to free up
        s->queue.pop_front();
        s->used += need;
        q->charge = need;
        q->admitted = true;
        q->t_admit = now_s();
        q->slot = s->free_slots.back();
        s->free_slots.pop_back();
        s->inflight += 1;
        (void)v;
        out.push_back(q);
    }
    return out;
}

// launch one wave (lock NOT held; the requests are owned by the wave)
lnf_status launch_wave(Server *s, Wave *w)
{
    lnf_ctx *ctx = s->ctx;
    cudaStream_t st = s->streams[w->stream_idx];
    FilterPack &pk = s->pack;
    std::memset(&pk, 0, sizeof(int) * 16);
    // every request is its own launch on the wave's stream, sized for its own
    // filter and radius (a shared launch would run every job at the largest
    // job's shared memory and occupancy); a specialised kernel takes the
    // request when it covers it (with this stream's own work counter), else
    // the generic kernel
    u32 *fast_counter = ctx->d_counter + 10 + w->stream_idx;
    EntropyPack ep;
    std::memset(&ep, 0, sizeof ep);
    cudaEventCreateWithFlags(&w->ev_start, cudaEventDefault);
    cudaEventCreateWithFlags(&w->ev_done, cudaEventDefault);
    cudaEventRecord(w->ev_start, st);
    for (int i = 0; i < (int)w->reqs.size(); ++i) {
        Req *q = w->reqs[i];
        Resident *v;
        {
            std::lock_guard<std::mutex> g(s->mu);
            v = &s->vols[q->r.vol_id];
        }
        if (lnf_fault(ctx, FAULT_OUTPUT) || cudaMallocAsync(&q->d_out, q->out_bytes, st) != cudaSuccess) {
            q->d_out = nullptr;
            return lnf_fail(ctx, LNF_ENOMEM, "serving: output allocation of %zu bytes failed", q->out_bytes);
        }
        u64 *oh = nullptr;
        if (q->r.want_entropy) {
            oh = s->hists + (size_t)q->slot * LNF_LEVELS_U16;
            const u32 levels = v->dtype == LNF_U8 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
            if (lnf_launch_zero(oh, levels, st) != cudaSuccess)
                return lnf_fail(ctx, LNF_ECUDA, "serving: histogram reset failed");
            const int k = ep.count++;
            ep.hist[k] = oh;
            ep.levels[k] = levels;
            ep.n[k] = req_voxels(q->r, *v);
            ep.H[k] = s->d_H + q->slot;
        }
        const bool roi = q->r.roi_dims[0] > 0;
        pk.n_jobs = 1;
        lnf_status r = lnf_make_job(ctx, pk, 0, q->r.filter_id, q->r.radius, v->d_vol, q->d_out, v->dims,
                                    v->dtype, roi ? q->r.roi_origin : nullptr, roi ? q->r.roi_dims : nullptr, v->vs,
                                    oh, v->pitch);
        if (r != LNF_OK)
            return r;
        if (lnf_fault(ctx, FAULT_LAUNCH))
            return lnf_fail(ctx, LNF_ECUDA, "injected fault: filter launch failed");
        int handled = 0;
        if (!ctx->no_fast) {
            FilterJob &j = pk.jobs[0];
            // sigma at r = 3..4: the tap kernel while few voxels pass the gate,
            // the generic kernel (its job marked gated) otherwise
            if (lnf_sparse_covers(j.filter, j.radius) && !ctx->no_gate && j.tmap_idx >= 0 && !j.aniso) {
                int sparse = 0;
                r = lnf_fast2_dispatch(ctx, j, &pk.tmaps[j.tmap_idx], st, &sparse, fast_counter, 2);
                if (r != LNF_OK)
                    return r;
                j.gated = sparse ? 1 : 0;
            }
            r = lnf_fast_dispatch(ctx, j, j.tmap_idx >= 0 ? &pk.tmaps[j.tmap_idx] : nullptr, st, &handled,
                                  fast_counter);
            if (r != LNF_OK)
                return r;
        }
        if (!handled && (r = lnf_run_pack_counter(ctx, pk, 0, st, nullptr)) != LNF_OK)
            return r;
    }
    if (lnf_launch_entropy_pack(ep, s->ent_part + (size_t)w->stream_idx * LNF_ENT_SPLIT * LNF_MAX_ENT,
                                s->ent_done + (size_t)w->stream_idx * LNF_MAX_ENT, st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "serving: entropy launch failed");
    for (Req *q : w->reqs) {
        if (q->r.out_host)
            cudaMemcpyAsync(q->r.out_host, q->d_out, q->out_bytes, cudaMemcpyDeviceToHost, st);
        if (q->r.want_entropy)
            cudaMemcpyAsync(s->h_H + q->slot, s->d_H + q->slot, sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    cudaEventRecord(w->ev_done, st);
    if (cudaLaunchHostFunc(st, wave_done_cb, w) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "serving: host callback enqueue failed");
    return LNF_OK;
}

void scheduler(Server *s)
{
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] {
            if (s->stop)
                return true;
            for (Wave *w : s->waves)
                if (w->done)
                    return true;
            return !s->queue.empty() && s->inflight < s->ctx->cfg.max_inflight && !s->free_slots.empty() &&
                   s->used + s->queue.front()->out_bytes <= s->ctx->cfg.hbm_budget_bytes;
        });
        retire(s);
        s->done_cv.notify_all();
        if (s->stop && s->waves.empty())
            break;
        if (s->stop)
            continue;
        std::vector<Req *> batch = admit(s);
        if (batch.empty())
            continue;
        Wave *w = new Wave();
        w->srv = s;
        w->reqs = batch;
        w->stream_idx = s->next_stream;
        s->next_stream = (s->next_stream + 1) % kStreams;
        for (Req *q : batch)
            q->wave = w;
        s->waves.push_back(w);
        lk.unlock();
        lnf_status r = launch_wave(s, w);
        lk.lock();
        if (r != LNF_OK) {
            // the wave did not reach the device whole: fail its requests.  What
            // it did enqueue finishes first, so that no slot (histogram, entropy)
            // or output is handed on while a kernel of this wave may still write it
            lk.unlock();
            cudaStreamSynchronize(s->streams[w->stream_idx]);
            lk.lock();
            s->last_err = lnf_last_error(s->ctx);
            for (Req *q : w->reqs) {
                if (q->d_out)
                    cudaFreeAsync(q->d_out, s->streams[w->stream_idx]);
                q->d_out = nullptr;
                q->status = r;
                q->t_finish = now_s();
                if (q->slot >= 0)
                    s->free_slots.push_back(q->slot);
                q->slot = -1;
                s->used -= q->charge;
                q->charge = 0;
                s->vols[q->r.vol_id].refs -= 1;
                s->inflight -= 1;
                q->wave = nullptr;
            }
            s->waves.erase(std::find(s->waves.begin(), s->waves.end(), w));
            if (w->ev_start)
                cudaEventDestroy(w->ev_start);
            if (w->ev_done)
                cudaEventDestroy(w->ev_done);
            delete w;
            s->done_cv.notify_all();
        }
    }
}

lnf_status ensure_server(lnf_ctx *ctx)
{
    if (ctx->srv)
        return LNF_OK;
    Server *s = new Server();
    s->ctx = ctx;
    const int slots = ctx->cfg.max_inflight;
    bool ok = true;
    for (int i = 0; i < kStreams && ok; ++i)
        ok = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMalloc(&s->hists, sizeof(u64) * LNF_LEVELS_U16 * slots) == cudaSuccess;
    ok = ok && cudaMalloc(&s->d_H, sizeof(double) * slots) == cudaSuccess;
    ok = ok && cudaHostAlloc(&s->h_H, sizeof(double) * slots, cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaMalloc(&s->ent_part, sizeof(double) * kStreams * LNF_ENT_SPLIT * LNF_MAX_ENT) == cudaSuccess;
    ok = ok && cudaMalloc(&s->ent_done, sizeof(u32) * kStreams * LNF_MAX_ENT) == cudaSuccess;
    ok = ok && cudaMemset(s->ent_done, 0, sizeof(u32) * kStreams * LNF_MAX_ENT) == cudaSuccess;
    if (ok) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (!ok) {
        for (auto st : s->streams)
            if (st)
                cudaStreamDestroy(st);
        cudaFree(s->hists);
        cudaFree(s->d_H);
        cudaFreeHost(s->h_H);
        cudaFree(s->ent_part);
        cudaFree(s->ent_done);
        delete s;
        return lnf_fail(ctx, LNF_ENOMEM, "serving: could not allocate the scheduler's buffers");
    }
    for (int i = slots - 1; i >= 0; --i)
        s->free_slots.push_back(i);
    s->thr = std::thread(scheduler, s);
    ctx->srv = s;
    return LNF_OK;
}

}  // namespace

void lnf_serve_shutdown(lnf_ctx *ctx)
{
    Server *s = ctx->srv;
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        for (Req *q : s->queue) {
            q->status = LNF_ECANCELLED;
            s->vols[q->r.vol_id].refs -= 1;
        }
        s->queue.clear();
    }
    s->cv.notify_all();
    s->thr.join();
    for (auto st : s->streams)
        cudaStreamSynchronize(st);
    for (auto &kv : s->reqs) {
        if (kv.second->d_out)
            cudaFreeAsync(kv.second->d_out, s->streams[0]);
        delete kv.second;
    }
    cudaStreamSynchronize(s->streams[0]);
    for (auto &kv : s->vols) {
        cudaFree(kv.second.d_vol);
        cudaFree(kv.second.vs.hist);
        cudaFree(kv.second.vs.st);
        cudaFree(kv.second.vs.prm);
        cudaFree(kv.second.vs.lut);
        cudaFree(kv.second.vs.pscr);
    }
    for (auto st : s->streams)
        cudaStreamDestroy(st);
    cudaFree(s->hists);
    cudaFree(s->d_H);
    cudaFreeHost(s->h_H);
    cudaFree(s->ent_part);
    cudaFree(s->ent_done);
    delete s;
    ctx->srv = nullptr;
}

#define CKS(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return lnf_fail(ctx, LNF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));             \
    } while (0)

extern "C" double lnf_now(void) { return now_s(); }

extern "C" lnf_status lnf_volume_register(lnf_ctx *ctx, const void *src, int src_is_host, const int64_t dims[3],
                                          int dtype, int *vol_id)
{
    LNF_RANGE("lnf_volume_register");
    if (!ctx || !vol_id)
        return LNF_EINVAL;
    lnf_status st = lnf_check_volume(ctx, src, dims, dtype);
    if (st != LNF_OK)
        return st;
    if ((st = ensure_server(ctx)) != LNF_OK)
        return st;
    Server *s = ctx->srv;
    Resident v;
    v.dims[0] = dims[0];
    v.dims[1] = dims[1];
    v.dims[2] = dims[2];
    v.dtype = dtype;
    const size_t es = dtype == LNF_U8 ? 1 : 2;
    // rows padded to a multiple of 16 bytes, so that every resident volume can be
    // read by TMA (the specialised kernels) whatever its width
    v.pitch = (int64_t)(((size_t)dims[0] * es + 15) / 16 * 16 / es);
    v.bytes = (size_t)v.pitch * dims[1] * dims[2] * es;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->used + v.bytes > ctx->cfg.hbm_budget_bytes)
            return lnf_fail(ctx, LNF_EBUDGET, "registering %zu bytes exceeds the HBM budget (%zu of %llu in use)",
                            v.bytes, s->used, (unsigned long long)ctx->cfg.hbm_budget_bytes);
        s->used += v.bytes;
    }
    auto undo = [&](lnf_status e) {
        std::lock_guard<std::mutex> g(s->mu);
        s->used -= v.bytes;
        return e;
    };
    cudaStream_t st0 = s->streams[0];
    if (lnf_fault(ctx, FAULT_RESIDENT) || cudaMalloc(&v.d_vol, v.bytes) != cudaSuccess) {
        v.d_vol = nullptr;
        return undo(lnf_fail(ctx, LNF_ENOMEM, "resident volume allocation failed"));
    }
    if (cudaMalloc(&v.vs.hist, sizeof(u64) * LNF_LEVELS_U16) != cudaSuccess ||
        cudaMalloc(&v.vs.st, sizeof(DevStats)) != cudaSuccess ||
        cudaMalloc(&v.vs.prm, sizeof(DevParams)) != cudaSuccess ||
        cudaMalloc(&v.vs.lut, sizeof(u32) * LNF_LEVELS_U16) != cudaSuccess ||
        cudaMalloc(&v.vs.pscr, lnf_param_scratch_bytes()) != cudaSuccess ||
        cudaMemset(v.vs.pscr, 0, lnf_param_scratch_bytes()) != cudaSuccess) {
        cudaFree(v.d_vol);
        return undo(lnf_fail(ctx, LNF_ENOMEM, "resident volume scratch allocation failed"));
    }
    // the statistics read dense rows: the caller's device buffer itself, or a
    // dense staging copy of a host buffer; then the rows go to their padded places
    const size_t row = (size_t)dims[0] * es;
    const void *dense = src;
    void *tmp = nullptr;
    if (src_is_host) {
        if (v.pitch == dims[0]) {
            dense = v.d_vol;   // already dense: stage in place
        } else if (cudaMalloc(&tmp, row * dims[1] * dims[2]) != cudaSuccess) {
            cudaFree(v.d_vol);
            return undo(lnf_fail(ctx, LNF_ENOMEM, "resident volume staging allocation failed"));
        } else {
            dense = tmp;
        }
        if (cudaMemcpyAsync(const_cast<void *>(dense), src, row * dims[1] * dims[2], cudaMemcpyHostToDevice, st0) !=
            cudaSuccess) {
            cudaFree(tmp);
            cudaFree(v.d_vol);
            return undo(lnf_fail(ctx, LNF_ECUDA, "resident volume upload failed"));
        }
    }
    if ((st = lnf_analyze(ctx, dense, v.dims, dtype, v.vs, st0)) != LNF_OK) {
        cudaStreamSynchronize(st0);
        cudaFree(tmp);
        cudaFree(v.d_vol);
        return undo(st);
    }
    if (dense != v.d_vol &&
        cudaMemcpy2DAsync(v.d_vol, (size_t)v.pitch * es, dense, row, row, (size_t)dims[1] * dims[2],
                          cudaMemcpyDeviceToDevice, st0) != cudaSuccess) {
        cudaStreamSynchronize(st0);
        cudaFree(tmp);
        cudaFree(v.d_vol);
        return undo(lnf_fail(ctx, LNF_ECUDA, "resident volume copy failed"));
    }
    const cudaError_t done = cudaStreamSynchronize(st0);
    cudaFree(tmp);
    if (done != cudaSuccess)
        return undo(lnf_fail(ctx, LNF_ECUDA, "statistics of the resident volume failed"));

    std::lock_guard<std::mutex> g(s->mu);
    *vol_id = s->next_vol++;
    s->vols[*vol_id] = v;
    return LNF_OK;
}

extern "C" lnf_status lnf_volume_unregister(lnf_ctx *ctx, int vol_id)
{
    if (!ctx || !ctx->srv)
        return LNF_EINVAL;
    Server *s = ctx->srv;
    Resident v;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->vols.find(vol_id);
        if (it == s->vols.end())
            return lnf_fail(ctx, LNF_ENOTFOUND, "no resident volume %d", vol_id);
        if (it->second.refs > 0)
            return lnf_fail(ctx, LNF_EPENDING, "volume %d still has %d requests", vol_id, it->second.refs);
        v = it->second;
        s->vols.erase(it);
        s->used -= v.bytes;
    }
    for (auto st : s->streams)
        cudaStreamSynchronize(st);
    cudaFree(v.d_vol);
    cudaFree(v.vs.hist);
    cudaFree(v.vs.st);
    cudaFree(v.vs.prm);
    cudaFree(v.vs.lut);
    cudaFree(v.vs.pscr);
    return LNF_OK;
}

extern "C" lnf_status lnf_submit(lnf_ctx *ctx, const lnf_request *req, uint64_t *ticket)
{
    LNF_RANGE("lnf_submit");
    if (!ctx || !req || !ticket)
        return LNF_EINVAL;
    lnf_status st = ensure_server(ctx);
    if (st != LNF_OK)
        return st;
    Server *s = ctx->srv;
    if (req->filter_id < LNF_MEAN || req->filter_id > LNF_ENTROPY_LOCAL || req->radius < 0 || req->radius > LNF_MAX_RADIUS)
        return lnf_fail(ctx, LNF_EINVAL, "request: filter %d / radius %d out of range", req->filter_id, req->radius);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->vols.find(req->vol_id);
    if (it == s->vols.end())
        return lnf_fail(ctx, LNF_ENOTFOUND, "request: no resident volume %d", req->vol_id);
    Resident &v = it->second;
    const bool roi = req->roi_dims[0] > 0 || req->roi_dims[1] > 0 || req->roi_dims[2] > 0;
    if (roi)
        for (int a = 0; a < 3; ++a)
            if (req->roi_dims[a] < 1 || req->roi_origin[a] < 0 || req->roi_origin[a] + req->roi_dims[a] > v.dims[a])
                return lnf_fail(ctx, LNF_EINVAL, "request: ROI axis %d outside volume %d", a, req->vol_id);
    Req *q = new Req();
    q->r = *req;
    if (!roi)
        std::memset(q->r.roi_dims, 0, sizeof q->r.roi_dims);
    q->out_bytes = req_voxels(q->r, v) * (v.dtype == LNF_U8 ? 1 : 2);
    size_t resident = 0;
    for (auto &kv : s->vols)
        resident += kv.second.bytes;
    if (resident + q->out_bytes > ctx->cfg.hbm_budget_bytes) {
        delete q;
        return lnf_fail(ctx, LNF_EBUDGET, "request output of %zu bytes can never fit the HBM budget",
                        (size_t)req_voxels(*req, v) * (v.dtype == LNF_U8 ? 1 : 2));
    }
    q->ticket = s->next_ticket++;
    v.refs += 1;
    s->reqs[q->ticket] = q;
    s->queue.push_back(q);
    *ticket = q->ticket;
    lk.unlock();
    s->cv.notify_all();
    return LNF_OK;
}

static void fill_result(const Req *q, lnf_result *res)
{
    if (!res)
        return;
    std::memset(res, 0, sizeof *res);
    res->status = q->status;
    res->entropy = q->entropy;
    res->t_admit = q->t_admit;
    res->t_start = q->t_start;
    res->t_finish = q->t_finish;
}

extern "C" lnf_status lnf_poll(lnf_ctx *ctx, uint64_t ticket, lnf_result *res)
{
    if (!ctx || !ctx->srv)
        return LNF_EINVAL;
    Server *s = ctx->srv;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return LNF_ENOTFOUND;
    fill_result(it->second, res);
    return it->second->status == LNF_EPENDING ? LNF_EPENDING : LNF_OK;
}

extern "C" lnf_status lnf_wait(lnf_ctx *ctx, uint64_t ticket, double timeout_s, lnf_result *res)
{
    LNF_RANGE("lnf_wait");
    if (!ctx || !ctx->srv)
        return LNF_EINVAL;
    Server *s = ctx->srv;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return LNF_ENOTFOUND;
    Req *q = it->second;
    const bool done = s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                          [&] { return q->status != LNF_EPENDING; });
    fill_result(q, res);
    return done ? LNF_OK : LNF_ETIMEOUT;
}

extern "C" lnf_status lnf_result_copy(lnf_ctx *ctx, uint64_t ticket, void *dst_host, size_t bytes)
{
    LNF_RANGE("lnf_result_copy");
    if (!ctx || !ctx->srv || !dst_host)
        return LNF_EINVAL;
    Server *s = ctx->srv;
    void *src = nullptr;
    size_t n = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end())
            return LNF_ENOTFOUND;
        Req *q = it->second;
        if (q->status == LNF_EPENDING)
            return LNF_EPENDING;
        if (q->status != LNF_OK || !q->d_out)
            return lnf_fail(ctx, LNF_EINVAL, "ticket %llu has no device result", (unsigned long long)ticket);
        if (bytes < q->out_bytes)
            return lnf_fail(ctx, LNF_EINVAL, "destination holds %zu bytes, result is %zu", bytes, q->out_bytes);
        src = q->d_out;
        n = q->out_bytes;
    }
    CKS(cudaMemcpy(dst_host, src, n, cudaMemcpyDeviceToHost));
    return LNF_OK;
}

extern "C" lnf_status lnf_cancel(lnf_ctx *ctx, uint64_t ticket)
{
    if (!ctx || !ctx->srv)
        return LNF_EINVAL;
    Server *s = ctx->srv;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return LNF_ENOTFOUND;
    Req *q = it->second;
    if (q->admitted || q->status != LNF_EPENDING)
        return LNF_EPENDING;
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), q));
    q->status = LNF_ECANCELLED;
    q->t_finish = now_s();
    s->vols[q->r.vol_id].refs -= 1;
    s->done_cv.notify_all();
    return LNF_OK;
}

extern "C" lnf_status lnf_release(lnf_ctx *ctx, uint64_t ticket)
{
    if (!ctx || !ctx->srv)
        return LNF_EINVAL;
    Server *s = ctx->srv;
    void *d = nullptr;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end())
            return LNF_ENOTFOUND;
        Req *q = it->second;
        if (q->status == LNF_EPENDING)
            return LNF_EPENDING;
        d = q->d_out;
        s->used -= q->charge;
        delete q;
        s->reqs.erase(it);
    }
    if (d)
        cudaFreeAsync(d, s->streams[0]);   // the wave that wrote it has finished
    s->cv.notify_all();
    return LNF_OK;
}

extern "C" lnf_status lnf_serving_stats(lnf_ctx *ctx, uint64_t *budget_used, int *queued, int *inflight)
{
    if (!ctx)
        return LNF_EINVAL;
    if (!ctx->srv) {
        if (budget_used)
            *budget_used = 0;
        if (queued)
            *queued = 0;
        if (inflight)
            *inflight = 0;
        return LNF_OK;
    }
    Server *s = ctx->srv;
    std::lock_guard<std::mutex> g(s->mu);
    if (budget_used)
        *budget_used = s->used;
    if (queued)
        *queued = (int)s->queue.size();
    if (inflight)
        *inflight = s->inflight;
    return LNF_OK;
}
