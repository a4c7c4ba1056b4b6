// Host-side context of liblnf (internal).
#pragma once

#include "lnf.h"
#include "lnf_internal.cuh"

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

// NVTX ranges around the entry points and the filter launches (header-only
// NVTX 3: free when no profiler is attached)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define LNF_RANGE(name) NvtxRange lnf_range_(name)
#else
#define LNF_RANGE(name) ((void)0)
#endif

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                    CUtensorMapFloatOOBfill);

// Device scratch of one analysed volume: histogram, stats, parameters, weights.
struct VolScratch {
    u64 *hist = nullptr;
    DevStats *st = nullptr;
    DevParams *prm = nullptr;
    u32 *lut = nullptr;
    void *pscr = nullptr;       // parameter-derivation scratch (zeroed once)
};

// Host-side fault injection (testing).  LNF_FAULT, read when a context is
// created, lists sites as "site" (every time) or "site@n" (the n-th time only,
// counted from 1), separated by commas; at a listed site the library behaves as
// if the CUDA call there had failed.  No device code is involved.
enum FaultSite {
    FAULT_SCRATCH = 0,   // lnf_create: the context's scratch allocation
    FAULT_RESIDENT,      // lnf_volume_register: the resident copy's allocation
    FAULT_OUTPUT,        // serving: a request's output allocation
    FAULT_STAGE,         // plain / batched calls: the padded staging copy's allocation
    FAULT_LAUNCH,        // plain / served calls: a filter launch
    FAULT_NSITES
};

struct FaultPlan {
    int64_t nth[FAULT_NSITES] = {};            // 0: off, -1: every time, n: the n-th time
    std::atomic<int64_t> seen[FAULT_NSITES] = {};
};

struct BatchEntry;
// batch.cu
#define LNF_BATCH_STREAMS 8   // side streams made per context
#define LNF_BATCH_CHAINS 8    // chains side by side by default
struct Server;          // serve.cu

struct lnf_ctx {
    lnf_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 1;
    int zchunk = 64;            // z chunk length of a work item (generic kernel)
    int fast_zlen = 0;          // z chunk length of a work item (specialised kernels; 0: automatic)
    bool no_tma = false;        // testing: force plain loads
    bool no_fast = false;       // testing: force the generic kernel
    bool no_gate = false;       // testing: never launch the gate-first kernel (the ring kernels work)
    int gate_mask = 0;          // filter ids a launched gate-first kernel covers (during a multi-filter call)
    VolScratch vs;              // scratch of plain calls
    std::vector<VolScratch> pool;   // scratch of batched / resident volumes
    u64 *out_hist = nullptr;    // LNF_MAX_PACK output histograms of 65536 bins
    double *d_H = nullptr;
    u32 *d_err = nullptr;
    unsigned long long *d_lt = nullptr;   // local entropy filter's table, LNF_LT_MAX + 1 entries
    u32 *d_counter = nullptr;   // work counters: [0] generic, [1..4] serving streams (generic),
                                // [8] paper's filter, [9] comparison filters, [10..13] serving
                                // streams (specialised), [14] fused kernel, [15] the self-test's status word
    // batched launches: the side streams that carry a batch's job chains side by
    // side (one chain per input volume, volume v on stream v % bchains), the fork /
    // join events, and two work counters per job (ring kernel, gate-first kernel)
    // so that chains running at once share none; made on first use
    int bchains = 0;
    cudaStream_t bstream[LNF_BATCH_STREAMS] = {};
    cudaEvent_t bfork = nullptr;
    cudaEvent_t bjoin[LNF_BATCH_STREAMS] = {};
    u32 *d_bcounter = nullptr;      // 2 x LNF_MAX_PACK
    double *d_ent_part = nullptr;   // entropy reduction partials (LNF_ENT_SPLIT x LNF_MAX_ENT)
    u32 *d_ent_done = nullptr;      // entropy reduction tickets (LNF_MAX_ENT)
    PFN_encodeTiled encode = nullptr;
    FilterPack pack;            // host staging of the kernel-parameter pack
    // host-buffer entry points: device staging
    void *st_in = nullptr;
    size_t st_in_cap = 0;
    std::vector<void *> st_out;
    std::vector<size_t> st_out_cap;
    cudaStream_t copy_stream = nullptr;        // device-to-host copies that overlap the filters
    std::vector<cudaEvent_t> filter_done;      // one per filter of a multi-filter call
    // plain calls: a copy of an input TMA cannot address, rows padded to 16 bytes
    void *pitched = nullptr;
    size_t pitched_cap = 0;
    // float32 volumes: the level volumes (input and output, 16-bit) and the range word
    void *f32_lv = nullptr;
    size_t f32_lv_cap = 0;
    u32 *d_range = nullptr;
    // batched graph cache
    std::vector<BatchEntry *> batches;   // owned; freed by lnf_batch_cache_clear
    // autotuner choice for batched launches (0 = not tuned yet)
    int tuned_zchunk = 0;
    // autotuned z length of the specialised kernels' work items, per job class
    // (dtype, filter, radius; see batch.cu), and the candidates' times
    std::map<int, int> tuned_zlen;
    std::map<int, std::vector<float>> tuned_zlen_ms;
    // profiling: events around launches of the plain path, launch counter
    bool prof = false;
    int64_t prof_launches = 0;
    struct ProfRec {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_free;
    FaultPlan fault;            // host-side fault injection (testing)
    // serving
    Server *srv = nullptr;
    std::mutex err_mu;
    std::string err, err_copy;
};

lnf_status lnf_fail(lnf_ctx *ctx, lnf_status s, const char *fmt, ...);
// Parse an LNF_FAULT list into `plan` (false: an unknown site or a bad count)
bool lnf_fault_parse(const char *spec, FaultPlan &plan);
// Whether the injected fault at `site` fires now (counts the visit)
inline bool lnf_fault(lnf_ctx *ctx, FaultSite site)
{
    const int64_t n = ctx->fault.nth[site];
    if (n == 0)
        return false;
    const int64_t k = ctx->fault.seen[site].fetch_add(1) + 1;
    return n < 0 || k == n;
}
lnf_status lnf_check_volume(lnf_ctx *ctx, const void *p, const int64_t dims[3], int dtype);
ParamCfg lnf_param_cfg(const lnf_ctx *ctx);
// the local entropy filter's table t[0..LNF_LT_MAX] to ctx->d_lt (lnf_create)
lnf_status lnf_lt_upload(lnf_ctx *ctx);
lnf_status lnf_scratch_pool(lnf_ctx *ctx, size_t n);
lnf_status lnf_analyze(lnf_ctx *ctx, const void *in, const int64_t dims[3], int dtype, VolScratch &vs,
                       cudaStream_t stream);
// `pitch`: the input's row stride in elements (0: dense rows, = dims[0]);
// `rad3` / `off3`: per-axis radii and cluster offsets (x, y, z) of an
// anisotropic job (null: `radius` and the context's offset on every axis)
lnf_status lnf_make_job(lnf_ctx *ctx, FilterPack &pk, int idx, int filter, int radius, const void *in, void *out,
                        const int64_t dims[3], int dtype, const int64_t *roi_o, const int64_t *roi_d,
                        const VolScratch &vs, u64 *out_hist, int64_t pitch = 0, const int *rad3 = nullptr,
                        const int *off3 = nullptr);
// 3D TMA map of a volume with row stride `pitch` elements, box {box_w, box_h, 1};
// false when the volume does not meet TMA's alignment rules or encoding fails
bool lnf_encode_box(lnf_ctx *ctx, const void *in, int nx, int ny, int nz, int pitch, int dtype, unsigned box_w,
                    unsigned box_h, CUtensorMap *map);
lnf_status lnf_run_pack(lnf_ctx *ctx, FilterPack &pk, int persistent, cudaStream_t stream);
lnf_status lnf_run_pack_counter(lnf_ctx *ctx, FilterPack &pk, int persistent, cudaStream_t stream, u32 *counter);
lnf_status lnf_run_one(lnf_ctx *ctx, int filter, int radius, const void *in, void *out, const int64_t dims[3],
                       int dtype, const int64_t *roi_o, const int64_t *roi_d, const VolScratch &vs,
                       u64 *out_hist, cudaStream_t stream, int64_t pitch = 0, const int *rad3 = nullptr,
                       const int *off3 = nullptr, const void *orig = nullptr);
// Row length in bytes of the padded copy of an input TMA cannot address (0: the
// input itself is addressable: 16-byte-aligned base and row length)
size_t lnf_pitched_row(const void *in, const int64_t dims[3], int dtype);
// pitch.cu: copy `in` into `dst` (16-byte aligned) with rows padded to `prow`
// bytes (a multiple of 16), on `st`; with `skip_prm` the copy kernel returns at
// once while the gate-first kernel takes the volume (lnf_gate_mode(*skip_prm))
lnf_status lnf_copy_pitched(lnf_ctx *ctx, void *dst, size_t prow, const void *in, const int64_t dims[3], int dtype,
                            cudaStream_t st, const DevParams *skip_prm = nullptr);
// A padded copy that lnf_fast_dispatch enqueues between its job's gate-first and
// ring kernels (`done` set once enqueued).  Where the gate-first kernel was
// launched, the copy is skipped on the device while it takes the volume: only
// for a volume whose ring kernels are all launched beside the gate-first kernel
// (the caller's promise), since those return at once in that case.
struct PitchedCopy {
    void *dst;
    size_t prow;
    const void *src;
    const int64_t *dims;
    int dtype;
    const DevParams *prm;
    bool done;
};
// profiling helpers (api.cu): bracket one launch (or a group of `count` launches)
int lnf_prof_begin(lnf_ctx *ctx, cudaStream_t st);
void lnf_prof_end(lnf_ctx *ctx, int rec, const char *name, cudaStream_t st, int count);
// fast.cu: whether a specialised kernel covers this filter, radius and cluster
// offset (on an input TMA can address)
bool lnf_fast_covers(int filter, int radius, int offset);
// fast.cu: whether a specialised kernel takes this filter and radius only while
// few voxels pass the gate (launched with gated = 2 beside the generic kernel,
// whose job is marked FilterJob::gated)
bool lnf_sparse_covers(int filter, int radius);
// fast.cu: run the job through a specialised kernel if one covers it (*handled = the
// number of kernels launched: 1, or 2 with the gate-first kernel beside, else 0);
// `counter` is the launch's work counter (null: the context's own, for its stream)
// `allow_gate`: the gate-first kernel may take a whole-volume job, with
// `gate_counter` as its chunk counter (null: the context's own, which only calls
// on the context's stream may use); `pre`: a padded copy of the job's input to
// enqueue after the gate-first kernel and before the ring kernel
lnf_status lnf_fast_dispatch(lnf_ctx *ctx, const FilterJob &job, const CUtensorMap *tmap, cudaStream_t stream,
                             int *handled, u32 *counter = nullptr, int allow_gate = 0,
                             u32 *gate_counter = nullptr, PitchedCopy *pre = nullptr);
// `gated`: 1 if the gate-first kernel was launched for this job (the ring kernel
// returns at once when that one does the work); 2 for a job lnf_sparse_covers
// names (the kernel returns at once unless few voxels pass)
lnf_status lnf_fast2_dispatch(lnf_ctx *ctx, const FilterJob &job, const CUtensorMap *tmap, cudaStream_t stream,
                              int *handled, u32 *counter = nullptr, int gated = 0);
// fast2_box.cu: the mean / entropy-filter job through its box kernel
lnf_status lnf_fast2_box(lnf_ctx *ctx, const FilterJob &job, cudaStream_t stream, u32 *counter, int *handled,
                         int gated);
// gate.cu: whether the gate-first kernel covers `filter` on the job's volume (a
// whole volume, isotropic radius 1..4, the paper's filter at cluster offset 1),
// and its launch for the filters whose outputs are given (outs / hists indexed
// by filter id 0..4, null where not requested); *handled = 1 if launched;
// `counter`: the launch's chunk counter (null: the context's own, for its stream)
bool lnf_gate_covers(const FilterJob &j, int filter);
// the entropy filter with local probabilities (LNF_ENTROPY_LOCAL) of a whole
// volume through the gate-first kernel; *handled = 1 if launched (the generic
// kernel then skips the job while the gate takes the volume: FilterJob::gated)
lnf_status lnf_gate_launch_eloc(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, int *handled);
lnf_status lnf_gate_launch(lnf_ctx *ctx, const FilterJob &j, void *const outs[5], u64 *const hists[5],
                           cudaStream_t st, int *handled, u32 *counter = nullptr);
// render.cu: one ray per pixel (see lnf_render)
cudaError_t lnf_launch_render(const void *vol, const int64_t dims[3], int64_t pitch, int dtype, int view,
                              int filter, int radius, int offset, const DevParams *prm, const u32 *lut,
                              unsigned char *image, int *depth, u32 *value, cudaStream_t st);
// f32.cu: range (min key, max key, non-finite count), quantisation to and from 65536 levels
cudaError_t lnf_launch_f32_range(const float *in, u64 n, u32 *range, int num_sms, cudaStream_t st);
cudaError_t lnf_launch_f32_quantize(const float *in, u64 n, const u32 *range, uint16_t *q, int num_sms,
                                    cudaStream_t st);
cudaError_t lnf_launch_f32_dequantize(const uint16_t *q, u64 n, const u32 *range, float *out, int num_sms,
                                      cudaStream_t st);
// batch.cu
void lnf_batch_cache_clear(lnf_ctx *ctx);
// the batch streams, events and per-job counters (made on a context's first batch)
void lnf_batch_streams_free(lnf_ctx *ctx);
// serve.cu
void lnf_serve_shutdown(lnf_ctx *ctx);
