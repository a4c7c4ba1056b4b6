/*
 * lnf.h -- C ABI of the GB300 (sm_103a) local noise filter library.
 *
 * Implements the data-parallel hot path of arXiv 1807.03119, "Real-time Local
 * Noise Filter in 3D Visualization of CT Data": the paper's spatially variant
 * filter (section "Our Method", Eq. 2-3: the mean of nine axis-cross "average
 * clusters", one at the voxel and eight at the diagonal offsets (+-d,+-d,+-d))
 * and the four comparison filters of section "3D Spatial Noise Filters" (mean
 * Eq. 4, sigma Eq. 5, Okada Eq. 6, entropy Eq. 7), all gated by the Otsu
 * threshold (Eq. 1), applied to every voxel of a CT volume; plus the image
 * entropy measure the paper uses to compare them (Fig. 4).
 *
 * Conventions shared by every entry point
 *   - A volume is a dense grid of nx*ny*nz grey values, uint8 or uint16,
 *     laid out x-fastest: idx = (z*ny + y)*nx + x.  dims = {nx, ny, nz}.
 *   - Kernel size M = 2*radius + 1 (Eq. 3 needs M odd), 0 <= radius <= 8.
 *   - Outside the volume, samples repeat the border value (clamp to edge).
 *   - An average a/b is rounded to the input type half-up: floor((2a+b)/(2b)).
 *   - Noise gate: a voxel is kept only if its own value P0 >= T and the
 *     unrounded filter value is >= T (compared as sum >= T*count); otherwise
 *     the output is 0 ("0, otherwise" of Eq. 6 and Eq. 7).  T is the Otsu
 *     threshold of the whole volume (Eq. 1; ties to the smallest level; a
 *     single-level volume gives T = that level), a fixed value, or 0.
 *   - All arithmetic on the filter path is exact integer arithmetic; results
 *     are bit-exact with the CPU oracle of this repository.
 *
 * Memory and streams
 *   - Unless a name ends in _host, volume pointers are DEVICE pointers owned by
 *     the caller.  The output must not overlap the input (LNF_EINVAL).
 *   - The library owns its scratch (histograms, parameter block, weight table,
 *     staging buffers, resident volumes) and frees it in lnf_destroy.
 *   - Device work is enqueued on the context's stream (lnf_config.stream, a
 *     cudaStream_t; NULL = the legacy default stream).  Device-pointer entry
 *     points return once the work is enqueued; they never synchronise the
 *     host, except where stated.
 *   - Errors are returned as lnf_status codes; the library never aborts.
 *     lnf_last_error() gives a human-readable message for the last failure.
 *
 * Threading: a context may be used by one host thread at a time, except for
 * lnf_submit / lnf_poll / lnf_cancel, which are thread-safe.
 */
#ifndef LNF_H
#define LNF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lnf_status {
    LNF_OK = 0,
    LNF_EINVAL = 1,     /* bad argument */
    LNF_ENOMEM = 2,     /* device or host allocation failed */
    LNF_EBUDGET = 3,    /* request can never fit the context's HBM budget */
    LNF_EPENDING = 4,   /* lnf_poll: request not finished yet */
    LNF_ECUDA = 5,      /* a CUDA runtime call failed (message in lnf_last_error) */
    LNF_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
    LNF_ENOTFOUND = 7,  /* unknown volume id or ticket */
    LNF_ECANCELLED = 8  /* the request was cancelled before it ran */
} lnf_status;

typedef enum lnf_dtype { LNF_U8 = 0, LNF_U16 = 1 } lnf_dtype;

/* Filter ids in the order of the paper's Fig. 5. */
typedef enum lnf_filter_id {
    LNF_MEAN = 0,     /* Eq. 4: mean of the M^3 cube */
    LNF_SIGMA = 1,    /* Eq. 5: mean of cube voxels with |P_i - P0| <= k*sigma (global sigma) */
    LNF_ENTROPY = 2,  /* Eq. 7: P0 if the cube's criterion -sum p_i log2 p_i exceeds T_e, else 0 */
    LNF_OKADA = 3,    /* Eq. 6: mean of the centre and its axis-cross neighbours with |P0 - P_i| < T_d */
    LNF_OURS = 4,     /* Eq. 2-3: mean of the nine average clusters S_0..S_8 */
    /* Cluster-layout variants of the paper's filter ("Our Method" carries a
       commented-out S_0; the conclusion proposes other layouts): the same nine
       cluster centres and combination, each cluster being */
    LNF_OURS_CROSS7 = 5,  /* its centre and axis cross of arm r, averaged (r = 1: (P0 + 6 neighbours) / 7) */
    LNF_OURS_CUBE = 6,    /* the M^3 cube around its centre, averaged */
    LNF_SIGMA_LOCAL = 7,  /* Eq. 5 with the local sigma of the M^3 cube (Lee's original, "Related Work"):
                             |P_i - P0| <= k sigma_cube, k = sigma_k */
    LNF_ENTROPY_LOCAL = 8 /* entropy filter with the cube's own grey-level probabilities (the kernel
                             entropy of "Related Work"): with c_g cube voxels at level g, keep P0 iff
                             P0 >= T and t[m] - sum_g t[c_g] > m theta, t[c] = round(2^22 c log2 c)
                             (40-bit repeated-squaring log2), theta = entropy_local_te_q */
} lnf_filter_id;

typedef enum lnf_threshold_mode {
    LNF_THRESH_OTSU = 0,   /* Eq. 1 on the whole volume (default, as in the paper's evaluation) */
    LNF_THRESH_FIXED = 1,  /* threshold_value */
    LNF_THRESH_NONE = 2    /* T = 0: the gate always passes */
} lnf_threshold_mode;

#define LNF_MAX_RADIUS 8
#define LNF_TD_AUTO (-1)        /* okada_td: floor(sigma) + 1, i.e. |P0 - P_i| <= sigma */
#define LNF_TE_AUTO (-2)        /* entropy_te_q: the expected criterion of a kernel */
#define LNF_TE_PASS_ALL (-1)    /* entropy_te_q: every voxel passes the entropy test */

/* Context configuration.  lnf_config_default() fills the defaults. */
typedef struct lnf_config {
    void *stream;               /* cudaStream_t all work is enqueued on (NULL = default stream) */
    uint64_t hbm_budget_bytes;  /* serving: device bytes for resident volumes + in-flight outputs
                                   (0 = 40 GiB) */
    int32_t max_inflight;       /* serving: requests on the device at once (0 = 64) */
    int32_t threshold_mode;     /* lnf_threshold_mode */
    uint32_t threshold_value;   /* T for LNF_THRESH_FIXED */
    int32_t sigma_k;            /* sigma band half-width in units of sigma (Eq. 5 uses 2) */
    int64_t okada_td;           /* T_d (>= 0) or LNF_TD_AUTO */
    int64_t entropy_te_q;       /* T_e in weight units (>= 0), LNF_TE_AUTO or LNF_TE_PASS_ALL */
    int32_t cluster_offset;     /* d of the diagonal clusters (paper: 1, distance sqrt(3)); 0..8 */
    int32_t autotune;           /* 1: pick tile shapes by measurement on first use */
    int64_t entropy_local_te_q; /* theta of LNF_ENTROPY_LOCAL in 2^-22 bits (>= 0), LNF_TE_AUTO
                                   (log2(m) / 2: floor(t[m] / 2m)) or LNF_TE_PASS_ALL */
} lnf_config;

/* Parameters derived from a volume's statistics (read back by lnf_get_params). */
typedef struct lnf_params {
    uint64_t n_voxels;          /* N */
    uint64_t sum;               /* S = sum P */
    uint64_t sum_sq;            /* Q = sum P^2 */
    uint32_t min_value, max_value;
    uint32_t threshold;         /* T (Eq. 1 or fixed or 0) */
    uint32_t sigma_band;        /* delta: |P_i - P0| <= k sigma  <=>  |P_i - P0| <= delta */
    int64_t okada_td;           /* T_d in use */
    uint64_t weight_sum;        /* sum_v h[v] w[v]: the expected criterion per voxel, times N */
    double input_entropy;       /* Shannon entropy of the input histogram, bits */
} lnf_params;

typedef struct lnf_ctx lnf_ctx;

/* Fill *cfg with defaults: Otsu gate, sigma_k 2, T_d and T_e automatic, d = 1. */
void lnf_config_default(lnf_config *cfg);

/* Create a context on the current CUDA device.  Allocates the fixed scratch
 * (about 3 MiB).  Returns LNF_EINVAL for a bad config, LNF_ENOMEM/LNF_ECUDA.
 *
 * Testing: the environment variable LNF_FAULT, read here, injects host-side
 * failures into this context.  It lists sites, separated by commas, each as
 * "site" (every time) or "site@n" (the n-th time only, from 1):
 *   scratch   scratch allocation of an analysed volume   -> LNF_ENOMEM
 *   resident  lnf_volume_register's resident copy        -> LNF_ENOMEM, budget restored
 *   output    a served request's output allocation       -> that request ends LNF_ENOMEM
 *   launch    a filter launch (plain call, served request) -> LNF_ECUDA
 *   stage     the padded copy of an input TMA cannot read -> none: the generic kernel runs
 * An unknown site or a bad count returns LNF_EINVAL before the device is touched. */
lnf_status lnf_create(const lnf_config *cfg, lnf_ctx **out);

/* Wait for the context's work, stop its scheduler and free everything it owns. */
void lnf_destroy(lnf_ctx *ctx);

/* Change the stream later calls enqueue on (a cudaStream_t). */
lnf_status lnf_set_stream(lnf_ctx *ctx, void *stream);

/* Message of the last failed call on this context (valid until the next call). */
const char *lnf_last_error(lnf_ctx *ctx);

/*
 * Filter one volume: out[v] = filter(in)[v] for every voxel v.
 * Runs on the device: the statistics pass (histogram, S, Q, min, max), the
 * parameter derivation (Otsu T, sigma band, T_d, entropy weights), then the
 * filter.  in/out: device buffers of nx*ny*nz elements of `dtype`, x-fastest.
 * Enqueued on the context's stream; no host synchronisation.
 * Errors: LNF_EINVAL (filter_id, radius, dtype, dims < 1, null or overlapping
 * buffers, more than 2^32 - 1 voxels), LNF_ECUDA.
 */
lnf_status lnf_filter_volume(lnf_ctx *ctx, int filter_id, int radius, const void *in, void *out,
                             const int64_t dims[3], int dtype);

/*
 * Filter one volume with several filters at the same radius, computing the
 * statistics once: outs[i] = filter_ids[i](in).  If d_entropy is not NULL it is
 * a DEVICE array of n+1 doubles that receives the image entropy (Fig. 4) of the
 * input and of each output, in that order; the output histograms are fused
 * into the filter kernels.  Enqueued; no host synchronisation.  The outputs must
 * not overlap the input or one another (LNF_EINVAL): mean, sigma, entropy filter
 * and Okada may be computed together in one pass.
 */
lnf_status lnf_filter_multi(lnf_ctx *ctx, int radius, const void *in, const int64_t dims[3], int dtype,
                            int n, const int *filter_ids, void *const *outs, double *d_entropy);

/*
 * The same with HOST buffers (pageable or, faster, pinned): copies `in` to the
 * device, runs lnf_filter_multi and copies the outputs back into outs[i] and
 * the n+1 entropies into entropy (host, may be NULL).  Synchronous.
 */
lnf_status lnf_filter_multi_host(lnf_ctx *ctx, int radius, const void *in, const int64_t dims[3], int dtype,
                                 int n, const int *filter_ids, void *const *outs, double *entropy);

/*
 * Filter a region of interest: out receives roi_dims[0]*roi_dims[1]*roi_dims[2]
 * voxels, x-fastest, equal to the crop at roi_origin of the whole-volume
 * result (halo samples come from the whole volume; the statistics are those of
 * the whole volume; clamping happens only at the volume's own border).
 */
lnf_status lnf_filter_roi(lnf_ctx *ctx, int filter_id, int radius, const void *in, const int64_t dims[3],
                          int dtype, const int64_t roi_origin[3], const int64_t roi_dims[3], void *out);

/*
 * Anisotropic voxel spacing.  The paper's volumes are isotropic; for a grid
 * whose spacing differs per axis every filter takes a radius and a cluster
 * offset per axis (x, y, z): the cube of M^3 voxels (mean Eq. 4, sigma Eq. 5,
 * entropy Eq. 7, local sigma) becomes the box of Mx*My*Mz voxels, M_a = 2 r_a + 1;
 * the Okada cross (Eq. 6) has arm r_a along axis a; a cluster of the paper's
 * filter (Eq. 2-3) averages its x-, y- and z-lines of Mx, My and Mz voxels (so
 * A = U / (9 (Mx + My + Mz))) and the diagonal clusters sit at (+-dx, +-dy, +-dz);
 * the entropy threshold's default kernel has Mx*My*Mz voxels.  Equal axes give
 * exactly lnf_filter_volume.
 *
 * radius: 3 radii in 0..LNF_MAX_RADIUS (host array).  offset: 3 cluster offsets
 * in 0..8 (host array), or NULL for the context's cluster_offset on every axis.
 * Other arguments, layout, ownership and errors as lnf_filter_volume.  Jobs
 * with unequal axes run in the generic kernel.
 */
lnf_status lnf_filter_volume_aniso(lnf_ctx *ctx, int filter_id, const int radius[3], const int offset[3],
                                   const void *in, void *out, const int64_t dims[3], int dtype);

/*
 * Per-axis radii, in voxels, of a physical extent on a grid of voxel spacing
 * spacing[3] (x, y, z; same unit as extent): radius[a] = floor(extent /
 * spacing[a] + 1/2) in IEEE double (round half up).  Host only; no context.
 * Errors: LNF_EINVAL for a null pointer, extent < 0 or not finite, a spacing
 * <= 0 or not finite, or a radius above LNF_MAX_RADIUS.
 */
lnf_status lnf_spacing_radii(double extent, const double spacing[3], int radius[3]);

/*
 * float32 volumes.  The paper filters grey levels; a float32 volume is filtered
 * on 65536 levels spanning its own range, in IEEE single precision with
 * round-to-nearest at every step (no fused operations):
 *   lo = min, hi = max over the volume, d = hi - lo;
 *   level q = floor((v - lo) * (65535 / d) + 1/2)   (every q = 0 when d = 0);
 *   the 16-bit pipeline (statistics, Otsu T, the filter) runs on the levels;
 *   out = lo + q * (d / 65535), so a gated voxel becomes lo.
 * in/out: device float32 buffers of nx*ny*nz values, x-fastest.  radius and
 * offset as lnf_filter_volume_aniso (equal radii: the paper's isotropic
 * filter).  Synchronises the stream once (the range is checked on the host).
 * Errors: LNF_EINVAL for a non-finite value, a range wider than float32 holds,
 * and as lnf_filter_volume_aniso; LNF_ENOMEM for the level buffers (4 bytes per
 * voxel, kept by the context); LNF_ECUDA.
 */
lnf_status lnf_filter_volume_f32(lnf_ctx *ctx, int filter_id, const int radius[3], const int offset[3],
                                 const float *in, float *out, const int64_t dims[3]);

/*
 * Image entropy (the paper's Fig. 4 measure) of a volume:
 * H = -sum_v (c_v/N) log2(c_v/N) over its grey-level histogram, accumulated in
 * FP64.  vol is a device buffer; *H is a HOST double.  Synchronises the stream.
 */
lnf_status lnf_entropy(lnf_ctx *ctx, const void *vol, const int64_t dims[3], int dtype, double *H);

/*
 * Read back the parameters derived for the last volume analysed on this
 * context and, if weights is not NULL, its entropy-filter weight table
 * (256 or 65536 uint32 entries, host memory).  Synchronises the stream.
 */
lnf_status lnf_get_params(lnf_ctx *ctx, lnf_params *out, uint32_t *weights);
/* It returns LNF_ETIMEOUT if a kernel's bounded wait gave up since the context
 * was created, LNF_ECUDA if a debug build's bounds check failed. */

/*
 * Debug builds.  A library compiled with LNF_DEBUG_CHECKS makes its kernels
 * check, before each access, the TMA box coordinates (innermost coordinate on a
 * 16-byte boundary, destination on a 128-byte one), the gate-first kernel's
 * list, histogram-window and voxel indices and the generic kernel's taps in its
 * staged planes; a failed check records LNF_DERR_BADJOB in the context's error
 * word and skips the access.
 *
 * lnf_debug_checks: 1 for such a build, else 0.
 * lnf_debug_poll: debug builds wait for the context's stream and return
 *   LNF_ECUDA if a check failed since the last poll (the record is cleared);
 *   release builds return LNF_OK at once.  NULL ctx: LNF_EINVAL.
 */
int lnf_debug_checks(void);
lnf_status lnf_debug_poll(lnf_ctx *ctx);

/*
 * Ray-cast the volume with a filter deciding at each candidate surface point:
 * the paper's use of its filter (sections "Introduction" and "3D Spatial
 * Noise Filters": the first sample at or above the threshold is a candidate;
 * the filter keeps it as structure, ending the ray, or rejects it as noise,
 * and the ray goes on; the surface is shaded with a 3D Sobel normal and Phong
 * illumination).  Orthographic rays along one of the six axis directions,
 * one per voxel column, samples at voxel centres; headlight Phong in IEEE
 * double: c = (g . d)/|g| (1 when g = 0), I = (0.1 + 0.7 max(c,0)) + 0.2 s^16
 * with s = 2c^2 - 1 when c > 0 and s > 0, pixel = min(255, floor(255 I + 1/2)).
 *   filter_id, radius  as lnf_filter_volume; the parameters (T, sigma band,
 *              T_d, entropy weights) are derived from the whole volume first
 *   in         device buffer of nx*ny*nz voxels (x-fastest)
 *   view       0..5 = rays along +x, -x, +y, -y, +z, -z; image axes (u, w) =
 *              (y, z) for +-x, (x, z) for +-y, (x, y) for +-z; pixel w*W + u
 *   image      device, W*H bytes: the shaded surface, 0 where no surface
 *   depth      device, W*H int32: step of the hit along the ray, -1 for none
 *              (NULL: not written)
 *   value      device, W*H uint32: the filter's output at the hit, 0 for none
 *              (NULL: not written)
 * Enqueued on the context's stream.  Returns LNF_EINVAL for a bad filter,
 * radius, view, dtype, dims or a NULL image.
 */
lnf_status lnf_render(lnf_ctx *ctx, int filter_id, int radius, const void *in, const int64_t dims[3], int dtype,
                      int view, uint8_t *image, int32_t *depth, uint32_t *value);

/*
 * Failure-detection self-test (no counterpart in the paper): launches one
 * kernel that waits, through the same bounded wait the filter kernels use on
 * their TMA barriers, on a barrier that nothing will ever complete.  The wait
 * must give up after limit_ms, record the failure in a device status word and
 * return, leaving the context usable.  elapsed_ms (may be NULL) receives the
 * host-side time of the call.  Returns LNF_ETIMEOUT when the wait gave up as
 * designed (the expected outcome), LNF_OK if it somehow completed,
 * LNF_EINVAL for limit_ms outside (0, 2000], LNF_ECUDA if the launch failed.
 * Synchronises the context's stream.
 */
lnf_status lnf_selftest_wait(lnf_ctx *ctx, double limit_ms, double *elapsed_ms);

/*
 * Image entropy of a volume, like lnf_entropy, for callers that must not
 * allocate device memory: no cudaMalloc, cudaFree or allocating library call
 * is made, and no lnf_ctx is needed (creating one allocates).  Typical users:
 * a render or acquisition loop that cannot take the device-wide stall an
 * allocation can cause, or code running while another component owns all of
 * the GPU's free memory.  The paper has no counterpart; it is a delivery
 * variant of the histogram + entropy steps.
 *   vol        device buffer of nx*ny*nz uint8/uint16 voxels (x-fastest)
 *   d_entropy  DEVICE pointer to one double that receives H
 *   stream     cudaStream_t the three kernels are enqueued on (NULL = default)
 * Scratch: one file-scope device array of 65536 uint32 counters (256 KiB),
 * present on every GPU that loads the library until the process exits.  The
 * first call on a device (with that device current) looks up the array's
 * address and has CUDA load all of this entry point's kernels (under lazy
 * module loading a kernel is otherwise loaded, possibly allocating, at its
 * first launch); make that first call before any stream capture.  The looked-up
 * address does not survive cudaDeviceReset.  Every call zeroes and reuses
 * the same array, so calls that overlap on the GPU race: order them on one
 * stream.  Returns LNF_EINVAL for null pointers, a bad dtype, dims < 1 or more
 * than 2^32 - 1 voxels (the counters are 32-bit), LNF_ECUDA if a launch fails
 * or if a CUDA error was already pending from earlier work (that error is
 * left set for the caller).  Asynchronous: read *d_entropy after
 * synchronising the stream.
 */
lnf_status lnf_entropy_noalloc(const void *vol, const int64_t dims[3], int dtype, double *d_entropy,
                               void *stream);

/* ------------------------------------------------------------------ batched */

/* One filter job of a batch.  All pointers are device pointers. */
typedef struct lnf_job {
    const void *in;             /* whole volume */
    void *out;                  /* roi_dims voxels (whole volume if roi_dims[0] == 0) */
    int64_t dims[3];
    int64_t roi_origin[3];
    int64_t roi_dims[3];        /* {0,0,0}: the whole volume */
    int32_t dtype;
    int32_t filter_id;
    int32_t radius;
    int32_t reserved;
    double *d_entropy;          /* optional device double: image entropy of the output */
} lnf_job;

/*
 * Run a batch of jobs (different volumes, sizes, dtypes, filters and radii):
 * one batched statistics launch and one batched parameter launch over the
 * distinct input volumes, then the jobs a specialised kernel covers as its
 * launches (a whole volume of the paper's filter also gets the gate-first
 * kernel, which takes the job on the device while few voxels pass the gate),
 * and ONE persistent launch of the generic kernel over the flattened tile list
 * of all other jobs, then one entropy launch.  The specialised launches run as
 * one chain per input volume, the chains side by side on the context's batch
 * streams (forked from and joined back into its stream), so the outputs of
 * different jobs must not overlap (not checked: overlapping outputs race).
 * The sequence is captured once
 * into a CUDA graph and replayed when the same batch (same pointers and
 * shapes) is run again.  With lnf_config.autotune set, the first batch times
 * the candidate z lengths of the specialised kernels' work items per job class
 * and the generic kernel's z chunk (lnf_get_tuning).  Enqueued; no host
 * synchronisation (the autotuner's first run synchronises).
 */
lnf_status lnf_filter_batch(lnf_ctx *ctx, const lnf_job *jobs, int n_jobs);

/*
 * The autotuner's choices on this context.  For up to `cap` job classes:
 * classes[k] = (dtype * 16 + filter_id) * 16 + radius, zlen[k] = the chosen z
 * length (planes) of a specialised work item, and, if ms is not NULL,
 * ms[4k .. 4k+3] = the class's batch time (ms) with z lengths 4, 8, 16, 32.
 * *n = the number of tuned classes (may exceed cap); *generic_zchunk (if not
 * NULL) = the generic kernel's tuned z chunk, 0 if not tuned.  Host arrays.
 */
lnf_status lnf_get_tuning(lnf_ctx *ctx, int32_t *classes, int32_t *zlen, float *ms, int cap, int *n,
                          int32_t *generic_zchunk);

/* ------------------------------------------------------------------ serving */

/* Copy a volume (device or host pointer, see `src_is_host`) into library-owned
 * device memory charged to the HBM budget, compute its statistics and
 * parameters once, and return its id.  Synchronous. */
lnf_status lnf_volume_register(lnf_ctx *ctx, const void *src, int src_is_host, const int64_t dims[3],
                               int dtype, int *vol_id);

/* Free a resident volume once no request uses it. */
lnf_status lnf_volume_unregister(lnf_ctx *ctx, int vol_id);

typedef struct lnf_request {
    int32_t vol_id;
    int32_t filter_id;
    int32_t radius;
    int32_t want_entropy;       /* also compute the output's image entropy */
    int64_t roi_origin[3];
    int64_t roi_dims[3];        /* {0,0,0}: the whole volume */
    void *out_host;             /* HOST buffer for the result (roi voxels), or NULL to keep it
                                   on the device until lnf_result_copy */
    double arrival_time;        /* seconds on the lnf_now() clock, recorded for latency */
} lnf_request;

typedef struct lnf_result {
    int32_t status;             /* LNF_OK, LNF_EPENDING, LNF_ECANCELLED, ... */
    int32_t reserved;
    double entropy;             /* image entropy of the output if requested */
    double t_admit, t_start, t_finish;  /* seconds on the lnf_now() clock; t_start/t_finish are the
                                           device start (CUDA events) and completion of the request's wave */
} lnf_result;

/*
 * Serving (continuous batching): queue a request against a resident volume
 * and return a ticket at once.  A scheduler thread admits queued requests as
 * in-flight slots and HBM budget free up and launches each admitted group as
 * one batched launch on one of several streams, so that groups overlap on the
 * device while later requests keep arriving.  LNF_EBUDGET if the request's
 * output alone exceeds the budget.  Thread-safe.
 */
lnf_status lnf_submit(lnf_ctx *ctx, const lnf_request *req, uint64_t *ticket);

/* Status of a ticket: LNF_EPENDING until done, then the request's status and
 * timings in *res.  A finished ticket may be polled again until released. */
lnf_status lnf_poll(lnf_ctx *ctx, uint64_t ticket, lnf_result *res);

/* Block until the ticket finishes or timeout_s elapses (LNF_ETIMEOUT). */
lnf_status lnf_wait(lnf_ctx *ctx, uint64_t ticket, double timeout_s, lnf_result *res);

/* Copy a finished request's device result to host memory (when out_host was NULL). */
lnf_status lnf_result_copy(lnf_ctx *ctx, uint64_t ticket, void *dst_host, size_t bytes);

/* Cancel a request that has not been admitted yet (LNF_EPENDING if it has). */
lnf_status lnf_cancel(lnf_ctx *ctx, uint64_t ticket);

/* Forget a finished ticket and free its device result. */
lnf_status lnf_release(lnf_ctx *ctx, uint64_t ticket);

/* The library's clock in seconds (CLOCK_MONOTONIC; Python's time.monotonic()),
 * the clock of lnf_request.arrival_time and of the lnf_result timings. */
double lnf_now(void);

/* Serving counters: bytes of the budget in use and requests queued / in flight. */
lnf_status lnf_serving_stats(lnf_ctx *ctx, uint64_t *budget_used, int *queued, int *inflight);

/* ------------------------------------------------------------------ profiling */

/* Per-kind device time of the launches made while profiling was on. */
typedef struct lnf_kernel_time {
    char name[24];              /* "stats", "params", "filter:ours", "entropy", ... */
    int32_t launches;           /* kernels of this kind launched */
    int32_t reserved;
    double total_ms;            /* sum of CUDA-event durations on the launching stream */
} lnf_kernel_time;

/* Turn profiling on (1) or off (0) and clear its records.  While on, every
 * kernel launch of the plain path is bracketed by CUDA events recorded on the
 * stream it is launched on, and every kernel launch is counted. */
lnf_status lnf_profile_enable(lnf_ctx *ctx, int on);

/* Synchronise, then return up to `max` per-kind records in `out` (*n set to
 * the number of kinds) and the total number of kernels launched since
 * profiling was enabled in *launches. */
lnf_status lnf_profile_read(lnf_ctx *ctx, lnf_kernel_time *out, int max, int *n, int64_t *launches);

/* Library version string. */
const char *lnf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LNF_H */
