// Internal declarations shared by the CUDA translation units of liblnf.
// Nothing here is part of the public C ABI (include/lnf.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

typedef unsigned long long u64;
typedef unsigned int u32;

#define LNF_LEVELS_U8 256
#define LNF_LEVELS_U16 65536

// Size of one volume's statistics pass; the pass itself accumulates only the
// grey-level histogram (sum P, sum P^2, min and max follow from it in the
// parameter kernels).
struct DevStats {
    u64 N;          // voxel count (set before the pass)
    u32 levels;     // 256 or 65536
    u32 pad;
};

// Per-volume parameter derivation settings (from lnf_config).
struct ParamCfg {
    int threshold_mode;         // 0 Otsu, 1 fixed, 2 none
    u32 threshold_value;
    int sigma_k;
    int pad;
    long long okada_td;         // >= 0, or -1 = auto
    long long entropy_te;       // >= 0, -1 = pass all, -2 = auto (per radius)
    long long entropy_local_te; // local entropy filter's theta: >= 0, -1 = pass all, -2 = auto
    const unsigned long long *lt;   // its table t[c] = round(2^22 c log2 c), c = 0..LNF_LT_MAX
};

// Parameters derived on the device from the histogram (one per volume).
struct DevParams {
    u64 N, S, Q;
    u32 minv, maxv;
    u32 T;                      // gate threshold (Eq. 1 / fixed / 0)
    u32 delta;                  // sigma band: |P_i - P0| <= delta
    long long td;               // Okada: |P0 - P_i| < td
    u64 hw_sum;                 // sum_v h[v] w[v]
    long long te_cfg;           // entropy threshold setting (see ParamCfg)
    u32 levels;
    u32 valid;                  // 1 once written
    double H_in;                // image entropy of the input
    u32 sigma_k;                // k of the sigma bands (global: in delta; local: applied per cube)
    u32 pad;
    u64 n_pass;                 // voxels whose own value passes the gate (P0 >= T)
    long long lte_cfg;          // local entropy filter's theta setting (see ParamCfg)
    const unsigned long long *lt;   // its table (see ParamCfg)
};

// Entries of the local entropy filter's table: cubes of up to 17^3 voxels
// (radius 8 on every axis).
#define LNF_LT_MAX (17 * 17 * 17)

// Whether the gate-first kernel (gate.cuh) does the work of the filters it is
// launched for: it streams the volume once and evaluates only the voxels that
// pass the gate (every other output is 0), so while they are at most 1/32 of
// the volume; the plane-ring kernels, launched beside, return at once then.
__host__ __device__ inline bool lnf_gate_mode(const DevParams &P)
{
    return P.n_pass * 32ull <= P.N;
}

// One unit of filter work: a volume (or ROI of it) with a filter and radius.
struct FilterJob {
    const void *in;
    void *out;
    int nx, ny, nz;             // whole volume
    int pitch;                  // input row stride in elements (>= nx)
    int ox, oy, oz;             // ROI origin
    int bx, by, bz;             // ROI dims (= output dims)
    int dtype;                  // 0 u8, 1 u16
    int filter;                 // lnf_filter_id
    int radius;                 // r (anisotropic jobs: the largest of rad[])
    int offset;                 // cluster offset d (anisotropic jobs: the largest of off[])
    int aniso;                  // 1: per-axis radii rad[] and offsets off[] (x, y, z)
    int rad[3];
    int off[3];
    const DevParams *prm;
    const u32 *lut;             // entropy weights, levels entries
    u64 *out_hist;              // output histogram (levels entries) or null
    int tmap_idx;               // index of the job's TMA map in the pack, -1: plain loads
    const void *orig;           // the caller's dense volume when `in` is a row-padded copy of it (or null)
    int gated;                  // 1: a gate-first kernel was launched for the job; the generic kernel
                                // skips its work while the gate takes the volume (lnf_gate_mode)
    int tiles_x, tiles_y, zchunks;
    int item_begin;             // first flattened work item of this job
};

// Up to kMaxJobs jobs and their TMA maps, passed BY VALUE as a
// __grid_constant__ kernel parameter (so a captured graph owns its copy).
#define LNF_MAX_PACK 64
struct FilterPack {
    int n_jobs;
    int total_items;
    int pad[14];
    CUtensorMap tmaps[LNF_MAX_PACK];    // 64-byte aligned
    FilterJob jobs[LNF_MAX_PACK];
};

// Device error word: set (never trapped) when a bounded wait gives up.
#define LNF_DERR_TIMEOUT 1u
#define LNF_DERR_BADJOB 2u

// ----------------------------------------------------------------- exact division
// floor(x / D) for 0 <= x <= XMAX as one 64-bit multiply (and a shift):
// q = (x * m) >> (32 + s) with m = ceil(2^(32+s) / D).  Writing x = qD + r,
// x m / 2^(32+s) = x / D + x e / (D 2^(32+s)) with e = m D - 2^(32+s) < D, so
// the floor is exact whenever XMAX * e < 2^(32+s) (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994); the smallest
// such s is chosen at compile time and the condition is checked statically.
template <unsigned long long D, unsigned long long XMAX>
struct ExactDiv {
    static constexpr unsigned long long mult(int s) { return ((1ull << (32 + s)) + D - 1) / D; }
    static constexpr bool ok(int s)
    {
        return mult(s) < (1ull << 32) && (mult(s) * D - (1ull << (32 + s))) * XMAX < (1ull << (32 + s));
    }
    static constexpr int pick(int s) { return s > 20 ? -1 : (ok(s) ? s : pick(s + 1)); }
    static constexpr int S = pick(0);
    static_assert(S >= 0, "no exact 32-bit multiplier for this divisor and range");
    static constexpr unsigned long long M = mult(S < 0 ? 0 : S);
    // floor((x + add) / D); add is folded into the multiply-add
    template <unsigned long long ADD>
    static __device__ __forceinline__ unsigned int div_add(unsigned int x)
    {
        static_assert(ADD <= XMAX, "offset beyond the proven range");
        return (unsigned int)(((unsigned long long)x * M + ADD * M) >> (32 + S));
    }
};

// ----------------------------------------------------------------- PTX helpers
namespace lnfdev {

__device__ __forceinline__ u32 smem_u32(const void *p)
{
    return static_cast<u32>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(u64 *bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(u64 *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u64 *bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase with a time limit; on timeout set the error
// word and return false (the caller then stops issuing work and exits).
__device__ __forceinline__ bool mbar_wait_bounded(u64 *bar, u32 parity, u32 *err, u64 limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity))
        return true;
    u64 t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (global_ns() - t0 > limit_ns) {
            if (err)
                atomicOr(err, LNF_DERR_TIMEOUT);
            return false;
        }
    }
}

// TMA: load a 3D box of the tensor map at element coordinates (x, y, z) into
// shared memory, completing `bytes` on the mbarrier.  x * elem_size must be a
// multiple of 16 bytes (the caller guarantees it).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, u64 *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<u64>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Debug builds (compiled with LNF_DEBUG_CHECKS): kernels check the indexes of
// the accesses named at each call before making them; a failed check records
// LNF_DERR_BADJOB in the error word and the access is skipped.  Release builds
// compile the checks away (both helpers return true).
__device__ __forceinline__ bool lnf_dbg_ok(bool ok, u32 *err)
{
#ifdef LNF_DEBUG_CHECKS
    if (!ok && err)
        atomicOr(err, LNF_DERR_BADJOB);
    return ok;
#else
    (void)ok;
    (void)err;
    return true;
#endif
}

// ... a TMA load: its innermost coordinate starts on a 16-byte boundary (x
// times the element size; a load left out leaves its mbarrier incomplete, so the
// kernel's bounded wait ends it) and its destination on a 128-byte one
__device__ __forceinline__ bool lnf_dbg_tma(int x, int elem_size, const void *dst, u32 *err)
{
    return lnf_dbg_ok(((x * elem_size) & 15) == 0 && (smem_u32(dst) & 127u) == 0u, err);
}

// TMA: prefetch a 3D box of the tensor map into L2 (no shared memory, no
// completion to wait for); used to keep DRAM reads in flight further ahead
// than the shared-memory ring allows.
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global [%0, {%1, %2, %3}];"
                 ::"l"(reinterpret_cast<u64>(map)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(map)) : "memory");
}

}  // namespace lnfdev

// ----------------------------------------------------------------- launchers
// (defined in stats.cu / filter.cu; all enqueue on `stream`)
cudaError_t lnf_launch_stats(const void *vol, u64 n, int dtype, u64 *hist, int num_sms, cudaStream_t stream);
cudaError_t lnf_launch_stats_init(u64 *hist, u32 levels, DevStats *st, u64 n, cudaStream_t stream);
// parameter derivation: two launches over chunks of 256 grey levels; pscr is
// per-volume device scratch of lnf_param_scratch_bytes() bytes, zeroed once
cudaError_t lnf_launch_params(const u64 *hist, const DevStats *st, const ParamCfg &cfg, DevParams *prm,
                              u32 *lut, void *pscr, int dtype, cudaStream_t stream);
size_t lnf_param_scratch_bytes();
cudaError_t lnf_launch_entropy(const u64 *hist, u32 levels, u64 n, double *H, cudaStream_t stream);
cudaError_t lnf_launch_zero(u64 *p, u64 count, cudaStream_t stream);

// Batched forms: arrays of volumes, one CTA group per volume.
struct StatsJob {
    const void *vol;
    u64 n;
    int dtype;
    int pad;
    u64 *hist;
    DevStats *st;
    DevParams *prm;
    u32 *lut;
    void *pscr;     // parameter scratch (lnf_param_scratch_bytes)
};
struct StatsPack {
    int n_jobs;
    int pad[3];
    StatsJob jobs[LNF_MAX_PACK];
};
cudaError_t lnf_launch_stats_batched(const StatsPack &pk, int ctas_per_job, cudaStream_t stream);
cudaError_t lnf_launch_stats_init_batched(const StatsPack &pk, cudaStream_t stream);
cudaError_t lnf_launch_params_batched(const StatsPack &pk, const ParamCfg &cfg, cudaStream_t stream);
// One CTA per entry: H[i] = entropy of histogram hists[i] (levels[i] bins, n[i] voxels).
#define LNF_MAX_ENT 128
struct EntropyPack {
    int count;
    int pad;
    const u64 *hist[LNF_MAX_ENT];
    u64 n[LNF_MAX_ENT];
    double *H[LNF_MAX_ENT];
    u32 levels[LNF_MAX_ENT];
};
// part: LNF_ENT_SPLIT * LNF_MAX_ENT doubles, done: LNF_MAX_ENT counters (zeroed once, reset by the kernel)
#define LNF_ENT_SPLIT 16
cudaError_t lnf_launch_entropy_pack(const EntropyPack &pk, double *part, u32 *done, cudaStream_t stream);

// Filter launch helpers (filter.cu).
int lnf_halo(int filter, int radius, int offset);
size_t lnf_filter_smem_bytes(int filter, int radius, int offset, int dtype);
void lnf_filter_decompose(FilterJob &j, int zchunk_len);
void lnf_filter_box(int filter, int radius, int offset, int dtype, unsigned *box_w, unsigned *box_h);
int lnf_filter_items(const FilterJob &j);
int lnf_filter_threads();
int lnf_filter_occupancy(size_t smem);
// Launch `grid` CTAs over the `total_items` work items of the jobs (device
// array sorted by item_begin).  persistent != 0: CTAs claim items from
// *d_counter (which must be 0 at launch); else CTA b takes b, b+grid, ...
cudaError_t lnf_filter_run(const FilterPack &pk, size_t smem, int grid, int persistent, u32 *d_counter, u32 *d_err,
                           cudaStream_t stream);
