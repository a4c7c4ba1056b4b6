// Filter kernels: a z-marching tile pipeline.
//
// A CTA owns an output tile of TX x TY columns and marches along z over a
// chunk of planes.  Input planes (tile + halo, x-halo widened to a 16-byte
// boundary) stream into a ring of shared-memory slots, by TMA
// (cp.async.bulk.tensor.3d, one mbarrier per slot, bounded waits) when the
// volume's row pitch allows it, else by plain coalesced loads staged through
// registers.  Border clamping: z by clamping the plane index; x and y by a
// small in-shared-memory fix-up on border tiles (TMA fills out-of-range cells
// with zeros, the filters need the border value).
//
// This file holds the generic compute: every filter evaluated per output
// voxel by direct enumeration of its taps from the ring (runtime filter id,
// radius and cluster offset), exact integer arithmetic, round-half-up to the
// input type, the noise gate, and a fused per-CTA output histogram (for the
// image entropy of the result, Fig. 4) flushed once per job.
#include "lnf_internal.cuh"
#include "filter_eval.cuh"

namespace {

using namespace lnfeval;

constexpr int kThreads = 256;
constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kHistWin16 = 4096;     // shared-memory histogram window for 16-bit outputs

struct Geo {
    int h;          // halo in y and z (and the x halo actually used)
    int E;          // TMA x alignment in elements (16 bytes)
    int PW, PH;     // plane width / height in elements
    int pstride;    // plane stride in elements (128-byte multiple)
    int NP;         // ring slots
};

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

__host__ __device__ inline Geo make_geo(int h, int esize)
{
    Geo g;
    g.h = h;
    g.E = 16 / esize;
    g.PW = round_up(kTX + 2 * h + g.E - 1, g.E);
    g.PH = kTY + 2 * h;
    g.pstride = round_up(g.PW * g.PH * esize, 128) / esize;
    g.NP = 2 * h + 3;
    return g;
}

// the paper's filter and its cluster-layout variants reach r past the cluster
// centres at offset d (anisotropic jobs: the largest radius and offset, a bound
// on the reach along every axis)
__host__ __device__ inline int job_halo(int filter, int r, int d)
{
    return (filter >= 4 && filter <= 6) ? r + d : r;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }


// ------------------------------------------------------------------ histogram

struct HistState {
    int job;        // job whose counts the shared histogram holds (-1 none)
    u32 base;       // first value of the 16-bit window
    u32 zeros;      // per-thread count of zero outputs
};

template <typename T>
__device__ __forceinline__ void hist_add(u32 *sh_hist, const HistState &hs, u64 *gh, u32 v, u32 &zeros)
{
    if (v == 0) {
        ++zeros;
        return;
    }
    if (sizeof(T) == 1) {
        atomicAdd(&sh_hist[v], 1u);
    } else {
        u32 o = v - hs.base;
        if (o < (u32)kHistWin16)
            atomicAdd(&sh_hist[o], 1u);
        else if (v < 65536u)   // always true for valid outputs
            atomicAdd(&gh[v], 1ull);
    }
}

// flush the shared histogram of job `hs.job` (all threads participate)
__device__ void hist_flush(u32 *sh_hist, HistState &hs, const FilterPack &pk, u32 &zeros)
{
    if (hs.job >= 0) {
        const FilterJob &J = pk.jobs[hs.job];
        u64 *gh = J.out_hist;
        const int bins = J.dtype == 0 ? LNF_LEVELS_U8 : kHistWin16;
        // zeros: warp sum then one atomic per warp
        u32 z = zeros;
        for (int o = 16; o > 0; o >>= 1)
            z += __shfl_xor_sync(0xFFFFFFFFu, z, o);
        if (gh && (threadIdx.x & 31) == 0 && z)
            atomicAdd(&gh[0], (u64)z);
        __syncthreads();
        for (int i = threadIdx.x; i < bins; i += blockDim.x) {
            u32 c = sh_hist[i];
            if (c && gh)
                atomicAdd(&gh[(J.dtype == 0 ? 0u : hs.base) + i], (u64)c);
            sh_hist[i] = 0;
        }
    } else {
        for (int i = threadIdx.x; i < kHistWin16; i += blockDim.x)
            sh_hist[i] = 0;
    }
    zeros = 0;
    __syncthreads();
}

// ------------------------------------------------------------------ generic compute

template <typename T>
struct Ring {
    const T *base;      // shared memory ring
    int pstride, PW, NP;
    int slot0;          // slot of the plane at dz = 0 for the current step
    int col, row;       // this thread's centre column / row in the plane
    int PH;             // rows of a plane (debug checks)
    u32 *err;           // error word (debug checks)
    __device__ __forceinline__ u32 at(int dx, int dy, int dz) const
    {
        int s = slot0 + dz;
        s = s < 0 ? s + NP : (s >= NP ? s - NP : s);
        // debug builds: the tap inside the staged plane and the ring
        if (!lnfdev::lnf_dbg_ok(s >= 0 && s < NP && row + dy >= 0 && row + dy < PH && col + dx >= 0 && col + dx < PW, err))
            return 0;
        return base[s * pstride + (row + dy) * PW + col + dx];
    }
};

// ------------------------------------------------------------------ plane loading

template <typename T>
__device__ __forceinline__ void fixup_plane(T *pl, const Geo &g, int px0, int py0, int nx, int ny)
{
    // x: replicate the border columns into out-of-range columns
    const int left = px0 < 0 ? min(-px0, g.PW) : 0;
    const int right_start = max(0, min(g.PW, nx - px0));
    const int right = g.PW - right_start;
    const int ncol = left + right;
    if (ncol > 0) {
        for (int e = threadIdx.x; e < ncol * g.PH; e += blockDim.x) {
            const int row = e / ncol;
            const int k = e - row * ncol;
            const int col = k < left ? k : right_start + (k - left);
            const int src = clampi(px0 + col, 0, nx - 1) - px0;
            pl[row * g.PW + col] = pl[row * g.PW + src];
        }
    }
    __syncthreads();
    const int top = py0 < 0 ? min(-py0, g.PH) : 0;
    const int bot_start = max(0, min(g.PH, ny - py0));
    const int bot = g.PH - bot_start;
    const int nrow = top + bot;
    if (nrow > 0) {
        for (int e = threadIdx.x; e < nrow * g.PW; e += blockDim.x) {
            const int k = e / g.PW;
            const int col = e - k * g.PW;
            const int row = k < top ? k : bot_start + (k - top);
            const int src = clampi(py0 + row, 0, ny - 1) - py0;
            pl[row * g.PW + col] = pl[src * g.PW + col];
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ one work item

template <typename T>
__device__ void process_item(const FilterJob &J, const CUtensorMap *tmap, int item_local, unsigned char *smem,
                             u32 *sh_hist, HistState &hs, u32 &zeros, u32 *err, int *s_abort)
{
    using namespace lnfdev;
    const int h = job_halo(J.filter, J.radius, J.offset);
    const Geo g = make_geo(h, sizeof(T));
    T *ring = reinterpret_cast<T *>(smem);
    u64 *bars = reinterpret_cast<u64 *>(smem + (size_t)g.NP * g.pstride * sizeof(T));

    const int zc_len = (J.bz + J.zchunks - 1) / J.zchunks;
    const int tx = item_local % J.tiles_x;
    const int rest = item_local / J.tiles_x;
    const int ty = rest % J.tiles_y;
    const int zci = rest / J.tiles_y;
    const int lx0 = tx * kTX, ly0 = ty * kTY;
    const int lz0 = zci * zc_len;
    const int lz1 = min(J.bz, lz0 + zc_len);
    if (lz0 >= lz1)
        return;
    const int x0 = J.ox + lx0, y0 = J.oy + ly0, z0 = J.oz + lz0;
    const int px0 = ((x0 - h) >= 0 ? (x0 - h) / g.E : -((h - x0 + g.E - 1) / g.E)) * g.E;   // floor to E
    const int py0 = y0 - h;
    const int cx0 = x0 - px0;
    const bool border = px0 < 0 || px0 + g.PW > J.nx || py0 < 0 || py0 + g.PH > J.ny;
    const int nplanes = (lz1 - lz0) + 2 * h;   // plane p <-> z = z0 - h + p
    const bool use_tma = tmap != nullptr;
    const T *vin = static_cast<const T *>(J.in);
    const u32 plane_bytes = (u32)(g.PW * g.PH * sizeof(T));

    // parameters of this job
    const DevParams &P = *J.prm;
    const StepParams sp = J.aniso ? make_step_params3(P, J.rad, J.off, J.lut)
                                  : make_step_params(P, J.radius, J.offset, J.lut);
    // stage loader for plain loads
    auto load_plane_plain = [&](int p, T *dst) {
        const int z = clampi(z0 - h + p, 0, J.nz - 1);
        const size_t zoff = (size_t)z * J.ny * J.pitch;
        for (int e = threadIdx.x; e < g.PW * g.PH; e += blockDim.x) {
            const int row = e / g.PW;
            const int col = e - row * g.PW;
            const int yy = clampi(py0 + row, 0, J.ny - 1);
            const int xx = clampi(px0 + col, 0, J.nx - 1);
            dst[row * g.PW + col] = vin[zoff + (size_t)yy * J.pitch + xx];
        }
    };

    if (use_tma) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < g.NP; ++s)
                mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            const int pre = min(g.NP, nplanes);
            for (int p = 0; p < pre; ++p) {
                const int z = clampi(z0 - h + p, 0, J.nz - 1);
                mbar_arrive_expect_tx(&bars[p], plane_bytes);
                if (lnf_dbg_tma(px0, (int)sizeof(T), ring + (size_t)p * g.pstride, err))
                    tma_load_3d(ring + (size_t)p * g.pstride, tmap, &bars[p], px0, py0, z);
            }
        }
    } else {
        for (int p = 0; p < min(2 * h + 1, nplanes); ++p)
            load_plane_plain(p, ring + (size_t)p * g.pstride);
        __syncthreads();
    }

    const int tl = threadIdx.x % kTX, tr = threadIdx.x / kTX;
    const bool active = (lx0 + tl) < J.bx && (ly0 + tr) < J.by;
    Ring<T> R;
    R.base = ring;
    R.pstride = g.pstride;
    R.PW = g.PW;
    R.NP = g.NP;
    R.col = cx0 + tl;
    R.row = h + tr;
    R.PH = g.PH;
    R.err = err;
    T *vout = static_cast<T *>(J.out);
    u64 *gh = J.out_hist;

    bool ok = true;
    for (int s = 0; s < lz1 - lz0; ++s) {
        // make planes up to s + 2h resident
        if (use_tma) {
            // one thread waits for the TMA completions; the barrier orders the
            // data before every thread's reads
            const int pfirst = s == 0 ? 0 : s + 2 * h;
            if (threadIdx.x == 0)
                for (int p = pfirst; p <= s + 2 * h; ++p)
                    if (!mbar_wait_bounded(&bars[p % g.NP], (u32)((p / g.NP) & 1), err))
                        *s_abort = 1;
            __syncthreads();
            if (*s_abort) {
                ok = false;
                break;
            }
            if (border)
                for (int p = pfirst; p <= s + 2 * h; ++p)
                    fixup_plane<T>(ring + (size_t)(p % g.NP) * g.pstride, g, px0, py0, J.nx, J.ny);
        }
        // compute output plane z = z0 + s from planes s .. s + 2h
        R.slot0 = (s + h) % g.NP;
        if (active) {
            const u32 f = eval_filter(J.filter, R, sp);
            const size_t o = ((size_t)(lz0 + s) * J.by + (ly0 + tr)) * J.bx + (lx0 + tl);
            vout[o] = (T)f;
            if (gh)
                hist_add<T>(sh_hist, hs, gh, f, zeros);
        }
        __syncthreads();   // everyone is done with plane s
        if (use_tma) {
            const int p = s + g.NP;   // refill the slot plane s occupied
            if (threadIdx.x == 0 && p < nplanes) {
                const int z = clampi(z0 - h + p, 0, J.nz - 1);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[p % g.NP], plane_bytes);
                if (lnf_dbg_tma(px0, (int)sizeof(T), ring + (size_t)(p % g.NP) * g.pstride, err))
                    tma_load_3d(ring + (size_t)(p % g.NP) * g.pstride, tmap, &bars[p % g.NP], px0, py0, z);
            }
        } else {
            const int p = s + 2 * h + 1;
            if (p < nplanes) {
                load_plane_plain(p, ring + (size_t)(p % g.NP) * g.pstride);
                __syncthreads();
            }
        }
    }
    if (use_tma) {
        if (!ok) {
            // a wait gave up: give this CTA's copies still in flight a bounded
            // time to land before the shared memory is released
            if (threadIdx.x == 0) {
                const u64 t0 = global_ns();
                while (global_ns() - t0 < 2000000ull) {
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int sl = 0; sl < g.NP; ++sl)
                mbar_inval(&bars[sl]);
        __syncthreads();
    }
}

__device__ __forceinline__ int find_job(const FilterPack &pk, int item)
{
    int lo = 0, hi = pk.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pk.jobs[mid].item_begin <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) k_filter(const __grid_constant__ FilterPack pk, u32 *counter,
                                                    u32 *err, int persistent)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations: keep the ring 128-byte aligned whatever the static layout
    unsigned char *smem = smem_raw + ((128 - (lnfdev::smem_u32(smem_raw) & 127)) & 127);
    __shared__ u32 sh_hist[kHistWin16];
    __shared__ int s_item, s_abort;
    HistState hs;
    hs.job = -1;
    hs.base = 0;
    u32 zeros = 0;
    if (threadIdx.x == 0)
        s_abort = 0;
    const int total_items = pk.total_items;
    hist_flush(sh_hist, hs, pk, zeros);   // zero the shared histogram
    for (int k = 0;; ++k) {
        int item;
        if (persistent) {
            if (threadIdx.x == 0)
                s_item = (int)atomicAdd(counter, 1u);
            __syncthreads();
            item = s_item;
            __syncthreads();
        } else {
            item = blockIdx.x + k * gridDim.x;
        }
        if (item >= total_items || s_abort)
            break;
        const int j = find_job(pk, item);
        const FilterJob &J = pk.jobs[j];
        if (j != hs.job) {
            hist_flush(sh_hist, hs, pk, zeros);
            hs.job = j;
            hs.base = J.dtype == 0 ? 0u : J.prm->minv;
        }
        if (J.gated && lnf_gate_mode(*J.prm))
            continue;   // the gate-first kernel writes this job's output (uniform over the CTA)
        const int local = item - J.item_begin;
        const CUtensorMap *tm = J.tmap_idx >= 0 ? &pk.tmaps[J.tmap_idx] : nullptr;
        if (J.dtype == 0)
            process_item<uint8_t>(J, tm, local, smem, sh_hist, hs, zeros, err, &s_abort);
        else
            process_item<uint16_t>(J, tm, local, smem, sh_hist, hs, zeros, err, &s_abort);
    }
    hist_flush(sh_hist, hs, pk, zeros);
}

}  // namespace

// ------------------------------------------------------------------ host helpers

int lnf_halo(int filter, int radius, int offset) { return job_halo(filter, radius, offset); }

size_t lnf_filter_smem_bytes(int filter, int radius, int offset, int dtype)
{
    const int es = dtype == 0 ? 1 : 2;
    const Geo g = make_geo(job_halo(filter, radius, offset), es);
    return (size_t)g.NP * g.pstride * es + (size_t)g.NP * sizeof(u64) + 128;   // + alignment slack
}

// tiles, z chunks and the TMA box of one job (item_begin is set by the caller)
void lnf_filter_decompose(FilterJob &j, int zchunk_len)
{
    j.tiles_x = (j.bx + kTX - 1) / kTX;
    j.tiles_y = (j.by + kTY - 1) / kTY;
    if (zchunk_len < 1)
        zchunk_len = 64;
    j.zchunks = (j.bz + zchunk_len - 1) / zchunk_len;
    if (j.zchunks < 1)
        j.zchunks = 1;
}

void lnf_filter_box(int filter, int radius, int offset, int dtype, unsigned *box_w, unsigned *box_h)
{
    const Geo g = make_geo(job_halo(filter, radius, offset), dtype == 0 ? 1 : 2);
    *box_w = (unsigned)g.PW;
    *box_h = (unsigned)g.PH;
}

int lnf_filter_items(const FilterJob &j) { return j.tiles_x * j.tiles_y * j.zchunks; }

int lnf_filter_threads() { return kThreads; }

cudaError_t lnf_filter_run(const FilterPack &pk, size_t smem, int grid, int persistent, u32 *d_counter, u32 *d_err,
                           cudaStream_t stream)
{
    cudaError_t e = cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    k_filter<<<grid, kThreads, smem, stream>>>(pk, d_counter, d_err, persistent);
    return cudaGetLastError();
}

int lnf_filter_occupancy(size_t smem)
{
    int n = 0;
    if (cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_filter, kThreads, smem) != cudaSuccess || n < 1)
        return 1;
    return n;
}
