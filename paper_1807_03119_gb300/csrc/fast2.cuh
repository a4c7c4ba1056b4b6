// Specialised kernels for the four comparison filters on volumes whose row
// pitch allows TMA (whole volumes or regions of interest); every other job
// runs on the generic kernel (filter.cu).  This header holds the shared
// driver; fast2_box.cu (mean, entropy filter) and fast2_tap.cu (sigma, Okada,
// and the dispatch) hold the two kernel bodies and compile in parallel.
//
//   box kernel  -- mean (Eq. 4) and entropy filter (Eq. 7): B = sum over the
//                  M^3 cube of q(P), q = identity or the fixed-point weight
//                  w[P].  Per step the lane keeps the z line sum Bz of each of
//                  its voxels as a running sum (one plane in, one out); the x
//                  box Sx of Bz takes the neighbouring columns from the
//                  adjacent lanes (shuffles) and goes to a shared Sx plane
//                  (tile rows - R .. 31 + R, the halo rows summed by R warps
//                  at each end); the y box of Sx is a running sum down the
//                  lane's rows.  The part of the x box beyond the tile comes
//                  from a few lanes per warp that keep the z sums of the R
//                  border columns of one row and store their prefix sums in
//                  the Sx plane's spare columns, for the edge lanes to add.
//   tap kernel  -- sigma (Eq. 5) and Okada (Eq. 6): data-dependent selection,
//                  so every tap is tested; each lane owns 4 x 4 voxels and
//                  reuses every loaded row segment across its voxels and
//                  offsets, accumulating value and count in one packed word.
//
// Shared driver: a CTA owns a 128 x 32 output tile and marches along z; input
// planes (tile + halo, x halo widened to 16 bytes) stream into a ring of
// shared-memory slots by TMA with one mbarrier per slot and bounded waits;
// border tiles replicate the volume's edge into out-of-range cells.
#pragma once
#include "lnf_ctx.h"

#include <algorithm>
#include <cstring>

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRows = 4;
constexpr int kTX = 128;
constexpr int kTY = kWarps * kRows;
constexpr int kPF = 2;
constexpr int kHistWin = 4096;
constexpr int kL2Ahead = 6;              // planes prefetched into L2 beyond the shared-memory ring

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T, int R, int PF = kPF>
struct Geo2 {
    static constexpr int H = R;                            // halo in y and z
    static constexpr int XH = 16 / sizeof(T);              // x halo, 16 bytes (>= R for R <= 8)
    static constexpr int PW = kTX + 2 * XH;
    static constexpr int PH = kTY + 2 * H;
    static constexpr int ROWB = PW * sizeof(T);
    static constexpr int PBYTES = ((PW * PH * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int NP = 2 * R + 2 + PF;
    static constexpr int M = 2 * R + 1;
    static constexpr int RING = NP * PBYTES;
    // box kernel: Sx plane of (kTY + 2R) rows x (kTX + 8) u32, own cells at column offset 4;
    // offsets 0..R-1 and kTX+4..kTX+3+R hold the border prefix sums
    static constexpr int BW = kTX + 8;
    static constexpr int BZ = (kTY + 2 * R) * BW * 4;
};

// four voxels at columns col..col+3 of a shared row, unpacked
template <typename T>
__device__ __forceinline__ void ld4(const unsigned char *row, int col, u32 v[4])
{
    if (sizeof(T) == 2) {
        const uint2 w = *reinterpret_cast<const uint2 *>(row + col * 2);
        v[0] = w.x & 0xFFFFu;
        v[1] = w.x >> 16;
        v[2] = w.y & 0xFFFFu;
        v[3] = w.y >> 16;
    } else {
        const u32 w = *reinterpret_cast<const u32 *>(row + col);
        v[0] = w & 0xFFu;
        v[1] = (w >> 8) & 0xFFu;
        v[2] = (w >> 16) & 0xFFu;
        v[3] = w >> 24;
    }
}

template <typename T>
__device__ __forceinline__ u32 ld1(const unsigned char *row, int col)
{
    return sizeof(T) == 2 ? (u32) reinterpret_cast<const uint16_t *>(row)[col] : (u32)row[col];
}

template <typename T, int R>
__device__ void fixup2(unsigned char *pl, int px0, int py0, int nx, int ny)
{
    typedef Geo2<T, R> G;
    T *p = reinterpret_cast<T *>(pl);
    const int left = px0 < 0 ? min(-px0, G::PW) : 0;
    const int right_start = max(0, min(G::PW, nx - px0));
    const int ncol = left + (G::PW - right_start);
    if (ncol > 0)
        for (int e = threadIdx.x; e < ncol * G::PH; e += blockDim.x) {
            const int row = e / ncol;
            const int k = e - row * ncol;
            const int col = k < left ? k : right_start + (k - left);
            p[row * G::PW + col] = p[row * G::PW + clampi(px0 + col, 0, nx - 1) - px0];
        }
    __syncthreads();
    const int top = py0 < 0 ? min(-py0, G::PH) : 0;
    const int bot_start = max(0, min(G::PH, ny - py0));
    const int nrow = top + (G::PH - bot_start);
    if (nrow > 0)
        for (int e = threadIdx.x; e < nrow * G::PW; e += blockDim.x) {
            const int k = e / G::PW;
            const int col = e - k * G::PW;
            const int row = k < top ? k : bot_start + (k - top);
            p[row * G::PW + col] = p[(clampi(py0 + row, 0, ny - 1) - py0) * G::PW + col];
        }
    __syncthreads();
}

struct Args2 {
    const void *in;
    void *out;
    int nx, ny, nz;
    // output region [o, o + b) (the whole volume unless a region of interest),
    // tiled from column xs = ox rounded down to TMA's 16-byte rule
    int ox, oy, oz, bx, by, bz, xs, xend, yend;
    int roi;                              // 1: masked per-voxel stores (ROI-shaped output or odd width)
    int tiles_x, tiles_y, zlen;
    int total_items;
    int filter;
    const DevParams *prm;
    const u32 *lut;
    u64 *out_hist;
    u32 *counter;
    u32 *err;
    u32 one;        // always 1; a multiplier the compiler cannot fold, so that adds
                    // written as multiply-adds issue on the FMA pipe (see tap_items)
    int gated;      // 1: launched beside the gate-first kernel, which takes the job while few voxels
                    // pass the gate (lnf_gate_mode); 2: launched beside the generic kernel, which
                    // takes the job unless few voxels pass
};

// shared histogram of nonzero outputs (window [hbase, hbase + bins)), zero count by difference
struct Hist2 {
    u32 *sh;
    u32 base;
    u32 bins;
    u32 nonzero, written;
    u64 *gh;
};

__device__ __forceinline__ void hist4(Hist2 &h, const u32 f[4])
{
    h.written += 4;
    if (!h.gh)
        return;
    const bool nz = (f[0] | f[1] | f[2] | f[3]) != 0;
    if (__any_sync(__activemask(), nz)) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (f[k]) {
                ++h.nonzero;
                const u32 b = f[k] - h.base;
                if (b < h.bins)
                    atomicAdd(&h.sh[b], 1u);
                else if (f[k] < 65536u)   // always true for valid outputs
                    atomicAdd(&h.gh[f[k]], 1ull);
            }
    }
}

template <typename T>
__device__ __forceinline__ void store4(const Args2 &a, int z, int y, int x, const u32 f[4])
{
    const size_t o = ((size_t)z * a.ny + y) * a.nx + x;
    if (sizeof(T) == 2)
        *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(a.out) + o) =
            make_uint2(f[0] | (f[1] << 16), f[2] | (f[3] << 16));
    else
        *reinterpret_cast<u32 *>(static_cast<uint8_t *>(a.out) + o) = f[0] | (f[1] << 8) | (f[2] << 16) | (f[3] << 24);
}

// a region of interest: masked stores of the lane's four voxels, one at a time
// (the tile starts at xs <= ox, so some lanes lie left of the region)
template <typename T>
__device__ __forceinline__ void store_roi(const Args2 &a, Hist2 &h, int z, int y, int x, const u32 f[4])
{
    if (y >= a.yend)
        return;
    const long long ob = ((long long)(z - a.oz) * a.by + (y - a.oy)) * a.bx - a.ox;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int xk = x + k;
        if (xk < a.ox || xk >= a.xend)
            continue;
        static_cast<T *>(a.out)[ob + xk] = (T)f[k];
        h.written += 1;
        if (h.gh && f[k]) {
            ++h.nonzero;
            const u32 b = f[k] - h.base;
            if (b < h.bins)
                atomicAdd(&h.sh[b], 1u);
            else if (f[k] < 65536u)   // always true for valid outputs
                atomicAdd(&h.gh[f[k]], 1ull);
        }
    }
}

// ------------------------------------------------------------------ the two kernel bodies

constexpr int kBoxPF = 1;            // box kernel: one plane prefetched (two CTAs per SM fit)
constexpr int kLutWin16 = 4096;      // box kernel (entropy): window of the weight table in shared
                                     // memory (16-bit data: all 12-bit levels from the minimum)
constexpr int kEntHist16 = 1024;     // ... and of its output histogram (the rest goes to global atomics)

// box kernel body (fast2_box.cu): mean (ENT = false) and entropy filter (ENT = true)
template <typename T, int R, bool ENT, bool MASK>
__device__ void box_items(const Args2 &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item, int *s_abort,
                          Hist2 &hist, const u32 *lut_sh, u32 lut_base);
// tap kernel (fast2_tap.cu): the taps of one voxel, and the most voxels with
// P0 >= T a block lists per step (beyond it every warp takes the dense form,
// which tests every tap of all its voxels while reusing each loaded row)
template <int R, int FILTER>
struct TapCoop {
    static constexpr int TAPS = FILTER == LNF_SIGMA ? (2 * R + 1) * (2 * R + 1) * (2 * R + 1) : 6 * R + 1;
    static constexpr int PER_LANE = (TAPS + 31) / 32;
    static constexpr int CAP = 1024;
    // the list (cells and destinations, 16 bits each), the warps' counts, and one
    // 16-bit output per voxel of the block step
    static constexpr int BYTES = CAP * 4 + 64 + kWarps * 32 * 16 * 2;
};
// tap kernel body (fast2_tap.cu): sigma and Okada; `wl`: the block's candidate
// area (TapCoop::BYTES): CAP cells, CAP destinations, one 32-bit count per warp,
// then the outputs of the step (16 per lane)
template <typename T, int R, int FILTER, bool MASK>
__device__ void tap_items(const Args2 &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item, int *s_abort,
                          Hist2 &hist, const u32 *recip, uint16_t *wl);

// ------------------------------------------------------------------ kernels

template <typename T, int R, int FILTER>
struct K2Smem {
    static constexpr bool BOX = FILTER == LNF_MEAN || FILTER == LNF_ENTROPY;
    typedef Geo2<T, R, BOX ? kBoxPF : kPF> G;
    static constexpr int HWIN = sizeof(T) == 1 ? 256 : (FILTER == LNF_ENTROPY ? kEntHist16 : kHistWin);
    static constexpr int LWIN = sizeof(T) == 1 ? 256 : kLutWin16;
    static constexpr int HISTB = HWIN * 4;
    static constexpr int NTAB = (2 * R + 1) * (2 * R + 1) * (2 * R + 1) + 1;   // counts 0 .. M^3
    static constexpr int LUTB = FILTER == LNF_ENTROPY ? LWIN * 4 : (BOX ? 0 : ((NTAB * 4 + 15) / 16) * 16);
    static constexpr int MAIN = G::RING + (BOX ? G::BZ : 0) + G::NP * 8;
    static constexpr int COOPB = BOX ? 0 : TapCoop<R, FILTER>::BYTES;
    static constexpr int TOTAL = 128 + MAIN + 64 + HISTB + LUTB + COOPB;
};

// MASK: masked per-voxel stores (a region of interest, an odd width), else dense
// 4-voxel vector stores
template <typename T, int R, int FILTER, bool MASK>
__global__ void __launch_bounds__(kThreads, (K2Smem<T, R, FILTER>::BOX && R > 2) ? 1 : 2)
    k_fast2(const __grid_constant__ CUtensorMap tmap, const Args2 a)
{
    typedef K2Smem<T, R, FILTER> S;
    if (a.gated == 1 && lnf_gate_mode(*a.prm))
        return;   // few voxels pass the gate: the gate-first kernel does the work
    if (a.gated == 2 && !lnf_gate_mode(*a.prm))
        return;   // many voxels pass: the generic kernel launched beside does the work
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128 - (lnfdev::smem_u32(smem_raw) & 127)) & 127);
    __shared__ int s_item, s_abort;
    u32 *hsh = reinterpret_cast<u32 *>(smem + S::MAIN + 64);
    u32 *lut_sh = reinterpret_cast<u32 *>(smem + S::MAIN + 64 + S::HISTB);
    uint16_t *wl = reinterpret_cast<uint16_t *>(smem + S::MAIN + 64 + S::HISTB + S::LUTB);
    const u32 bins = (u32)S::HWIN;
    Hist2 h;
    h.sh = hsh;
    h.bins = bins;
    // nonzero outputs are >= T (gate), so the window starts there for 16-bit data
    h.base = sizeof(T) == 1 ? 0u : max(a.prm->T, a.prm->minv);
    h.nonzero = 0;
    h.written = 0;
    h.gh = a.out_hist;
    for (int i = threadIdx.x; i < (int)bins; i += blockDim.x)
        hsh[i] = 0;
    u32 lut_base = 0;
    if (FILTER == LNF_ENTROPY) {
        lut_base = sizeof(T) == 1 ? 0u : a.prm->minv;
        const int nl = S::LWIN;
        for (int i = threadIdx.x; i < nl; i += blockDim.x)
            lut_sh[i] = (lut_base + i < (sizeof(T) == 1 ? 256u : 65536u)) ? a.lut[lut_base + i] : 0u;
    }
    if (!S::BOX)   // reciprocals of the voxel counts a tap filter can select
        for (int n = threadIdx.x; n < S::NTAB; n += blockDim.x)
            lut_sh[n] = (n <= 1 || n >= 256) ? 0u : (u32)((0x100000000ull + n - 1) / n);
    if (threadIdx.x == 0)
        s_abort = 0;
    __syncthreads();
    if constexpr (FILTER == LNF_MEAN)
        box_items<T, R, false, MASK>(a, &tmap, smem, &s_item, &s_abort, h, lut_sh, lut_base);
    else if constexpr (FILTER == LNF_ENTROPY)
        box_items<T, R, true, MASK>(a, &tmap, smem, &s_item, &s_abort, h, lut_sh, lut_base);
    else
        tap_items<T, R, FILTER, MASK>(a, &tmap, smem, &s_item, &s_abort, h, lut_sh, wl);
    if (a.out_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < (int)bins; i += blockDim.x)
            if (hsh[i])
                atomicAdd(&a.out_hist[h.base + i], (u64)hsh[i]);
        u32 zeros = h.written - h.nonzero;
        for (int o = 16; o > 0; o >>= 1)
            zeros += __shfl_xor_sync(0xFFFFFFFFu, zeros, o);
        if ((threadIdx.x & 31) == 0 && zeros)
            atomicAdd(&a.out_hist[0], (u64)zeros);
    }
}

template <typename T, int R, int FILTER>
lnf_status launch2(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, u32 *counter, int *handled, int gated)
{
    typedef K2Smem<T, R, FILTER> S;
    typedef typename S::G G;
    CUtensorMap map;   // this kernel's own descriptor: box = its tile + halo
    if (!lnf_encode_box(ctx, j.in, j.nx, j.ny, j.nz, j.pitch, j.dtype, G::PW, G::PH, &map))
        return LNF_OK;
    const CUtensorMap *tmap = &map;
    Args2 a;
    std::memset(&a, 0, sizeof a);
    a.in = j.in;
    a.out = j.out;
    a.nx = j.nx;
    a.ny = j.ny;
    a.nz = j.nz;
    a.ox = j.ox;
    a.oy = j.oy;
    a.oz = j.oz;
    a.bx = j.bx;
    a.by = j.by;
    a.bz = j.bz;
    a.xs = j.ox - j.ox % (16 / (int)sizeof(T));
    a.xend = j.ox + j.bx;
    a.yend = j.oy + j.by;
    // dense 4-voxel vector stores need rows that start on 4-voxel boundaries of an
    // aligned output; anything else (a region of interest, an odd width) takes the
    // masked per-voxel stores
    const bool whole = !(j.ox || j.oy || j.oz || j.bx != j.nx || j.by != j.ny || j.bz != j.nz);
    const bool vec = j.nx % 4 == 0 && reinterpret_cast<uintptr_t>(j.out) % (4 * sizeof(T)) == 0;
    a.roi = whole && vec ? 0 : 1;
    a.tiles_x = (a.xend - a.xs + kTX - 1) / kTX;
    a.tiles_y = (j.by + kTY - 1) / kTY;
    a.filter = FILTER;
    a.prm = j.prm;
    a.lut = j.lut;
    a.out_hist = j.out_hist;
    a.counter = counter ? counter : ctx->d_counter + 9;
    a.err = ctx->d_err;
    a.one = 1u;
    a.gated = gated;
    void (*kern)(const CUtensorMap, const Args2) = a.roi ? k_fast2<T, R, FILTER, true> : k_fast2<T, R, FILTER, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::TOTAL) !=
        cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast2 kernel: shared memory attribute (%d bytes)", S::TOTAL);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, S::TOTAL);
    if (occ < 1)
        occ = 1;
    const int cap = ctx->num_sms * occ;
    if (ctx->fast_zlen > 0) {
        a.zlen = ctx->fast_zlen;
    } else if (S::BOX) {
        // the longest of 64, 32, 16 planes that still gives every CTA three items
        a.zlen = 16;
        for (int zl : {64, 32})
            if ((long long)a.tiles_x * a.tiles_y * ((j.bz + zl - 1) / zl) >= 3ll * cap) {
                a.zlen = zl;
                break;
            }
    } else {
        a.zlen = 16;
    }
    // the tap kernels' work is concentrated where voxels pass the gate: shorter
    // z chunks (four times the work items) keep one heavy item from setting the end
    if (!S::BOX)
        a.zlen = std::max(1, a.zlen / 4);
    a.total_items = a.tiles_x * a.tiles_y * ((j.bz + a.zlen - 1) / a.zlen);
    const int grid = std::min(a.total_items, cap);
    if (cudaMemsetAsync(a.counter, 0, sizeof(u32), st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast2 kernel: counter reset");
    kern<<<grid, kThreads, S::TOTAL, st>>>(*tmap, a);
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast2 kernel launch failed");
    *handled = 1;
    return LNF_OK;
}

template <typename T, int FILTER>
lnf_status by_radius(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, u32 *counter, int *handled, int gated)
{
    switch (j.radius) {
    case 1: return launch2<T, 1, FILTER>(ctx, j, st, counter, handled, gated);
    case 2: return launch2<T, 2, FILTER>(ctx, j, st, counter, handled, gated);
    case 3: return launch2<T, 3, FILTER>(ctx, j, st, counter, handled, gated);
    default: return launch2<T, 4, FILTER>(ctx, j, st, counter, handled, gated);
    }
}

}  // namespace
