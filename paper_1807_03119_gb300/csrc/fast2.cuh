// Specialised kernels for the four comparison filters on volumes whose row
// pitch allows TMA (whole volumes or regions of interest); every other job
// runs on the generic kernel (filter.cu).  Included by fast2_box.cu (mean,
// entropy filter) and fast2_tap.cu (sigma, Okada, and the dispatch), two
// translation units that compile in parallel.
//
//   box kernel  -- mean (Eq. 4) and entropy filter (Eq. 7): B = sum over the
//                  M^3 cube of q(P), q = identity or the fixed-point weight
//                  w[P].  Per step the lane keeps the z line sum Bz of each of
//                  its voxels as a running sum (one plane in, one out), the
//                  CTA writes the Bz plane (tile + halo) to shared memory, and
//                  each lane forms the 2D box of Bz over its 4 x 4 voxels with
//                  running sums in registers.
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
    // box kernel: Bz plane of (kTY + 2R) rows x (kTX + 8) u32, own cells at column offset 4
    static constexpr int BW = kTX + 8;
    static constexpr int BZ = (kTY + 2 * R) * BW * 4;
    static constexpr int NHALO = 2 * R * (kTY + 2 * R) + 2 * R * kTX;
    static constexpr int HS = (NHALO + kThreads - 1) / kThreads;
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

// ------------------------------------------------------------------ box kernel body

constexpr int kBoxPF = 1;            // box kernel: one plane prefetched (two CTAs per SM fit)
constexpr int kBoxWin = 2048;        // box kernel (entropy): histogram / weight windows

template <typename T, int R, bool ENT>
struct BoxBody {
    typedef Geo2<T, R, kBoxPF> G;
    // per-thread state
    u32 bz[kRows][4];
    u32 hz[G::HS];
    int hcol[G::HS], hrow[G::HS];   // halo cell coordinates relative to the tile (-R..)
    u32 te;                          // entropy threshold
    const u32 *lut_sh;
    u32 lut_base;
    const u32 *lut_g;

    __device__ __forceinline__ u32 q(u32 v) const
    {
        if (!ENT)
            return v;
        const u32 o = v - lut_base;
        return o < (u32)kBoxWin ? lut_sh[o] : __ldg(lut_g + v);
    }
};

template <typename T, int R, bool ENT, bool MASK>
__device__ void box_items(const Args2 &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item, int *s_abort,
                          Hist2 &hist, const u32 *lut_sh, u32 lut_base)
{
    using namespace lnfdev;
    typedef Geo2<T, R, kBoxPF> G;
    unsigned char *ring = smem;
    u32 *bzp = reinterpret_cast<u32 *>(smem + G::RING);
    u64 *bars = reinterpret_cast<u64 *>(smem + G::RING + G::BZ);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = G::XH + 4 * lane;
    const int r0 = G::H + kRows * warp;
    const DevParams &P = *a.prm;
    const u32 T_ = P.T;
    constexpr u32 M3 = (u32)(G::M * G::M * G::M);
    typedef ExactDiv<M3, (unsigned long long)M3 * 65536ull> MDiv;
    u32 te = 0;
    if (ENT) {
        if (P.te_cfg == -2)
            te = (u32)(((unsigned __int128)M3 * P.hw_sum) / P.N);
        else
            te = P.te_cfg < 0 ? 0u : (P.te_cfg > 0xFFFFFFFFll ? 0xFFFFFFFFu : (u32)P.te_cfg);
    }
    const bool pass_all = ENT && P.te_cfg == -1;
    BoxBody<T, R, ENT> B;
    B.lut_sh = lut_sh;
    B.lut_base = lut_base;
    B.lut_g = a.lut;
    // halo cells of the Bz plane handled by this thread
#pragma unroll
    for (int j = 0; j < G::HS; ++j) {
        int k = threadIdx.x + j * kThreads;
        int col = 0, row = 0;
        if (k < G::NHALO) {
            const int nside = 2 * R * (kTY + 2 * R);
            if (k < nside) {
                const int c = k % (2 * R);
                col = c < R ? -R + c : kTX + (c - R);
                row = k / (2 * R) - R;
            } else {
                k -= nside;
                const int ri = k / kTX;
                col = k % kTX;
                row = ri < R ? -R + ri : kTY + (ri - R);
            }
        } else {
            col = 0;
            row = 0;   // duplicate of an own cell: computed but never written
        }
        B.hcol[j] = col;
        B.hrow[j] = row;
    }
    const bool hvalid_last = threadIdx.x + (G::HS - 1) * kThreads < G::NHALO;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::NP; ++s)
            mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0)
            *s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = *s_item;
        __syncthreads();
        if (item >= a.total_items || *s_abort)
            break;
        const int tx = item % a.tiles_x;
        const int rest = item / a.tiles_x;
        const int ty = rest % a.tiles_y;
        const int zc = rest / a.tiles_y;
        const int x0 = a.xs + tx * kTX, y0 = a.oy + ty * kTY;
        const int z0 = a.oz + zc * a.zlen, z1 = min(a.oz + a.bz, z0 + a.zlen);
        const int px0 = x0 - G::XH, py0 = y0 - G::H;
        const bool border = px0 < 0 || px0 + G::PW > a.nx || py0 < 0 || py0 + G::PH > a.ny;
        const int nplanes = (z1 - z0) + 2 * R;   // plane p <-> z = z0 - R + p
        const u32 pbytes = G::PW * G::PH * sizeof(T);
        auto issue = [&](int p) {
            const int slot = p % G::NP;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[slot], pbytes);
            tma_load_3d(ring + slot * G::PBYTES, tmap, &bars[slot], px0, py0, clampi(z0 - R + p, 0, a.nz - 1));
        };
        auto prefetch = [&](int p) {   // thread 0 only: plane p into L2
            if (p < nplanes)
                tma_prefetch_3d(tmap, max(px0, 0), max(py0, 0), clampi(z0 - R + p, 0, a.nz - 1));
        };
        if (threadIdx.x == 0) {
            for (int p = 0; p < min(G::NP, nplanes); ++p)
                issue(p);
            for (int p = G::NP; p < G::NP + kL2Ahead; ++p)
                prefetch(p);
        }
        bool ok = true;
        for (int s = 0; s < z1 - z0; ++s) {
            // one thread waits for the TMA completions; the barrier orders the
            // data before every thread's reads
            const int pfirst = s == 0 ? 0 : s + 2 * R;
            if (threadIdx.x == 0)
                for (int p = pfirst; p <= s + 2 * R; ++p)
                    if (!mbar_wait_bounded(&bars[p % G::NP], (u32)((p / G::NP) & 1), a.err))
                        *s_abort = 1;
            __syncthreads();
            if (*s_abort) {
                ok = false;
                break;
            }
            if (border)
                for (int p = pfirst; p <= s + 2 * R; ++p)
                    fixup2<T, R>(ring + (p % G::NP) * G::PBYTES, px0, py0, a.nx, a.ny);
            // ---- z line sums of q(P): initialise, then one plane in and one out
            if (s == 0) {
#pragma unroll
                for (int i = 0; i < kRows; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        B.bz[i][k] = 0;
#pragma unroll
                for (int j = 0; j < G::HS; ++j)
                    B.hz[j] = 0;
                for (int p = 0; p <= 2 * R; ++p) {
                    const unsigned char *pl = ring + (p % G::NP) * G::PBYTES;
#pragma unroll
                    for (int i = 0; i < kRows; ++i) {
                        u32 v[4];
                        ld4<T>(pl + (r0 + i) * G::ROWB, c0, v);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            B.bz[i][k] += B.q(v[k]);
                    }
#pragma unroll
                    for (int j = 0; j < G::HS; ++j)
                        B.hz[j] += B.q(ld1<T>(pl + (G::H + B.hrow[j]) * G::ROWB, G::XH + B.hcol[j]));
                }
            } else {
                const unsigned char *pn = ring + ((s + 2 * R) % G::NP) * G::PBYTES;
                const unsigned char *po = ring + ((s - 1) % G::NP) * G::PBYTES;
#pragma unroll
                for (int i = 0; i < kRows; ++i) {
                    u32 vn[4], vo[4];
                    ld4<T>(pn + (r0 + i) * G::ROWB, c0, vn);
                    ld4<T>(po + (r0 + i) * G::ROWB, c0, vo);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        B.bz[i][k] += B.q(vn[k]) - B.q(vo[k]);
                }
#pragma unroll
                for (int j = 0; j < G::HS; ++j) {
                    const int rr = (G::H + B.hrow[j]) * G::ROWB, cc = G::XH + B.hcol[j];
                    B.hz[j] += B.q(ld1<T>(pn + rr, cc)) - B.q(ld1<T>(po + rr, cc));
                }
            }
            // ---- Bz plane to shared memory (own cells + halo)
#pragma unroll
            for (int i = 0; i < kRows; ++i)
                *reinterpret_cast<uint4 *>(bzp + (R + kRows * warp + i) * G::BW + 4 + 4 * lane) =
                    make_uint4(B.bz[i][0], B.bz[i][1], B.bz[i][2], B.bz[i][3]);
#pragma unroll
            for (int j = 0; j < G::HS; ++j)
                if (j < G::HS - 1 || hvalid_last)
                    bzp[(R + B.hrow[j]) * G::BW + 4 + B.hcol[j]] = B.hz[j];
            __syncthreads();
            // plane s-1 was last read by the z line sums above: refill its slot
            if (threadIdx.x == 0 && s >= 1 && s - 1 + G::NP < nplanes) {
                issue(s - 1 + G::NP);
                prefetch(s - 1 + G::NP + kL2Ahead);
            }
            // ---- 2D box of Bz over the lane's 4 x 4 voxels
            u32 box[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    box[i][k] = 0;
#pragma unroll
            for (int rr = 0; rr < kRows + 2 * R; ++rr) {   // Bz rows y0w - R .. y0w + 3 + R
                const u32 *row = bzp + (kRows * warp + rr) * G::BW + 4 * lane;   // column x - 4
                const uint4 a0 = *reinterpret_cast<const uint4 *>(row);
                const uint4 a1 = *reinterpret_cast<const uint4 *>(row + 4);
                const uint4 a2 = *reinterpret_cast<const uint4 *>(row + 8);
                const u32 w[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
                u32 sx[4];
                sx[0] = 0;
#pragma unroll
                for (int d = -R; d <= R; ++d)
                    sx[0] += w[4 + d];
#pragma unroll
                for (int k = 1; k < 4; ++k)
                    sx[k] = sx[k - 1] + w[4 + k + R] - w[4 + k - 1 - R];
#pragma unroll
                for (int i = 0; i < kRows; ++i)
                    if (rr - R - i >= -R && rr - R - i <= R)
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            box[i][k] += sx[k];
            }
            // ---- gate, round / select, store, histogram
            const int z = z0 + s;
            const unsigned char *pc = ring + ((s + R) % G::NP) * G::PBYTES;
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                u32 p0[4];
                ld4<T>(pc + (r0 + i) * G::ROWB, c0, p0);
                u32 f[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (ENT)
                        f[k] = (p0[k] >= T_ && (pass_all || box[i][k] > te)) ? p0[k] : 0u;
                    else   // round(B / M^3) half up = floor((B + (M^3 - 1)/2) / M^3), M^3 odd
                        f[k] = (p0[k] >= T_ && box[i][k] >= M3 * T_) ? MDiv::template div_add<(M3 - 1) / 2>(box[i][k])
                                                                     : 0u;
                }
                const int y = y0 + kRows * warp + i, x = x0 + 4 * lane;
                if (MASK) {
                    store_roi<T>(a, hist, z, y, x, f);
                } else if (y < a.ny && x < a.nx) {
                    store4<T>(a, z, y, x, f);
                    hist4(hist, f);
                }
            }
            // the next step's first barrier orders these Bz-plane reads before
            // that step's Bz-plane writes
        }
        if (!ok) {
            if (threadIdx.x == 0) {
                const u64 t0 = global_ns();
                while (global_ns() - t0 < 2000000ull) {
                }
            }
            __syncthreads();
            break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int sl = 0; sl < G::NP; ++sl) {
                mbar_inval(&bars[sl]);
                mbar_init(&bars[sl], 1);
            }
            fence_mbar_init();
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ tap kernel body

// SIGMA: |P_i - P0| <= delta over the cube; OKADA: centre + axis cross, |P0 - P_i| < td.
// Value and count are accumulated in one word: acc += (v << CS) | 1.
template <typename T, int R>
struct TapPack {
    static constexpr int M3 = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    static constexpr int CS = M3 < 256 ? 8 : (M3 < 1024 ? 10 : 13);
    static constexpr unsigned long long MAXV = sizeof(T) == 1 ? 255ull : 65535ull;
    static constexpr bool PACK = MAXV * M3 * (1ull << CS) < (1ull << 32);
};

template <typename T, int R, int FILTER, bool MASK>
__device__ void tap_items(const Args2 &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item, int *s_abort,
                          Hist2 &hist, const u32 *recip)
{
    using namespace lnfdev;
    typedef Geo2<T, R> G;
    typedef TapPack<T, R> TP;
    unsigned char *ring = smem;
    u64 *bars = reinterpret_cast<u64 *>(smem + G::RING);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = G::XH + 4 * lane;
    const int r0 = G::H + kRows * warp;
    const DevParams &P = *a.prm;
    const u32 T_ = P.T;
    const u32 dl = min(P.delta, 65535u);
    const long long td = P.td;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::NP; ++s)
            mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0)
            *s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = *s_item;
        __syncthreads();
        if (item >= a.total_items || *s_abort)
            break;
        const int tx = item % a.tiles_x;
        const int rest = item / a.tiles_x;
        const int ty = rest % a.tiles_y;
        const int zc = rest / a.tiles_y;
        const int x0 = a.xs + tx * kTX, y0 = a.oy + ty * kTY;
        const int z0 = a.oz + zc * a.zlen, z1 = min(a.oz + a.bz, z0 + a.zlen);
        const int px0 = x0 - G::XH, py0 = y0 - G::H;
        const bool border = px0 < 0 || px0 + G::PW > a.nx || py0 < 0 || py0 + G::PH > a.ny;
        const int nplanes = (z1 - z0) + 2 * R;
        const u32 pbytes = G::PW * G::PH * sizeof(T);
        auto issue = [&](int p) {
            const int slot = p % G::NP;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[slot], pbytes);
            tma_load_3d(ring + slot * G::PBYTES, tmap, &bars[slot], px0, py0, clampi(z0 - R + p, 0, a.nz - 1));
        };
        auto prefetch = [&](int p) {   // thread 0 only: plane p into L2
            if (p < nplanes)
                tma_prefetch_3d(tmap, max(px0, 0), max(py0, 0), clampi(z0 - R + p, 0, a.nz - 1));
        };
        if (threadIdx.x == 0) {
            for (int p = 0; p < min(G::NP, nplanes); ++p)
                issue(p);
            for (int p = G::NP; p < G::NP + kL2Ahead; ++p)
                prefetch(p);
        }
        bool ok = true;
        for (int s = 0; s < z1 - z0; ++s) {
            // one thread waits for the TMA completions; the barrier orders the
            // data before every thread's reads
            const int pfirst = s == 0 ? 0 : s + 2 * R;
            if (threadIdx.x == 0)
                for (int p = pfirst; p <= s + 2 * R; ++p)
                    if (!mbar_wait_bounded(&bars[p % G::NP], (u32)((p / G::NP) & 1), a.err))
                        *s_abort = 1;
            __syncthreads();
            if (*s_abort) {
                ok = false;
                break;
            }
            // plane s-1 was last read at step s-1, which every thread has finished
            if (threadIdx.x == 0 && s >= 1 && s - 1 + G::NP < nplanes) {
                issue(s - 1 + G::NP);
                prefetch(s - 1 + G::NP + kL2Ahead);
            }
            if (border)
                for (int p = pfirst; p <= s + 2 * R; ++p)
                    fixup2<T, R>(ring + (p % G::NP) * G::PBYTES, px0, py0, a.nx, a.ny);
            const unsigned char *pc = ring + ((s + R) % G::NP) * G::PBYTES;   // plane z
            u32 p0[kRows][4], lo[kRows][4], wd[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                ld4<T>(pc + (r0 + i) * G::ROWB, c0, p0[i]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (FILTER == LNF_SIGMA) {   // band [P0 - delta, P0 + delta] as (v - lo) <= width
                        lo[i][k] = p0[i][k] > dl ? p0[i][k] - dl : 0u;
                        wd[i][k] = p0[i][k] - lo[i][k] + dl;
                    } else {                     // |P0 - v| < td  as (v - lo) <= width, td >= 1
                        const u32 t1 = td > 65536 ? 65535u : (u32)(td - 1);
                        lo[i][k] = p0[i][k] > t1 ? p0[i][k] - t1 : 0u;
                        wd[i][k] = p0[i][k] - lo[i][k] + t1;
                    }
                }
            }
            u32 acc[kRows][4], cnt[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[i][k] = 0;
                    cnt[i][k] = 0;
                }
            // per tap and voxel: d = v - lo (multiply-add: FMA pipe), in-band test
            // (compare: ALU pipe), accumulate (alternately FMA and ALU pipe), so
            // that the integer work is split between the two half-rate pipes
            const u32 one = a.one;
            u32 nlo[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    nlo[i][k] = 0u - lo[i][k];
            auto take = [&](int i, int k, u32 v, u32 pv) {
                if (TP::PACK) {
                    // d = v - lo: a plain add (ALU) for even voxels, a multiply-add by
                    // the runtime 1 (FMA pipe) for odd ones; the in-band test is a
                    // compare (ALU) and the accumulate a predicated multiply-add (FMA)
                    u32 d;
                    if (k & 1)
                        asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(v), "r"(one), "r"(nlo[i][k]));
                    else
                        d = v + nlo[i][k];
                    asm(
                        "{\n\t.reg .pred p;\n\tsetp.le.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %4, %0;\n\t}"
                        : "+r"(acc[i][k])
                        : "r"(d), "r"(wd[i][k]), "r"(pv), "r"(one));
                } else {
                    if (v - lo[i][k] <= wd[i][k]) {
                        acc[i][k] += v;
                        cnt[i][k] += 1;
                    }
                }
            };
            if (FILTER == LNF_SIGMA) {
#pragma unroll 1
                for (int dz = -R; dz <= R; ++dz) {
                    const unsigned char *pl = ring + ((s + R + dz) % G::NP) * G::PBYTES;
#pragma unroll
                    for (int rr = 0; rr < kRows + 2 * R; ++rr) {   // rows r0 - R .. r0 + 3 + R
                        u32 v[12], pv[12];
                        const unsigned char *row = pl + (r0 - R + rr) * G::ROWB;
                        ld4<T>(row, c0 - 4, v);
                        ld4<T>(row, c0, v + 4);
                        ld4<T>(row, c0 + 4, v + 8);
#pragma unroll
                        for (int e = 0; e < 12; ++e)
                            pv[e] = TP::PACK ? ((v[e] << TP::CS) | 1u) : v[e];
#pragma unroll
                        for (int i = 0; i < kRows; ++i) {
                            const int dy = rr - R - i;
                            if (dy < -R || dy > R)
                                continue;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
#pragma unroll
                                for (int dx = -R; dx <= R; ++dx)
                                    take(i, k, v[4 + k + dx], pv[4 + k + dx]);
                        }
                    }
                }
            } else if (td > 0) {   // Okada: centre + cross of arm R (td == 0 selects nothing)
#pragma unroll
                for (int i = 0; i < kRows; ++i) {
                    const unsigned char *row = pc + (r0 + i) * G::ROWB;
                    u32 v[12];
                    ld4<T>(row, c0 - 4, v);
                    ld4<T>(row, c0, v + 4);
                    ld4<T>(row, c0 + 4, v + 8);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        auto pk = [&](u32 x) { return TP::PACK ? ((x << TP::CS) | 1u) : x; };
                        take(i, k, v[4 + k], pk(v[4 + k]));   // the centre itself
#pragma unroll
                        for (int t = 1; t <= R; ++t) {
                            take(i, k, v[4 + k - t], pk(v[4 + k - t]));
                            take(i, k, v[4 + k + t], pk(v[4 + k + t]));
                        }
                    }
                }
#pragma unroll
                for (int t = 1; t <= R; ++t) {
#pragma unroll
                    for (int sg = -1; sg <= 1; sg += 2) {
                        const unsigned char *plz = ring + ((s + R + sg * t) % G::NP) * G::PBYTES;
#pragma unroll
                        for (int i = 0; i < kRows; ++i) {
                            u32 vy[4], vz[4];
                            ld4<T>(pc + (r0 + i + sg * t) * G::ROWB, c0, vy);
                            ld4<T>(plz + (r0 + i) * G::ROWB, c0, vz);
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                take(i, k, vy[k], TP::PACK ? ((vy[k] << TP::CS) | 1u) : vy[k]);
                                take(i, k, vz[k], TP::PACK ? ((vz[k] << TP::CS) | 1u) : vz[k]);
                            }
                        }
                    }
                }
            }
            // ---- gate, round, store, histogram
            // round(sm / n) half up = floor((sm + floor(n/2)) / n) = (x * recip[n]) >> 32
            // with recip[n] = ceil(2^32 / n): exact when x e < 2^32 (e = recip n - 2^32 < n);
            // x < n 2^16 gives x e < n^2 2^16, so counts below 256 use the table
            // and larger ones (sigma at radius >= 3) divide
            const int z = z0 + s;
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                u32 f[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const u32 n = TP::PACK ? (acc[i][k] & ((1u << TP::CS) - 1u)) : cnt[i][k];
                    const u32 sm = TP::PACK ? (acc[i][k] >> TP::CS) : acc[i][k];
                    const u32 x = sm + (n >> 1);
                    const u32 q = n == 1 ? sm : (n < 256 ? __umulhi(x, recip[n]) : x / n);
                    f[k] = (n && p0[i][k] >= T_ && (u64)sm >= (u64)n * T_) ? q : 0u;
                }
                const int y = y0 + kRows * warp + i, x = x0 + 4 * lane;
                if (MASK) {
                    store_roi<T>(a, hist, z, y, x, f);
                } else if (y < a.ny && x < a.nx) {
                    store4<T>(a, z, y, x, f);
                    hist4(hist, f);
                }
            }
        }
        if (!ok) {
            if (threadIdx.x == 0) {
                const u64 t0 = global_ns();
                while (global_ns() - t0 < 2000000ull) {
                }
            }
            __syncthreads();
            break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int sl = 0; sl < G::NP; ++sl) {
                mbar_inval(&bars[sl]);
                mbar_init(&bars[sl], 1);
            }
            fence_mbar_init();
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ kernels

template <typename T, int R, int FILTER>
struct K2Smem {
    static constexpr bool BOX = FILTER == LNF_MEAN || FILTER == LNF_ENTROPY;
    typedef Geo2<T, R, BOX ? kBoxPF : kPF> G;
    static constexpr int HWIN = sizeof(T) == 1 ? 256 : (FILTER == LNF_ENTROPY ? kBoxWin : kHistWin);
    static constexpr int LWIN = sizeof(T) == 1 ? 256 : kBoxWin;
    static constexpr int HISTB = HWIN * 4;
    static constexpr int NTAB = (2 * R + 1) * (2 * R + 1) * (2 * R + 1) + 1;   // counts 0 .. M^3
    static constexpr int LUTB = FILTER == LNF_ENTROPY ? LWIN * 4 : (BOX ? 0 : ((NTAB * 4 + 15) / 16) * 16);
    static constexpr int MAIN = G::RING + (BOX ? G::BZ : 0) + G::NP * 8;
    static constexpr int TOTAL = 128 + MAIN + 64 + HISTB + LUTB;
};

// MASK: masked per-voxel stores (a region of interest, an odd width), else dense
// 4-voxel vector stores
template <typename T, int R, int FILTER, bool MASK>
__global__ void __launch_bounds__(kThreads, (K2Smem<T, R, FILTER>::BOX && R > 2) ? 1 : 2)
    k_fast2(const __grid_constant__ CUtensorMap tmap, const Args2 a)
{
    typedef K2Smem<T, R, FILTER> S;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128 - (lnfdev::smem_u32(smem_raw) & 127)) & 127);
    __shared__ int s_item, s_abort;
    u32 *hsh = reinterpret_cast<u32 *>(smem + S::MAIN + 64);
    u32 *lut_sh = reinterpret_cast<u32 *>(smem + S::MAIN + 64 + S::HISTB);
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
    if (FILTER == LNF_MEAN)
        box_items<T, R, false, MASK>(a, &tmap, smem, &s_item, &s_abort, h, lut_sh, lut_base);
    else if (FILTER == LNF_ENTROPY)
        box_items<T, R, true, MASK>(a, &tmap, smem, &s_item, &s_abort, h, lut_sh, lut_base);
    else
        tap_items<T, R, FILTER, MASK>(a, &tmap, smem, &s_item, &s_abort, h, lut_sh);
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
lnf_status launch2(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, u32 *counter, int *handled)
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
    a.zlen = ctx->fast_zlen > 0 ? ctx->fast_zlen : 16;
    a.total_items = a.tiles_x * a.tiles_y * ((j.bz + a.zlen - 1) / a.zlen);
    a.filter = FILTER;
    a.prm = j.prm;
    a.lut = j.lut;
    a.out_hist = j.out_hist;
    a.counter = counter ? counter : ctx->d_counter + 9;
    a.err = ctx->d_err;
    a.one = 1u;
    void (*kern)(const CUtensorMap, const Args2) = a.roi ? k_fast2<T, R, FILTER, true> : k_fast2<T, R, FILTER, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::TOTAL) !=
        cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast2 kernel: shared memory attribute (%d bytes)", S::TOTAL);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, S::TOTAL);
    if (occ < 1)
        occ = 1;
    const int grid = std::min(a.total_items, ctx->num_sms * occ);
    if (cudaMemsetAsync(a.counter, 0, sizeof(u32), st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast2 kernel: counter reset");
    kern<<<grid, kThreads, S::TOTAL, st>>>(*tmap, a);
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast2 kernel launch failed");
    *handled = 1;
    return LNF_OK;
}

template <typename T, int FILTER>
lnf_status by_radius(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, u32 *counter, int *handled)
{
    switch (j.radius) {
    case 1: return launch2<T, 1, FILTER>(ctx, j, st, counter, handled);
    case 2: return launch2<T, 2, FILTER>(ctx, j, st, counter, handled);
    case 3: return launch2<T, 3, FILTER>(ctx, j, st, counter, handled);
    default: return launch2<T, 4, FILTER>(ctx, j, st, counter, handled);
    }
}

}  // namespace
