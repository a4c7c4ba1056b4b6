// Specialised kernel for the paper's filter (Eq. 2-3) at radius 1..4 with the
// diagonal clusters at distance sqrt(3) (offset d = 1), for whole volumes
// whose row pitch allows TMA.  lnf_fast_dispatch routes such jobs here; every
// other job goes to the generic kernel (filter.cu).
//
// Algebra (exact, integer): with the line sums Lx, Ly, Lz of M = 2r+1 voxels,
//   G = Lx + Ly + Lz                       (the unnormalised cluster S at a voxel)
//   U = G + T_x T_y T_z G                  (S_0 plus the eight diagonal clusters)
// where T_a f(c) = f(c - e_a) + f(c + e_a).  With C = T_x T_y G,
//   U(z) = G(z) + C(z-1) + C(z+1),
// and the output is round(U / 27M), gated by P0 >= T and U >= 27M T.
//
// Mapping: a CTA owns a 128 x 32 output tile and marches along z over a chunk
// of planes; the input planes (tile + halo) stream into a ring of shared
// memory slots by TMA.  Each lane owns 4 consecutive columns of 4 rows.
// Shared-memory bandwidth is what bounds this kernel, so each value is read
// from shared memory as few times as possible:
//   * z: Lz is a running sum held in registers (one term in, one out per
//     step); the output needs two accumulators per voxel, A = G(z-1) + C(z-2)
//     and B = C(z-1), so the z direction costs no shared memory beyond the
//     new and the old plane.
//   * y: a lane reads its rows and R rows on each side of the current plane
//     once; Ly is a running sum down that window, and the lane's own rows
//     are kept as P0 for the next step's outputs.
//   * x: Lx takes the neighbouring columns from the adjacent lanes
//     (shuffles); lanes 0 and 31 read the columns beyond the tile.
//   * C = T_x T_y G: T_y from the lane's rows and the neighbouring warps'
//     boundary rows (the only G values that pass through shared memory),
//     T_x across lanes.  The one-voxel ring around the tile is computed by
//     the first and last warp (rows above and below, vectorised) and by a
//     few lanes per warp (the two ring columns, voxel by voxel).
//     Two barriers per step.
// Line sums are formed on packed pairs of 16-bit lanes (two voxels per 32-bit
// add) whenever 3M * max <= 65535, which keeps every lane exact; otherwise
// the same code runs on unpacked 32-bit pairs.
#include "lnf_ctx.h"

#include <algorithm>
#include <cstring>

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRows = 4;                  // rows per lane
constexpr int kTX = 128;                  // 32 lanes x 4 columns
constexpr int kTY = kWarps * kRows;       // 32

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------------------------ packed pairs

// two adjacent voxels in the 16-bit lanes of one register (exact while every
// final lane value stays within 0..65535)
struct Narrow {
    typedef u32 P;
    static __device__ __forceinline__ P word(u32 w) { return w; }
    static __device__ __forceinline__ P shift(P a, P b) { return __funnelshift_r(a, b, 16); }   // (a.hi, b.lo)
    static __device__ __forceinline__ P add3(P a, P b, P c) { return a + b + c; }
    static __device__ __forceinline__ P addsub(P a, P b, P c) { return a + b - c; }
    static __device__ __forceinline__ P zero() { return 0u; }
    static __device__ __forceinline__ u32 lo(P a) { return a & 0xFFFFu; }
    static __device__ __forceinline__ u32 hi(P a) { return a >> 16; }
};

// the same pair unpacked into two 32-bit registers (any 16-bit data)
struct Wide {
    struct P {
        u32 l, h;
    };
    static __device__ __forceinline__ P word(u32 w) { return P{w & 0xFFFFu, w >> 16}; }
    static __device__ __forceinline__ P shift(P a, P b) { return P{a.h, b.l}; }
    static __device__ __forceinline__ P add3(P a, P b, P c) { return P{a.l + b.l + c.l, a.h + b.h + c.h}; }
    static __device__ __forceinline__ P addsub(P a, P b, P c) { return P{a.l + b.l - c.l, a.h + b.h - c.h}; }
    static __device__ __forceinline__ P zero() { return P{0u, 0u}; }
    static __device__ __forceinline__ u32 lo(P a) { return a.l; }
    static __device__ __forceinline__ u32 hi(P a) { return a.h; }
};

// loads from a shared-memory row (byte pointer) at element column `col`
template <typename T>
struct Ld;

template <>
struct Ld<uint16_t> {
    // columns col..col+3 as two words (col multiple of 4)
    static __device__ __forceinline__ void quad(const unsigned char *row, int col, u32 &a, u32 &b)
    {
        const uint2 w = *reinterpret_cast<const uint2 *>(row + col * 2);
        a = w.x;
        b = w.y;
    }
    // columns col, col+1 as one word (col even)
    static __device__ __forceinline__ u32 pair(const unsigned char *row, int col)
    {
        return *reinterpret_cast<const u32 *>(row + col * 2);
    }
};

template <>
struct Ld<uint8_t> {
    static __device__ __forceinline__ void quad(const unsigned char *row, int col, u32 &a, u32 &b)
    {
        const u32 w = *reinterpret_cast<const u32 *>(row + col);
        a = __byte_perm(w, 0u, 0x4140);
        b = __byte_perm(w, 0u, 0x4342);
    }
    static __device__ __forceinline__ u32 pair(const unsigned char *row, int col)
    {
        const u32 w = *reinterpret_cast<const unsigned short *>(row + col);
        return __byte_perm(w, 0u, 0x4140);
    }
};

// ------------------------------------------------------------------ geometry

constexpr int kPFo = 1;                  // planes prefetched into shared memory (two CTAs per SM fit)
constexpr int kL2Ahead = 6;              // planes prefetched into L2 beyond the shared-memory ring
constexpr int kGW = kTX + 8;             // G plane row: columns -1 .. 128 at offsets 3 .. 132

template <typename T, int R>
struct FGeo {
    static constexpr int H = R + 1;                        // halo in y and z
    static constexpr int XH = 16 / sizeof(T);              // x halo (16 bytes)
    static constexpr int PW = kTX + 2 * XH;                // plane width (elements)
    static constexpr int PH = kTY + 2 * H;                 // plane height
    static constexpr int ROWB = PW * sizeof(T);            // row bytes (multiple of 16)
    static constexpr int PBYTES = ((PW * PH * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int NP = 2 * R + 2 + kPFo;            // ring slots
    static constexpr int M = 2 * R + 1;
    static constexpr int RING = NP * PBYTES;
    static constexpr int GPLANE = (kTY + 2) * kGW * 4;
    // output histogram window: all 8-bit levels; 4096 16-bit levels where two
    // CTAs per SM still fit, else 2048
    static constexpr int HWIN = sizeof(T) == 1 ? 256 : (R <= 2 ? 4096 : 2048);
    static constexpr int HIST = (HWIN + 32) * 4;   // + one bin per lane counting zeros
    static constexpr int SMEM = 128 + RING + GPLANE + HIST + NP * 8 + 64;
};

// fix the out-of-volume cells of a freshly loaded plane by replicating the
// border; only the halo the kernel reads (H columns / rows on each side) is fixed
template <typename T, int R>
__device__ void fixup(unsigned char *pl, int px0, int py0, int nx, int ny)
{
    typedef FGeo<T, R> G;
    T *p = reinterpret_cast<T *>(pl);
    constexpr int HC = G::H;                       // columns read left of XH / right of XH + kTX - 1
    constexpr int NC = 2 * HC;
    const bool fix_l = px0 + G::XH - HC < 0, fix_r = px0 + G::XH + kTX + HC > nx;
    if (fix_l || fix_r || px0 + G::XH + kTX > nx)
        for (int e = threadIdx.x; e < NC * G::PH; e += blockDim.x) {
            const int row = e / NC;               // constant divisor
            const int k = e - row * NC;
            const int col = k < HC ? G::XH - HC + k : G::XH + kTX + (k - HC);
            const int vx = px0 + col;
            if (vx < 0 || vx >= nx)
                p[row * G::PW + col] = p[row * G::PW + clampi(vx, 0, nx - 1) - px0];
        }
    // columns inside the tile but beyond the volume (a ragged last tile)
    if (px0 + G::XH + kTX > nx)
        for (int e = threadIdx.x; e < kTX * G::PH; e += blockDim.x) {
            const int row = e / kTX;
            const int col = G::XH + (e - row * kTX);
            if (px0 + col >= nx)
                p[row * G::PW + col] = p[row * G::PW + nx - 1 - px0];
        }
    __syncthreads();
    const int top = py0 < 0 ? min(-py0, G::PH) : 0;
    const int bot0 = max(top, min(G::PH, ny - py0));
    const int nfix = top + (G::PH - bot0);
    for (int e = threadIdx.x; e < nfix * G::PW; e += blockDim.x) {
        const int k = e / G::PW;                  // constant divisor
        const int col = e - k * G::PW;
        const int row = k < top ? k : bot0 + (k - top);
        p[row * G::PW + col] = p[(clampi(py0 + row, 0, ny - 1) - py0) * G::PW + col];
    }
    __syncthreads();
}

// ------------------------------------------------------------------ per-row sums

__host__ __device__ constexpr int fl2(int o) { return o >= 0 ? o / 2 : -((-o + 1) / 2); }   // floor(o / 2)

// sum over o = -R..R of the pair at column base+o, from the aligned words wd[k]
// = pair at column base+2k (valid for k in [-(R+1)/2, (R+1)/2])
template <int R, class PK>
__device__ __forceinline__ typename PK::P window_sum(const typename PK::P *wd)
{
    typename PK::P acc = PK::zero();
#pragma unroll
    for (int o = -R; o <= R; o += 2) {
        // two terms per add3: the pair at o and (if o < R) the one at o + 1
        const typename PK::P t0 = (o & 1) == 0 ? wd[fl2(o)] : PK::shift(wd[fl2(o)], wd[fl2(o) + 1]);
        if (o < R) {
            const int o1 = o + 1;
            const typename PK::P t1 =
                (o1 & 1) == 0 ? wd[fl2(o1)] : PK::shift(wd[fl2(o1)], wd[fl2(o1) + 1]);
            acc = PK::add3(acc, t0, t1);
        } else {
            acc = PK::add3(acc, t0, PK::zero());
        }
    }
    return acc;
}

template <typename T, class PK>
__device__ __forceinline__ void quad_pairs(const unsigned char *row, int c0, typename PK::P &a, typename PK::P &b)
{
    u32 q0, q1;
    Ld<T>::quad(row, c0, q0, q1);
    a = PK::word(q0);
    b = PK::word(q1);
}

template <typename T>
__device__ __forceinline__ u32 ld1(const unsigned char *row, int col)
{
    return sizeof(T) == 2 ? (u32) reinterpret_cast<const uint16_t *>(row)[col] : (u32)row[col];
}

// ------------------------------------------------------------------ the kernel

struct FastArgs {
    const void *in;
    void *out;
    int nx, ny, nz;
    // output region [o, o + b) (the whole volume unless a region of interest),
    // tiled from column xs = ox rounded down to TMA's 16-byte rule
    int ox, oy, oz, bx, by, bz, xs, xend, yend;
    int roi;                              // 1: masked per-voxel stores (ROI-shaped output or odd width)
    int tiles_x, tiles_y, zchunks, zlen;
    int total_items;
    const DevParams *prm;
    u64 *out_hist;
    u32 *counter;
    u32 *err;
    int gated;                            // 1: launched beside the gate-first kernel, which may take the job
};

// the ring-column cell (tile column -1 or kTX, tile row -1 .. kTY) a lane
// computes: warp w takes tile rows 4w-1 .. 4w+2 (the last warp also kTY-1 and
// kTY), two lanes per row, one per side; consecutive rows fall in distinct banks
__device__ __forceinline__ bool ring_cell(int warp, int lane, int &row, int &col)
{
    const int j = lane >> 1;
    row = kRows * warp - 1 + j;
    col = (lane & 1) ? kTX : -1;
    return j < (warp == kWarps - 1 ? kRows + 2 : kRows);
}

// Lx of the lane's pairs A (c0, c0+1) and B (c0+2, c0+3) of one row, from the
// lane's own words w0, w1 and its neighbours' words (shuffles); lanes 0 and 31
// take the words beyond the tile from the row itself: the quad at column ec,
// which every lane of a half-warp shares (one broadcast read, no branch)
template <typename T, int R, class PK>
__device__ __forceinline__ void lx_lanes(const unsigned char *row, int ec, int lane, u32 w0, u32 w1,
                                         typename PK::P &lxA, typename PK::P &lxB)
{
    typedef typename PK::P P;
    constexpr int A = (R + 1) / 2;   // words needed on each side
    u32 e0, e1;
    Ld<T>::quad(row, ec, e0, e1);
    u32 l1 = __shfl_up_sync(0xFFFFFFFFu, w1, 1), r0 = __shfl_down_sync(0xFFFFFFFFu, w0, 1);
    if (lane == 0)
        l1 = e1;
    if (lane == 31)
        r0 = e0;
    P w[2 * A + 2];   // w[A + k] = pair at column c0 + 2k
    w[A - 1] = PK::word(l1);
    w[A] = PK::word(w0);
    w[A + 1] = PK::word(w1);
    w[A + 2] = PK::word(r0);
    if (A == 2) {
        u32 l0 = __shfl_up_sync(0xFFFFFFFFu, w0, 1), r1 = __shfl_down_sync(0xFFFFFFFFu, w1, 1);
        if (lane == 0)
            l0 = e0;
        if (lane == 31)
            r1 = e1;
        w[0] = PK::word(l0);
        w[2 * A + 1] = PK::word(r1);
    }
    lxA = window_sum<R, PK>(&w[A]);
    lxB = window_sum<R, PK>(&w[A + 1]);
}

template <typename T, int R, class PK, bool MASK>
__device__ void ours_items(const FastArgs &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item,
                           int *s_abort, u32 *hist, u32 hbase)
{
    using namespace lnfdev;
    typedef FGeo<T, R> G;
    typedef typename PK::P P;
    constexpr int NW = kRows + 2 * R;                 // rows a lane reads per plane: its own and R each side
    unsigned char *ring = smem;
    u32 *gp = reinterpret_cast<u32 *>(smem + G::RING);                      // G plane
    u64 *bars = reinterpret_cast<u64 *>(smem + G::RING + G::GPLANE + G::HIST);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = G::XH + 4 * lane;                   // first own column (plane coords)
    const int r0 = G::H + kRows * warp;                // first own row (plane coords)
    const int gr0 = 1 + kRows * warp;                  // first own row in the G plane
    const int gc0 = 4 + 4 * lane;                      // first own column in the G plane
    // the quad beyond the tile (read by lanes 0 / 31, shared by their half-warps)
    const int ec = lane < 16 ? G::XH - 4 : G::XH + kTX;
    const int egc = lane < 16 ? 3 : 4 + kTX;           // ... and its ring column in the G plane
    // the first and the last warp also compute the ring row above / below the tile
    const bool xtop = warp == 0, xbot = warp == kWarps - 1;
    const int xr = xtop ? r0 - 1 : r0 + kRows;         // plane row of that ring row
    const int xly = xtop ? r0 - R - 1 : r0 + kRows + R;   // the row its Ly needs beyond the window
    const int xg = xtop ? 0 : kTY + 1;                 // its G-plane row
    int hr = 0, hc = 0;
    const bool hv = ring_cell(warp, lane, hr, hc);     // ring-column cell of this lane, if any;
    if (!hv)                                           // the others shadow lane 0 / 1 (same reads)
        ring_cell(warp, lane & 1, hr, hc);
    const int hpr = G::H + hr, hpc = G::XH + hc;       // ... in plane coordinates

    const u32 T_ = a.prm->T;
    const u32 KT = 27u * G::M * T_;
    // round(U / 27M) half up = floor((2U + 27M) / 54M) = floor((U + (27M - 1)/2) / 27M)
    // (27M is odd); U < 27M * 65536 for any 16-bit input
    typedef ExactDiv<27ull * G::M, 27ull * G::M * 65536ull> Div;
    constexpr unsigned long long HALF = (27ull * G::M - 1) / 2;
    const u32 hbins = G::HWIN;
    const u32 hlim = hbase + hbins;   // nonzero outputs lie in [hbase, 65535]
    const u32 hzero = hbins + lane;   // this lane's zero bin (zeros never meet in one bin)
    // outputs are averages, so none exceeds maxv: values above the window occur
    // only when maxv >= hbase + hbins
    const bool hcheck = a.prm->maxv >= hlim;

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
        // plane p <-> z = z0 - 1 - R + p; G planes g = z0-1 .. z1 (steps s = 0 .. z1-z0+1)
        const int nplanes = (z1 - z0 + 2) + 2 * R;
        const int nsteps = z1 - z0 + 2;
        const u32 pbytes = G::PW * G::PH * sizeof(T);

        auto issue = [&](int p) {   // thread 0 only
            const int slot = p % G::NP;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[slot], pbytes);
            if (lnf_dbg_tma(px0, (int)sizeof(T), ring + slot * G::PBYTES, a.err))
                tma_load_3d(ring + slot * G::PBYTES, tmap, &bars[slot], px0, py0, clampi(z0 - 1 - R + p, 0, a.nz - 1));
        };
        auto prefetch = [&](int p) {   // thread 0 only: plane p into L2
            if (p < nplanes)
                tma_prefetch_3d(tmap, max(px0, 0), max(py0, 0), clampi(z0 - 1 - R + p, 0, a.nz - 1));
        };
        if (threadIdx.x == 0) {
            for (int p = 0; p < min(G::NP, nplanes); ++p)
                issue(p);
            for (int p = G::NP; p < G::NP + kL2Ahead; ++p)
                prefetch(p);
        }

        P lzA[kRows], lzB[kRows];                 // running z line sums of the own pairs
        P lzxA = PK::zero(), lzxB = PK::zero();   // ... of the ring row (first / last warp)
        u32 lzh = 0;                              // ... of the ring-column cell
        u32 accA[kRows][4], accB[kRows][4];       // z accumulators
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                accB[i][k] = 0;
        }
        bool ok = true;

        for (int s = 0; s < nsteps; ++s) {
            // planes needed: s-1 (old) .. s+2R (new); plane p is the (p / NP)-th
            // load into its slot since the barriers were initialised
            // one thread waits for the TMA completions; the barrier then
            // orders the data before every thread's reads (and keeps the other
            // warps off the issue slots while the planes arrive)
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
                    fixup<T, R>(ring + (p % G::NP) * G::PBYTES, px0, py0, a.nx, a.ny);
            const unsigned char *pg = ring + ((s + R) % G::NP) * G::PBYTES;   // G plane g = z0-1+s
            const unsigned char *pn = ring + ((s + 2 * R) % G::NP) * G::PBYTES;
            const unsigned char *po = ring + ((s + G::NP - 1) % G::NP) * G::PBYTES;

            // ---- Lz: initialise at the first step, then one plane in, one out
            if (s == 0) {
#pragma unroll
                for (int i = 0; i < kRows; ++i) {
                    lzA[i] = PK::zero();
                    lzB[i] = PK::zero();
                }
                lzxA = lzxB = PK::zero();
                lzh = 0;
                for (int d = 0; d <= 2 * R; ++d) {
                    const unsigned char *pl = ring + (d % G::NP) * G::PBYTES;
#pragma unroll
                    for (int i = 0; i < kRows; ++i) {
                        P qa, qb;
                        quad_pairs<T, PK>(pl + (r0 + i) * G::ROWB, c0, qa, qb);
                        lzA[i] = PK::add3(lzA[i], qa, PK::zero());
                        lzB[i] = PK::add3(lzB[i], qb, PK::zero());
                    }
                    if (xtop || xbot) {
                        P qa, qb;
                        quad_pairs<T, PK>(pl + xr * G::ROWB, c0, qa, qb);
                        lzxA = PK::add3(lzxA, qa, PK::zero());
                        lzxB = PK::add3(lzxB, qb, PK::zero());
                    }
                    lzh += ld1<T>(pl + hpr * G::ROWB, hpc);
                }
            } else {
#pragma unroll
                for (int i = 0; i < kRows; ++i) {
                    P na, nb, oa, ob;
                    quad_pairs<T, PK>(pn + (r0 + i) * G::ROWB, c0, na, nb);
                    quad_pairs<T, PK>(po + (r0 + i) * G::ROWB, c0, oa, ob);
                    lzA[i] = PK::addsub(lzA[i], na, oa);
                    lzB[i] = PK::addsub(lzB[i], nb, ob);
                }
                if (xtop || xbot) {
                    P na, nb, oa, ob;
                    quad_pairs<T, PK>(pn + xr * G::ROWB, c0, na, nb);
                    quad_pairs<T, PK>(po + xr * G::ROWB, c0, oa, ob);
                    lzxA = PK::addsub(lzxA, na, oa);
                    lzxB = PK::addsub(lzxB, nb, ob);
                }
                lzh += ld1<T>(pn + hpr * G::ROWB, hpc) - ld1<T>(po + hpr * G::ROWB, hpc);
            }

            // ---- the lane's window of plane g: rows r0-R .. r0+3+R, read once
            u32 rw[NW][2];
#pragma unroll
            for (int j = 0; j < NW; ++j)
                Ld<T>::quad(pg + (r0 - R + j) * G::ROWB, c0, rw[j][0], rw[j][1]);

            // ---- G of the own voxels (packed pairs): Ly running down the window
            u32 g[kRows][4];
            P lyA = PK::zero(), lyB = PK::zero();
#pragma unroll
            for (int j = 0; j <= 2 * R; ++j) {
                lyA = PK::add3(lyA, PK::word(rw[j][0]), PK::zero());
                lyB = PK::add3(lyB, PK::word(rw[j][1]), PK::zero());
            }
            const P ly0A = lyA, ly0B = lyB;
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                if (i > 0) {
                    lyA = PK::addsub(lyA, PK::word(rw[i + 2 * R][0]), PK::word(rw[i - 1][0]));
                    lyB = PK::addsub(lyB, PK::word(rw[i + 2 * R][1]), PK::word(rw[i - 1][1]));
                }
                P lxA, lxB;
                lx_lanes<T, R, PK>(pg + (r0 + i) * G::ROWB, ec, lane, rw[R + i][0], rw[R + i][1], lxA, lxB);
                const P gA = PK::add3(lxA, lyA, lzA[i]);
                const P gB = PK::add3(lxB, lyB, lzB[i]);
                g[i][0] = PK::lo(gA);
                g[i][1] = PK::hi(gA);
                g[i][2] = PK::lo(gB);
                g[i][3] = PK::hi(gB);
            }
            // rows other warps need: the first and the last own row
            if (warp > 0)
                *reinterpret_cast<uint4 *>(gp + gr0 * kGW + gc0) = make_uint4(g[0][0], g[0][1], g[0][2], g[0][3]);
            if (warp < kWarps - 1)
                *reinterpret_cast<uint4 *>(gp + (gr0 + kRows - 1) * kGW + gc0) =
                    make_uint4(g[kRows - 1][0], g[kRows - 1][1], g[kRows - 1][2], g[kRows - 1][3]);
            // ---- the ring row (first / last warp)
            if (xtop || xbot) {
                u32 ea, eb;
                Ld<T>::quad(pg + xly * G::ROWB, c0, ea, eb);
                P xlyA, xlyB, lxA, lxB;
                if (xtop) {
                    xlyA = PK::addsub(ly0A, PK::word(ea), PK::word(rw[2 * R][0]));
                    xlyB = PK::addsub(ly0B, PK::word(eb), PK::word(rw[2 * R][1]));
                    lx_lanes<T, R, PK>(pg + xr * G::ROWB, ec, lane, rw[R - 1][0], rw[R - 1][1], lxA, lxB);
                } else {
                    xlyA = PK::addsub(lyA, PK::word(ea), PK::word(rw[kRows - 1][0]));
                    xlyB = PK::addsub(lyB, PK::word(eb), PK::word(rw[kRows - 1][1]));
                    lx_lanes<T, R, PK>(pg + xr * G::ROWB, ec, lane, rw[R + kRows][0], rw[R + kRows][1], lxA,
                                       lxB);
                }
                const P gA = PK::add3(lxA, xlyA, lzxA);
                const P gB = PK::add3(lxB, xlyB, lzxB);
                *reinterpret_cast<uint4 *>(gp + xg * kGW + gc0) =
                    make_uint4(PK::lo(gA), PK::hi(gA), PK::lo(gB), PK::hi(gB));
            }
            // ---- the ring-column cell, one voxel
            {
                u32 gx = lzh;
#pragma unroll
                for (int d = -R; d <= R; ++d)
                    gx += ld1<T>(pg + hpr * G::ROWB, hpc + d) + ld1<T>(pg + (hpr + d) * G::ROWB, hpc);
                if (hv)
                    gp[(1 + hr) * kGW + 4 + hc] = gx;
            }
            __syncthreads();
            // plane s-1 (the oldest) is no longer read: refill its slot
            if (threadIdx.x == 0 && s >= 1 && s - 1 + G::NP < nplanes) {
                issue(s - 1 + G::NP);
                prefetch(s - 1 + G::NP + kL2Ahead);
            }

            // ---- C = T_x T_y G: T_y from the own rows and the neighbouring rows,
            // T_x across lanes (the edge lanes take the ring columns)
            const uint4 gn = *reinterpret_cast<const uint4 *>(gp + (gr0 - 1) * kGW + gc0);
            const uint4 gs = *reinterpret_cast<const uint4 *>(gp + (gr0 + kRows) * kGW + gc0);
            u32 eg[kRows + 2];
#pragma unroll
            for (int d = 0; d < kRows + 2; ++d)
                eg[d] = gp[(gr0 - 1 + d) * kGW + egc];
            const int zout = z0 - 2 + s;
            const bool emit = s >= 2;
            const unsigned char *pc = ring + ((s + R - 1) % G::NP) * G::PBYTES;   // plane z = g - 1
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                u32 ty_[4];
                if (i == 0) {
                    ty_[0] = gn.x + g[1][0];
                    ty_[1] = gn.y + g[1][1];
                    ty_[2] = gn.z + g[1][2];
                    ty_[3] = gn.w + g[1][3];
                } else if (i == kRows - 1) {
                    ty_[0] = g[i - 1][0] + gs.x;
                    ty_[1] = g[i - 1][1] + gs.y;
                    ty_[2] = g[i - 1][2] + gs.z;
                    ty_[3] = g[i - 1][3] + gs.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        ty_[k] = g[i - 1][k] + g[i + 1][k];
                }
                const u32 tye = eg[i] + eg[i + 2];
                u32 tl = __shfl_up_sync(0xFFFFFFFFu, ty_[3], 1);
                u32 tr = __shfl_down_sync(0xFFFFFFFFu, ty_[0], 1);
                if (lane == 0)
                    tl = tye;
                if (lane == 31)
                    tr = tye;
                u32 c[4];
                c[0] = tl + ty_[1];
                c[1] = ty_[0] + ty_[2];
                c[2] = ty_[1] + ty_[3];
                c[3] = ty_[2] + tr;
                if (emit) {
                    const int y = y0 + kRows * warp + i;
                    const int x = x0 + 4 * lane;
                    u32 q0, q1;
                    Ld<T>::quad(pc + (r0 + i) * G::ROWB, c0, q0, q1);
                    const u32 p0[4] = {q0 & 0xFFFFu, q0 >> 16, q1 & 0xFFFFu, q1 >> 16};
                    u32 f[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const u32 U = accA[i][k] + c[k];
                        f[k] = (p0[k] >= T_ && U >= KT) ? Div::template div_add<HALF>(U) : 0u;
                    }
                    if (MASK) {
                        // a region of interest or an odd width: masked stores, one voxel at a time
                        // (the tile starts at xs <= ox, so some lanes lie left of it)
                        const long long ob = ((long long)(zout - a.oz) * a.by + (y - a.oy)) * a.bx - a.ox;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int xk = x + k;
                            if (y >= a.yend || xk < a.ox || xk >= a.xend)
                                continue;
                            static_cast<T *>(a.out)[ob + xk] = (T)f[k];
                            if (hist) {
                                if (f[k] >= hlim) {
                                    if (f[k] < 65536u)   // always true for valid outputs
                                        atomicAdd(&a.out_hist[f[k]], 1ull);
                                } else {
                                    atomicAdd(&hist[min(f[k] - hbase, hzero)], 1u);
                                }
                            }
                        }
                    } else if (y < a.ny && x < a.nx) {
                        const size_t o = ((size_t)zout * a.ny + y) * a.nx + x;
                        if (sizeof(T) == 2) {
                            *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(a.out) + o) =
                                make_uint2(f[0] | (f[1] << 16), f[2] | (f[3] << 16));
                        } else {
                            *reinterpret_cast<u32 *>(static_cast<uint8_t *>(a.out) + o) =
                                f[0] | (f[1] << 8) | (f[2] << 16) | (f[3] << 24);
                        }
                        if (hist) {
                            // window bins for nonzero outputs (hbase >= 1), the
                            // lane's zero bin for zeros; values above the window
                            // (rare) go to the global histogram
                            if (hcheck && __any_sync(__activemask(), max(max(f[0], f[1]), max(f[2], f[3])) >= hlim)) {
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    if (f[k] >= hlim) {
                                        if (f[k] < 65536u)   // always true for valid outputs
                                            atomicAdd(&a.out_hist[f[k]], 1ull);
                                    } else {
                                        atomicAdd(&hist[min(f[k] - hbase, hzero)], 1u);
                                    }
                                }
                            } else {
                                // f - hbase wraps to a large value for a zero
#pragma unroll
                                for (int k = 0; k < 4; ++k)
                                    atomicAdd(&hist[min(f[k] - hbase, hzero)], 1u);
                            }
                        }
                    }
                }
                // advance the z accumulators: A <- B + G(g), B <- C(g)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    accA[i][k] = accB[i][k] + g[i][k];
                    accB[i][k] = c[k];
                }
            }
            // the next step's first barrier orders these G-plane reads before
            // that step's G-plane writes
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
        // all issued planes were waited for; re-arm the barriers for the next item
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

// Work-item z length (planes per item) when neither the autotuner nor the
// caller set one: the longest of 64, 32 and 16 planes that still gives every CTA
// of the persistent grid three items or more.  Longer items repeat fewer of the
// 2R + 2 warm-up planes of their z march; enough items keep the grid balanced
// (measured: 512^3 uint16 is fastest at 32, the 1024^3 uint8 volume at 64).
static int auto_zlen(int tiles, int depth, int grid)
{
    for (int zl : {64, 32})
        if ((long long)tiles * ((depth + zl - 1) / zl) >= 3ll * grid)
            return zl;
    return 16;
}

// MASK: masked per-voxel stores (a region of interest, an odd width), else dense
// 4-voxel vector stores
template <typename T, int R, bool MASK>
__global__ void __launch_bounds__(kThreads, 2) k_ours_fast(const __grid_constant__ CUtensorMap tmap, const FastArgs a)
{
    typedef FGeo<T, R> G;
    if (a.gated && lnf_gate_mode(*a.prm))
        return;   // few voxels pass the gate: the gate-first kernel does the work
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128 - (lnfdev::smem_u32(smem_raw) & 127)) & 127);
    __shared__ int s_item, s_abort;
    u32 *hist = reinterpret_cast<u32 *>(smem + G::RING + G::GPLANE);
    constexpr int bins = G::HWIN;
    for (int i = threadIdx.x; i < bins + 32; i += blockDim.x)
        hist[i] = 0;
    if (threadIdx.x == 0)
        s_abort = 0;
    __syncthreads();
    // a nonzero output passed the gate and averages voxels >= minv, so it is
    // >= max(T, minv); the window starts there (and at 1 at least, keeping the
    // zeros out of it)
    const u32 hbase = sizeof(T) == 1 ? 1u : max(1u, max(a.prm->T, a.prm->minv));
    const u32 M = 2 * R + 1;
    const bool narrow = 3u * M * a.prm->maxv <= 65535u;
    if (narrow)
        ours_items<T, R, Narrow, MASK>(a, &tmap, smem, &s_item, &s_abort, a.out_hist ? hist : nullptr,
                                 hbase);
    else
        ours_items<T, R, Wide, MASK>(a, &tmap, smem, &s_item, &s_abort, a.out_hist ? hist : nullptr,
                               hbase);
    if (a.out_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < bins; i += blockDim.x)
            if (hist[i])
                atomicAdd(&a.out_hist[hbase + i], (u64)hist[i]);
        if (threadIdx.x < 32) {   // the zero bins
            u32 z = hist[bins + threadIdx.x];
            for (int o = 16; o > 0; o >>= 1)
                z += __shfl_xor_sync(0xFFFFFFFFu, z, o);
            if (threadIdx.x == 0 && z)
                atomicAdd(&a.out_hist[0], (u64)z);
        }
    }
}

template <typename T, int R>
lnf_status launch(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st, u64 *out_hist, u32 *counter, int *handled,
                  int gated)
{
    typedef FGeo<T, R> G;
    // this kernel's own descriptor: box = its tile + halo
    CUtensorMap map;
    if (!lnf_encode_box(ctx, j.in, j.nx, j.ny, j.nz, j.pitch, j.dtype, G::PW, G::PH, &map))
        return LNF_OK;   // not handled: the generic kernel runs instead
    const CUtensorMap *tmap = &map;
    FastArgs a;
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
    a.prm = j.prm;
    a.out_hist = out_hist;
    a.counter = counter ? counter : ctx->d_counter + 8;
    a.err = ctx->d_err;
    a.gated = gated;
    void (*kern)(const CUtensorMap, const FastArgs) = a.roi ? k_ours_fast<T, R, true> : k_ours_fast<T, R, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast kernel: shared memory attribute");
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, G::SMEM);
    if (occ < 1)
        occ = 1;
    const int cap = ctx->num_sms * occ;
    a.zlen = ctx->fast_zlen > 0 ? ctx->fast_zlen : auto_zlen(a.tiles_x * a.tiles_y, j.bz, cap);
    a.zchunks = (j.bz + a.zlen - 1) / a.zlen;
    a.total_items = a.tiles_x * a.tiles_y * a.zchunks;
    const int grid = std::min(a.total_items, cap);
    if (cudaMemsetAsync(a.counter, 0, sizeof(u32), st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast kernel: counter reset");
    kern<<<grid, kThreads, G::SMEM, st>>>(*tmap, a);
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fast kernel launch failed");
    *handled = 1;
    return LNF_OK;
}

}  // namespace

bool lnf_sparse_covers(int filter, int radius)
{
    // sigma at r = 3..4: the tap kernel only while few voxels pass the gate (it
    // evaluates the listed voxels alone), the generic kernel beside it otherwise
    return filter == LNF_SIGMA && radius >= 3 && radius <= 4;
}

bool lnf_fast_covers(int filter, int radius, int offset)
{
    if (radius < 1 || radius > 4)
        return false;
    switch (filter) {
    case LNF_OURS: return offset == 1;
    case LNF_SIGMA: return radius <= 2;   // dense r = 3..4 (343, 729 taps per voxel): the generic kernel is
                                          // faster; sparse ones take the tap kernel (lnf_sparse_covers)
    case LNF_MEAN:
    case LNF_ENTROPY:
    case LNF_OKADA: return true;
    default: return false;
    }
}

lnf_status lnf_fast_dispatch(lnf_ctx *ctx, const FilterJob &job, const CUtensorMap *tmap, cudaStream_t stream,
                             int *handled, u32 *counter, int allow_gate, u32 *gate_counter, PitchedCopy *pre)
{
    *handled = 0;
    if (!tmap || job.aniso || !lnf_fast_covers(job.filter, job.radius, job.offset))
        return LNF_OK;
    // Whole volumes also get the gate-first kernels, which take the job when few
    // voxels pass the gate (decided on the device); the ring kernel then returns
    // at once.  A multi-filter call may have launched them for this filter
    // already.  A single comparison filter stays on its ring kernel: the
    // gate-first evaluation computes the four cube filters together, which for
    // one filter alone is slower.
    const bool in_multi = (ctx->gate_mask >> job.filter) & 1;
    const bool own_gate = allow_gate && !in_multi && !ctx->no_gate && job.filter == LNF_OURS &&
                          lnf_gate_covers(job, job.filter);
    lnf_status s = LNF_OK;
    // the gate-first kernels first: whether they could be launched decides whether
    // the ring kernel may leave the job to them
    int own = 0;
    if (own_gate) {
        static const char *names[5] = {"gate:mean", "gate:sigma", "gate:entropy", "gate:okada", "gate:ours"};
        void *outs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        u64 *hists[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        outs[job.filter] = job.out;
        hists[job.filter] = job.out_hist;
        const int rec = lnf_prof_begin(ctx, stream);   // the gate kernels alone (counted by the caller)
        s = lnf_gate_launch(ctx, job, outs, hists, stream, &own, gate_counter);
        lnf_prof_end(ctx, rec, names[job.filter], stream, 0);
        if (s != LNF_OK)
            return s;
    }
    const int gated = in_multi || own ? 1 : 0;
    if (pre) {
        s = lnf_copy_pitched(ctx, pre->dst, pre->prow, pre->src, pre->dims, pre->dtype, stream,
                             own ? pre->prm : nullptr);
        if (s != LNF_OK)
            return s;
        pre->done = true;
    }
    if (job.filter != LNF_OURS) {
        s = lnf_fast2_dispatch(ctx, job, tmap, stream, handled, counter, gated);
    } else {
        u64 *oh = job.out_hist;
        if (job.dtype == LNF_U8) {
            switch (job.radius) {
            case 1: s = launch<uint8_t, 1>(ctx, job, stream, oh, counter, handled, gated); break;
            case 2: s = launch<uint8_t, 2>(ctx, job, stream, oh, counter, handled, gated); break;
            case 3: s = launch<uint8_t, 3>(ctx, job, stream, oh, counter, handled, gated); break;
            default: s = launch<uint8_t, 4>(ctx, job, stream, oh, counter, handled, gated); break;
            }
        } else {
            switch (job.radius) {
            case 1: s = launch<uint16_t, 1>(ctx, job, stream, oh, counter, handled, gated); break;
            case 2: s = launch<uint16_t, 2>(ctx, job, stream, oh, counter, handled, gated); break;
            case 3: s = launch<uint16_t, 3>(ctx, job, stream, oh, counter, handled, gated); break;
            default: s = launch<uint16_t, 4>(ctx, job, stream, oh, counter, handled, gated); break;
            }
        }
    }
    if (s != LNF_OK)
        return s;
    // where the gate kernels may write this output, the ring kernel must be there
    // to take the dense case: no other kernel may write it
    if (gated && !*handled)
        return lnf_fail(ctx, LNF_ECUDA, "ring kernel not launchable beside the gate-first kernels");
    if (own)
        *handled = 3;   // the two gate kernels and the ring kernel
    return s;
}
