// The box kernels of fast2.cuh: mean (Eq. 4) and entropy filter (Eq. 7).
#include "fast2.cuh"

namespace {

// ------------------------------------------------------------------ box kernel body


// q(P): the voxel itself (mean) or its fixed-point weight w[P] (entropy filter),
// from the shared window of the weight table or, outside it, from global memory
template <typename T, int R, bool ENT>
struct BoxBody {
    const u32 *lut_sh;
    u32 lut_base;
    const u32 *lut_g;

    __device__ __forceinline__ u32 q(u32 v) const
    {
        if (!ENT)
            return v;
        const u32 o = v - lut_base;
        return o < (u32)(sizeof(T) == 1 ? 256 : kLutWin16) ? lut_sh[o] : __ldg(lut_g + v);
    }
};

template <typename T, int R, bool ENT, bool MASK>
__device__ void box_items(const Args2 &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item, int *s_abort,
                          Hist2 &hist, const u32 *lut_sh, u32 lut_base)
{
    using namespace lnfdev;
    typedef Geo2<T, R, kBoxPF> G;
    constexpr int SR = kTY + 2 * R;           // rows of the Sx plane: tile rows -R .. kTY-1+R
    unsigned char *ring = smem;
    u32 *sxp = reinterpret_cast<u32 *>(smem + G::RING);   // Sx plane, own columns at offsets 4 .. 4+kTX-1
    u64 *bars = reinterpret_cast<u64 *>(smem + G::RING + G::BZ);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = G::XH + 4 * lane;          // plane column of the lane's first voxel
    const int r0 = G::H + kRows * warp;       // plane row of the lane's first row
    const int sc0 = 4 + 4 * lane;             // its column offset in the Sx plane
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
    // the halo row of the Sx plane this warp also sums (R warps at each end)
    const bool xrow = warp < R || warp >= kWarps - R;
    const int xtr = warp < R ? -R + warp : kTY + warp - (kWarps - R);   // tile row
    const int xpr = G::H + xtr;                                       // plane row
    // the border columns beyond the tile (tile columns -R..-1 or kTX..kTX+R-1)
    // of one tile row, summed by one lane: warp w takes tile rows 5w-R .. 5w-R+4,
    // lane = 2 j + side; the other lanes shadow a valid cell (same addresses)
    const bool hv = lane < 10 && 5 * warp + (lane >> 1) < SR;
    const int htr = hv ? 5 * warp + (lane >> 1) - R : -R;
    const int hside = lane & 1;
    const int hpr = G::H + htr;
    const int hpc = hside ? G::XH + kTX : G::XH - R;                 // plane column of its first cell
    // edge lanes read the border prefix sums from their side of the Sx plane
    const int hpo = lane < 16 ? 0 : 4 + kTX;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::NP; ++s)
            mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Sx of one row of the lane's four voxels: the x box of width M over the
    // z line sums, neighbours from the adjacent lanes (nothing past the tile:
    // the edge lanes add the border part later)
    auto sx_row = [&](const u32 b[4], u32 out[4]) {
        u32 v[4 + 2 * R];   // v[j + R] = z line sum at own column j, j = -R .. 3+R
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            const u32 l = __shfl_up_sync(0xFFFFFFFFu, b[4 - m], 1);
            const u32 r = __shfl_down_sync(0xFFFFFFFFu, b[m - 1], 1);
            v[R - m] = lane == 0 ? 0u : l;
            v[3 + R + m] = lane == 31 ? 0u : r;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            v[R + k] = b[k];
        u32 acc = 0;
#pragma unroll
        for (int j = 0; j <= 2 * R; ++j)
            acc += v[j];
        out[0] = acc;
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            acc += v[k + 2 * R] - v[k - 1];
            out[k] = acc;
        }
    };

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
            if (lnf_dbg_tma(px0, (int)sizeof(T), ring + slot * G::PBYTES, a.err))
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
        u32 bz[kRows][4];   // z line sums of q(P): the lane's voxels
        u32 xz[4];          // ... of its halo row
        u32 hz[R];          // ... of its border cells
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
            // ---- z line sums: initialise, then one plane in and one out
            if (s == 0) {
#pragma unroll
                for (int i = 0; i < kRows; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        bz[i][k] = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    xz[k] = 0;
#pragma unroll
                for (int m = 0; m < R; ++m)
                    hz[m] = 0;
                for (int p = 0; p <= 2 * R; ++p) {
                    const unsigned char *pl = ring + (p % G::NP) * G::PBYTES;
#pragma unroll
                    for (int i = 0; i < kRows; ++i) {
                        u32 v[4];
                        ld4<T>(pl + (r0 + i) * G::ROWB, c0, v);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            bz[i][k] += B.q(v[k]);
                    }
                    if (xrow) {
                        u32 v[4];
                        ld4<T>(pl + xpr * G::ROWB, c0, v);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            xz[k] += B.q(v[k]);
                    }
#pragma unroll
                    for (int m = 0; m < R; ++m)
                        hz[m] += B.q(ld1<T>(pl + hpr * G::ROWB, hpc + m));
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
                        bz[i][k] += B.q(vn[k]) - B.q(vo[k]);
                }
                if (xrow) {
                    u32 vn[4], vo[4];
                    ld4<T>(pn + xpr * G::ROWB, c0, vn);
                    ld4<T>(po + xpr * G::ROWB, c0, vo);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        xz[k] += B.q(vn[k]) - B.q(vo[k]);
                }
#pragma unroll
                for (int m = 0; m < R; ++m)
                    hz[m] += B.q(ld1<T>(pn + hpr * G::ROWB, hpc + m)) - B.q(ld1<T>(po + hpr * G::ROWB, hpc + m));
            }
            // ---- Sx rows (own, halo) to the Sx plane; border prefix sums to its spare columns
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                u32 o[4];
                sx_row(bz[i], o);
                *reinterpret_cast<uint4 *>(sxp + (kRows * warp + i + R) * G::BW + sc0) = make_uint4(o[0], o[1], o[2], o[3]);
            }
            if (xrow) {
                u32 o[4];
                sx_row(xz, o);
                *reinterpret_cast<uint4 *>(sxp + (xtr + R) * G::BW + sc0) = make_uint4(o[0], o[1], o[2], o[3]);
            }
            if (hv) {
                // left: part of Sx(c) beyond the tile = sum of cells m >= c (c = 0 .. R-1)
                // right: part of Sx(kTX-1-j) beyond the tile = sum of cells m <= R-1-j
                u32 *row = sxp + (htr + R) * G::BW;
                u32 run = 0;
                if (hside == 0) {
#pragma unroll
                    for (int c = R - 1; c >= 0; --c) {
                        run += hz[c];
                        row[c] = run;
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < R; ++m) {
                        run += hz[m];
                        row[4 + kTX + (R - 1 - m)] = run;
                    }
                }
            }
            __syncthreads();
            // plane s-1 was last read by the z line sums above: refill its slot
            if (threadIdx.x == 0 && s >= 1 && s - 1 + G::NP < nplanes) {
                issue(s - 1 + G::NP);
                prefetch(s - 1 + G::NP + kL2Ahead);
            }
            // ---- y box of Sx over the lane's rows (and of the border sums for the edge lanes)
            u32 box[kRows][4], hy[kRows][4];
            {
                u32 w[kRows + 2 * R][4], e[kRows + 2 * R][4];
#pragma unroll
                for (int rr = 0; rr < kRows + 2 * R; ++rr) {   // Sx rows of tile rows 4w-R .. 4w+3+R
                    const u32 *row = sxp + (kRows * warp + rr) * G::BW;
                    const uint4 q4 = *reinterpret_cast<const uint4 *>(row + sc0);
                    const uint4 h4 = *reinterpret_cast<const uint4 *>(row + hpo);
                    w[rr][0] = q4.x;
                    w[rr][1] = q4.y;
                    w[rr][2] = q4.z;
                    w[rr][3] = q4.w;
                    e[rr][0] = h4.x;
                    e[rr][1] = h4.y;
                    e[rr][2] = h4.z;
                    e[rr][3] = h4.w;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    u32 acc = 0, acch = 0;
#pragma unroll
                    for (int rr = 0; rr <= 2 * R; ++rr) {
                        acc += w[rr][k];
                        acch += e[rr][k];
                    }
                    box[0][k] = acc;
                    hy[0][k] = acch;
#pragma unroll
                    for (int i = 1; i < kRows; ++i) {
                        acc += w[i + 2 * R][k] - w[i - 1][k];
                        acch += e[i + 2 * R][k] - e[i - 1][k];
                        box[i][k] = acc;
                        hy[i][k] = acch;
                    }
                }
            }
            // the edge lanes add the part of the box beyond the tile
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k < R && lane == 0)
                        box[i][k] += hy[i][k];
                    if (3 - k < R && lane == 31)   // own column 124 + k = kTX - 1 - (3 - k)
                        box[i][k] += hy[i][3 - k];
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
            // the next step's first barrier orders these Sx-plane reads before
            // that step's Sx-plane writes
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

}  // namespace

lnf_status lnf_fast2_box(lnf_ctx *ctx, const FilterJob &job, cudaStream_t stream, u32 *counter, int *handled,
                         int gated)
{
    const bool u8 = job.dtype == LNF_U8;
    if (job.filter == LNF_MEAN)
        return u8 ? by_radius<uint8_t, LNF_MEAN>(ctx, job, stream, counter, handled, gated)
                  : by_radius<uint16_t, LNF_MEAN>(ctx, job, stream, counter, handled, gated);
    return u8 ? by_radius<uint8_t, LNF_ENTROPY>(ctx, job, stream, counter, handled, gated)
              : by_radius<uint16_t, LNF_ENTROPY>(ctx, job, stream, counter, handled, gated);
}
