// The four cube filters of a multi-filter call in one pass: mean (Eq. 4),
// sigma (Eq. 5), entropy filter (Eq. 7) and Okada (Eq. 6) at radius 1..2 all
// read the M^3 cube around a voxel (Okada its axis cross, a subset), and all
// output 0 unless the voxel's own value P0 >= T.  While few voxels pass that
// gate (lnf_fused_mode), this kernel streams the volume once through the plane
// ring of the tap kernels (fast2.cuh), writes zeros for every voxel of the four
// outputs, lists each block step's passing voxels in shared memory and
// evaluates them with one warp each: every lane loads a few taps of the cube
// once and accumulates all four filters from them (box sum, sigma band, Okada
// band on the cross taps, entropy weights), then a butterfly sum per filter;
// lane 0 writes the four outputs over the zeros (a block barrier orders the two
// writes) and counts the nonzero ones into the global histograms.  A step with
// more passing voxels than the list holds is evaluated in rounds.
#include "fast2.cuh"

namespace {

constexpr int kFCap = 1024;          // listed voxels per round
constexpr int kFLut = 4096;          // entropy weights kept in shared memory (from the minimum level)

struct FusedArgs {
    const void *in;
    void *out[4];                    // mean, sigma, entropy filter, Okada
    u64 *hist[4];                    // their output histograms (null: not wanted)
    int nx, ny, nz;
    int tiles_x, tiles_y, zlen, total_items;
    const DevParams *prm;
    const u32 *lut;
    u32 *counter;
    u32 *err;
};

template <int R>
struct FTaps {
    static constexpr int M = 2 * R + 1;
    static constexpr int TAPS = M * M * M;
    static constexpr int PER_LANE = (TAPS + 31) / 32;
};

template <typename T, int R>
struct FSmem {
    typedef Geo2<T, R> G;
    static constexpr int BARS = ((G::NP * 8 + 15) / 16) * 16;
    static constexpr int LUTB = kFLut * 4;
    static constexpr int RECB = ((FTaps<R>::TAPS + 1) * 4 + 15) / 16 * 16;
    static constexpr int LSTB = kFCap * 2;
    static constexpr int TOTAL = 128 + G::RING + BARS + LUTB + RECB + LSTB + 64;
};

template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2) k_fused4(const __grid_constant__ CUtensorMap tmap, const FusedArgs a)
{
    using namespace lnfdev;
    typedef Geo2<T, R> G;
    typedef FSmem<T, R> S;
    typedef FTaps<R> F;
    const DevParams &P = *a.prm;
    if (!lnf_fused_mode(P))
        return;   // the four ring kernels do the work
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    __shared__ int s_item, s_abort;
    unsigned char *ring = smem;
    u64 *bars = reinterpret_cast<u64 *>(smem + G::RING);
    u32 *lut_sh = reinterpret_cast<u32 *>(smem + G::RING + S::BARS);
    u32 *recip = reinterpret_cast<u32 *>(smem + G::RING + S::BARS + S::LUTB);
    uint16_t *lst = reinterpret_cast<uint16_t *>(smem + G::RING + S::BARS + S::LUTB + S::RECB);
    u32 *s_wt = reinterpret_cast<u32 *>(smem + G::RING + S::BARS + S::LUTB + S::RECB + S::LSTB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = G::XH + 4 * lane;
    const int r0 = G::H + kRows * warp;
    const u32 T_ = P.T;
    const u32 lbase = sizeof(T) == 1 ? 0u : P.minv;
    for (int i = threadIdx.x; i < kFLut; i += blockDim.x)
        lut_sh[i] = (lbase + i < (sizeof(T) == 1 ? 256u : 65536u)) ? a.lut[lbase + i] : 0u;
    for (int n = threadIdx.x; n <= F::TAPS; n += blockDim.x)
        recip[n] = n <= 1 ? 0u : (u32)((0x100000000ull + n - 1) / n);
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int sl = 0; sl < G::NP; ++sl)
            mbar_init(&bars[sl], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // the filters' parameters: the sigma band |v - P0| <= delta, the Okada band
    // |P0 - v| < td (nothing when td <= 0), the entropy threshold (default: the
    // expected criterion of a cube of M^3 voxels)
    const u32 dl = min(P.delta, 65535u);
    const long long td = P.td;
    const u32 th = td > 65536 ? 65535u : (td > 0 ? (u32)(td - 1) : 0u);
    long long te = P.te_cfg;
    if (te == -2)
        te = (long long)(((unsigned __int128)F::TAPS * P.hw_sum) / P.N);
    constexpr u32 M3 = (u32)F::TAPS;
    // this lane's taps t = lane + 32 j of the cube: plane index (0 .. 2R), in-plane
    // byte offset, and whether the tap lies on the Okada cross
    int tdz[F::PER_LANE], tin[F::PER_LANE];
    bool tcross[F::PER_LANE];
#pragma unroll
    for (int j = 0; j < F::PER_LANE; ++j) {
        const int t = lane + 32 * j < F::TAPS ? lane + 32 * j : 0;
        const int dx = t % F::M - R, dy = (t / F::M) % F::M - R, dz = t / (F::M * F::M) - R;
        tdz[j] = dz + R;
        tin[j] = dy * G::ROWB + dx * (int)sizeof(T);
        tcross[j] = (dx == 0 && dy == 0) || (dx == 0 && dz == 0) || (dy == 0 && dz == 0);
    }
    u32 written = 0, nz[4] = {0u, 0u, 0u, 0u};

    for (;;) {
        if (threadIdx.x == 0)
            s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.total_items || s_abort)
            break;
        const int tx = item % a.tiles_x;
        const int rest = item / a.tiles_x;
        const int ty = rest % a.tiles_y;
        const int zc = rest / a.tiles_y;
        const int x0 = tx * kTX, y0 = ty * kTY;
        const int z0 = zc * a.zlen, z1 = min(a.nz, z0 + a.zlen);
        const int px0 = x0 - G::XH, py0 = y0 - G::H;
        const bool border = px0 < 0 || px0 + G::PW > a.nx || py0 < 0 || py0 + G::PH > a.ny;
        const int nplanes = (z1 - z0) + 2 * R;
        const u32 pbytes = G::PW * G::PH * sizeof(T);
        auto issue = [&](int p) {
            const int slot = p % G::NP;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[slot], pbytes);
            tma_load_3d(ring + slot * G::PBYTES, &tmap, &bars[slot], px0, py0, clampi(z0 - R + p, 0, a.nz - 1));
        };
        auto prefetch = [&](int p) {
            if (p < nplanes)
                tma_prefetch_3d(&tmap, max(px0, 0), max(py0, 0), clampi(z0 - R + p, 0, a.nz - 1));
        };
        if (threadIdx.x == 0) {
            for (int p = 0; p < min(G::NP, nplanes); ++p)
                issue(p);
            for (int p = G::NP; p < G::NP + kL2Ahead; ++p)
                prefetch(p);
        }
        bool ok = true;
        for (int s = 0; s < z1 - z0; ++s) {
            const int pfirst = s == 0 ? 0 : s + 2 * R;
            if (threadIdx.x == 0)
                for (int p = pfirst; p <= s + 2 * R; ++p)
                    if (!mbar_wait_bounded(&bars[p % G::NP], (u32)((p / G::NP) & 1), a.err))
                        s_abort = 1;
            __syncthreads();
            if (s_abort) {
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
            const int z = z0 + s;
            // zeros for the lane's voxels in every output; its passing voxels listed
            u32 cm = 0;
            const int x = x0 + 4 * lane;
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                const int y = y0 + kRows * warp + i;
                if (y >= a.ny || x >= a.nx)
                    continue;
                u32 p0[4];
                ld4<T>(pc + (r0 + i) * G::ROWB, c0, p0);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (p0[k] >= T_)
                        cm |= 1u << (4 * i + k);
                const size_t o = ((size_t)z * a.ny + y) * a.nx + x;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    if (sizeof(T) == 2)
                        *reinterpret_cast<uint2 *>(static_cast<uint16_t *>(a.out[f]) + o) = make_uint2(0u, 0u);
                    else
                        *reinterpret_cast<u32 *>(static_cast<uint8_t *>(a.out[f]) + o) = 0u;
                }
                written += 4;
            }
            const u32 cnt = (u32)__popc(cm);
            u32 incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o)
                    incl += t;
            }
            if (lane == 31)
                s_wt[warp] = incl;
            __syncthreads();
            u32 wbase = 0, ctot = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const u32 v = s_wt[w];
                wbase += w < warp ? v : 0u;
                ctot += v;
            }
            if (ctot == 0)
                continue;   // uniform: nothing passes in this block step
            // the byte offsets of the ring slots of planes z - R .. z + R from plane z,
            // and this lane's taps from a voxel's cell
            int poff[2 * R + 1];
#pragma unroll
            for (int d = 0; d <= 2 * R; ++d)
                poff[d] = (int)(ring - pc) + ((s + d) % G::NP) * G::PBYTES;
            int toff[F::PER_LANE];
#pragma unroll
            for (int j = 0; j < F::PER_LANE; ++j) {
                int sel = poff[0];
#pragma unroll
                for (int d = 1; d <= 2 * R; ++d)
                    sel = tdz[j] == d ? poff[d] : sel;
                toff[j] = sel + tin[j];
            }
            for (u32 r0c = 0; r0c < ctot; r0c += kFCap) {   // rounds of at most kFCap voxels
                {
                    u32 m = cm, pos = wbase + incl - cnt;
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        if (pos >= r0c && pos < r0c + kFCap)
                            lst[pos - r0c] =
                                (uint16_t)((r0 + (b >> 2)) * G::ROWB + (c0 + (b & 3)) * (int)sizeof(T));
                        ++pos;
                    }
                }
                __syncthreads();   // the list is complete, and every zero is written
                const u32 nc = min((u32)kFCap, ctot - r0c);
                for (u32 c = warp; c < nc; c += kWarps) {
                    const int cell = lst[c];
                    const u32 P0 = sizeof(T) == 2 ? (u32)*reinterpret_cast<const uint16_t *>(pc + cell) : (u32)pc[cell];
                    const u32 slo = P0 > dl ? P0 - dl : 0u, swd = P0 - slo + dl;
                    const u32 olo = P0 > th ? P0 - th : 0u, owd = P0 - olo + th;
                    u32 B = 0, Sg = 0, Ok = 0, E = 0;
#pragma unroll
                    for (int j = 0; j < F::PER_LANE; ++j) {
                        if (lane + 32 * j >= F::TAPS)
                            continue;
                        const unsigned char *q = pc + cell + toff[j];
                        const u32 v = sizeof(T) == 2 ? (u32)*reinterpret_cast<const uint16_t *>(q) : (u32)*q;
                        B += v;
                        if (v - slo <= swd)
                            Sg += (v << 8) | 1u;   // value and count (count < 256)
                        if (tcross[j] && v - olo <= owd)
                            Ok += (v << 8) | 1u;
                        const u32 lo = v - lbase;
                        E += lo < (u32)kFLut ? lut_sh[lo] : __ldg(a.lut + v);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        B += __shfl_xor_sync(0xFFFFFFFFu, B, o);
                        Sg += __shfl_xor_sync(0xFFFFFFFFu, Sg, o);
                        Ok += __shfl_xor_sync(0xFFFFFFFFu, Ok, o);
                        E += __shfl_xor_sync(0xFFFFFFFFu, E, o);
                    }
                    if (lane == 0) {
                        // outputs (P0 >= T holds for every listed voxel): round half up
                        // of each mean; the sigma and Okada means by the reciprocal
                        // table (exact: x < n 2^16, recip n - 2^32 < n, n < 256)
                        const u32 fm = B >= M3 * T_ ? (2u * B + M3) / (2u * M3) : 0u;
                        u32 fs, fo;
                        {
                            const u32 n = Sg & 0xFFu, sm = Sg >> 8;
                            const u32 q = n == 1 ? sm : __umulhi(sm + (n >> 1), recip[n]);
                            fs = (n && (u64)sm >= (u64)n * T_) ? q : 0u;
                        }
                        {
                            const u32 n = Ok & 0xFFu, sm = Ok >> 8;
                            const u32 q = n == 1 ? sm : __umulhi(sm + (n >> 1), recip[n]);
                            fo = (td > 0 && n && (u64)sm >= (u64)n * T_) ? q : 0u;
                        }
                        const u32 fe = (long long)E > te ? P0 : 0u;
                        const int row = cell / G::ROWB;
                        const int col = (cell - row * G::ROWB) / (int)sizeof(T);
                        const size_t o = ((size_t)z * a.ny + (py0 + row)) * a.nx + (px0 + col);
                        const u32 fv[4] = {fm, fs, fe, fo};
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            static_cast<T *>(a.out[f])[o] = (T)fv[f];
                            if (fv[f] && a.hist[f]) {
                                ++nz[f];
                                atomicAdd(&a.hist[f][fv[f]], 1ull);
                            }
                        }
                    }
                }
                if (r0c + kFCap < ctot)
                    __syncthreads();   // the next round rewrites the list
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
    // zeros of each output: the voxels written minus the nonzero ones
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!a.hist[f])
            continue;
        u32 zeros = written - nz[f];
        for (int o = 16; o > 0; o >>= 1)
            zeros += __shfl_xor_sync(0xFFFFFFFFu, zeros, o);
        if (lane == 0 && zeros)
            atomicAdd(&a.hist[f][0], (u64)zeros);
    }
}

template <typename T, int R>
lnf_status launch_fused(lnf_ctx *ctx, const FilterJob &j, void *const outs[4], u64 *const hists[4], cudaStream_t st,
                        int *handled)
{
    typedef FSmem<T, R> S;
    typedef typename S::G G;
    CUtensorMap map;
    if (!lnf_encode_box(ctx, j.in, j.nx, j.ny, j.nz, j.pitch, j.dtype, G::PW, G::PH, &map))
        return LNF_OK;
    FusedArgs a;
    std::memset(&a, 0, sizeof a);
    a.in = j.in;
    for (int f = 0; f < 4; ++f) {
        a.out[f] = outs[f];
        a.hist[f] = hists[f];
    }
    a.nx = j.nx;
    a.ny = j.ny;
    a.nz = j.nz;
    a.tiles_x = (j.nx + kTX - 1) / kTX;
    a.tiles_y = (j.ny + kTY - 1) / kTY;
    a.zlen = std::max(1, (ctx->fast_zlen > 0 ? ctx->fast_zlen : 16) / 4);
    a.total_items = a.tiles_x * a.tiles_y * ((j.nz + a.zlen - 1) / a.zlen);
    a.prm = j.prm;
    a.lut = j.lut;
    a.counter = ctx->d_counter + 14;
    a.err = ctx->d_err;
    if (cudaFuncSetAttribute(k_fused4<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::TOTAL) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fused kernel: shared memory attribute (%d bytes)", S::TOTAL);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused4<T, R>, kThreads, S::TOTAL);
    if (occ < 1)
        occ = 1;
    const int grid = std::min(a.total_items, ctx->num_sms * occ);
    if (cudaMemsetAsync(a.counter, 0, sizeof(u32), st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fused kernel: counter reset");
    k_fused4<T, R><<<grid, kThreads, S::TOTAL, st>>>(map, a);
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "fused kernel launch failed");
    *handled = 1;
    return LNF_OK;
}

}  // namespace

// Launch the fused kernel for a whole-volume job whose input TMA can read, at
// radius 1..2, with dense-row outputs a 4-voxel vector store can write; outs /
// hists in the order mean, sigma, entropy filter, Okada.  *handled = 1 if launched.
lnf_status lnf_fused_launch(lnf_ctx *ctx, const FilterJob &j, void *const outs[4], u64 *const hists[4],
                            cudaStream_t st, int *handled)
{
    *handled = 0;
    if (j.aniso || j.radius < 1 || j.radius > 2 || j.pitch != j.nx || j.nx % 4 != 0)
        return LNF_OK;
    const size_t es = j.dtype == LNF_U8 ? 1 : 2;
    for (int f = 0; f < 4; ++f)
        if (!outs[f] || reinterpret_cast<uintptr_t>(outs[f]) % (4 * es) != 0)
            return LNF_OK;
    if (j.dtype == LNF_U8)
        return j.radius == 1 ? launch_fused<uint8_t, 1>(ctx, j, outs, hists, st, handled)
                             : launch_fused<uint8_t, 2>(ctx, j, outs, hists, st, handled);
    return j.radius == 1 ? launch_fused<uint16_t, 1>(ctx, j, outs, hists, st, handled)
                         : launch_fused<uint16_t, 2>(ctx, j, outs, hists, st, handled);
}
