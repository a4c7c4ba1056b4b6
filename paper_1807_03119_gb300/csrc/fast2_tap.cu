// The tap kernels of fast2.cuh: sigma (Eq. 5) and Okada (Eq. 6); and the
// dispatch of the four comparison filters to the specialised kernels.
#include "fast2.cuh"

namespace {

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

// four voxels at columns col..col+3 of a shared row as packed tap words
// (v << CS) | 1; for CS = 8 one byte permute per voxel builds the word from the
// loaded bytes directly
template <typename T, int CS>
__device__ __forceinline__ void ld4p(const unsigned char *row, int col, u32 pv[4])
{
    if (CS == 8 && sizeof(T) == 2) {
        const uint2 w = *reinterpret_cast<const uint2 *>(row + col * 2);
        pv[0] = __byte_perm(w.x, 1u, 0x5104);   // bytes: 1, v.lo, v.hi, 0
        pv[1] = __byte_perm(w.x, 1u, 0x5324);
        pv[2] = __byte_perm(w.y, 1u, 0x5104);
        pv[3] = __byte_perm(w.y, 1u, 0x5324);
    } else if (CS == 8) {
        const u32 w = *reinterpret_cast<const u32 *>(row + col);
        pv[0] = __byte_perm(w, 1u, 0x5504);     // bytes: 1, v, 0, 0
        pv[1] = __byte_perm(w, 1u, 0x5514);
        pv[2] = __byte_perm(w, 1u, 0x5524);
        pv[3] = __byte_perm(w, 1u, 0x5534);
    } else {
        u32 v[4];
        ld4<T>(row, col, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            pv[k] = (v[k] << CS) | 1u;
    }
}

template <typename T, int R, int FILTER, bool MASK>
__device__ void tap_items(const Args2 &a, const CUtensorMap *tmap, unsigned char *smem, int *s_item, int *s_abort,
                          Hist2 &hist, const u32 *recip, uint16_t *wl)
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
    // sigma, a warp per listed voxel: lane's taps t = lane + 32 j of the M^3 cube,
    // as a plane index (0 .. 2R, plane z - R + index) and an in-plane byte offset
    constexpr int TPL = (FILTER == LNF_SIGMA && TapCoop<R, FILTER>::TAPS > 32) ? TapCoop<R, FILTER>::PER_LANE : 1;
    int tdz[TPL], tin[TPL];
#pragma unroll
    for (int j = 0; j < TPL; ++j) {
        constexpr int M = 2 * R + 1;
        const int t = lane + 32 * j < TapCoop<R, FILTER>::TAPS ? lane + 32 * j : 0;
        tdz[j] = t / (M * M);
        tin[j] = ((t / M) % M - R) * G::ROWB + (t % M - R) * (int)sizeof(T);
    }

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
            u32 p0[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
                ld4<T>(pc + (r0 + i) * G::ROWB, c0, p0[i]);
            // the band of a centre value as (v - lo) <= width: sigma [P0 - delta, P0 + delta],
            // Okada |P0 - v| < td (td >= 1)
            auto band = [&](u32 c, u32 &blo, u32 &bwd) {
                const u32 h = FILTER == LNF_SIGMA ? dl : (td > 65536 ? 65535u : (u32)(td - 1));
                blo = c > h ? c - h : 0u;
                bwd = c - blo + h;
            };
            // round(sm / n) half up = floor((sm + floor(n/2)) / n) = (x * recip[n]) >> 32
            // with recip[n] = ceil(2^32 / n): exact when x e < 2^32 (e = recip n - 2^32 < n);
            // x < n 2^16 gives x e < n^2 2^16, so counts below 256 use the table
            // and larger ones (sigma at radius >= 3) divide; then the gate
            auto finish = [&](u32 sm, u32 n, u32 P0) -> u32 {
                const u32 x = sm + (n >> 1);
                constexpr bool SMALL = TapCoop<R, FILTER>::TAPS < 256;   // every count has a table entry
                const u32 q = n == 1 ? sm : ((SMALL || n < 256) ? __umulhi(x, recip[n]) : x / n);
                return (n && P0 >= T_ && (u64)sm >= (u64)n * T_) ? q : 0u;
            };
            u32 fo[kRows][4];   // this step's outputs
            // Gate first: a voxel with P0 < T is 0 whatever its band, so only the
            // voxels with P0 >= T need their taps.  The block lists this step's
            // such voxels in shared memory and all eight warps share them out (the
            // per-step barrier would otherwise hold every warp to the slowest one):
            // with more taps than lanes a whole warp evaluates one voxel (each lane
            // a few taps, a butterfly sum of the packed value and count), else one
            // thread evaluates one voxel.  Beyond TapCoop::CAP voxels every warp
            // takes the dense form below, which tests every tap of all 16 voxels of
            // every lane.  (Okada at r >= 3, whose 6r + 1 taps per voxel are cheap,
            // keeps the dense form: the listed one would cost it registers.)
            typedef TapCoop<R, FILTER> TC;
            constexpr bool COOP = FILTER == LNF_SIGMA || R <= 2;
            u32 cm = 0, cnt = 0, incl = 0, wbase = 0, ctot = 0xFFFFFFFFu;
            uint16_t *wdst = wl + TC::CAP;                                   // destinations
            u32 *s_wt = reinterpret_cast<u32 *>(wl + 2 * TC::CAP);          // the warps' counts
            uint16_t *wres = wl + 2 * TC::CAP + 32;                         // outputs, 16 per lane
            if constexpr (COOP) {
#pragma unroll
                for (int i = 0; i < kRows; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (p0[i][k] >= T_)
                            cm |= 1u << (4 * i + k);
                if (FILTER == LNF_OKADA && td <= 0)
                    cm = 0;   // Okada selects nothing: every output is 0
                cnt = (u32)__popc(cm);
                incl = cnt;   // inclusive prefix of the lanes' counts
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o)
                        incl += t;
                }
                if (lane == 31)
                    s_wt[warp] = incl;
                __syncthreads();
                ctot = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    const u32 v = s_wt[w];
                    wbase += w < warp ? v : 0u;
                    ctot += v;
                }
            }
            if (COOP && ctot <= (u32)TC::CAP) {
#pragma unroll
                for (int i = 0; i < kRows; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        fo[i][k] = 0u;
                {
                    u32 m = cm, pos = wbase + incl - cnt;
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        // the voxel's byte offset in a plane (< 2^16: a plane is smaller),
                        // and where its output goes
                        wl[pos] = (uint16_t)((r0 + (b >> 2)) * G::ROWB + (c0 + (b & 3)) * (int)sizeof(T));
                        wdst[pos] = (uint16_t)((warp * 32 + lane) * 16 + b);
                        ++pos;
                    }
                }
                __syncthreads();
                static_assert(G::PBYTES <= 65536, "a plane's byte offsets fit the 16-bit list entries");
                auto cell_of = [](u32 e) { return (int)e; };
                auto val = [&](const unsigned char *q) {
                    return sizeof(T) == 2 ? (u32)*reinterpret_cast<const uint16_t *>(q) : (u32)*q;
                };
                // the byte offsets of the ring slots of planes z - R .. z + R from plane z
                int poff[2 * R + 1];
#pragma unroll
                for (int d = 0; d <= 2 * R; ++d)
                    poff[d] = (int)(ring - pc) + ((s + d) % G::NP) * G::PBYTES;
                // the byte offset of tap t from the centre's cell in plane z
                auto tap_off = [&](int t) {
                    int dx = 0, dy = 0, dz = 0;
                    if (FILTER == LNF_SIGMA) {
                        constexpr int M = 2 * R + 1;
                        dz = t / (M * M) - R;
                        dy = (t / M) % M - R;
                        dx = t % M - R;
                    } else if (t > 0) {   // tap 0 is the centre; then the arms
                        const int arm = (t - 1) % 6, d = (t - 1) / 6 + 1;
                        const int sg = (arm & 1) ? d : -d;
                        dx = arm < 2 ? sg : 0;
                        dy = arm == 2 || arm == 3 ? sg : 0;
                        dz = arm >= 4 ? sg : 0;
                    }
                    return poff[dz + R] + dy * G::ROWB + dx * (int)sizeof(T);
                };
                if (TC::TAPS > 32) {   // a warp per voxel
                    if (ctot > (u32)warp) {
                        // this lane's taps: the in-plane part of the offset is fixed, the
                        // plane's slot is picked from this step's (no division per tap)
                        int toff[TC::PER_LANE];
#pragma unroll
                        for (int j = 0; j < TC::PER_LANE; ++j) {
                            int sel = poff[0];
#pragma unroll
                            for (int d = 1; d <= 2 * R; ++d)
                                sel = tdz[j] == d ? poff[d] : sel;
                            toff[j] = sel + tin[j];
                        }
                        for (u32 c = warp; c < ctot; c += kWarps) {
                            const int cell = cell_of(wl[c]);
                            const u32 P0 = val(pc + cell);
                            u32 blo, bwd;
                            band(P0, blo, bwd);
                            u32 acc = 0, nn = 0;   // packed (value << CS) + count, or value and count
#pragma unroll
                            for (int j = 0; j < TC::PER_LANE; ++j) {
                                if (lane + 32 * j >= TC::TAPS)
                                    continue;
                                const u32 v = val(pc + cell + toff[j]);
                                if (v - blo <= bwd) {
                                    if (TP::PACK) {
                                        acc += (v << TP::CS) | 1u;
                                    } else {
                                        acc += v;
                                        ++nn;
                                    }
                                }
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                                if (!TP::PACK)
                                    nn += __shfl_xor_sync(0xFFFFFFFFu, nn, o);
                            }
                            const u32 n = TP::PACK ? (acc & ((1u << TP::CS) - 1u)) : nn;
                            const u32 sm = TP::PACK ? (acc >> TP::CS) : acc;
                            if (lane == 0)
                                wres[wdst[c]] = (uint16_t)finish(sm, n, P0);
                        }
                    }
                } else {               // a thread per voxel, dealt round the warps
                    for (u32 c = warp + kWarps * lane; c < ctot; c += kThreads) {
                        const int cell = cell_of(wl[c]);
                        const u32 P0 = val(pc + cell);
                        u32 blo, bwd;
                        band(P0, blo, bwd);
                        u32 sm = 0, n = 0;
#pragma unroll
                        for (int t = 0; t < TC::TAPS; ++t) {
                            const u32 v = val(pc + cell + tap_off(t));
                            if (v - blo <= bwd) {
                                sm += v;
                                ++n;
                            }
                        }
                        wres[wdst[c]] = (uint16_t)finish(sm, n, P0);
                    }
                }
                __syncthreads();
                if (cm) {   // this lane's 16 outputs, two 16-byte loads; listed voxels only
                    const uint4 *rp = reinterpret_cast<const uint4 *>(wres + (warp * 32 + lane) * 16);
                    const uint4 q0 = rp[0], q1 = rp[1];
                    const u32 w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                    for (int i = 0; i < kRows; ++i)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int b = 4 * i + k;
                            const u32 f = (w[b >> 1] >> (16 * (b & 1))) & 0xFFFFu;
                            fo[i][k] = (cm >> b) & 1u ? f : 0u;
                        }
                }
            } else {
            u32 lo[kRows][4], wd[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    band(p0[i][k], lo[i][k], wd[i][k]);
            u32 acc[kRows][4], cnt[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[i][k] = 0;
                    cnt[i][k] = 0;
                }
            // per tap and voxel: d = pv - (lo << CS) (multiply-add: FMA pipe), in-band
            // test (compare: ALU pipe), accumulate (alternately FMA and ALU pipe), so
            // that the integer work is split between the two half-rate pipes.  On the
            // packed word pv = (v << CS) | 1 the band test v - lo <= wd reads
            // pv - (lo << CS) <= (wd << CS) + 1: for v >= lo both sides are the
            // shifted difference plus 1, and for v < lo the left side wraps above
            // 2^32 - 65535 * 2^CS, beyond any right side
            const u32 one = a.one;
            u32 nlo[kRows][4], wdp[kRows][4];
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    nlo[i][k] = TP::PACK ? 0u - (lo[i][k] << TP::CS) : 0u - lo[i][k];
                    wdp[i][k] = TP::PACK ? (wd[i][k] << TP::CS) + 1u : wd[i][k];
                }
            auto take = [&](int i, int k, u32 v, u32 pv) {
                if (TP::PACK) {
                    // d = pv - (lo << CS): a plain add (ALU) for even voxels, a
                    // multiply-add by the runtime 1 (FMA pipe) for odd ones; the
                    // in-band test is a compare (ALU) and the accumulate a predicated
                    // multiply-add (FMA)
                    u32 d;
                    if (k & 1)
                        asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(pv), "r"(one), "r"(nlo[i][k]));
                    else
                        d = pv + nlo[i][k];
                    asm(
                        "{\n\t.reg .pred p;\n\tsetp.le.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %4, %0;\n\t}"
                        : "+r"(acc[i][k])
                        : "r"(d), "r"(wdp[i][k]), "r"(pv), "r"(one));
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
                        if (TP::PACK) {   // the packed words only (the band test reads them)
                            ld4p<T, TP::CS>(row, c0 - 4, pv);
                            ld4p<T, TP::CS>(row, c0, pv + 4);
                            ld4p<T, TP::CS>(row, c0 + 4, pv + 8);
#pragma unroll
                            for (int e = 0; e < 12; ++e)
                                v[e] = pv[e];
                        } else {
                            ld4<T>(row, c0 - 4, v);
                            ld4<T>(row, c0, v + 4);
                            ld4<T>(row, c0 + 4, v + 8);
#pragma unroll
                            for (int e = 0; e < 12; ++e)
                                pv[e] = v[e];
                        }
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
                    u32 v[12];   // packed words (PACK) or values
                    if (TP::PACK) {
                        ld4p<T, TP::CS>(row, c0 - 4, v);
                        ld4p<T, TP::CS>(row, c0, v + 4);
                        ld4p<T, TP::CS>(row, c0 + 4, v + 8);
                    } else {
                        ld4<T>(row, c0 - 4, v);
                        ld4<T>(row, c0, v + 4);
                        ld4<T>(row, c0 + 4, v + 8);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        take(i, k, v[4 + k], v[4 + k]);   // the centre itself
#pragma unroll
                        for (int t = 1; t <= R; ++t) {
                            take(i, k, v[4 + k - t], v[4 + k - t]);
                            take(i, k, v[4 + k + t], v[4 + k + t]);
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
                            u32 vy[4], vz[4];   // packed words (PACK) or values
                            if (TP::PACK) {
                                ld4p<T, TP::CS>(pc + (r0 + i + sg * t) * G::ROWB, c0, vy);
                                ld4p<T, TP::CS>(plz + (r0 + i) * G::ROWB, c0, vz);
                            } else {
                                ld4<T>(pc + (r0 + i + sg * t) * G::ROWB, c0, vy);
                                ld4<T>(plz + (r0 + i) * G::ROWB, c0, vz);
                            }
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                take(i, k, vy[k], vy[k]);
                                take(i, k, vz[k], vz[k]);
                            }
                        }
                    }
                }
            }
            // ---- gate and round
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const u32 n = TP::PACK ? (acc[i][k] & ((1u << TP::CS) - 1u)) : cnt[i][k];
                    const u32 sm = TP::PACK ? (acc[i][k] >> TP::CS) : acc[i][k];
                    fo[i][k] = finish(sm, n, p0[i][k]);
                }
            }   // dense
            // ---- store, histogram
            const int z = z0 + s;
#pragma unroll
            for (int i = 0; i < kRows; ++i) {
                u32 f[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    f[k] = fo[i][k];
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

}  // namespace

// Route mean / sigma / entropy / Okada jobs on TMA-able volumes (whole or a
// region of interest) at radius 1..4 (sigma 1..2) to the specialised kernels.
lnf_status lnf_fast2_dispatch(lnf_ctx *ctx, const FilterJob &job, const CUtensorMap *tmap, cudaStream_t stream,
                              int *handled, u32 *counter, int gated)
{
    *handled = 0;
    if (!tmap || job.aniso || job.filter == LNF_OURS)
        return LNF_OK;
    if (gated == 2 ? !lnf_sparse_covers(job.filter, job.radius) : !lnf_fast_covers(job.filter, job.radius, job.offset))
        return LNF_OK;
    const bool u8 = job.dtype == LNF_U8;
    switch (job.filter) {
    case LNF_MEAN:
    case LNF_ENTROPY: return lnf_fast2_box(ctx, job, stream, counter, handled, gated);
    case LNF_SIGMA: return u8 ? by_radius<uint8_t, LNF_SIGMA>(ctx, job, stream, counter, handled, gated)
                              : by_radius<uint16_t, LNF_SIGMA>(ctx, job, stream, counter, handled, gated);
    case LNF_OKADA: return u8 ? by_radius<uint8_t, LNF_OKADA>(ctx, job, stream, counter, handled, gated)
                              : by_radius<uint16_t, LNF_OKADA>(ctx, job, stream, counter, handled, gated);
    default: return LNF_OK;
    }
}
