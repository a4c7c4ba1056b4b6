// Gate-first path for the paper's five filters on whole volumes: mean (Eq. 4),
// sigma (Eq. 5), entropy filter (Eq. 7), Okada (Eq. 6) and the paper's own
// filter (Eq. 2-3, nine clusters at offset d = 1), at radius 1..4.
//
// Every one of the five outputs is 0 where the voxel's own value P0 is below
// the noise threshold T, whatever its neighbourhood (§Our Method; the "0,
// otherwise" of Eq. 6 and Eq. 7).  While few voxels pass (lnf_gate_mode), the
// work splits into two kernels:
//   k_scan -- a stream over the volume: 16-byte vector loads (8 voxels), one
//     zero vector stored to every requested output, and one bit per voxel,
//     P0 >= T, into a bitmask.  It moves each byte once and needs no shared
//     memory or synchronisation, so it runs at the speed of a copy;
//   k_eval -- persistent warps take 1024-voxel chunks of the bitmask, gather
//     the set bits of a chunk into their own list (in-warp prefix sum) and
//     evaluate full rounds of 32 listed voxels, one per lane, carrying the rest
//     into the next chunk.  Each voxel's taps are read through L1 from the
//     input (taps at compile-time plane / row / column offsets); a voxel within
//     the filter's reach of a face takes a clamped path (clamp-to-edge
//     sampling).  Nonzero outputs overwrite the zeros.
// One launch pair serves any subset of the five filters: one read of the
// volume, one write per output.
//
// Output histograms: nonzero outputs (all >= max(1, T, min)) go to a shared
// window of 4096 16-bit bins per output (all 12-bit levels), the rest to
// global atomics; a bin that reaches 0x8000 moves 0x8000 to the global bin at
// once, so no bin overflows.  The zeros are N minus the nonzero outputs.
#pragma once
#include "lnf_ctx.h"

#include <algorithm>
#include <cstring>
#include <utility>

namespace gatek {

constexpr int kScanThreads = 256;
constexpr int kScanUnroll = 4;                       // vectors a thread loads before using them
constexpr int kEvalWarps = 8;
constexpr int kEvalThreads = kEvalWarps * 32;
constexpr int kChunkWords = 32;                      // bitmask words (32 voxels each) per chunk
constexpr int kChunkVox = kChunkWords * 32;          // voxels per chunk
constexpr int kListCap = kChunkVox + 32;             // a warp's list: one chunk plus 31 carried over
constexpr int kHistW = 4096;                         // shared histogram window per output (16-bit bins)
constexpr int kLutW = 4096;                          // entropy weights kept in shared memory (16-bit data)

// Multiplicity of the tap at offset (dx, dy, dz) in U, the sum over the nine
// clusters (the voxel and its eight diagonal neighbours at distance sqrt(3)) of
// their x-, y- and z-lines of M = 2R + 1 voxels (Eq. 2, Eq. 3).
__host__ __device__ constexpr int ours_weight(int R, int dx, int dy, int dz)
{
    int w = 0;
    for (int c = 0; c < 9; ++c) {
        const int cx = c == 0 ? 0 : (((c - 1) & 1) ? 1 : -1);
        const int cy = c == 0 ? 0 : (((c - 1) & 2) ? 1 : -1);
        const int cz = c == 0 ? 0 : (((c - 1) & 4) ? 1 : -1);
        if (dy == cy && dz == cz && dx - cx >= -R && dx - cx <= R)
            ++w;
        if (dx == cx && dz == cz && dy - cy >= -R && dy - cy <= R)
            ++w;
        if (dx == cx && dy == cy && dz - cz >= -R && dz - cz <= R)
            ++w;
    }
    return w;
}

// whether any tap of row (dy, dz) of the paper's filter has a nonzero multiplicity
__host__ __device__ constexpr bool ours_row(int R, int dy, int dz)
{
    for (int dx = -R - 1; dx <= R + 1; ++dx)
        if (ours_weight(R, dx, dy, dz))
            return true;
    return false;
}

enum { SET_OURS = 1, SET_CUBE = 2, SET_ALL = 3 };

template <typename T, int R, int SET>
struct GGeo {
    static constexpr bool OURS = (SET & SET_OURS) != 0;
    static constexpr bool CUBE = (SET & SET_CUBE) != 0;
    static constexpr int M = 2 * R + 1;
    static constexpr int H = OURS ? R + 1 : R;       // reach of the taps on each axis
    static constexpr int W = 2 * H + 1;
    static constexpr int CT = CUBE ? M * M * M : 0;  // cube taps
    static constexpr int ES = (int)sizeof(T);
    static constexpr int NOUT = (OURS ? 1 : 0) + (CUBE ? 4 : 0);
    static constexpr int LUTN = CUBE ? (ES == 1 ? 256 : kLutW) : 0;
    static constexpr int HISTB = NOUT * kHistW * 2;   // two 16-bit bins per 32-bit word
    static constexpr int LSTB = kEvalWarps * kListCap * 4;
    static constexpr int SMEM = HISTB + LUTN * 4 + LSTB;
    // sigma: value and count packed in one word (count in the low bits) while exact
    static constexpr int SSH = ES == 1 ? 10 : 8;
    static constexpr bool SPACK = CT < (1 << SSH) &&
                                  (unsigned long long)CT * (ES == 1 ? 255ull : 65535ull) * (1ull << SSH) <
                                      (1ull << 32);
};

// slot of a filter's output in the per-output arrays of a launch (the cube
// filters by id, the paper's filter after them)
template <int SET>
__host__ __device__ constexpr int oslot(int f)
{
    return f == LNF_OURS ? ((SET & SET_CUBE) ? 4 : 0) : f;
}

struct ScanArgs {
    const void *in;
    void *out[5];                  // by filter id; null: not requested
    u32 *mask;                     // one bit per voxel (P0 >= T), voxel i at bit i % 32 of word i / 32
    u64 n;                         // voxels
    u64 mask_bytes;                // bytes of the bitmask the evaluation reads (whole chunks)
    const DevParams *prm;
    u32 *counter;                  // the evaluation's chunk counter (reset here)
};

struct EvalArgs {
    const void *in;
    void *out[5];
    u64 *hist[5];                  // output histograms (null: not wanted)
    const u32 *mask;
    int nx, ny, nz;
    u32 nchunks;
    const DevParams *prm;
    const u32 *lut;
    u32 *counter;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ------------------------------------------------------------------ the scan

// the bits of the 8 voxels of a vector (16-bit: all four words; 8-bit: x, y)
// whose value is >= T; most vectors have none, found with one comparison
template <typename T>
__device__ __forceinline__ u32 pass_bits(const uint4 &w, u32 T_)
{
    u32 bits = 0;
    if (sizeof(T) == 2) {
        const u32 m = __vmaxu2(__vmaxu2(w.x, w.y), __vmaxu2(w.z, w.w));
        if (max(m & 0xFFFFu, m >> 16) >= T_) {
            const u32 ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int q = 0; q < 8; ++q)
                bits |= (((ww[q >> 1] >> (16 * (q & 1))) & 0xFFFFu) >= T_ ? 1u : 0u) << q;
        }
    } else {
        const u32 m2 = __vmaxu4(w.x, w.y);
        const u32 m1 = __vmaxu4(m2, m2 >> 16);
        if (max(m1 & 0xFFu, (m1 >> 8) & 0xFFu) >= T_) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                bits |= ((((q < 4 ? w.x : w.y) >> (8 * (q & 3))) & 0xFFu) >= T_ ? 1u : 0u) << q;
        }
    }
    return bits;
}

// one bit per voxel of the bitmask, written a byte (8 voxels) at a time
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan(const ScanArgs a)
{
    const DevParams &P = *a.prm;
    if (!lnf_gate_mode(P))
        return;   // many voxels pass the gate: the plane-ring kernels do the work
    const u32 T_ = P.T;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *a.counter = 0;   // the evaluation, next on the stream, claims chunks from 0
    unsigned char *mb = reinterpret_cast<unsigned char *>(a.mask);
    const u64 nvec = a.n / 8;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 v0 = blockIdx.x * (u64)blockDim.x + threadIdx.x; v0 < nvec; v0 += kScanUnroll * stride) {
        uint4 w[kScanUnroll];
#pragma unroll
        for (int k = 0; k < kScanUnroll; ++k) {
            const u64 v = v0 + k * stride;
            w[k] = make_uint4(0u, 0u, 0u, 0u);
            if (v < nvec) {
                if (sizeof(T) == 2) {
                    w[k] = __ldg(reinterpret_cast<const uint4 *>(a.in) + v);
                } else {
                    const uint2 h = __ldg(reinterpret_cast<const uint2 *>(a.in) + v);
                    w[k] = make_uint4(h.x, h.y, 0u, 0u);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kScanUnroll; ++k) {
            const u64 v = v0 + k * stride;
            if (v >= nvec)
                continue;
            const u32 bits = pass_bits<T>(w[k], T_);
#pragma unroll
            for (int f = 0; f < 5; ++f)
                if (a.out[f]) {
                    if (sizeof(T) == 2)
                        reinterpret_cast<uint4 *>(a.out[f])[v] = make_uint4(0u, 0u, 0u, 0u);
                    else
                        reinterpret_cast<uint2 *>(a.out[f])[v] = make_uint2(0u, 0u);
                }
            mb[v] = (unsigned char)bits;
        }
    }
    // the last voxels (n not a multiple of 8), and the bitmask's bytes beyond the
    // volume up to the end of the last chunk
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const u64 r = a.n - nvec * 8;
        u32 bits = 0;
        for (u64 q = 0; q < r; ++q) {
            const u64 i = nvec * 8 + q;
            const u32 val = sizeof(T) == 2 ? (u32) static_cast<const uint16_t *>(a.in)[i]
                                           : (u32) static_cast<const uint8_t *>(a.in)[i];
            bits |= (val >= T_ ? 1u : 0u) << q;
            for (int f = 0; f < 5; ++f)
                if (a.out[f])
                    static_cast<T *>(a.out[f])[i] = (T)0;
        }
        if (r)
            mb[nvec] = (unsigned char)bits;
        for (u64 b = (a.n + 7) / 8; b < a.mask_bytes; ++b)
            mb[b] = 0;
    }
}

// ------------------------------------------------------------------ the evaluation

// compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1
template <class F, int... I>
__device__ __forceinline__ void sfor_impl(F &f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F &&f)
{
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

template <typename T>
__device__ __forceinline__ u32 ldgv(const T *p)
{
    return (u32)__ldg(p);
}

// One voxel's sums for the filters of the set.  CLAMP = false: every tap is at a
// compile-time offset from the pointer of its plane and row; CLAMP = true: the
// voxel lies within reach H of a face, and each tap is clamped into the volume.
template <typename T, int R, int SET, bool LUTALL, bool CLAMP>
struct Sums {
    u32 U = 0, B = 0, S = 0, N = 0, O = 0, E = 0;
    // four partial sums per quantity at radius <= 2 (tap t adds into partial t % 4),
    // so that the adds form four short dependency chains instead of one long one
    static constexpr int NA = R <= 2 ? 4 : 1;

    __device__ __forceinline__ void run(const T *in, int x, int y, int z, int nx, int ny, int nz, u32 slo,
                                        u32 swd, u32 olo, u32 owd, const u32 *lut_sh, u32 lbase, const u32 *lut)
    {
        typedef GGeo<T, R, SET> G;
        const long long sxy = (long long)nx * ny;
        u32 u[4] = {0u, 0u, 0u, 0u};
        u32 b[4] = {0u, 0u, 0u, 0u}, sg[4] = {0u, 0u, 0u, 0u}, n[4] = {0u, 0u, 0u, 0u}, e[4] = {0u, 0u, 0u, 0u};
        u32 o[2] = {0u, 0u};
        // one row (plane dz, row dy) at a time: its pointer, then its taps
        sfor<G::W * G::W>([&](auto ri) {
            constexpr int rix = decltype(ri)::value;
            constexpr int dy = rix % G::W - G::H, dz = rix / G::W - G::H;
            constexpr bool row_cube = G::CUBE && dy >= -R && dy <= R && dz >= -R && dz <= R;
            constexpr bool row_ours = G::OURS && ours_row(R, dy, dz);
            if constexpr (row_cube || row_ours) {
                const T *rp;
                if constexpr (CLAMP)
                    rp = in + (clampi(z + dz, 0, nz - 1) * sxy + (long long)clampi(y + dy, 0, ny - 1) * nx);
                else
                    rp = in + ((long long)(z + dz) * sxy + (long long)(y + dy) * nx + x);
                sfor<G::W>([&](auto ci) {
                    constexpr int dx = decltype(ci)::value - G::H;
                    constexpr int t = rix * G::W + decltype(ci)::value;
                    constexpr int w = G::OURS ? ours_weight(R, dx, dy, dz) : 0;
                    constexpr bool cube = row_cube && dx >= -R && dx <= R;
                    if constexpr (w != 0 || cube) {
                        u32 v;
                        if constexpr (CLAMP)
                            v = ldgv<T>(rp + clampi(x + dx, 0, nx - 1));
                        else
                            v = ldgv<T>(rp + dx);
                        if constexpr (w != 0)
                            u[t % NA] += (u32)w * v;
                        if constexpr (cube) {
                            constexpr int q = t % NA;
                            constexpr bool cross = (dx == 0 && dy == 0) || (dx == 0 && dz == 0) || (dy == 0 && dz == 0);
                            b[q] += v;
                            if (v - slo <= swd) {
                                if constexpr (G::SPACK) {
                                    sg[q] += (v << G::SSH) | 1u;
                                } else {
                                    sg[q] += v;
                                    n[q] += 1u;
                                }
                            }
                            if constexpr (cross) {
                                if (v - olo <= owd)
                                    o[t % (NA > 1 ? 2 : 1)] += (v << 8) | 1u;
                            }
                            const u32 lo = v - lbase;
                            if constexpr (LUTALL)
                                e[q] += lut_sh[lo];
                            else
                                e[q] += lo < (u32)G::LUTN ? lut_sh[lo] : __ldg(lut + v);
                        }
                    }
                });
            }
        });
        U = (u[0] + u[1]) + (u[2] + u[3]);
        B = (b[0] + b[1]) + (b[2] + b[3]);
        S = (sg[0] + sg[1]) + (sg[2] + sg[3]);
        N = (n[0] + n[1]) + (n[2] + n[3]);
        E = (e[0] + e[1]) + (e[2] + e[3]);
        O = o[0] + o[1];
    }
};

// the sums of a voxel near a face, out of line so that the common path stays compact
template <typename T, int R, int SET>
__device__ __noinline__ void sums_clamped(Sums<T, R, SET, false, true> &sm, const T *in, int x, int y, int z,
                                          int nx, int ny, int nz, u32 slo, u32 swd, u32 olo, u32 owd,
                                          const u32 *lut_sh, u32 lbase, const u32 *lut)
{
    sm.run(in, x, y, z, nx, ny, nz, slo, swd, olo, owd, lut_sh, lbase, lut);
}

template <typename T, int R, int SET>
__global__ void __launch_bounds__(kEvalThreads, 2) k_eval(const EvalArgs a)
{
    typedef GGeo<T, R, SET> G;
    const DevParams &P = *a.prm;
    if (!lnf_gate_mode(P))
        return;
    extern __shared__ __align__(16) unsigned char smem[];
    u32 *hsh = reinterpret_cast<u32 *>(smem);                                  // NOUT windows of 16-bit bins
    u32 *lut_sh = reinterpret_cast<u32 *>(smem + G::HISTB);                    // LUTN entropy weights
    u32 *lst = reinterpret_cast<u32 *>(smem + G::HISTB + G::LUTN * 4);         // the warps' lists
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const T *in = static_cast<const T *>(a.in);

    // ---- parameters of the gates (the same values the ring kernels use)
    const u32 T_ = P.T;
    const u32 hbase = max(1u, max(T_, P.minv));   // nonzero outputs lie in [hbase, levels)
    const u32 dl = min(P.delta, 65535u);          // sigma band |v - P0| <= dl
    const long long td = P.td;                    // Okada band |P0 - v| < td
    const u32 th = td > 65536 ? 65535u : (td > 0 ? (u32)(td - 1) : 0u);
    long long te = P.te_cfg;                      // entropy filter: keep P0 iff E > te
    if (te == -2)
        te = (long long)(((unsigned __int128)(G::CT ? G::CT : 1) * P.hw_sum) / P.N);
    const u32 lbase = G::ES == 1 ? 0u : P.minv;
    const bool lutall = G::LUTN > 0 && (P.maxv - lbase) + 1u <= (u32)G::LUTN;
    for (int i = tid; i < G::NOUT * kHistW / 2; i += kEvalThreads)
        hsh[i] = 0;
    for (int i = tid; i < G::LUTN; i += kEvalThreads)
        lut_sh[i] = (lbase + i < (G::ES == 1 ? 256u : 65536u)) ? a.lut[lbase + i] : 0u;
    __syncthreads();

    typedef ExactDiv<27ull * G::M, 27ull * G::M * 65536ull> DivO;   // the paper's filter: U / 27M
    typedef ExactDiv<(unsigned long long)G::M * G::M * G::M,
                     (unsigned long long)G::M * G::M * G::M * 65536ull> DivM;   // mean: B / M^3
    constexpr u32 KO = 27u * G::M, KM = (u32)(G::M * G::M * G::M);
    const u32 KOT = KO * T_, KMT = KM * T_;
    const u32 nxny = (u32)a.nx * (u32)a.ny;
    u32 nzc[5] = {0u, 0u, 0u, 0u, 0u};
    u32 *L = lst + warp * kListCap;

    // one listed voxel (linear index i), evaluated by this lane
    auto eval_voxel = [&](u32 i) {
        const int z = (int)(i / nxny);
        const u32 rem = i - (u32)z * nxny;
        const int y = (int)(rem / (u32)a.nx);
        const int x = (int)(rem - (u32)y * (u32)a.nx);
        const u32 P0 = ldgv<T>(in + i);
        const u32 slo = P0 > dl ? P0 - dl : 0u, swd = P0 - slo + dl;
        const u32 olo = P0 > th ? P0 - th : 0u, owd = P0 - olo + th;
        const bool inner = x >= G::H && x + G::H < a.nx && y >= G::H && y + G::H < a.ny && z >= G::H &&
                           z + G::H < a.nz;
        u32 fv[5] = {0u, 0u, 0u, 0u, 0u};
        auto finish = [&](const auto &sm) {
            if constexpr (G::OURS)
                fv[LNF_OURS] = sm.U >= KOT ? DivO::template div_add<(27ull * G::M - 1) / 2>(sm.U) : 0u;
            if constexpr (G::CUBE) {
                fv[LNF_MEAN] = sm.B >= KMT ? DivM::template div_add<((unsigned long long)KM - 1) / 2>(sm.B) : 0u;
                const u32 n = G::SPACK ? (sm.S & ((1u << G::SSH) - 1u)) : sm.N;
                const u32 ssum = G::SPACK ? (sm.S >> G::SSH) : sm.S;
                fv[LNF_SIGMA] = (n && ssum >= n * T_) ? (ssum + (n >> 1)) / n : 0u;
                const u32 on = sm.O & 0xFFu, osum = sm.O >> 8;
                fv[LNF_OKADA] = (td > 0 && on && osum >= on * T_) ? (osum + (on >> 1)) / on : 0u;
                fv[LNF_ENTROPY] = (long long)sm.E > te ? P0 : 0u;
            }
        };
        if (inner) {
            if (lutall || !G::CUBE) {
                Sums<T, R, SET, true, false> sm;
                sm.run(in, x, y, z, a.nx, a.ny, a.nz, slo, swd, olo, owd, lut_sh, lbase, a.lut);
                finish(sm);
            } else {
                Sums<T, R, SET, false, false> sm;
                sm.run(in, x, y, z, a.nx, a.ny, a.nz, slo, swd, olo, owd, lut_sh, lbase, a.lut);
                finish(sm);
            }
        } else {
            Sums<T, R, SET, false, true> sm;
            sums_clamped<T, R, SET>(sm, in, x, y, z, a.nx, a.ny, a.nz, slo, swd, olo, owd, lut_sh, lbase, a.lut);
            finish(sm);
        }
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            if (!(((f == LNF_OURS) ? G::OURS : G::CUBE) && a.out[f]))
                continue;
            const u32 v = fv[f];
            if (!v)
                continue;
            static_cast<T *>(a.out[f])[i] = (T)v;
            ++nzc[f];
            if (a.hist[f]) {
                const u32 hb = v - hbase;
                if (hb < (u32)kHistW) {
                    // 16-bit bins: the add that makes a bin 0x8000 moves 0x8000 to the
                    // global bin, so that no bin passes 0xFFFF
                    u32 *wd = &hsh[oslot<SET>(f) * (kHistW / 2) + (hb >> 1)];
                    const u32 sh = 16u * (hb & 1u);
                    const u32 old = atomicAdd(wd, 1u << sh);
                    if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
                        atomicAdd(wd, 0u - (0x8000u << sh));
                        atomicAdd(&a.hist[f][v], 0x8000ull);
                    }
                } else if (v < 65536u) {   // always true for valid outputs
                    atomicAdd(&a.hist[f][v], 1ull);
                }
            }
        }
    };

    // ---- chunks of the bitmask: the set bits into this warp's list, then full rounds
    u32 nlist = 0;   // listed voxels not yet evaluated (the same in every lane)
    for (;;) {
        u32 c = 0;
        if (lane == 0)
            c = atomicAdd(a.counter, 1u);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        const bool done = c >= a.nchunks;
        if (!done) {
            const u32 w = a.mask[(u64)c * kChunkWords + lane];
            const u32 k = (u32)__popc(w);
            u32 incl = k;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const u32 t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d)
                    incl += t;
            }
            u32 pos = nlist + incl - k;
            const u32 base = c * (u32)kChunkVox + (u32)lane * 32u;
            u32 m = w;
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1u;
                L[pos++] = base + (u32)bit;
            }
            nlist += __shfl_sync(0xFFFFFFFFu, incl, 31);
            __syncwarp();
        }
        const u32 neval = done ? nlist : (nlist & ~31u);
        for (u32 e = (u32)lane; e < neval; e += 32)
            eval_voxel(L[e]);
        __syncwarp();
        const u32 rest = nlist - neval;   // at most 31: to the front of the list
        u32 keep = 0;
        if ((u32)lane < rest)
            keep = L[neval + lane];
        __syncwarp();
        if ((u32)lane < rest)
            L[lane] = keep;
        __syncwarp();
        nlist = rest;
        if (done)
            break;
    }

    // ---- histograms: the shared windows, and the zeros as N minus the nonzero outputs
    __syncthreads();
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        if (!(((f == LNF_OURS) ? G::OURS : G::CUBE) && a.out[f] && a.hist[f]))
            continue;
        const u32 *h = hsh + oslot<SET>(f) * (kHistW / 2);
        for (int i = tid; i < kHistW / 2; i += kEvalThreads) {
            const u32 w = h[i];
            if (w & 0xFFFFu)
                atomicAdd(&a.hist[f][hbase + 2 * i], (u64)(w & 0xFFFFu));
            if (w >> 16)
                atomicAdd(&a.hist[f][hbase + 2 * i + 1], (u64)(w >> 16));
        }
        const u32 nsum = __reduce_add_sync(0xFFFFFFFFu, nzc[f]);
        u64 add = 0ull - (u64)nsum;            // modulo 2^64: the bin ends at N - sum of nonzero
        if (blockIdx.x == 0 && warp == 0)
            add += P.N;
        if (lane == 0 && add)
            atomicAdd(&a.hist[f][0], add);
    }
}

// ------------------------------------------------------------------ launch

template <typename T, int R, int SET>
lnf_status eval_launch_t(lnf_ctx *ctx, const EvalArgs &a, cudaStream_t st)
{
    typedef GGeo<T, R, SET> G;
    if (cudaFuncSetAttribute(k_eval<T, R, SET>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) !=
        cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "gate evaluation kernel: shared memory attribute (%d bytes)", G::SMEM);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval<T, R, SET>, kEvalThreads, G::SMEM);
    const int grid = std::max(1, std::min((int)a.nchunks, ctx->num_sms * std::max(1, occ)));
    k_eval<T, R, SET><<<grid, kEvalThreads, G::SMEM, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? LNF_OK
                                             : lnf_fail(ctx, LNF_ECUDA, "gate evaluation kernel launch failed");
}

template <typename T, int SET>
lnf_status eval_by_radius(lnf_ctx *ctx, int radius, const EvalArgs &a, cudaStream_t st)
{
    switch (radius) {
    case 1: return eval_launch_t<T, 1, SET>(ctx, a, st);
    case 2: return eval_launch_t<T, 2, SET>(ctx, a, st);
    case 3: return eval_launch_t<T, 3, SET>(ctx, a, st);
    default: return eval_launch_t<T, 4, SET>(ctx, a, st);
    }
}

// The scan and the evaluation of one job (outs / hists by filter id).
template <typename T>
lnf_status gate_dispatch_t(lnf_ctx *ctx, const FilterJob &j, void *const outs[5], u64 *const hists[5],
                           cudaStream_t st, int *handled)
{
    const u64 n = (u64)j.nx * j.ny * j.nz;
    if (n >= (1ull << 32) || j.pitch != j.nx || reinterpret_cast<uintptr_t>(j.in) % 16 != 0)
        return LNF_OK;   // not handled: 32-bit voxel indices and dense aligned rows only
    for (int f = 0; f < 5; ++f)
        if (outs[f] && reinterpret_cast<uintptr_t>(outs[f]) % 16 != 0)
            return LNF_OK;
    const u64 nchunks = (n + kChunkVox - 1) / kChunkVox;
    const size_t mbytes = nchunks * kChunkVox / 8;
    if (ctx->gate_mask_cap < mbytes) {
        cudaFree(ctx->gate_mask_buf);   // waits for the work that still reads it
        ctx->gate_mask_buf = nullptr;
        ctx->gate_mask_cap = 0;
        if (cudaMalloc(&ctx->gate_mask_buf, mbytes) != cudaSuccess) {
            ctx->gate_mask_buf = nullptr;
            cudaGetLastError();
            return LNF_OK;   // no room for the bitmask: the ring kernels do the work
        }
        ctx->gate_mask_cap = mbytes;
    }
    u32 *mask = static_cast<u32 *>(ctx->gate_mask_buf);
    u32 *counter = ctx->d_counter + 14;
    ScanArgs sa;
    std::memset(&sa, 0, sizeof sa);
    sa.in = j.in;
    for (int f = 0; f < 5; ++f)
        sa.out[f] = outs[f];
    sa.mask = mask;
    sa.n = n;
    sa.mask_bytes = mbytes;
    sa.prm = j.prm;
    sa.counter = counter;
    const int sgrid = std::max(1, ctx->num_sms * 8);
    k_scan<T><<<sgrid, kScanThreads, 0, st>>>(sa);
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "gate scan kernel launch failed");
    EvalArgs ea;
    std::memset(&ea, 0, sizeof ea);
    ea.in = j.in;
    for (int f = 0; f < 5; ++f) {
        ea.out[f] = outs[f];
        ea.hist[f] = outs[f] ? hists[f] : nullptr;
    }
    ea.mask = mask;
    ea.nx = j.nx;
    ea.ny = j.ny;
    ea.nz = j.nz;
    ea.nchunks = (u32)nchunks;
    ea.prm = j.prm;
    ea.lut = j.lut;
    ea.counter = counter;
    const bool ours = outs[LNF_OURS] != nullptr;
    const bool cube = outs[0] || outs[1] || outs[2] || outs[3];
    lnf_status s;
    if (ours && cube)
        s = eval_by_radius<T, SET_ALL>(ctx, j.radius, ea, st);
    else if (ours)
        s = eval_by_radius<T, SET_OURS>(ctx, j.radius, ea, st);
    else
        s = eval_by_radius<T, SET_CUBE>(ctx, j.radius, ea, st);
    if (s == LNF_OK)
        *handled = 1;
    return s;
}

}  // namespace gatek
