// Gate-first path for the paper's five filters on whole volumes: mean (Eq. 4),
// sigma (Eq. 5), entropy filter (Eq. 7), Okada (Eq. 6) and the paper's own
// filter (Eq. 2-3, nine clusters at offset d = 1), at radius 1..4.
//
// Every one of the five outputs is 0 where the voxel's own value P0 is below
// the noise threshold T, whatever its neighbourhood (§Our Method; the "0,
// otherwise" of Eq. 6 and Eq. 7).  While few voxels pass (lnf_gate_mode), one
// persistent kernel streams the volume and evaluates only the passing voxels.
// Its warps claim chunks of 256 VL voxels in order (VL 16-byte vectors of 8
// voxels per lane); per chunk a warp
//   - loads the chunk (for the paper's filter alone: the next chunk's loads are
//     issued before this one is used, and the claim of the one after it is
//     read only at the end of the step, so that neither waits), stores one
//     zero vector to every requested output and keeps, per lane, the bits of
//     its voxels with P0 >= T;
//   - appends those voxels to its own list (in-warp prefix sum) and evaluates
//     full rounds of 32 listed voxels, one per lane, carrying up to 31 into
//     its next chunk (the warp zeroed them itself, so its nonzero outputs
//     follow the zeros in program order).
// A voxel's taps are read through L1 from the input, at compile-time plane /
// row / column offsets; the chunks a warp's neighbours in z were given a few
// hundred claims earlier, so those taps come from L2.  A voxel within the
// filter's reach of a face takes a clamped path (clamp-to-edge sampling).
// One launch serves any subset of the five filters: one read of the volume,
// one write per output.  A launch of set SET_ELOC instead evaluates the entropy
// filter with the cube's own grey-level probabilities (filter id 8, r = 1..2):
// each lane copies its voxel's M^3 values into its own column of shared memory
// and counts equal levels there by rank (the criterion t[m] - sum_g t[c_g]
// with t[c] = round(2^22 c log2 c) from the parameter block).
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

#ifndef LNF_GATE_MINB_CUBE
#define LNF_GATE_MINB_CUBE 2
#endif
#ifndef LNF_GATE_MINB_OURS
#define LNF_GATE_MINB_OURS 2
#endif
#ifndef LNF_GATE_VL_CUBE
#define LNF_GATE_VL_CUBE 2
#endif
#ifndef LNF_GATE_VL_OURS
#define LNF_GATE_VL_OURS 6
#endif
#ifndef LNF_GATE_PF_CUBE
#define LNF_GATE_PF_CUBE 0
#endif
#ifndef LNF_GATE_PF_OURS
#define LNF_GATE_PF_OURS 1
#endif

namespace gatek {

constexpr int kWarpsC = 8;                           // warps per CTA
constexpr int kThreadsC = kWarpsC * 32;
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

// filter sets of a launch: the paper's filter, the four cube filters, both, or
// the entropy filter with the cube's own grey-level probabilities (alone; its
// output takes the entropy filter's slot)
enum { SET_OURS = 1, SET_CUBE = 2, SET_ALL = 3, SET_ELOC = 4 };

// whether a launch of set SET writes the output slot of filter id f (0..4)
template <int SET>
__host__ __device__ constexpr bool gets(int f)
{
    return f == LNF_OURS ? (SET & SET_OURS) != 0
                         : (f == LNF_ENTROPY ? (SET & (SET_CUBE | SET_ELOC)) != 0 : (SET & SET_CUBE) != 0);
}

template <typename T, int R, int SET>
struct GGeo {
    static constexpr bool OURS = (SET & SET_OURS) != 0;
    static constexpr bool CUBE = (SET & SET_CUBE) != 0;
    static constexpr bool ELOC = (SET & SET_ELOC) != 0;
    static constexpr bool BOX = CUBE || ELOC;         // evaluates the M^3 cube
    static constexpr int M = 2 * R + 1;
    static constexpr int H = OURS ? R + 1 : R;       // reach of the taps on each axis
    static constexpr int W = 2 * H + 1;
    static constexpr int CT = BOX ? M * M * M : 0;   // cube taps
    static constexpr int ES = (int)sizeof(T);
    static constexpr int NOUT = (OURS ? 1 : 0) + (CUBE ? 4 : 0) + (ELOC ? 1 : 0);
    static constexpr int LUTN = CUBE ? (ES == 1 ? 256 : kLutW) : 0;
    static constexpr int HISTB = NOUT * kHistW * 2;   // two 16-bit bins per 32-bit word
    // chunks: VL 16-byte vectors of 8 voxels per lane; PF: the next chunk's loads
    // are issued before the current chunk is used
    static constexpr int VL = BOX ? LNF_GATE_VL_CUBE : LNF_GATE_VL_OURS;
    static constexpr bool PF = (BOX ? LNF_GATE_PF_CUBE : LNF_GATE_PF_OURS) != 0;
    static constexpr int CVEC = 32 * VL;            // vectors per chunk
    static constexpr int CVOX = CVEC * 8;           // voxels per chunk
    static constexpr int LCAP = CVOX + 32;          // a warp's list: one chunk plus 31 carried over
    static constexpr int LSTB = kWarpsC * LCAP * 4;
    // the local entropy filter: each lane's column of its voxel's cube values
    // (16-bit, value t of lane L at t * 32 + L in its warp's block), and the table
    // t[0..CT] of round(2^22 c log2 c)
    static constexpr int ELB = ELOC ? kWarpsC * CT * 32 * 2 : 0;
    static constexpr int LTB = ELOC ? ((CT + 1) * 8 + 15) / 16 * 16 : 0;
    static constexpr int SMEM = HISTB + LUTN * 4 + LSTB + ELB + LTB;
    // CTAs per SM the register budget aims for: the kernel waits on loads, so
    // more warps hide more of it where the evaluation needs fewer registers
    static constexpr int MINB = BOX ? LNF_GATE_MINB_CUBE : LNF_GATE_MINB_OURS;
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
    return (SET & SET_ELOC) ? 0 : (f == LNF_OURS ? ((SET & SET_CUBE) ? 4 : 0) : f);
}

struct GateArgs {
    const void *in;
    void *out[5];                  // by filter id; null: not requested
    u64 *hist[5];                  // output histograms (null: not wanted)
    int nx, ny, nz;
    u64 n;                         // voxels
    u32 nchunks;
    const DevParams *prm;
    const u32 *lut;
    u32 *counter;                  // chunk counter, 0 at launch
    u32 *err;                      // error word (debug builds' bounds checks)
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
// The paper's filter's taps are unrolled (two instructions each); the cube's
// are unrolled within a plane and looped over the planes, which keeps the code
// of a voxel small enough for the instruction cache.
template <typename T, int R, int SET, bool LUTALL, bool CLAMP>
struct Sums {
    u32 U = 0, B = 0, S = 0, N = 0, O = 0, E = 0;
    // four partial sums per quantity at radius <= 2 (tap t adds into partial t % 4),
    // so that the adds form four short dependency chains instead of one long one
    static constexpr int NA = R <= 2 ? 4 : 1;

    __device__ __forceinline__ const T *row(const T *in, int x, int y, int z, int dy, int dz, int nx, int ny,
                                            int nz, long long sxy) const
    {
        if constexpr (CLAMP)
            return in + (clampi(z + dz, 0, nz - 1) * sxy + (long long)clampi(y + dy, 0, ny - 1) * nx);
        else
            return in + ((long long)(z + dz) * sxy + (long long)(y + dy) * nx + x);
    }

    template <int DX>
    __device__ __forceinline__ u32 tap(const T *rp, int x, int nx) const
    {
        if constexpr (CLAMP)
            return ldgv<T>(rp + clampi(x + DX, 0, nx - 1));
        else
            return ldgv<T>(rp + DX);
    }

    __device__ __forceinline__ void run(const T *in, int x, int y, int z, int nx, int ny, int nz, u32 slo,
                                        u32 swd, u32 olo, u32 owd, const u32 *lut_sh, u32 lbase, const u32 *lut)
    {
        typedef GGeo<T, R, SET> G;
        const long long sxy = (long long)nx * ny;
        if constexpr (G::OURS) {
            u32 u[4] = {0u, 0u, 0u, 0u};
            sfor<G::W * G::W>([&](auto ri) {
                constexpr int rix = decltype(ri)::value;
                constexpr int dy = rix % G::W - G::H, dz = rix / G::W - G::H;
                if constexpr (ours_row(R, dy, dz)) {
                    const T *rp = row(in, x, y, z, dy, dz, nx, ny, nz, sxy);
                    sfor<G::W>([&](auto ci) {
                        constexpr int dx = decltype(ci)::value - G::H;
                        constexpr int w = ours_weight(R, dx, dy, dz);
                        if constexpr (w != 0)
                            u[(rix * G::W + decltype(ci)::value) % NA] += (u32)w * tap<dx>(rp, x, nx);
                    });
                }
            });
            U = (u[0] + u[1]) + (u[2] + u[3]);
        }
        if constexpr (G::CUBE) {
            u32 b[4] = {0u, 0u, 0u, 0u}, sg[4] = {0u, 0u, 0u, 0u}, n[4] = {0u, 0u, 0u, 0u}, e[4] = {0u, 0u, 0u, 0u};
            u32 o[2] = {0u, 0u};
#pragma unroll 1
            for (int dz = -R; dz <= R; ++dz) {
                const bool mid = dz == 0;   // the Okada cross has its x and y arms in this plane
                sfor<G::M * G::M>([&](auto ti) {
                    constexpr int t = decltype(ti)::value;
                    constexpr int q = t % NA;
                    constexpr int dx = t % G::M - R, dy = t / G::M - R;
                    const T *rp = row(in, x, y, z, dy, dz, nx, ny, nz, sxy);
                    const u32 v = tap<dx>(rp, x, nx);
                    b[q] += v;
                    if (v - slo <= swd) {
                        if constexpr (G::SPACK) {
                            sg[q] += (v << G::SSH) | 1u;
                        } else {
                            sg[q] += v;
                            n[q] += 1u;
                        }
                    }
                    constexpr bool zarm = dx == 0 && dy == 0;   // on the cross in every plane
                    constexpr bool xyarm = dx == 0 || dy == 0;  // on the cross in the middle plane
                    if constexpr (zarm) {
                        if (v - olo <= owd)
                            o[t & 1] += (v << 8) | 1u;
                    } else if constexpr (xyarm) {
                        if (mid && v - olo <= owd)
                            o[t & 1] += (v << 8) | 1u;
                    }
                    const u32 lo = v - lbase;
                    if constexpr (LUTALL)
                        e[q] += lut_sh[lo];
                    else
                        e[q] += lo < (u32)G::LUTN ? lut_sh[lo] : __ldg(lut + v);
                });
            }
            B = (b[0] + b[1]) + (b[2] + b[3]);
            S = (sg[0] + sg[1]) + (sg[2] + sg[3]);
            N = (n[0] + n[1]) + (n[2] + n[3]);
            E = (e[0] + e[1]) + (e[2] + e[3]);
            O = o[0] + o[1];
        }
    }
};

// The sums of a voxel near a face (taps clamped), or of any voxel whose levels'
// entropy weights do not all fit in shared memory: out of line, so that the
// common path stays compact.
template <typename T, int R, int SET>
__device__ __noinline__ void sums_clamped(Sums<T, R, SET, false, true> &sm, const T *in, int x, int y, int z,
                                          int nx, int ny, int nz, u32 slo, u32 swd, u32 olo, u32 owd,
                                          const u32 *lut_sh, u32 lbase, const u32 *lut)
{
    sm.run(in, x, y, z, nx, ny, nz, slo, swd, olo, owd, lut_sh, lbase, lut);
}

template <typename T, int R, int SET>
__global__ void __launch_bounds__(kThreadsC, GGeo<T, R, SET>::MINB) k_gate(const GateArgs a)
{
    typedef GGeo<T, R, SET> G;
    const DevParams &P = *a.prm;
    if (!lnf_gate_mode(P))
        return;   // many voxels pass the gate: the plane-ring kernels do the work
    extern __shared__ __align__(16) unsigned char smem[];
    u32 *hsh = reinterpret_cast<u32 *>(smem);                                  // NOUT windows of 16-bit bins
    u32 *lut_sh = reinterpret_cast<u32 *>(smem + G::HISTB);                    // LUTN entropy weights
    u32 *lst = reinterpret_cast<u32 *>(smem + G::HISTB + G::LUTN * 4);         // the warps' lists
    uint16_t *elb = reinterpret_cast<uint16_t *>(smem + G::HISTB + G::LUTN * 4 + G::LSTB);   // cube columns
    unsigned long long *lt_sh =
        reinterpret_cast<unsigned long long *>(smem + G::HISTB + G::LUTN * 4 + G::LSTB + G::ELB);   // t[c]
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
    for (int i = tid; i < G::NOUT * kHistW / 2; i += kThreadsC)
        hsh[i] = 0;
    for (int i = tid; i < G::LUTN; i += kThreadsC)
        lut_sh[i] = (lbase + i < (G::ES == 1 ? 256u : 65536u)) ? a.lut[lbase + i] : 0u;
    if constexpr (G::ELOC)
        for (int i = tid; i <= G::CT; i += kThreadsC)
            lt_sh[i] = P.lt ? P.lt[i] : 0ull;
    // the local entropy filter's theta (2^-22 bits): default floor(t[m] / 2m)
    long long lte = P.lte_cfg;
    if (G::ELOC && lte == -2)
        lte = P.lt ? (long long)(P.lt[G::CT] / (2ull * (u64)(G::CT ? G::CT : 1))) : 0;
    __syncthreads();

    typedef ExactDiv<27ull * G::M, 27ull * G::M * 65536ull> DivO;   // the paper's filter: U / 27M
    typedef ExactDiv<(unsigned long long)G::M * G::M * G::M,
                     (unsigned long long)G::M * G::M * G::M * 65536ull> DivM;   // mean: B / M^3
    constexpr u32 KO = 27u * G::M, KM = (u32)(G::M * G::M * G::M);
    const u32 KOT = KO * T_, KMT = KM * T_;
    const u32 nxny = (u32)a.nx * (u32)a.ny;
    const u64 nvec = a.n / 8;
    u32 nzc[5] = {0u, 0u, 0u, 0u, 0u};
    u32 *L = lst + warp * G::LCAP;

    // one listed voxel (linear index i), evaluated by this lane
    auto eval_voxel = [&](u32 i) {
        if (!lnfdev::lnf_dbg_ok(i < a.n, a.err))
            return;
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
        // debug builds: an interior voxel's taps lie within the volume's linear range
        const u64 reach = (u64)G::H * ((u64)nxny + (u64)a.nx + 1ull);
        if (inner && !lnfdev::lnf_dbg_ok((u64)i >= reach && (u64)i + reach < a.n, a.err))
            return;
        if constexpr (G::ELOC) {
            // the entropy filter with the cube's own probabilities: the lane's cube
            // values into its column, then m 2^22 H = t[m] - sum_g t[c_g], the sum taken
            // over the taps a as t[k_a] - t[k_a - 1] (k_a: taps up to a at a's level)
            uint16_t *col = elb + warp * (G::CT * 32) + lane;
            if (inner) {
                const T *c0 = in + i;
                const long long sxy = (long long)nxny;
                sfor<G::CT>([&](auto ti) {
                    constexpr int t = decltype(ti)::value;
                    constexpr int dx = t % G::M - R, dy = (t / G::M) % G::M - R, dz = t / (G::M * G::M) - R;
                    col[t * 32] = (uint16_t)ldgv<T>(c0 + (dz * sxy + (long long)dy * a.nx + dx));
                });
            } else {
                int t = 0;
                for (int dz = -R; dz <= R; ++dz)
                    for (int dy = -R; dy <= R; ++dy) {
                        const T *rp = in + ((long long)clampi(z + dz, 0, a.nz - 1) * nxny +
                                            (long long)clampi(y + dy, 0, a.ny - 1) * a.nx);
                        for (int dx = -R; dx <= R; ++dx, ++t)
                            col[t * 32] = (uint16_t)ldgv<T>(rp + clampi(x + dx, 0, a.nx - 1));
                    }
            }
            u64 K = 0;
            for (int t = 0; t < G::CT; ++t) {
                const u32 va = col[t * 32];
                u32 k = 1;
#pragma unroll 4
                for (int b = 0; b < t; ++b)
                    k += col[b * 32] == va ? 1u : 0u;
                K += lt_sh[k] - lt_sh[k - 1];
            }
            const long long crit = (long long)(lt_sh[G::CT] - K);
            fv[LNF_ENTROPY] = crit > (long long)G::CT * lte ? P0 : 0u;
        } else if (inner && (lutall || !G::CUBE)) {
            Sums<T, R, SET, true, false> sm;
            sm.run(in, x, y, z, a.nx, a.ny, a.nz, slo, swd, olo, owd, lut_sh, lbase, a.lut);
            finish(sm);
        } else {
            Sums<T, R, SET, false, true> sm;
            sums_clamped<T, R, SET>(sm, in, x, y, z, a.nx, a.ny, a.nz, slo, swd, olo, owd, lut_sh, lbase, a.lut);
            finish(sm);
        }
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            if (!(gets<SET>(f) && a.out[f]))
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
                    if (!lnfdev::lnf_dbg_ok(oslot<SET>(f) < G::NOUT, a.err))
                        continue;
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

    // ---- chunks: stream, list, evaluate full rounds
    auto claim = [&]() -> u32 {
        u32 c = 0;
        if (lane == 0)
            c = atomicAdd(a.counter, 1u);
        return __shfl_sync(0xFFFFFFFFu, c, 0);
    };
    // the lane's vectors of chunk c: chunk vector lane + 32 k (consecutive lanes,
    // consecutive 16 bytes)
    auto load_chunk = [&](u32 c, uint4 *w) {
#pragma unroll
        for (int k = 0; k < G::VL; ++k) {
            const u64 v = (u64)c * G::CVEC + lane + 32 * k;
            w[k] = make_uint4(0u, 0u, 0u, 0u);
            if (c < a.nchunks && v < nvec) {
                if (sizeof(T) == 2) {
                    w[k] = __ldg(reinterpret_cast<const uint4 *>(a.in) + v);
                } else {
                    const uint2 h = __ldg(reinterpret_cast<const uint2 *>(a.in) + v);
                    w[k] = make_uint4(h.x, h.y, 0u, 0u);
                }
            }
        }
    };
    u32 nlist = 0;   // listed voxels not yet evaluated (the same in every lane)
    uint4 w[G::VL], wn[G::VL];
    u32 c = claim();
    load_chunk(c, w);
    // with PF: the next chunk (its loads in flight while this one is used) and the
    // claim of the one after it, whose result is read only at the end of the step
    u32 cn = G::PF ? claim() : 0u;
    for (;;) {
        const bool done = c >= a.nchunks;
        u32 cnn = 0;
        if (!done) {
            if constexpr (G::PF) {
                load_chunk(cn, wn);
                if (lane == 0)
                    cnn = atomicAdd(a.counter, 1u);
            }
            static_assert(G::VL >= 1 && G::VL <= 8, "one pass bit per voxel of the lane's vectors");
            u64 word = 0;          // bit 8k + q: voxel 8 (chunk vector lane + 32 k) + q passes
#pragma unroll
            for (int k = 0; k < G::VL; ++k) {
                const u64 v = (u64)c * G::CVEC + lane + 32 * k;
                if (v < nvec) {
                    word |= (u64)pass_bits<T>(w[k], T_) << (8 * k);
#pragma unroll
                    for (int f = 0; f < 5; ++f)
                        if (gets<SET>(f) && a.out[f]) {
                            if (sizeof(T) == 2)
                                reinterpret_cast<uint4 *>(a.out[f])[v] = make_uint4(0u, 0u, 0u, 0u);
                            else
                                reinterpret_cast<uint2 *>(a.out[f])[v] = make_uint2(0u, 0u);
                        }
                } else if (v == nvec) {
                    // the last voxels (n not a multiple of 8), one by one
                    u32 bits = 0;
                    for (u32 q = 0; q < (u32)(a.n - nvec * 8); ++q) {
                        const u64 vi = nvec * 8 + q;
                        bits |= (ldgv<T>(in + vi) >= T_ ? 1u : 0u) << q;
                        for (int f = 0; f < 5; ++f)
                            if (gets<SET>(f) && a.out[f])
                                static_cast<T *>(a.out[f])[vi] = (T)0;
                    }
                    word |= (u64)bits << (8 * k);
                }
            }
            // the warp's list: an exclusive prefix sum of the lanes' counts
            const u32 cnt = (u32)__popcll(word);
            u32 incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const u32 t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d)
                    incl += t;
            }
            u32 pos = nlist + incl - cnt;
            while (word) {
                const int bit = __ffsll((long long)word) - 1;
                word &= word - 1ull;
                const u32 v = c * (u32)G::CVEC + (u32)lane + 32u * (u32)(bit >> 3);
                if (lnfdev::lnf_dbg_ok(pos < (u32)G::LCAP, a.err))
                    L[pos] = v * 8u + (u32)(bit & 7);
                ++pos;
            }
            nlist += __shfl_sync(0xFFFFFFFFu, incl, 31);
            __syncwarp();
        }
        const u32 neval = done ? nlist : (nlist & ~31u);
        for (u32 e = (u32)lane; e < neval; e += 32)
            if (lnfdev::lnf_dbg_ok(e < (u32)G::LCAP, a.err))
                eval_voxel(L[e]);
        __syncwarp();
        const u32 rest = nlist - neval;   // at most 31: to the front of the list
        u32 keep = 0;
        if ((u32)lane < rest && lnfdev::lnf_dbg_ok(neval + lane < (u32)G::LCAP, a.err))
            keep = L[neval + lane];
        __syncwarp();
        if ((u32)lane < rest)
            L[lane] = keep;
        __syncwarp();
        nlist = rest;
        if (done)
            break;
        if constexpr (G::PF) {
            c = cn;
            cn = __shfl_sync(0xFFFFFFFFu, cnn, 0);
#pragma unroll
            for (int k = 0; k < G::VL; ++k)
                w[k] = wn[k];
        } else {
            c = claim();
            load_chunk(c, w);
        }
    }

    // ---- histograms: the shared windows, and the zeros as N minus the nonzero outputs
    __syncthreads();
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        if (!(gets<SET>(f) && a.out[f] && a.hist[f]))
            continue;
        const u32 *h = hsh + oslot<SET>(f) * (kHistW / 2);
        for (int i = tid; i < kHistW / 2; i += kThreadsC) {
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
lnf_status gate_launch_t(lnf_ctx *ctx, const GateArgs &a0, cudaStream_t st)
{
    typedef GGeo<T, R, SET> G;
    GateArgs a = a0;
    a.nchunks = (u32)((a.n + G::CVOX - 1) / G::CVOX);
    if (cudaFuncSetAttribute(k_gate<T, R, SET>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM) !=
        cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "gate kernel: shared memory attribute (%d bytes)", G::SMEM);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gate<T, R, SET>, kThreadsC, G::SMEM);
    const int grid = std::max(1, std::min((int)((a.nchunks + kWarpsC - 1) / kWarpsC), ctx->num_sms * std::max(1, occ)));
    if (cudaMemsetAsync(a.counter, 0, sizeof(u32), st) != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "gate kernel: counter reset");
    k_gate<T, R, SET><<<grid, kThreadsC, G::SMEM, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? LNF_OK : lnf_fail(ctx, LNF_ECUDA, "gate kernel launch failed");
}

template <typename T, int SET>
lnf_status gate_by_radius(lnf_ctx *ctx, int radius, const GateArgs &a, cudaStream_t st)
{
    switch (radius) {
    case 1: return gate_launch_t<T, 1, SET>(ctx, a, st);
    case 2: return gate_launch_t<T, 2, SET>(ctx, a, st);
    case 3: return gate_launch_t<T, 3, SET>(ctx, a, st);
    default: return gate_launch_t<T, 4, SET>(ctx, a, st);
    }
}

// the local entropy filter at r = 1..2 (its cube's columns in shared memory
// bound the radius)
template <typename T>
lnf_status gate_eloc_by_radius(lnf_ctx *ctx, int radius, const GateArgs &a, cudaStream_t st)
{
    if (radius == 1)
        return gate_launch_t<T, 1, SET_ELOC>(ctx, a, st);
    return gate_launch_t<T, 2, SET_ELOC>(ctx, a, st);
}

// The gate kernel for one job (outs / hists by filter id; `eloc`: the entropy
// filter with the cube's own probabilities, its output in the entropy slot;
// `counter`: the chunk counter, null for the context's own).
template <typename T>
lnf_status gate_dispatch_t(lnf_ctx *ctx, const FilterJob &j, void *const outs[5], u64 *const hists[5],
                           cudaStream_t st, int *handled, bool eloc = false, u32 *counter = nullptr)
{
    const u64 n = (u64)j.nx * j.ny * j.nz;
    if (n >= (1ull << 32) || j.pitch != j.nx || reinterpret_cast<uintptr_t>(j.in) % 16 != 0)
        return LNF_OK;   // not handled: 32-bit voxel indices and dense aligned rows only
    for (int f = 0; f < 5; ++f)
        if (outs[f] && reinterpret_cast<uintptr_t>(outs[f]) % 16 != 0)
            return LNF_OK;
    GateArgs a;
    std::memset(&a, 0, sizeof a);
    a.in = j.in;
    for (int f = 0; f < 5; ++f) {
        a.out[f] = outs[f];
        a.hist[f] = outs[f] ? hists[f] : nullptr;
    }
    a.nx = j.nx;
    a.ny = j.ny;
    a.nz = j.nz;
    a.n = n;
    a.prm = j.prm;
    a.lut = j.lut;
    a.counter = counter ? counter : ctx->d_counter + 14;
    a.err = ctx->d_err;
    const bool ours = outs[LNF_OURS] != nullptr;
    const bool cube = outs[0] || outs[1] || outs[2] || outs[3];
    lnf_status s;
    if (eloc)
        s = (j.radius >= 1 && j.radius <= 2 && outs[LNF_ENTROPY] && !ours && !outs[0] && !outs[1] && !outs[3])
                ? gate_eloc_by_radius<T>(ctx, j.radius, a, st)
                : lnf_fail(ctx, LNF_EINVAL, "gate-first kernel: local entropy job not covered");
    else if (ours && cube)
        s = gate_by_radius<T, SET_ALL>(ctx, j.radius, a, st);
    else if (ours)
        s = gate_by_radius<T, SET_OURS>(ctx, j.radius, a, st);
    else
        s = gate_by_radius<T, SET_CUBE>(ctx, j.radius, a, st);
    if (s == LNF_OK)
        *handled = 1;
    return s;
}

}  // namespace gatek
