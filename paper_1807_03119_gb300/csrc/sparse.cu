// Gather kernels: the five filters on whole volumes where few voxels pass the
// noise gate.  Every filter outputs 0 unless the voxel's own value P0 >= T
// (Eq. 6/7 "0, otherwise"; the gate of Eq. 2-5), so only those voxels need
// their taps.  One pass streams the volume: each thread reads 8 voxels with one
// vector load, the warp lists the ones with P0 >= T in shared memory, then
// evaluates them one at a time with all 32 lanes -- each lane a few taps,
// read from global memory (the cube of a voxel is cached in L1 / L2 for its
// neighbours), a butterfly sum -- and each thread writes its 8 outputs with
// one vector store.  No plane ring, so many warps per SM hide the gathers.
// Taps of interior voxels are fixed offsets; voxels within the reach of the
// border clamp each coordinate.
//
// lnf_gather_mode (lnf_internal.cuh) decides on the device, from the count of
// passing voxels, whether this kernel or the plane-ring kernel of the same
// filter does the work; both are launched and the other returns at once.
#include "lnf_ctx.h"

namespace {

constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / 32;
constexpr int kVox = 8;                          // voxels per thread per pass
constexpr int kPass = kGThreads * kVox;          // voxels per block per pass
constexpr int kGHist = 4096;                     // shared histogram window (16-bit outputs)

// The taps of a filter at radius R: their count and the offset of tap t
// (d: the cluster offset of the paper's filter)
template <int R, int FILTER>
struct GTaps {
    static constexpr int M = 2 * R + 1;
    static constexpr int TAPS = FILTER == LNF_OKADA ? 6 * R + 1 : (FILTER == LNF_OURS ? 27 * M : M * M * M);
    static constexpr int PER_LANE = (TAPS + 31) / 32;
    static __device__ __forceinline__ void off(int t, int d, int &dx, int &dy, int &dz)
    {
        dx = dy = dz = 0;
        if (FILTER == LNF_OKADA) {   // the centre, then the arms (-x, +x, -y, +y, -z, +z) at 1..R
            if (t > 0) {
                const int arm = (t - 1) % 6, k = (t - 1) / 6 + 1;
                const int sg = (arm & 1) ? k : -k;
                dx = arm < 2 ? sg : 0;
                dy = arm == 2 || arm == 3 ? sg : 0;
                dz = arm >= 4 ? sg : 0;
            }
        } else if (FILTER == LNF_OURS) {   // 9 clusters x 3 lines x M voxels (Eq. 2-3)
            const int c = t / (3 * M), a = (t / M) % 3, k = t % M - R;
            if (c > 0) {
                dx = ((c - 1) & 1) ? d : -d;
                dy = ((c - 1) & 2) ? d : -d;
                dz = ((c - 1) & 4) ? d : -d;
            }
            dx += a == 0 ? k : 0;
            dy += a == 1 ? k : 0;
            dz += a == 2 ? k : 0;
        } else {   // the M^3 cube
            dx = t % M - R;
            dy = (t / M) % M - R;
            dz = t / (M * M) - R;
        }
    }
};

struct GatherArgs {
    const void *in;
    void *out;
    u32 nx, ny, nz, n;              // dims and voxel count (< 2^32)
    u32 plane;                      // nx * ny
    unsigned long long mx, mp;      // ceil(2^64 / nx), ceil(2^64 / plane): exact quotients of 32-bit indices
    int d;                          // cluster offset (the paper's filter)
    int reach;                      // largest tap offset per axis
    const DevParams *prm;
    const u32 *lut;
    u64 *out_hist;
};

template <typename T>
__device__ __forceinline__ u32 ldv(const T *p, u32 i)
{
    return (u32)__ldg(p + i);
}

template <typename T, int R, int FILTER>
__global__ void __launch_bounds__(kGThreads) k_gather(const GatherArgs a)
{
    typedef GTaps<R, FILTER> G;
    const DevParams &P = *a.prm;
    if (!lnf_gather_mode(P, FILTER))
        return;   // the plane-ring kernel of this filter does the work
    __shared__ u32 list[kGWarps][32 * kVox];    // per warp: its passing voxels' indices, then their outputs
    __shared__ u32 meta[kGWarps][32 * kVox];    // ... their values P0, bit 31 set for interior voxels
    __shared__ u32 hsh[kGHist];
    __shared__ u32 recip[G::TAPS + 1];          // ceil(2^32 / n): rounding of a mean over n taps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *in = static_cast<const T *>(a.in);
    T *out = static_cast<T *>(a.out);
    const u32 T_ = P.T;
    const u32 hbins = sizeof(T) == 1 ? 256u : (u32)kGHist;
    const u32 hbase = sizeof(T) == 1 ? 0u : max(T_, P.minv);   // nonzero outputs are >= T
    for (u32 i = threadIdx.x; i < hbins; i += blockDim.x)
        hsh[i] = 0;
    for (int i = threadIdx.x; i <= G::TAPS; i += blockDim.x)
        recip[i] = i <= 1 ? 0u : (u32)((0x100000000ull + i - 1) / i);
    __syncthreads();
    u32 written = 0, nonzero = 0;

    // the band of a centre value as (v - lo) <= width: sigma |v - P0| <= delta,
    // Okada |P0 - v| < td (td >= 1)
    const u32 dl = min(P.delta, 65535u);
    const long long td = P.td;
    const u32 hw = FILTER == LNF_SIGMA ? dl : (td > 65536 ? 65535u : (u32)(td - 1));
    // entropy filter: the threshold on the criterion (Eq. 7), default the
    // expectation over a cube of M^3 voxels
    long long te = P.te_cfg;
    if (FILTER == LNF_ENTROPY && te == -2)
        te = (long long)(((unsigned __int128)(G::M * G::M * G::M) * P.hw_sum) / P.N);
    // this lane's taps as offsets in the flat volume, for interior voxels (32-bit
    // when the plane is small enough; otherwise every voxel takes the clamped taps)
    const bool small = a.plane < (1u << 28);
    int toff[G::PER_LANE];
#pragma unroll
    for (int j = 0; j < G::PER_LANE; ++j) {
        int dx, dy, dz;
        G::off(lane + 32 * j < G::TAPS ? lane + 32 * j : 0, a.d, dx, dy, dz);
        toff[j] = small ? (dz * (int)a.plane + dy * (int)a.nx + dx) : 0;
    }
    const bool okada_none = FILTER == LNF_OKADA && td <= 0;   // Okada selects nothing: every output is 0
    const u32 rc = (u32)a.reach;

    // the taps of the voxel `idx` (value P0, interior or not) summed over the
    // warp: packed value and count (sigma, Okada), weights (entropy filter) or values
    auto taps = [&](u32 idx, u32 P0, bool inner, u32 &acc) {
        const u32 blo = P0 > hw ? P0 - hw : 0u, bwd = P0 - blo + hw;
        u32 x = 0, y = 0, z = 0;
        if (!inner) {
            z = a.plane == 1 ? idx : (u32)__umul64hi(idx, a.mp);
            const u32 rem = idx - z * a.plane;
            y = a.nx == 1 ? rem : (u32)__umul64hi(rem, a.mx);
            x = rem - y * a.nx;
        }
#pragma unroll
        for (int j = 0; j < G::PER_LANE; ++j) {
            const int t = lane + 32 * j;
            if (t >= G::TAPS)
                continue;
            u32 tv;
            if (inner) {
                tv = ldv(in, idx + (u32)toff[j]);
            } else {   // clamp to the volume's edge
                int dx, dy, dz;
                G::off(t, a.d, dx, dy, dz);
                const u32 xc = (u32)min(max((int)x + dx, 0), (int)a.nx - 1);
                const u32 yc = (u32)min(max((int)y + dy, 0), (int)a.ny - 1);
                const u32 zc = (u32)min(max((int)z + dz, 0), (int)a.nz - 1);
                tv = ldv(in, zc * a.plane + yc * a.nx + xc);
            }
            if (FILTER == LNF_SIGMA || FILTER == LNF_OKADA) {
                if (tv - blo <= bwd)
                    acc += (tv << 8) | 1u;   // value and count in one word (count < 256)
            } else if (FILTER == LNF_ENTROPY) {
                acc += __ldg(a.lut + tv);
            } else {
                acc += tv;
            }
        }
    };
    auto finish = [&](u32 acc, u32 P0) -> u32 {
        if (FILTER == LNF_SIGMA || FILTER == LNF_OKADA) {
            // round(sm / n) half up = (x * recip[n]) >> 32, x = sm + n / 2 (exact:
            // x < n 2^16 and recip n - 2^32 < n, n < 256)
            const u32 n = acc & 0xFFu, sm = acc >> 8;
            const u32 q = n == 1 ? sm : __umulhi(sm + (n >> 1), recip[n]);
            return (n && P0 >= T_ && (u64)sm >= (u64)n * T_) ? q : 0u;
        } else if (FILTER == LNF_ENTROPY) {
            return (P0 >= T_ && (long long)acc > te) ? P0 : 0u;
        } else {
            // mean (Eq. 4) over M^3, the paper's filter (Eq. 2-3) over 27 M line voxels:
            // round half up by a constant divisor
            constexpr u32 DEN = FILTER == LNF_OURS ? 27u * G::M : (u32)(G::M * G::M * G::M);
            return (P0 >= T_ && (u64)acc >= (u64)DEN * T_) ? (2u * acc + DEN) / (2u * DEN) : 0u;
        }
    };

    for (u64 base = (u64)blockIdx.x * kPass; base < a.n; base += (u64)gridDim.x * kPass) {
        // (64-bit: the pass start never wraps; every voxel index is below 2^32)
        const u64 i0w = base + (u64)threadIdx.x * kVox;
        const u32 i0 = (u32)min(i0w, (u64)a.n);
        u32 v[kVox];
        const bool full = i0w + kVox <= a.n;
        if (full) {
            if (sizeof(T) == 2) {
                const uint4 w = __ldg(reinterpret_cast<const uint4 *>(in + i0));
                const u32 ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    v[2 * k] = ww[k] & 0xFFFFu;
                    v[2 * k + 1] = ww[k] >> 16;
                }
            } else {
                const uint2 w = __ldg(reinterpret_cast<const uint2 *>(in + i0));
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    v[k] = (w.x >> (8 * k)) & 0xFFu;
                    v[4 + k] = (w.y >> (8 * k)) & 0xFFu;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < kVox; ++k)
                v[k] = i0w + k < a.n ? ldv(in, i0 + k) : 0u;
        }
        u32 cm = 0;
#pragma unroll
        for (int k = 0; k < kVox; ++k)
            if (v[k] >= T_ && i0w + k < a.n)
                cm |= 1u << k;
        if (okada_none)
            cm = 0;
        const u32 cnt = (u32)__popc(cm);
        u32 incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o)
                incl += t;
        }
        const u32 cw = __shfl_sync(0xFFFFFFFFu, incl, 31);
        u32 o[kVox];
#pragma unroll
        for (int k = 0; k < kVox; ++k)
            o[k] = 0u;
        if (cw) {
            u32 *lst = list[warp], *mt = meta[warp];
            if (cm) {   // the owner lists its voxels with their values and whether their taps stay inside
                const u32 z = a.plane == 1 ? i0 : (u32)__umul64hi(i0, a.mp);
                const u32 rem = i0 - z * a.plane;
                const u32 y = a.nx == 1 ? rem : (u32)__umul64hi(rem, a.mx);
                const u32 x = rem - y * a.nx;
                const bool yz_in = small && y >= rc && y + rc < a.ny && z >= rc && z + rc < a.nz;
                u32 m = cm, pos = incl - cnt;
                while (m) {
                    const int k = __ffs(m) - 1;
                    m &= m - 1;
                    // the 8 voxels of a pass may run past the row's end: the x of voxel
                    // k is x + k only while it stays in the row
                    const bool inner = yz_in && x + k < a.nx && x + k >= rc && x + k + rc < a.nx;
                    lst[pos] = i0 + k;
                    mt[pos] = v[k] | (inner ? 0x80000000u : 0u);
                    ++pos;
                }
            }
            __syncwarp();
            // two voxels at a time: independent loads and sums overlap
            for (u32 c = 0; c < cw; c += 2) {
                const bool two = c + 1 < cw;
                const u32 idx0 = lst[c], m0 = mt[c];
                const u32 idx1 = two ? lst[c + 1] : idx0, m1 = two ? mt[c + 1] : m0;
                u32 acc0 = 0, acc1 = 0;
                taps(idx0, m0 & 0xFFFFu, (m0 >> 31) != 0, acc0);
                if (two)
                    taps(idx1, m1 & 0xFFFFu, (m1 >> 31) != 0, acc1);
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    acc0 += __shfl_xor_sync(0xFFFFFFFFu, acc0, s);
                    acc1 += __shfl_xor_sync(0xFFFFFFFFu, acc1, s);
                }
                if (lane == 0)
                    lst[c] = finish(acc0, m0 & 0xFFFFu);   // the output replaces the entry
                if (lane == 1 && two)
                    lst[c + 1] = finish(acc1, m1 & 0xFFFFu);
            }
            __syncwarp();
            u32 m = cm, pos = incl - cnt;
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                const u32 f = lst[pos++];
#pragma unroll
                for (int q = 0; q < kVox; ++q)
                    o[q] = q == k ? f : o[q];
            }
            __syncwarp();   // the list is refilled at the next pass
        }
        if (full) {
            if (sizeof(T) == 2)
                __stcs(reinterpret_cast<uint4 *>(out + i0),
                       make_uint4(o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16), o[6] | (o[7] << 16)));
            else
                __stcs(reinterpret_cast<uint2 *>(out + i0),
                       make_uint2(o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24),
                                  o[4] | (o[5] << 8) | (o[6] << 16) | (o[7] << 24)));
            written += kVox;
        } else {
#pragma unroll
            for (int k = 0; k < kVox; ++k)
                if (i0w + k < a.n) {
                    out[i0 + k] = (T)o[k];
                    ++written;
                }
        }
        if (a.out_hist && cm) {   // nonzero outputs come only from listed voxels
#pragma unroll
            for (int k = 0; k < kVox; ++k)
                if (o[k]) {
                    ++nonzero;
                    const u32 b = o[k] - hbase;
                    if (b < hbins)
                        atomicAdd(&hsh[b], 1u);
                    else if (o[k] < 65536u)   // always true for valid outputs
                        atomicAdd(&a.out_hist[o[k]], 1ull);
                }
        }
    }
    if (a.out_hist) {
        __syncthreads();
        for (u32 i = threadIdx.x; i < hbins; i += blockDim.x)
            if (hsh[i])
                atomicAdd(&a.out_hist[hbase + i], (u64)hsh[i]);
        u32 zeros = written - nonzero;
        for (int s = 16; s > 0; s >>= 1)
            zeros += __shfl_xor_sync(0xFFFFFFFFu, zeros, s);
        if (lane == 0 && zeros)
            atomicAdd(&a.out_hist[0], (u64)zeros);
    }
}

template <typename T, int R, int FILTER>
lnf_status launch_gather(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st)
{
    GatherArgs a;
    a.in = j.in;
    a.out = j.out;
    a.nx = (u32)j.nx;
    a.ny = (u32)j.ny;
    a.nz = (u32)j.nz;
    a.plane = a.nx * a.ny;
    a.n = a.plane * a.nz;
    // ceil(2^64 / D) for D >= 2 (a divisor of 1 is taken apart in the kernel)
    auto magic = [](u32 D) { return D <= 1 ? 0ull : ~0ull / D + 1ull; };
    a.mx = magic(a.nx);
    a.mp = magic(a.plane);
    a.d = j.offset;
    a.reach = FILTER == LNF_OURS ? R + j.offset : R;
    a.prm = j.prm;
    a.lut = j.lut;
    a.out_hist = j.out_hist;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gather<T, R, FILTER>, kGThreads, 0);
    if (occ < 1)
        occ = 1;
    const u32 passes = (a.n + kPass - 1) / kPass;
    const int grid = (int)std::min<u32>(passes, (u32)(ctx->num_sms * occ));
    k_gather<T, R, FILTER><<<grid, kGThreads, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "gather kernel launch failed");
    return LNF_OK;
}

template <typename T, int R>
lnf_status by_filter(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st)
{
    switch (j.filter) {
    case LNF_MEAN: return launch_gather<T, R, LNF_MEAN>(ctx, j, st);
    case LNF_SIGMA: return launch_gather<T, R, LNF_SIGMA>(ctx, j, st);
    case LNF_ENTROPY: return launch_gather<T, R, LNF_ENTROPY>(ctx, j, st);
    case LNF_OKADA: return launch_gather<T, R, LNF_OKADA>(ctx, j, st);
    default: return launch_gather<T, R, LNF_OURS>(ctx, j, st);
    }
}

}  // namespace

bool lnf_gather_covers(const FilterJob &j)
{
    const bool whole = !(j.ox || j.oy || j.oz || j.bx != j.nx || j.by != j.ny || j.bz != j.nz);
    const size_t es = j.dtype == LNF_U8 ? 1 : 2;
    return whole && !j.aniso && j.filter >= LNF_MEAN && j.filter <= LNF_OURS && j.radius >= 1 && j.radius <= 2 &&
           j.pitch == j.nx && reinterpret_cast<uintptr_t>(j.in) % (8 * es) == 0 &&
           reinterpret_cast<uintptr_t>(j.out) % (8 * es) == 0;
}

lnf_status lnf_gather_launch(lnf_ctx *ctx, const FilterJob &j, cudaStream_t st)
{
    if (j.dtype == LNF_U8)
        return j.radius == 1 ? by_filter<uint8_t, 1>(ctx, j, st) : by_filter<uint8_t, 2>(ctx, j, st);
    return j.radius == 1 ? by_filter<uint16_t, 1>(ctx, j, st) : by_filter<uint16_t, 2>(ctx, j, st);
}
