// Statistics pre-pass and parameter derivation, on the device.
//
//   k_stats   : one read of the volume -> grey-level histogram h[v] (the
//               "normalized frequency distribution" the entropy filter
//               precomputes, section "Entropy Filter", and all the Otsu
//               threshold, Eq. 1, and the global sigma of the sigma filter,
//               Eq. 5, need: S = sum v h[v], Q = sum v^2 h[v], min and max
//               are taken from it).
//   k_param_totals / k_params : per chunk of 256 levels, then the last chunk
//               -> Otsu threshold T (Eq. 1) in exact integer arithmetic, sigma
//               band delta, Okada T_d, the fixed-point entropy weights w[v] of
//               Eq. 7, and the input image entropy.
//   k_entropy : image entropy H = -sum (c/N) log2(c/N) of a histogram (the
//               measure of the paper's Fig. 4), FP64 only in this reduction.
#include "lnf_internal.cuh"

typedef unsigned __int128 u128;
typedef __int128 i128;

namespace {

constexpr int kStatsThreads = 1024;
// CTA histograms in shared memory, laid out so that the lanes of a warp rarely
// meet in one bank (random grey levels otherwise collide about 3-4 deep):
//   8-bit  : one copy of the 256 bins per lane, bin v of lane L at word 32 v + L
//            (its own bank: no conflicts within a warp);
//   16-bit, chosen per CTA from the vectors its threads stream first:
//     low  : (7/8 of them hold only levels below 4096: 12-bit data) eight copies
//            of the levels v < 4096, bin v of lane group g = L % 8 at word
//            8 v + g (bank 8 (v % 4) + g); levels above to the global histogram;
//     wide : one copy of the levels v < 32768; levels above to the global
//            histogram.
// Both 16-bit layouts take 128 KB, which leaves L1 room for the loads in
// flight (larger CTA histograms measured slower).
constexpr int kLaneCopiesU8 = 32;
constexpr int kLowBinsU16 = 4096;
constexpr int kLowCopiesU16 = 8;
constexpr int kWideBinsU16 = 32768;
constexpr int kSmemWordsU8 = LNF_LEVELS_U8 * kLaneCopiesU8;
constexpr int kSmemWordsU16 = kWideBinsU16;
static_assert(kLowBinsU16 * kLowCopiesU16 == kSmemWordsU16, "both 16-bit layouts fill the same words");

// ------------------------------------------------------------------ init

__global__ void k_stats_init(u64 *hist, u32 levels, DevStats *st, u64 n)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < levels; i += gridDim.x * blockDim.x)
        hist[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->N = n;
        st->levels = levels;
        st->pad = 0;
    }
}

__global__ void k_stats_init_batched(const __grid_constant__ StatsPack pk)
{
    const StatsJob &j = pk.jobs[blockIdx.y];
    u32 levels = j.dtype == 0 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < levels; i += gridDim.x * blockDim.x)
        j.hist[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        DevStats *st = j.st;
        st->N = j.n;
        st->levels = levels;
        st->pad = 0;
    }
}

__global__ void k_zero(u64 *p, u64 count)
{
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < count; i += (u64)gridDim.x * blockDim.x)
        p[i] = 0;
}

// ------------------------------------------------------------------ stats

// one grey level into the CTA's histogram.  8-bit: word 32 v + lane.  16-bit:
// levels below `lim` to word v mul + lw (low layout: mul = 8, lw = L % 8,
// lim = 4096; wide layout: mul = 1, lw = 0, lim = 32768), the rest to the
// global histogram.
template <typename T>
__device__ __forceinline__ void stats_value(u32 v, u32 *sh, u32 lw, u32 mul, u32 lim, u64 *hist)
{
    if (sizeof(T) == 1) {
        atomicAdd(&sh[v * kLaneCopiesU8 + lw], 1u);
    } else if (v < lim) {
        atomicAdd(&sh[v * mul + lw], 1u);
    } else {
        atomicAdd(&hist[v], 1ull);
    }
}

template <typename T>
__device__ void stats_body(const T *vol, u64 n, u64 *hist, u64 cta, u64 nctas, u32 *sh)
{
    const u64 gtid = cta * blockDim.x + threadIdx.x;
    const u64 gsz = nctas * blockDim.x;
    // elements before the first 16-byte boundary
    u64 head = ((16 - (reinterpret_cast<uintptr_t>(vol) & 15)) & 15) / sizeof(T);
    if (head > n)
        head = n;
    const u64 nv = (n - head) * sizeof(T) / 16;
    const int words = sizeof(T) == 1 ? kSmemWordsU8 : kSmemWordsU16;
    for (int i = threadIdx.x; i < words; i += blockDim.x)
        sh[i] = 0;
    // 16-bit: the layout from the vector each thread streams first (contiguous
    // over the grid, so the sample costs no scattered reads; a thread without
    // one counts as low): low where 7/8 of the CTA's threads saw only levels
    // below 4096.  The count is also the barrier after the zeroing.
    bool lo = true;
    if (sizeof(T) == 2 && gtid < nv) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(vol + head) + gtid);
        lo = ((q.x | q.y | q.z | q.w) & 0xF000F000u) == 0u;
    }
    const bool low = __syncthreads_count(lo) * 8 >= (int)blockDim.x * 7;
    const u32 lane = threadIdx.x & 31;
    const u32 lw = sizeof(T) == 1 ? lane : (low ? lane % kLowCopiesU16 : 0u);
    const u32 mul = low ? (u32)kLowCopiesU16 : 1u;
    const u32 lim = low ? (u32)kLowBinsU16 : (u32)kWideBinsU16;

    for (u64 i = gtid; i < head; i += gsz)
        stats_value<T>(vol[i], sh, lw, mul, lim, hist);
    const uint4 *v4 = reinterpret_cast<const uint4 *>(vol + head);
    // four independent 16-byte loads in flight per thread before any is consumed
    constexpr int kU = 4;
    for (u64 i = gtid; i < nv; i += kU * gsz) {
        uint4 w[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const u64 j = i + u * gsz;
            w[u] = j < nv ? __ldcs(v4 + j) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (i + u * gsz >= nv)
                break;
            const u32 words4[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (sizeof(T) == 1) {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        stats_value<T>((words4[k] >> (8 * b)) & 0xFFu, sh, lw, mul, lim, hist);
                } else {
                    stats_value<T>(words4[k] & 0xFFFFu, sh, lw, mul, lim, hist);
                    stats_value<T>(words4[k] >> 16, sh, lw, mul, lim, hist);
                }
            }
        }
    }
    for (u64 i = head + nv * (16 / sizeof(T)) + gtid; i < n; i += gsz)
        stats_value<T>(vol[i], sh, lw, mul, lim, hist);
    __syncthreads();
    // the copies of each level added up, one global atomic per occupied level
    if (sizeof(T) == 1) {
        for (int v = threadIdx.x; v < LNF_LEVELS_U8; v += blockDim.x) {
            u32 c = 0;
            for (int r = 0; r < kLaneCopiesU8; ++r)
                c += sh[v * kLaneCopiesU8 + ((r + v) & 31)];
            if (c)
                atomicAdd(&hist[v], (u64)c);
        }
    } else {
        for (u32 v = threadIdx.x; v < lim; v += blockDim.x) {
            u32 c = 0;
            for (u32 r = 0; r < mul; ++r)
                c += sh[v * mul + r];
            if (c)
                atomicAdd(&hist[v], (u64)c);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kStatsThreads) k_stats(const T *vol, u64 n, u64 *hist)
{
    extern __shared__ u32 smem[];
    stats_body<T>(vol, n, hist, blockIdx.x, gridDim.x, smem);
}

__global__ void __launch_bounds__(kStatsThreads) k_stats_batched(const __grid_constant__ StatsPack pk)
{
    extern __shared__ u32 smem[];
    const StatsJob &j = pk.jobs[blockIdx.y];
    if (j.dtype == 0)
        stats_body<uint8_t>(static_cast<const uint8_t *>(j.vol), j.n, j.hist, blockIdx.x, gridDim.x, smem);
    else
        stats_body<uint16_t>(static_cast<const uint16_t *>(j.vol), j.n, j.hist, blockIdx.x, gridDim.x, smem);
}

// ------------------------------------------------------------------ exact helpers

// floor(sqrt(x)) for x < 2^112: an FP64 estimate, then exact integer correction
__device__ u64 isqrt_u128(u128 x)
{
    const double xd = (double)(u64)(x >> 64) * 18446744073709551616.0 + (double)(u64)x;
    u64 r = (u64)sqrt(xd);
    while (r > 0 && (u128)r * r > x)
        --r;
    while ((u128)(r + 1) * (r + 1) <= x)
        ++r;
    return r;
}

// Binary logarithm of x >= 1 in fixed point with 40 fractional bits, by the
// classical repeated-squaring method: x = 2^k m with m in [1,2) held with 62
// fractional bits; each squaring (truncated to 62 fractional bits) that
// reaches 2 yields a 1 bit and is halved.
__device__ u64 log2_fixed40(u64 x)
{
    const int k = 63 - __clzll(x);
    u64 m = k <= 62 ? (x << (62 - k)) : (x >> (k - 62));
    u64 res = (u64)k << 40;
    for (int i = 1; i <= 40; ++i) {
        const u64 lo = m * m;
        const u64 hi = __umul64hi(m, m);
        m = (hi << 2) | (lo >> 62);
        if (m >= (1ull << 63)) {
            m >>= 1;
            res |= 1ull << (40 - i);
        }
    }
    return res;
}

// J(t) = S0^2/n0 + S1^2/n1 split as q + fnum/fden with fnum/fden in [0, 2).
struct OtsuJ {
    u128 q;
    u64 fnum, fden;
    u32 t;          // 0 = no candidate
};

__device__ __forceinline__ OtsuJ otsu_j(u64 n0, u64 s0, u64 N, u64 S, u32 t)
{
    const u64 n1 = N - n0, s1 = S - s0;
    const u128 a = (u128)s0 * s0, b = (u128)s1 * s1;
    const u128 q0 = a / n0, q1 = b / n1;
    const u64 r0 = (u64)(a - q0 * n0), r1 = (u64)(b - q1 * n1);
    OtsuJ j;
    j.q = q0 + q1;
    j.fnum = r0 * n1 + r1 * n0;   // < 2 n0 n1 <= 2^63
    j.fden = n0 * n1;             // <= N^2/4 < 2^62
    j.t = t;
    return j;
}

// sign(J_a - J_b), exactly
__device__ __forceinline__ int otsu_cmp(const OtsuJ &a, const OtsuJ &b)
{
    const i128 dq = (i128)a.q - (i128)b.q;
    if (dq >= 2)
        return 1;
    if (dq <= -2)
        return -1;
    const i128 x = dq * (i128)a.fden * (i128)b.fden + (i128)a.fnum * (i128)b.fden - (i128)b.fnum * (i128)a.fden;
    return x > 0 ? 1 : (x < 0 ? -1 : 0);
}

// better = larger J; equal J -> smaller t; t == 0 never wins
__device__ __forceinline__ bool otsu_better(const OtsuJ &a, const OtsuJ &b)
{
    if (a.t == 0)
        return false;
    if (b.t == 0)
        return true;
    int c = otsu_cmp(a, b);
    return c > 0 || (c == 0 && a.t < b.t);
}

// ---- parameter derivation over chunks of 256 grey levels, one level per
// thread (a 16-bit histogram has 256 chunks, an 8-bit one a single chunk): the
// exact per-level work (128-bit Otsu quotients, the fixed-point logarithm)
// runs on as many threads as there are levels
constexpr int kChunk = 256;
constexpr int kPThreads = 256;

struct ParamPartial {          // one per chunk
    u128 q;                    // best Otsu candidate of the chunk (see OtsuJ)
    u64 fnum, fden;
    u32 t, pad;
    u64 hw;                    // sum of h[v] w[v] over the chunk
    double H;                  // sum of -p log2 p over the chunk
};

struct ParamScratch {
    u64 tot_n[LNF_LEVELS_U16 / kChunk];   // per chunk: sum h[v]
    u64 tot_s[LNF_LEVELS_U16 / kChunk];   //            sum v h[v]
    u64 tot_q[LNF_LEVELS_U16 / kChunk];   //            sum v^2 h[v]
    u32 lo[LNF_LEVELS_U16 / kChunk];      //            first occupied level (0xFFFFFFFF: none)
    u32 hi[LNF_LEVELS_U16 / kChunk];      //            last occupied level (0: none)
    ParamPartial part[LNF_LEVELS_U16 / kChunk];
    u32 done;                  // chunks finished (reset by the last one)
    u32 pad[3];
};

__device__ __forceinline__ int n_chunks(u32 levels) { return (int)((levels + kChunk - 1) / kChunk); }

// pass 1: per chunk, the count, sum and sum of squares of its levels and its
// first and last occupied level
__device__ void chunk_totals(const u64 *hist, u32 levels, ParamScratch *ps, int c)
{
    __shared__ u64 rn[kPThreads / 32], rs[kPThreads / 32], rq[kPThreads / 32];
    __shared__ u32 rlo[kPThreads / 32], rhi[kPThreads / 32];
    u64 n = 0, s = 0, q = 0;
    u32 lo = 0xFFFFFFFFu, hi = 0;
    for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
        const u32 v = c * kChunk + i;
        if (v < levels) {
            const u64 h = hist[v];
            n += h;
            s += h * v;
            q += h * ((u64)v * v);
            if (h) {
                lo = min(lo, v);
                hi = max(hi, v);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        rn[threadIdx.x >> 5] = n;
        rs[threadIdx.x >> 5] = s;
        rq[threadIdx.x >> 5] = q;
        rlo[threadIdx.x >> 5] = lo;
        rhi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 tn = 0, ts = 0, tq = 0;
        u32 tlo = 0xFFFFFFFFu, thi = 0;
        for (int w = 0; w < kPThreads / 32; ++w) {
            tn += rn[w];
            ts += rs[w];
            tq += rq[w];
            tlo = min(tlo, rlo[w]);
            thi = max(thi, rhi[w]);
        }
        ps->tot_n[c] = tn;
        ps->tot_s[c] = ts;
        ps->tot_q[c] = tq;
        ps->lo[c] = tlo;
        ps->hi[c] = thi;
    }
}

struct PSmem {
    u64 h[kChunk];
    u64 pn[kPThreads], ps[kPThreads], pq[kPThreads];
    u32 plo[kPThreads], phi[kPThreads];
    u128 q[kPThreads];
    u64 fnum[kPThreads], fden[kPThreads];
    u32 t[kPThreads];
    u64 hw[kPThreads];
    double d[kPThreads];
    int last;
};

// pass 2: per chunk, the Otsu candidates, the weights and partial sums; the
// last chunk to finish reduces all chunks and writes the parameter block.
__device__ void chunk_params(const u64 *hist, const DevStats *st, const ParamCfg &cfg, DevParams *prm, u32 *lut,
                             ParamScratch *ps, int c, PSmem &sm)
{
    const int tid = threadIdx.x;
    const u32 L = st->levels;
    const u64 N = st->N;
    const int nc = n_chunks(L);
    // prefix of the chunks before this one (c < kPThreads: one total per thread),
    // and the whole volume's S = sum P, Q = sum P^2, min and max over all chunks
    u64 n0 = 0, s0 = 0, S = 0, Q = 0;
    u32 minv = 0xFFFFFFFFu, maxv = 0;
    {
        u64 an = 0, as = 0, ss = 0, sq = 0;
        u32 mn = 0xFFFFFFFFu, mx = 0;
        for (int k = tid; k < nc; k += blockDim.x) {
            if (k < c) {
                an += ps->tot_n[k];
                as += ps->tot_s[k];
            }
            ss += ps->tot_s[k];
            sq += ps->tot_q[k];
            mn = min(mn, ps->lo[k]);
            mx = max(mx, ps->hi[k]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            an += __shfl_xor_sync(0xFFFFFFFFu, an, o);
            as += __shfl_xor_sync(0xFFFFFFFFu, as, o);
            ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
            sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
            mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        }
        if ((tid & 31) == 0) {
            sm.pn[tid >> 5] = an;
            sm.ps[tid >> 5] = as;
            sm.pq[tid >> 5] = sq;
            sm.hw[tid >> 5] = ss;
            sm.plo[tid >> 5] = mn;
            sm.phi[tid >> 5] = mx;
        }
        __syncthreads();
        for (int w = 0; w < kPThreads / 32; ++w) {
            n0 += sm.pn[w];
            s0 += sm.ps[w];
            S += sm.hw[w];
            Q += sm.pq[w];
            minv = min(minv, sm.plo[w]);
            maxv = max(maxv, sm.phi[w]);
        }
        __syncthreads();
    }
    for (int i = tid; i < kChunk; i += blockDim.x) {
        const u32 v = c * kChunk + i;
        sm.h[i] = v < L ? hist[v] : 0ull;
    }
    __syncthreads();
    // each thread owns 4 consecutive levels of the chunk
    constexpr int PER = kChunk / kPThreads;
    u64 ln = 0, ls = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const u32 v = c * kChunk + tid * PER + k;
        ln += sm.h[tid * PER + k];
        ls += sm.h[tid * PER + k] * v;
    }
    sm.pn[tid] = ln;
    sm.ps[tid] = ls;
    __syncthreads();
    for (int off = 1; off < kPThreads; off <<= 1) {
        u64 an = 0, as = 0;
        if (tid >= off) {
            an = sm.pn[tid - off];
            as = sm.ps[tid - off];
        }
        __syncthreads();
        sm.pn[tid] += an;
        sm.ps[tid] += as;
        __syncthreads();
    }
    u64 cn = n0 + sm.pn[tid] - ln, cs = s0 + sm.ps[tid] - ls;
    // Otsu (Eq. 1) candidates t = v + 1 at occupied levels v
    OtsuJ best;
    best.t = 0;
    best.q = 0;
    best.fnum = 0;
    best.fden = 1;
    const u64 lgN = log2_fixed40(N);
    u64 hw = 0;
    double hsum = 0.0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const u32 v = c * kChunk + tid * PER + k;
        const u64 h = sm.h[tid * PER + k];
        cn += h;
        cs += h * v;
        u32 w = 0;
        if (h) {
            if (v + 1 <= L - 1 && cn != N) {
                OtsuJ j = otsu_j(cn, cs, N, S, v + 1);
                if (otsu_better(j, best))
                    best = j;
            }
            // entropy weight (Eq. 7, fixed point) and the Shannon term
            const u64 D = lgN - log2_fixed40(h);
            const u128 num = (((u128)h * D) << 22) + ((u128)N << 39);
            w = (u32)(num / ((u128)N << 40));
            const double p = (double)h / (double)N;
            hsum += -p * log2(p);
        }
        if (v < L)
            lut[v] = w;
        hw += h * (u64)w;
    }
    sm.q[tid] = best.q;
    sm.fnum[tid] = best.fnum;
    sm.fden[tid] = best.fden;
    sm.t[tid] = best.t;
    sm.hw[tid] = hw;
    sm.d[tid] = hsum;
    __syncthreads();
    for (int off = kPThreads / 2; off > 0; off >>= 1) {
        if (tid < off) {
            OtsuJ a{sm.q[tid], sm.fnum[tid], sm.fden[tid], sm.t[tid]};
            OtsuJ b{sm.q[tid + off], sm.fnum[tid + off], sm.fden[tid + off], sm.t[tid + off]};
            if (otsu_better(b, a)) {
                sm.q[tid] = b.q;
                sm.fnum[tid] = b.fnum;
                sm.fden[tid] = b.fden;
                sm.t[tid] = b.t;
            }
            sm.hw[tid] += sm.hw[tid + off];
            sm.d[tid] += sm.d[tid + off];
        }
        __syncthreads();
    }
    if (tid == 0) {
        ParamPartial &pp = ps->part[c];
        pp.q = sm.q[0];
        pp.fnum = sm.fnum[0];
        pp.fden = sm.fden[0];
        pp.t = sm.t[0];
        pp.hw = sm.hw[0];
        pp.H = sm.d[0];
        __threadfence();
        const u32 ticket = atomicAdd(&ps->done, 1u);
        sm.last = ticket == (u32)nc - 1;
    }
    __syncthreads();
    if (!sm.last)
        return;
    // the last chunk: reduce the chunks (tree over the CTA, exact comparisons)
    __threadfence();
    {
        OtsuJ j;
        j.t = 0;
        j.q = 0;
        j.fnum = 0;
        j.fden = 1;
        u64 hwp = 0;
        double Hp = 0.0;
        if (tid < nc) {
            // written by other CTAs of this launch: read past L1
            const ParamPartial *pp = &ps->part[tid];
            const u64 *q64 = reinterpret_cast<const u64 *>(&pp->q);
            j.q = ((u128)__ldcg(q64 + 1) << 64) | (u128)__ldcg(q64);
            j.fnum = __ldcg(&pp->fnum);
            j.fden = __ldcg(&pp->fden);
            j.t = __ldcg(&pp->t);
            hwp = __ldcg(&pp->hw);
            Hp = __ldcg(&pp->H);
        }
        __syncthreads();
        sm.q[tid] = j.q;
        sm.fnum[tid] = j.fnum;
        sm.fden[tid] = j.fden;
        sm.t[tid] = j.t;
        sm.hw[tid] = hwp;
        sm.d[tid] = Hp;
        __syncthreads();
        for (int off = kPThreads / 2; off > 0; off >>= 1) {
            if (tid < off) {
                OtsuJ a{sm.q[tid], sm.fnum[tid], sm.fden[tid], sm.t[tid]};
                OtsuJ b2{sm.q[tid + off], sm.fnum[tid + off], sm.fden[tid + off], sm.t[tid + off]};
                if (otsu_better(b2, a)) {
                    sm.q[tid] = b2.q;
                    sm.fnum[tid] = b2.fnum;
                    sm.fden[tid] = b2.fden;
                    sm.t[tid] = b2.t;
                }
                sm.hw[tid] += sm.hw[tid + off];
                sm.d[tid] += sm.d[tid + off];
            }
            __syncthreads();
        }
    }
    // the gate threshold, and how many voxels pass it: the chunks above T's
    // chunk whole, then the levels of T's own chunk from T up
    const u32 t_best = sm.t[0];
    const u64 hws = sm.hw[0];
    const double Hs = sm.d[0];
    const u32 T_gate = cfg.threshold_mode == 0 ? (t_best ? t_best : minv)
                                               : (cfg.threshold_mode == 1 ? cfg.threshold_value : 0u);
    {
        const int cT = (int)(T_gate / kChunk);
        u64 np = 0;
        for (int cc = tid; cc < nc; cc += blockDim.x)
            if (cc > cT)
                np += __ldcg(&ps->tot_n[cc]);
        for (u32 v = (u32)cT * kChunk + tid; v < min((u32)(cT + 1) * kChunk, L); v += blockDim.x)
            if (v >= T_gate)
                np += hist[v];
        __syncthreads();
        sm.hw[tid] = np;
        __syncthreads();
        for (int off = kPThreads / 2; off > 0; off >>= 1) {
            if (tid < off)
                sm.hw[tid] += sm.hw[tid + off];
            __syncthreads();
        }
    }
    if (tid != 0)
        return;
    OtsuJ b;
    b.t = t_best;
    ps->done = 0;
    const u32 t_otsu = b.t ? b.t : minv;   // single level: T = that level
    const u128 var_num = (u128)N * Q - (u128)S * S;   // N^2 sigma^2
    const u128 nn = (u128)N * N;
    const u128 k2 = (u128)cfg.sigma_k * (u128)cfg.sigma_k;
    const u64 delta = isqrt_u128((k2 * var_num) / nn);
    const u64 sig = isqrt_u128(var_num / nn);
    DevParams p;
    p.N = N;
    p.S = S;
    p.Q = Q;
    p.minv = minv;
    p.maxv = maxv;
    p.T = cfg.threshold_mode == 0 ? t_otsu : (cfg.threshold_mode == 1 ? cfg.threshold_value : 0u);
    p.delta = delta > 0xFFFFFFFFull ? 0xFFFFFFFFu : (u32)delta;
    p.td = cfg.okada_td >= 0 ? cfg.okada_td : (long long)(sig + 1);
    p.hw_sum = hws;
    p.te_cfg = cfg.entropy_te;
    p.levels = L;
    p.valid = 1;
    p.H_in = Hs;
    p.sigma_k = (u32)cfg.sigma_k;
    p.pad = 0;
    p.n_pass = sm.hw[0];
    p.lte_cfg = cfg.entropy_local_te;
    p.lt = cfg.lt;
    *prm = p;
}

__global__ void __launch_bounds__(kPThreads) k_param_totals(const u64 *hist, const DevStats *st, ParamScratch *ps)
{
    if ((int)blockIdx.x < n_chunks(st->levels))
        chunk_totals(hist, st->levels, ps, blockIdx.x);
}

__global__ void __launch_bounds__(kPThreads) k_params(const u64 *hist, const DevStats *st, ParamCfg cfg,
                                                      DevParams *prm, u32 *lut, ParamScratch *ps)
{
    __shared__ PSmem sm;
    if ((int)blockIdx.x < n_chunks(st->levels))
        chunk_params(hist, st, cfg, prm, lut, ps, blockIdx.x, sm);
}

__global__ void __launch_bounds__(kPThreads) k_param_totals_batched(const __grid_constant__ StatsPack pk)
{
    const StatsJob &j = pk.jobs[blockIdx.y];
    const u32 levels = j.dtype == 0 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
    if ((int)blockIdx.x < n_chunks(levels))
        chunk_totals(j.hist, levels, reinterpret_cast<ParamScratch *>(j.pscr), blockIdx.x);
}

__global__ void __launch_bounds__(kPThreads) k_params_batched(const __grid_constant__ StatsPack pk, ParamCfg cfg)
{
    __shared__ PSmem sm;
    const StatsJob &j = pk.jobs[blockIdx.y];
    const u32 levels = j.dtype == 0 ? LNF_LEVELS_U8 : LNF_LEVELS_U16;
    if ((int)blockIdx.x < n_chunks(levels))
        chunk_params(j.hist, j.st, cfg, j.prm, j.lut, reinterpret_cast<ParamScratch *>(j.pscr), blockIdx.x, sm);
}

// ------------------------------------------------------------------ entropy

__device__ void entropy_body(const u64 *hist, u32 levels, u64 n, double *H, double *sd)
{
    const int tid = threadIdx.x;
    double acc = 0.0;
    const double Nd = (double)n;
    for (u32 v = tid; v < levels; v += blockDim.x) {
        const u64 c = hist[v];
        if (c) {
            const double p = (double)c / Nd;
            acc += -p * log2(p);
        }
    }
    sd[tid] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (tid < off)
            sd[tid] += sd[tid + off];
        __syncthreads();
    }
    if (tid == 0)
        *H = sd[0];
}

__global__ void __launch_bounds__(1024) k_entropy(const u64 *hist, u32 levels, u64 n, double *H)
{
    __shared__ double sd[1024];
    entropy_body(hist, levels, n, H, sd);
}

// one histogram per blockIdx.y, split over gridDim.x CTAs; partial sums in
// `part` (gridDim.x doubles per histogram), the last CTA of each histogram
// adds them in order and writes H
__global__ void __launch_bounds__(256) k_entropy_pack(const __grid_constant__ EntropyPack pk, double *part,
                                                      u32 *done)
{
    __shared__ double sd[256];
    __shared__ int last;
    const int i = blockIdx.y;
    const u64 *h = pk.hist[i];
    const u32 levels = pk.levels[i];
    const double Nd = (double)pk.n[i];
    double acc = 0.0;
    for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < levels; v += gridDim.x * blockDim.x) {
        const u64 c = h[v];
        if (c) {
            const double p = (double)c / Nd;
            acc += -p * log2(p);
        }
    }
    sd[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            sd[threadIdx.x] += sd[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[i * gridDim.x + blockIdx.x] = sd[0];
        __threadfence();
        last = atomicAdd(&done[i], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double H = 0.0;
        for (u32 b = 0; b < gridDim.x; ++b)
            H += __ldcg(&part[i * gridDim.x + b]);
        *pk.H[i] = H;
        done[i] = 0;
    }
}

size_t stats_smem_bytes(int dtype)
{
    return sizeof(u32) * (dtype == 0 ? kSmemWordsU8 : kSmemWordsU16);
}

}  // namespace

// ------------------------------------------------------------------ launchers

cudaError_t lnf_launch_stats_init(u64 *hist, u32 levels, DevStats *st, u64 n, cudaStream_t stream)
{
    k_stats_init<<<(levels + 255) / 256, 256, 0, stream>>>(hist, levels, st, n);
    return cudaGetLastError();
}

cudaError_t lnf_launch_zero(u64 *p, u64 count, cudaStream_t stream)
{
    int blocks = (int)((count + 255) / 256);
    if (blocks > 1024)
        blocks = 1024;
    if (blocks < 1)
        blocks = 1;
    k_zero<<<blocks, 256, 0, stream>>>(p, count);
    return cudaGetLastError();
}

cudaError_t lnf_launch_stats(const void *vol, u64 n, int dtype, u64 *hist, int num_sms, cudaStream_t stream)
{
    const size_t smem = stats_smem_bytes(dtype);
    cudaError_t e;
    if (dtype == 0) {
        e = cudaFuncSetAttribute(k_stats<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        u64 want = (n + 16ull * kStatsThreads - 1) / (16ull * kStatsThreads);
        int grid = (int)(want < (u64)(2 * num_sms) ? (want ? want : 1) : 2 * num_sms);
        k_stats<uint8_t><<<grid, kStatsThreads, smem, stream>>>(static_cast<const uint8_t *>(vol), n, hist);
    } else {
        e = cudaFuncSetAttribute(k_stats<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        u64 want = (n + 8ull * kStatsThreads - 1) / (8ull * kStatsThreads);
        int grid = (int)(want < (u64)num_sms ? (want ? want : 1) : num_sms);
        k_stats<uint16_t><<<grid, kStatsThreads, smem, stream>>>(static_cast<const uint16_t *>(vol), n, hist);
    }
    return cudaGetLastError();
}

size_t lnf_param_scratch_bytes() { return sizeof(ParamScratch); }

cudaError_t lnf_launch_params(const u64 *hist, const DevStats *st, const ParamCfg &cfg, DevParams *prm, u32 *lut,
                              void *pscr, int dtype, cudaStream_t stream)
{
    const int nc = dtype == 0 ? 1 : LNF_LEVELS_U16 / kChunk;
    ParamScratch *ps = static_cast<ParamScratch *>(pscr);
    k_param_totals<<<nc, kPThreads, 0, stream>>>(hist, st, ps);
    k_params<<<nc, kPThreads, 0, stream>>>(hist, st, cfg, prm, lut, ps);
    return cudaGetLastError();
}

cudaError_t lnf_launch_entropy(const u64 *hist, u32 levels, u64 n, double *H, cudaStream_t stream)
{
    k_entropy<<<1, 1024, 0, stream>>>(hist, levels, n, H);
    return cudaGetLastError();
}

cudaError_t lnf_launch_stats_init_batched(const StatsPack &pk, cudaStream_t stream)
{
    if (pk.n_jobs <= 0)
        return cudaSuccess;
    dim3 grid(16, pk.n_jobs);
    k_stats_init_batched<<<grid, 256, 0, stream>>>(pk);
    return cudaGetLastError();
}

cudaError_t lnf_launch_stats_batched(const StatsPack &pk, int ctas_per_job, cudaStream_t stream)
{
    if (pk.n_jobs <= 0)
        return cudaSuccess;
    const size_t smem = stats_smem_bytes(1);
    cudaError_t e = cudaFuncSetAttribute(k_stats_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid(ctas_per_job, pk.n_jobs);
    k_stats_batched<<<grid, kStatsThreads, smem, stream>>>(pk);
    return cudaGetLastError();
}

cudaError_t lnf_launch_params_batched(const StatsPack &pk, const ParamCfg &cfg, cudaStream_t stream)
{
    if (pk.n_jobs <= 0)
        return cudaSuccess;
    dim3 grid(LNF_LEVELS_U16 / kChunk, pk.n_jobs);
    k_param_totals_batched<<<grid, kPThreads, 0, stream>>>(pk);
    k_params_batched<<<grid, kPThreads, 0, stream>>>(pk, cfg);
    return cudaGetLastError();
}

cudaError_t lnf_launch_entropy_pack(const EntropyPack &pk, double *part, u32 *done, cudaStream_t stream)
{
    if (pk.count <= 0)
        return cudaSuccess;
    dim3 grid(LNF_ENT_SPLIT, pk.count);
    k_entropy_pack<<<grid, 256, 0, stream>>>(pk, part, done);
    return cudaGetLastError();
}
