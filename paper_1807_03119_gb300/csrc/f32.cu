// float32 volumes.  The paper filters grey levels (8- or 16-bit CT data); a
// float32 volume is filtered on 65536 levels spanning its own range:
//
//   lo = min v, hi = max v, d = hi - lo             (finite values only)
//   level q(v) = floor((v - lo) * (65535 / d) + 1/2)  (q = 0 everywhere when d = 0)
//   the 16-bit pipeline runs on the levels (statistics, Otsu T, every filter)
//   value(q) = lo + q * (d / 65535)
//
// Every operation is IEEE single precision with round-to-nearest, written with
// the explicit-rounding intrinsics so that no step is fused or reordered: a
// CPU doing the same float32 operations in the same order gets the same bits.
// A gated voxel (level 0) comes back as lo, the lowest value of the volume.
//
// Kernels: the range (an exact min / max through order-preserving integer
// keys, with a count of non-finite values), the quantisation and the
// dequantisation; all three are HBM-bound grid-stride loops with 16-byte loads
// where the buffer allows.
#include "lnf_internal.cuh"

namespace {

constexpr int kThreads = 512;

// order-preserving map of a non-NaN float to an unsigned key, and back
__device__ __forceinline__ u32 fkey(float f)
{
    const u32 b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float fkey_inv(u32 k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ bool finite(float f) { return (__float_as_uint(f) & 0x7F800000u) != 0x7F800000u; }

__global__ void k_range_init(u32 *range)
{
    range[0] = 0xFFFFFFFFu;   // min key
    range[1] = 0u;            // max key
    range[2] = 0u;            // non-finite values
    range[3] = 0u;
}

__global__ void __launch_bounds__(kThreads) k_range(const float *in, u64 n, u32 *range)
{
    u32 kmin = 0xFFFFFFFFu, kmax = 0u, bad = 0u;
    const u64 tid = blockIdx.x * (u64)blockDim.x + threadIdx.x, stride = (u64)gridDim.x * blockDim.x;
    auto take = [&](float f) {
        if (finite(f)) {
            const u32 k = fkey(f);
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        } else {
            ++bad;
        }
    };
    const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    const u64 n4 = vec ? n / 4 : 0;
    for (u64 i = tid; i < n4; i += stride) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(in) + i);
        take(v.x);
        take(v.y);
        take(v.z);
        take(v.w);
    }
    for (u64 i = n4 * 4 + tid; i < n; i += stride)
        take(in[i]);
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xFFFFFFFFu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xFFFFFFFFu, kmax, o));
        bad += __shfl_xor_sync(0xFFFFFFFFu, bad, o);
    }
    __shared__ u32 smin[kThreads / 32], smax[kThreads / 32], sbad[kThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        smin[w] = kmin;
        smax[w] = kmax;
        sbad[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThreads / 32; ++i) {
            kmin = min(kmin, smin[i]);
            kmax = max(kmax, smax[i]);
            bad += sbad[i];
        }
        atomicMin(&range[0], kmin);
        atomicMax(&range[1], kmax);
        if (bad)
            atomicAdd(&range[2], bad);
    }
}

struct Map {
    float lo, d;
};

__device__ __forceinline__ Map load_map(const u32 *range)
{
    Map m;
    m.lo = fkey_inv(range[0]);
    m.d = __fsub_rn(fkey_inv(range[1]), m.lo);
    return m;
}

__device__ __forceinline__ u32 level(float v, float lo, float sc)
{
    const float t = __fadd_rn(__fmul_rn(__fsub_rn(v, lo), sc), 0.5f);
    return (u32)fminf(floorf(t), 65535.0f);   // t >= 1/2: v >= lo
}

__global__ void __launch_bounds__(kThreads) k_quantize(const float *in, u64 n, const u32 *range, uint16_t *q)
{
    const Map m = load_map(range);
    const float sc = m.d > 0.0f ? __fdiv_rn(65535.0f, m.d) : 0.0f;   // d = 0: every level is 0
    const u64 tid = blockIdx.x * (u64)blockDim.x + threadIdx.x, stride = (u64)gridDim.x * blockDim.x;
    const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0 && (reinterpret_cast<uintptr_t>(q) & 7) == 0;
    const u64 n4 = vec ? n / 4 : 0;
    for (u64 i = tid; i < n4; i += stride) {
        const float4 v = __ldcs(reinterpret_cast<const float4 *>(in) + i);
        const u32 a = level(v.x, m.lo, sc), b = level(v.y, m.lo, sc), c = level(v.z, m.lo, sc),
                  e = level(v.w, m.lo, sc);
        reinterpret_cast<uint2 *>(q)[i] = make_uint2(a | (b << 16), c | (e << 16));
    }
    for (u64 i = n4 * 4 + tid; i < n; i += stride)
        q[i] = (uint16_t)level(in[i], m.lo, sc);
}

__global__ void __launch_bounds__(kThreads) k_dequantize(const uint16_t *q, u64 n, const u32 *range, float *out)
{
    const Map m = load_map(range);
    const float step = __fdiv_rn(m.d, 65535.0f);
    const u64 tid = blockIdx.x * (u64)blockDim.x + threadIdx.x, stride = (u64)gridDim.x * blockDim.x;
    auto value = [&](u32 l) { return __fadd_rn(m.lo, __fmul_rn((float)l, step)); };
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0 && (reinterpret_cast<uintptr_t>(q) & 7) == 0;
    const u64 n4 = vec ? n / 4 : 0;
    for (u64 i = tid; i < n4; i += stride) {
        const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(q) + i);
        __stcs(reinterpret_cast<float4 *>(out) + i,
               make_float4(value(w.x & 0xFFFFu), value(w.x >> 16), value(w.y & 0xFFFFu), value(w.y >> 16)));
    }
    for (u64 i = n4 * 4 + tid; i < n; i += stride)
        out[i] = value(q[i]);
}

int grid_for(u64 n, int num_sms)
{
    const u64 want = (n / 4 + kThreads - 1) / kThreads;
    const u64 cap = (u64)num_sms * 4;   // 4 CTAs of 512 threads per SM
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

// range[0..3]: min key, max key, count of non-finite values, unused
cudaError_t lnf_launch_f32_range(const float *in, u64 n, u32 *range, int num_sms, cudaStream_t st)
{
    k_range_init<<<1, 1, 0, st>>>(range);
    k_range<<<grid_for(n, num_sms), kThreads, 0, st>>>(in, n, range);
    return cudaGetLastError();
}

cudaError_t lnf_launch_f32_quantize(const float *in, u64 n, const u32 *range, uint16_t *q, int num_sms,
                                    cudaStream_t st)
{
    k_quantize<<<grid_for(n, num_sms), kThreads, 0, st>>>(in, n, range, q);
    return cudaGetLastError();
}

cudaError_t lnf_launch_f32_dequantize(const uint16_t *q, u64 n, const u32 *range, float *out, int num_sms,
                                      cudaStream_t st)
{
    k_dequantize<<<grid_for(n, num_sms), kThreads, 0, st>>>(q, n, range, out);
    return cudaGetLastError();
}
