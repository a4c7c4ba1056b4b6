// Row-padded copy of a volume that TMA cannot address (its base is not 16-byte
// aligned or its row length in bytes is not a multiple of 16): rows of
// `row_bytes` bytes are copied into rows of `prow` bytes (a multiple of 16) so
// that the plane-ring kernels can read it with TMA.  The copy can be told to
// return at once while the gate-first kernel takes the volume (lnf_gate_mode):
// the ring kernels that read the copy then return at once too.
#include "lnf_ctx.h"

#include <algorithm>

namespace {

__device__ __forceinline__ uint4 shfl_down4(uint4 v)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
    v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
    v.z = __shfl_down_sync(0xffffffffu, v.z, 1);
    v.w = __shfl_down_sync(0xffffffffu, v.w, 1);
    return v;
}

// One warp per 512-byte segment of a row: lane t writes the 16 bytes at offset
// 16 t of the segment.  The segment's source starts o bytes past a 16-byte
// boundary a0 (o is the same for the whole warp); lane t loads the aligned block
// a0 + 16 t, takes block a0 + 16 (t + 1) from lane t + 1 (lane 31 loads
// a0 + 512 itself) and shifts that 32-byte window down by o bytes.  A block is
// loaded only if it holds a byte of the volume (block < end; every block is at
// or past the one that holds the volume's first byte): an aligned 16-byte block
// never crosses the edge of an allocation, so no load leaves the volume's
// allocation.  Bytes of a loaded block outside the row go to the destination's
// row padding or are not stored; a store is made only at offsets below
// row_bytes, which with prow a multiple of 16 keeps it inside its padded row.
__global__ void __launch_bounds__(256) k_copy_pitched(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                                      u64 row_bytes, u64 prow, u64 rows, const DevParams *skip)
{
    if (skip && lnf_gate_mode(*skip))
        return;   // the gate-first kernel takes the volume: nothing reads the copy
    const uintptr_t base = reinterpret_cast<uintptr_t>(src);
    const uintptr_t end = base + row_bytes * rows;
    const u64 segs = (row_bytes + 511) / 512;
    const u64 work = rows * segs;
    const u32 lane = threadIdx.x & 31u;
    const u64 nwarps = (u64)gridDim.x * (blockDim.x >> 5);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (u64 w = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < work; w += nwarps) {
        const u64 r = w / segs;
        const u64 off0 = (w - r * segs) * 512;
        const uintptr_t s = base + r * row_bytes + off0;
        const uintptr_t a0 = s & ~(uintptr_t)15;
        const u32 o = (u32)(s - a0);
        const uintptr_t blk = a0 + 16u * lane;
        const uint4 lo = blk < end ? *reinterpret_cast<const uint4 *>(blk) : zero;
        uint4 hi = shfl_down4(lo);   // every lane of the warp takes part
        if (lane == 31u) {
            const uintptr_t b = a0 + 512;
            hi = (o != 0u && b < end) ? *reinterpret_cast<const uint4 *>(b) : zero;
        }
        const u32 win[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        const u32 ws = o >> 2, bs = (o & 3u) * 8u;
        u32 v[5];
#pragma unroll
        for (int i = 0; i < 5; ++i)
            v[i] = ws == 0u ? win[i] : ws == 1u ? win[i + 1] : ws == 2u ? win[i + 2] : win[i + 3];
        uint4 out;
        out.x = __funnelshift_r(v[0], v[1], bs);
        out.y = __funnelshift_r(v[1], v[2], bs);
        out.z = __funnelshift_r(v[2], v[3], bs);
        out.w = __funnelshift_r(v[3], v[4], bs);
        const u64 off = off0 + 16u * lane;
        if (off < row_bytes)
            *reinterpret_cast<uint4 *>(dst + r * prow + off) = out;
    }
}

}  // namespace

lnf_status lnf_copy_pitched(lnf_ctx *ctx, void *dst, size_t prow, const void *in, const int64_t dims[3], int dtype,
                            cudaStream_t st, const DevParams *skip_prm)
{
    const u64 row = (u64)dims[0] * (dtype == LNF_U8 ? 1u : 2u);
    const u64 rows = (u64)dims[1] * dims[2];
    if (prow % 16 != 0 || prow < row || reinterpret_cast<uintptr_t>(dst) % 16 != 0)
        return lnf_fail(ctx, LNF_EINVAL, "padded copy: destination rows not 16-byte aligned");
    const u64 work = rows * ((row + 511) / 512);
    const u64 grid = std::min<u64>((work + 7) / 8, (u64)ctx->num_sms * 8);
    if (grid == 0)
        return LNF_OK;
    k_copy_pitched<<<(unsigned)grid, 256, 0, st>>>(static_cast<const uint8_t *>(in), static_cast<uint8_t *>(dst), row,
                                                 prow, rows, skip_prm);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return lnf_fail(ctx, LNF_ECUDA, "padded copy: %s", cudaGetErrorString(e));
    return LNF_OK;
}
