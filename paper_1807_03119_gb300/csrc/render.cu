// Ray caster: the paper's use of its filter ("Introduction", "3D Spatial Noise
// Filters").  Each pixel's ray marches through the volume; the first sample at
// or above the threshold T is a candidate surface point, where the chosen
// filter decides between structure and noise; a candidate the filter keeps
// (gated output not 0) ends the ray and is shaded with the normal of a 3D
// Sobel operator and headlight Phong illumination; a rejected candidate is
// noise and the ray goes on.
//
// Orthographic rays along one of the six axis directions (view 0..5 = +x, -x,
// +y, -y, +z, -z), one per voxel column, samples at voxel centres; image axes
// (u, w) = (y, z) for +-x, (x, z) for +-y, (x, y) for +-z, pixel w * W + u.
// Shading in IEEE double with explicitly rounded operations (no fused
// multiply-add): c = (g . d) / |g| (1 when g = 0), I = (0.1 + 0.7 max(c, 0))
// + 0.2 s^16 with s = 2c^2 - 1 when c > 0 and s > 0, pixel = min(255,
// floor(255 I + 1/2)); 0 where no surface is found.
//
// Mapping: one thread per ray, a CTA of 8 warps over 32 x 8 pixels (u
// fastest, so a warp's rays read consecutive voxels of a row).  Each lane
// scans ahead to its next candidate with 8 loads in flight, then the warp
// evaluates all its lanes' candidates together; the filter at a candidate is
// the per-voxel evaluation of filter_eval.cuh over clamped global reads.
#include "lnf_ctx.h"
#include "filter_eval.cuh"

namespace {

using namespace lnfeval;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// clamp-to-edge reads of the volume at offsets from a centre voxel
template <typename T>
struct GlobalSampler {
    const T *v;
    int nx, ny, nz;
    long long pitch;   // elements per row
    int x, y, z;
    __device__ __forceinline__ u32 at(int dx, int dy, int dz) const
    {
        const int xx = clampi(x + dx, 0, nx - 1), yy = clampi(y + dy, 0, ny - 1), zz = clampi(z + dz, 0, nz - 1);
        return (u32)__ldg(v + ((long long)zz * ny + yy) * pitch + xx);
    }
};

struct RenderArgs {
    const void *vol;
    int nx, ny, nz;
    long long pitch;
    int view;
    int W, H, len;
    int filter, radius, offset;
    const DevParams *prm;
    const u32 *lut;
    unsigned char *image;
    int *depth;        // may be null
    u32 *value;        // may be null
};

constexpr int kAhead = 8;   // samples loaded before the first is tested

template <typename T>
__device__ unsigned char shade(const GlobalSampler<T> &S, int view)
{
    long long gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int k = -1; k <= 1; ++k)
#pragma unroll
        for (int j = -1; j <= 1; ++j)
#pragma unroll
            for (int i = -1; i <= 1; ++i) {
                const long long P = S.at(i, j, k);
                const long long bj = j == 0 ? 2 : 1, bk = k == 0 ? 2 : 1, bi = i == 0 ? 2 : 1;
                gx += i * bj * bk * P;
                gy += j * bi * bk * P;
                gz += k * bi * bj * P;
            }
    const long long ga = view < 2 ? gx : (view < 4 ? gy : gz);
    const long long along = (view & 1) ? -ga : ga;   // g . d
    const long long n2 = gx * gx + gy * gy + gz * gz;
    const double c = n2 > 0 ? __ddiv_rn((double)along, __dsqrt_rn((double)n2)) : 1.0;
    const double diff = c > 0.0 ? c : 0.0;
    double spec = 0.0;
    if (c > 0.0) {
        double s = __dadd_rn(__dmul_rn(2.0, __dmul_rn(c, c)), -1.0);
        if (s > 0.0) {
            s = __dmul_rn(s, s);
            s = __dmul_rn(s, s);
            s = __dmul_rn(s, s);
            s = __dmul_rn(s, s);
            spec = s;
        }
    }
    const double I = __dadd_rn(__dadd_rn(0.1, __dmul_rn(0.7, diff)), __dmul_rn(0.2, spec));
    const double q = floor(__dadd_rn(__dmul_rn(255.0, I), 0.5));
    return q >= 255.0 ? (unsigned char)255 : (unsigned char)q;
}

template <typename T>
__global__ void __launch_bounds__(256) k_render(const RenderArgs a)
{
    // every lane stays to the end (the warp votes below); lanes past the
    // image's edge read nothing and write nothing
    const bool active = blockIdx.x * 32 + (threadIdx.x & 31) < a.W && blockIdx.y * 8 + (threadIdx.x >> 5) < a.H;
    const int u = active ? blockIdx.x * 32 + (threadIdx.x & 31) : 0;
    const int w = active ? blockIdx.y * 8 + (threadIdx.x >> 5) : 0;
    const StepParams sp = make_step_params(*a.prm, a.radius, a.offset, a.lut);
    const T *vol = static_cast<const T *>(a.vol);
    // the voxel at step 0 and the step along the ray
    int x0, y0, z0, sx = 0, sy = 0, sz = 0;
    switch (a.view) {
    case 0: x0 = 0; y0 = u; z0 = w; sx = 1; break;
    case 1: x0 = a.nx - 1; y0 = u; z0 = w; sx = -1; break;
    case 2: x0 = u; y0 = 0; z0 = w; sy = 1; break;
    case 3: x0 = u; y0 = a.ny - 1; z0 = w; sy = -1; break;
    case 4: x0 = u; y0 = w; z0 = 0; sz = 1; break;
    default: x0 = u; y0 = w; z0 = a.nz - 1; sz = -1; break;
    }
    const long long off0 = ((long long)z0 * a.ny + y0) * a.pitch + x0;
    const long long step = (long long)sx + (long long)sy * a.pitch + (long long)sz * a.pitch * a.ny;
    // each lane scans ahead to its next candidate (8 samples in flight), then
    // the warp evaluates all its lanes' candidates in one pass, so a warp runs
    // as many filter evaluations as its busiest lane needs, not their sum
    int hit = -1;
    u32 val = 0;
    int k = 0;
    bool done = !active;
    for (;;) {
        while (!done) {
            u32 smp[kAhead];
#pragma unroll
            for (int j = 0; j < kAhead; ++j)
                smp[j] = k + j < a.len ? (u32)__ldg(vol + off0 + (long long)(k + j) * step) : 0u;
            int first = kAhead;
#pragma unroll
            for (int j = kAhead - 1; j >= 0; --j)
                if (k + j < a.len && smp[j] >= sp.T)
                    first = j;
            if (first < kAhead) {
                k += first;   // a candidate: at or above the threshold
                break;
            }
            k += kAhead;
            if (k >= a.len)
                done = true;   // no surface along this ray
        }
        if (!__any_sync(0xFFFFFFFFu, !done))
            break;
        if (!done) {
            const GlobalSampler<T> S{vol, a.nx, a.ny, a.nz, a.pitch, x0 + k * sx, y0 + k * sy, z0 + k * sz};
            const u32 f = eval_filter(a.filter, S, sp);
            if (f != 0) {   // the filter keeps it: the surface
                hit = k;
                val = f;
                done = true;
            } else if (++k >= a.len) {   // noise: the ray goes on
                done = true;
            }
        }
    }
    unsigned char pix = 0;
    if (hit >= 0) {
        const GlobalSampler<T> S{vol, a.nx, a.ny, a.nz, a.pitch, x0 + hit * sx, y0 + hit * sy, z0 + hit * sz};
        pix = shade<T>(S, a.view);
    }
    if (!active)
        return;
    const long long o = (long long)w * a.W + u;
    a.image[o] = pix;
    if (a.depth)
        a.depth[o] = hit;
    if (a.value)
        a.value[o] = val;
}

}  // namespace

cudaError_t lnf_launch_render(const void *vol, const int64_t dims[3], int64_t pitch, int dtype, int view,
                              int filter, int radius, int offset, const DevParams *prm, const u32 *lut,
                              unsigned char *image, int *depth, u32 *value, cudaStream_t st)
{
    RenderArgs a;
    a.vol = vol;
    a.nx = (int)dims[0];
    a.ny = (int)dims[1];
    a.nz = (int)dims[2];
    a.pitch = pitch;
    a.view = view;
    a.W = view < 2 ? a.ny : a.nx;
    a.H = view < 4 ? a.nz : a.ny;
    a.len = view < 2 ? a.nx : (view < 4 ? a.ny : a.nz);
    a.filter = filter;
    a.radius = radius;
    a.offset = offset;
    a.prm = prm;
    a.lut = lut;
    a.image = image;
    a.depth = depth;
    a.value = value;
    const dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
    if (dtype == LNF_U8)
        k_render<uint8_t><<<grid, 256, 0, st>>>(a);
    else
        k_render<uint16_t><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}
