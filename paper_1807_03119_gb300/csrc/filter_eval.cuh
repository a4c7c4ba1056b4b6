// Per-voxel evaluation of the five filters by direct enumeration of their
// taps, shared by the generic filter kernel (filter.cu, reading a shared-memory
// plane ring) and the ray caster (render.cu, reading the volume in global
// memory): exact integer sums, round-half-up to the input type and the noise
// gate (P0 >= T and the unrounded value >= T, cross-multiplied).  The sampler
// S gives R.at(dx, dy, dz) = P at the centre voxel plus (dx, dy, dz), with
// clamp-to-edge at the volume's borders.
#pragma once
#include "lnf_internal.cuh"

namespace lnfeval {

__device__ __forceinline__ u32 rnd_div(u64 a, u64 b) { return (u32)((2 * a + b) / (2 * b)); }

struct StepParams {
    u32 T;
    u32 delta;
    u32 k;              // sigma_k, for the local sigma filter
    long long td;
    long long te;
    int r, d;
    const u32 *lut;
};

template <class S>
__device__ __forceinline__ u32 eval_filter(int filter, const S &R, const StepParams &p)
{
    const int r = p.r;
    const int M = 2 * r + 1;
    const u32 P0 = R.at(0, 0, 0);
    switch (filter) {
    case 0: {   // mean, Eq. 4
        u64 B = 0;
        for (int k = -r; k <= r; ++k)
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i)
                    B += R.at(i, j, k);
        const u64 n = (u64)M * M * M;
        if (P0 < p.T || B < n * p.T)
            return 0;
        return rnd_div(B, n);
    }
    case 1: {   // sigma, Eq. 5: |P_i - P0| <= delta over the cube
        u64 s = 0;
        u32 n = 0;
        const u32 dl = min(p.delta, 65535u);      // every value lies within 65535
        const u32 lo = P0 > dl ? P0 - dl : 0u;
        const u32 width = (P0 - lo) + dl;         // band [lo, lo + width]
        for (int k = -r; k <= r; ++k)
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i) {
                    const u32 v = R.at(i, j, k);
                    if (v - lo <= width) {
                        s += v;
                        ++n;
                    }
                }
        if (P0 < p.T || s < (u64)n * p.T)
            return 0;
        return rnd_div(s, n);
    }
    case 2: {   // entropy, Eq. 7
        u64 E = 0;
        for (int k = -r; k <= r; ++k)
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i)
                    E += __ldg(p.lut + R.at(i, j, k));
        if (P0 < p.T)
            return 0;
        return (long long)E > p.te ? P0 : 0u;
    }
    case 3: {   // Okada, Eq. 6: centre + axis cross of arm r, |P0 - P_i| < T_d
        u64 s = 0;
        u32 n = 0;
        if (p.td > 0) {
            s = P0;
            n = 1;
            for (int t = 1; t <= r; ++t) {
                const u32 v[6] = {R.at(t, 0, 0), R.at(-t, 0, 0), R.at(0, t, 0),
                                  R.at(0, -t, 0), R.at(0, 0, t), R.at(0, 0, -t)};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const long long df = (long long)P0 - (long long)v[q];
                    if ((df < 0 ? -df : df) < p.td) {
                        s += v[q];
                        ++n;
                    }
                }
            }
        }
        if (n == 0 || P0 < p.T || s < (u64)n * p.T)
            return 0;
        return rnd_div(s, n);
    }
    case 7: {   // sigma with the local standard deviation of the cube (Lee's original):
        // m^2 (P_i - P0)^2 <= k^2 (m S2 - S1^2), exactly
        u64 S1 = 0, S2 = 0;
        for (int k = -r; k <= r; ++k)
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i) {
                    const u64 v = R.at(i, j, k);
                    S1 += v;
                    S2 += v * v;
                }
        const unsigned __int128 m = (unsigned __int128)M * M * M;
        const unsigned __int128 rhs = (unsigned __int128)p.k * p.k * (m * S2 - (unsigned __int128)S1 * S1);
        u64 s = 0;
        u32 n = 0;
        for (int k = -r; k <= r; ++k)
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i) {
                    const u32 v = R.at(i, j, k);
                    const u64 d = v > P0 ? v - P0 : P0 - v;
                    if (m * m * d * d <= rhs) {
                        s += v;
                        ++n;
                    }
                }
        if (P0 < p.T || s < (u64)n * p.T)
            return 0;
        return rnd_div(s, n);
    }
    case 5:     // cluster-layout variants of the paper's filter: the nine cluster
    case 6: {   // centres of Eq. 2-3, each cluster its axis cross of arm r (5) or its M^3 cube (6)
        u64 U = 0;
        const int d = p.d;
        for (int c = 0; c < 9; ++c) {
            int cx = 0, cy = 0, cz = 0;
            if (c > 0) {
                cx = (c - 1) & 1 ? d : -d;
                cy = (c - 1) & 2 ? d : -d;
                cz = (c - 1) & 4 ? d : -d;
            }
            if (filter == 5) {
                U += R.at(cx, cy, cz);
                for (int t = 1; t <= r; ++t)
                    U += R.at(cx - t, cy, cz) + R.at(cx + t, cy, cz) + R.at(cx, cy - t, cz) + R.at(cx, cy + t, cz) +
                         R.at(cx, cy, cz - t) + R.at(cx, cy, cz + t);
            } else {
                for (int k = -r; k <= r; ++k)
                    for (int j = -r; j <= r; ++j)
                        for (int i = -r; i <= r; ++i)
                            U += R.at(cx + i, cy + j, cz + k);
            }
        }
        const u64 den = 9ull * (filter == 5 ? 6ull * r + 1 : (u64)M * M * M);
        if (P0 < p.T || U < den * p.T)
            return 0;
        return rnd_div(U, den);
    }
    default: {  // the paper's filter, Eq. 2-3: nine average clusters
        u64 U = 0;
        const int d = p.d;
        for (int c = 0; c < 9; ++c) {
            int cx = 0, cy = 0, cz = 0;
            if (c > 0) {
                cx = (c - 1) & 1 ? d : -d;
                cy = (c - 1) & 2 ? d : -d;
                cz = (c - 1) & 4 ? d : -d;
            }
            for (int t = -r; t <= r; ++t)
                U += R.at(cx + t, cy, cz) + R.at(cx, cy + t, cz) + R.at(cx, cy, cz + t);
        }
        const u64 den = 27ull * M;
        if (P0 < p.T || U < den * p.T)
            return 0;
        return rnd_div(U, den);
    }
    }
}

// the scalars a job's evaluation needs, from the device parameter block; the
// entropy threshold T_e (Eq. 7) defaults to the expected criterion of a kernel
// of M^3 voxels, floor(M^3 sum h w / N)
__device__ __forceinline__ StepParams make_step_params(const DevParams &P, int radius, int offset, const u32 *lut)
{
    StepParams sp;
    sp.T = P.T;
    sp.delta = P.delta;
    sp.k = P.sigma_k;
    sp.td = P.td;
    sp.r = radius;
    sp.d = offset;
    sp.lut = lut;
    const u64 M = 2 * radius + 1;
    if (P.te_cfg == -2) {
        const unsigned __int128 num = (unsigned __int128)(M * M * M) * P.hw_sum;
        sp.te = (long long)(num / P.N);
    } else {
        sp.te = P.te_cfg;
    }
    return sp;
}

}  // namespace lnfeval
