// Per-voxel evaluation of the five filters by direct enumeration of their
// taps, shared by the generic filter kernel (filter.cu, reading a shared-memory
// plane ring) and the ray caster (render.cu, reading the volume in global
// memory): exact integer sums, round-half-up to the input type and the noise
// gate (P0 >= T and the unrounded value >= T, cross-multiplied).  The sampler
// S gives R.at(dx, dy, dz) = P at the centre voxel plus (dx, dy, dz), with
// clamp-to-edge at the volume's borders.
//
// Radii and cluster offsets are per axis (x, y, z), for volumes of anisotropic
// voxel spacing: the cube of M^3 voxels becomes the box of Mx My Mz voxels
// (M_a = 2 r_a + 1), the Okada cross has arm r_a along axis a, and a cluster of
// the paper's filter averages its lines of Mx, My and Mz voxels, the diagonal
// clusters sitting at (+-dx, +-dy, +-dz).  Equal axes give the paper's forms.
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
    int r[3], d[3];     // radius and cluster offset per axis (x, y, z)
    const u32 *lut;
    const unsigned long long *lt;   // local entropy filter: t[c] = round(2^22 c log2 c)
    long long lte;                  // ... and its theta (2^-22 bits)
};

template <class S>
__device__ __forceinline__ u32 eval_filter(int filter, const S &R, const StepParams &p)
{
    const int rx = p.r[0], ry = p.r[1], rz = p.r[2];
    const u64 box = (u64)(2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1);   // voxels of the box
    const u32 P0 = R.at(0, 0, 0);
    // every filter is 0 below the noise gate (Eq. 6 / Eq. 7 "0, otherwise", and
    // the same test in each case below): a gated voxel needs none of its taps,
    // and a warp whose voxels are all gated skips the tap loops
    if (P0 < p.T)
        return 0;
    switch (filter) {
    case 0: {   // mean, Eq. 4
        u64 B = 0;
        for (int k = -rz; k <= rz; ++k)
            for (int j = -ry; j <= ry; ++j)
                for (int i = -rx; i <= rx; ++i)
                    B += R.at(i, j, k);
        if (P0 < p.T || B < box * p.T)
            return 0;
        return rnd_div(B, box);
    }
    case 1: {   // sigma, Eq. 5: |P_i - P0| <= delta over the box
        u64 s = 0;
        u32 n = 0;
        const u32 dl = min(p.delta, 65535u);      // every value lies within 65535
        const u32 lo = P0 > dl ? P0 - dl : 0u;
        const u32 width = (P0 - lo) + dl;         // band [lo, lo + width]
        for (int k = -rz; k <= rz; ++k)
            for (int j = -ry; j <= ry; ++j)
                for (int i = -rx; i <= rx; ++i) {
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
        for (int k = -rz; k <= rz; ++k)
            for (int j = -ry; j <= ry; ++j)
                for (int i = -rx; i <= rx; ++i)
                    E += __ldg(p.lut + R.at(i, j, k));
        if (P0 < p.T)
            return 0;
        return (long long)E > p.te ? P0 : 0u;
    }
    case 3: {   // Okada, Eq. 6: centre + axis cross of arm r_a, |P0 - P_i| < T_d
        u64 s = 0;
        u32 n = 0;
        if (p.td > 0) {
            s = P0;
            n = 1;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                for (int t = 1; t <= p.r[a]; ++t) {
                    const u32 v[2] = {R.at(a == 0 ? t : 0, a == 1 ? t : 0, a == 2 ? t : 0),
                                      R.at(a == 0 ? -t : 0, a == 1 ? -t : 0, a == 2 ? -t : 0)};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
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
    case 7: {   // sigma with the local standard deviation of the box (Lee's original):
        // m^2 (P_i - P0)^2 <= k^2 (m S2 - S1^2), exactly
        u64 S1 = 0, S2 = 0;
        for (int k = -rz; k <= rz; ++k)
            for (int j = -ry; j <= ry; ++j)
                for (int i = -rx; i <= rx; ++i) {
                    const u64 v = R.at(i, j, k);
                    S1 += v;
                    S2 += v * v;
                }
        const unsigned __int128 m = box;
        const unsigned __int128 rhs = (unsigned __int128)p.k * p.k * (m * S2 - (unsigned __int128)S1 * S1);
        u64 s = 0;
        u32 n = 0;
        for (int k = -rz; k <= rz; ++k)
            for (int j = -ry; j <= ry; ++j)
                for (int i = -rx; i <= rx; ++i) {
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
    case 8: {   // entropy filter with the box's own grey-level probabilities: with c_g of
        // the m box voxels at level g, m 2^22 H = t[m] - sum_g t[c_g].  The sum is
        // taken as the telescoping sum over the taps a of t[k_a] - t[k_a - 1], k_a
        // the taps up to a (enumeration order) at a's level.  P0 >= T first.
        if (P0 < p.T)
            return 0;
        const int m = (int)box;
        u64 K = 0;
        int a = 0;
        for (int ka = -rz; ka <= rz; ++ka)
            for (int ja = -ry; ja <= ry; ++ja)
                for (int ia = -rx; ia <= rx; ++ia, ++a) {
                    const u32 va = R.at(ia, ja, ka);
                    // taps b <= a at level va (a itself included)
                    auto rank = [&]() -> u32 {
                        u32 k = 0;
                        int b = 0;
                        for (int kb = -rz; kb <= rz; ++kb)
                            for (int jb = -ry; jb <= ry; ++jb)
                                for (int ib = -rx; ib <= rx; ++ib, ++b) {
                                    if (b > a)
                                        return k;
                                    k += R.at(ib, jb, kb) == va;
                                }
                        return k;
                    };
                    const u32 k = rank();
                    K += __ldg(p.lt + k) - __ldg(p.lt + k - 1);
                }
        const long long crit = (long long)(__ldg(p.lt + m) - K);
        return crit > (long long)m * p.lte ? P0 : 0u;
    }
    case 5:     // cluster-layout variants of the paper's filter: the nine cluster
    case 6: {   // centres of Eq. 2-3, each cluster its axis cross of arms r_a (5) or its box (6)
        u64 U = 0;
        for (int c = 0; c < 9; ++c) {
            int cx = 0, cy = 0, cz = 0;
            if (c > 0) {
                cx = (c - 1) & 1 ? p.d[0] : -p.d[0];
                cy = (c - 1) & 2 ? p.d[1] : -p.d[1];
                cz = (c - 1) & 4 ? p.d[2] : -p.d[2];
            }
            if (filter == 5) {
                U += R.at(cx, cy, cz);
                for (int t = 1; t <= rx; ++t)
                    U += R.at(cx - t, cy, cz) + R.at(cx + t, cy, cz);
                for (int t = 1; t <= ry; ++t)
                    U += R.at(cx, cy - t, cz) + R.at(cx, cy + t, cz);
                for (int t = 1; t <= rz; ++t)
                    U += R.at(cx, cy, cz - t) + R.at(cx, cy, cz + t);
            } else {
                for (int k = -rz; k <= rz; ++k)
                    for (int j = -ry; j <= ry; ++j)
                        for (int i = -rx; i <= rx; ++i)
                            U += R.at(cx + i, cy + j, cz + k);
            }
        }
        const u64 den = 9ull * (filter == 5 ? 1ull + 2ull * (rx + ry + rz) : box);
        if (P0 < p.T || U < den * p.T)
            return 0;
        return rnd_div(U, den);
    }
    default: {  // the paper's filter, Eq. 2-3: nine average clusters
        u64 U = 0;
        for (int c = 0; c < 9; ++c) {
            int cx = 0, cy = 0, cz = 0;
            if (c > 0) {
                cx = (c - 1) & 1 ? p.d[0] : -p.d[0];
                cy = (c - 1) & 2 ? p.d[1] : -p.d[1];
                cz = (c - 1) & 4 ? p.d[2] : -p.d[2];
            }
            for (int t = -rx; t <= rx; ++t)
                U += R.at(cx + t, cy, cz);
            for (int t = -ry; t <= ry; ++t)
                U += R.at(cx, cy + t, cz);
            for (int t = -rz; t <= rz; ++t)
                U += R.at(cx, cy, cz + t);
        }
        const u64 den = 9ull * (u64)(2 * rx + 1 + 2 * ry + 1 + 2 * rz + 1);
        if (P0 < p.T || U < den * p.T)
            return 0;
        return rnd_div(U, den);
    }
    }
}

// the scalars a job's evaluation needs, from the device parameter block and the
// per-axis radii and offsets; the entropy threshold T_e (Eq. 7) defaults to the
// expected criterion of a kernel of m = Mx My Mz voxels, floor(m sum h w / N)
__device__ __forceinline__ StepParams make_step_params3(const DevParams &P, const int rad[3], const int off[3],
                                                        const u32 *lut)
{
    StepParams sp;
    sp.T = P.T;
    sp.delta = P.delta;
    sp.k = P.sigma_k;
    sp.td = P.td;
    u64 m = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        sp.r[a] = rad[a];
        sp.d[a] = off[a];
        m *= (u64)(2 * rad[a] + 1);
    }
    sp.lut = lut;
    if (P.te_cfg == -2) {
        const unsigned __int128 num = (unsigned __int128)m * P.hw_sum;
        sp.te = (long long)(num / P.N);
    } else {
        sp.te = P.te_cfg;
    }
    // the local entropy filter: default theta log2(m) / 2 as floor(t[m] / 2m)
    sp.lt = P.lt;
    if (P.lte_cfg == -2)
        sp.lte = (P.lt && m <= LNF_LT_MAX) ? (long long)(__ldg(P.lt + m) / (2 * m)) : 0;
    else
        sp.lte = P.lte_cfg;
    return sp;
}

// ... with the same radius and offset on every axis (the paper's forms)
__device__ __forceinline__ StepParams make_step_params(const DevParams &P, int radius, int offset, const u32 *lut)
{
    const int rad[3] = {radius, radius, radius}, off[3] = {offset, offset, offset};
    return make_step_params3(P, rad, off, lut);
}

}  // namespace lnfeval
