/*
 * Plain, slow CPU oracle for the local noise filter of arXiv 1807.03119
 * ("Real-time Local Noise Filter in 3D Visualization of CT Data").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code with the
 * CUDA path: every filter is evaluated here by literal enumeration of every tap
 * of its definition, one output voxel at a time, in exact integer arithmetic.
 *
 * Conventions (the paper is silent on them; each is a stated reading):
 *   - volume layout x-fastest: idx = (z*ny + y)*nx + x;
 *   - clamp-to-edge sampling outside the volume;
 *   - rounding of an average a/b to the input type is round-half-up,
 *     floor((2a + b) / (2b));
 *   - noise gate: a voxel is kept only if its own value P0 >= T and the
 *     unrounded filter value is >= T (cross-multiplied: sum >= T*count);
 *     otherwise the output is 0 (the "0, otherwise" branch of Eq. 6 / Eq. 7).
 *
 * Filter ids follow the order of the paper's Fig. 5: 0 mean, 1 sigma,
 * 2 entropy, 3 Okada, 4 the paper's own filter ("ours"); 5 and 6 are two
 * cluster-layout variants of it (see filter_ours_variant); 7 is the sigma
 * filter with the local standard deviation (see filter_sigma_local); 8 is the
 * entropy filter with the cube's own grey-level probabilities (see
 * filter_entropy_local).
 */
#include <stdint.h>
#include <stddef.h>

typedef struct oracle_params {
    int32_t filter_id;     /* 0..4 the paper's five (Fig. 5 order), 5..7 the variants below */
    int32_t radius;        /* r >= 0, kernel size M = 2r+1 (Eq. 3 needs M odd) */
    int32_t offset;        /* d: diagonal cluster offset, (+-d,+-d,+-d); d=1 is distance sqrt(3) */
    uint32_t threshold;    /* T: Otsu (Eq. 1) or fixed; 0 disables the gate */
    uint32_t sigma_band;   /* delta: |P_i - P0| <= delta  (delta = floor(2 sigma), Eq. 5) */
    int64_t okada_td;      /* T_d: |P0 - P_i| < T_d (Eq. 6) */
    int64_t entropy_te;    /* T_e (fixed point): keep P0 iff E > T_e (Eq. 7) */
    const uint32_t *entropy_w; /* w[v] = fixed-point -p_v log2 p_v, one entry per grey level */
    int32_t sigma_k;       /* k of the local sigma filter: |P_i - P0| <= k sigma_local */
    /* anisotropic voxel spacing: when `aniso` is set, radius and cluster offset
     * are taken per axis (x, y, z) from rad[] and off[] instead of radius and
     * offset; M_a = 2 rad[a] + 1 voxels along axis a */
    int32_t aniso;
    int32_t rad[3];
    int32_t off[3];
    /* entropy filter with local probabilities (id 8): entropy_lt[c] =
     * round(2^22 c log2 c) for c = 0..m (m voxels in the cube), and the
     * threshold theta in 2^-22 bits: keep P0 iff lt[m] - sum_g lt[c_g] > m theta */
    const uint64_t *entropy_lt;
    int64_t entropy_lte;
} oracle_params;

/* largest cube of the local entropy filter: radius 8 on every axis */
#define ORACLE_MAX_CUBE (17 * 17 * 17)

typedef struct vol_view {
    const void *data;
    int64_t nx, ny, nz;
    int dtype;             /* 0 = uint8, 1 = uint16 */
} vol_view;

static int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* P(x,y,z) with clamp-to-edge. */
static uint32_t sample(const vol_view *v, int64_t x, int64_t y, int64_t z)
{
    x = clampi(x, 0, v->nx - 1);
    y = clampi(y, 0, v->ny - 1);
    z = clampi(z, 0, v->nz - 1);
    int64_t idx = (z * v->ny + y) * v->nx + x;
    if (v->dtype == 0)
        return ((const uint8_t *)v->data)[idx];
    return ((const uint16_t *)v->data)[idx];
}

/* The per-axis radii r[a] and cluster offsets d[a] (a = x, y, z) of a filter;
 * the isotropic filters of the paper have r[a] = radius and d[a] = offset. */
static void axis_extents(const oracle_params *p, int r[3], int d[3])
{
    for (int a = 0; a < 3; ++a) {
        r[a] = p->aniso ? p->rad[a] : p->radius;
        d[a] = p->aniso ? p->off[a] : p->offset;
    }
}

/* round-half-up of a/b, b > 0 */
static uint32_t round_div(uint64_t a, uint64_t b)
{
    return (uint32_t)((2 * a + b) / (2 * b));
}

/* Eq. 2 without its 1/(3M) factor: the x-, y- and z-line sums through the
 * cluster centre c, of M_a = 2 r[a] + 1 voxels along axis a, with offsets
 * Delta_i = i - (M_a - 1)/2 (Eq. 3).  The centre voxel therefore enters three
 * times.  (Isotropic: M voxels per line, 3M in all.) */
static uint64_t cluster_line_sum(const vol_view *v, const int r[3], int64_t cx, int64_t cy, int64_t cz)
{
    uint64_t s = 0;
    for (int i = 0; i < 2 * r[0] + 1; ++i) {
        int64_t di = i - r[0];
        s += sample(v, cx + di, cy, cz);
    }
    for (int i = 0; i < 2 * r[1] + 1; ++i) {
        int64_t di = i - r[1];
        s += sample(v, cx, cy + di, cz);
    }
    for (int i = 0; i < 2 * r[2] + 1; ++i) {
        int64_t di = i - r[2];
        s += sample(v, cx, cy, cz + di);
    }
    return s;
}

/* The paper's filter (section "Our Method"): the average cluster S_0 at the
 * voxel and eight more S_1..S_8 centred at the diagonal offsets (+-d,+-d,+-d);
 * the voxel is replaced by the mean of the nine cluster averages.  Each S_k is
 * its line sum over the 3M voxels of its three lines (Mx + My + Mz with
 * per-axis radii), so A = U / (9 * 3M). */
static uint32_t filter_ours(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    uint64_t U = cluster_line_sum(v, r, x, y, z);           /* S_0 */
    for (int sz = -1; sz <= 1; sz += 2)
        for (int sy = -1; sy <= 1; sy += 2)
            for (int sx = -1; sx <= 1; sx += 2)
                U += cluster_line_sum(v, r, x + sx * d[0], y + sy * d[1], z + sz * d[2]); /* S_1..S_8 */
    uint64_t den = 9ull * (uint64_t)(2 * r[0] + 1 + 2 * r[1] + 1 + 2 * r[2] + 1);
    uint32_t P0 = sample(v, x, y, z);
    if (P0 < p->threshold || U < den * (uint64_t)p->threshold)
        return 0;
    return round_div(U, den);
}

/* Mean (low-pass) filter, Eq. 4: average over the M^3 cube (Mx x My x Mz). */
static uint32_t filter_mean(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    uint64_t B = 0, n = 0;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i) {
                B += sample(v, x + i, y + j, z + k);
                n += 1;
            }
    uint32_t P0 = sample(v, x, y, z);
    if (P0 < p->threshold || B < n * (uint64_t)p->threshold)
        return 0;
    return round_div(B, n);
}

/* Sigma filter, Eq. 5 (reading: band centred on P0, closed interval
 * |P_i - P0| <= delta, over the M^3 cube; P0 always qualifies). */
static uint32_t filter_sigma(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    uint32_t P0 = sample(v, x, y, z);
    uint64_t s = 0, n = 0;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i) {
                uint32_t Pi = sample(v, x + i, y + j, z + k);
                int64_t diff = (int64_t)Pi - (int64_t)P0;
                if (diff < 0)
                    diff = -diff;
                if (diff <= (int64_t)p->sigma_band) {
                    s += Pi;
                    n += 1;
                }
            }
    if (P0 < p->threshold || s < n * (uint64_t)p->threshold)
        return 0;
    return round_div(s, n);
}

/* Sigma filter with the local standard deviation (Lee's original form, named
 * in "Related Work"): the band |P_i - P0| <= k sigma_local, where sigma_local
 * is the population standard deviation of the M^3 cube itself; with m = M^3,
 * S1 and S2 the sum and the sum of squares over the cube,
 *   (P_i - P0)^2 <= k^2 (m S2 - S1^2) / m^2  <=>  m^2 (P_i - P0)^2 <= k^2 (m S2 - S1^2),
 * compared exactly in integers; then as filter_sigma (mean of the band, gate). */
static uint32_t filter_sigma_local(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], dd[3];
    axis_extents(p, r, dd);
    const uint32_t P0 = sample(v, x, y, z);
    const unsigned __int128 m = (unsigned __int128)(2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1);
    unsigned __int128 S1 = 0, S2 = 0;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i) {
                const uint64_t Pi = sample(v, x + i, y + j, z + k);
                S1 += Pi;
                S2 += (unsigned __int128)Pi * Pi;
            }
    const unsigned __int128 kk = (unsigned __int128)p->sigma_k * p->sigma_k;
    const unsigned __int128 rhs = kk * (m * S2 - S1 * S1);
    uint64_t s = 0, n = 0;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i) {
                const uint32_t Pi = sample(v, x + i, y + j, z + k);
                const unsigned __int128 d = Pi > P0 ? Pi - P0 : P0 - Pi;
                if (m * m * d * d <= rhs) {
                    s += Pi;
                    n += 1;
                }
            }
    if (P0 < p->threshold || s < n * (uint64_t)p->threshold)
        return 0;
    return round_div(s, n);
}

/* Okada filter, Eq. 6 (reading: the centre and its axis-cross neighbours of
 * arm r, i.e. the six direct neighbours at M = 3; strict |P0 - P_i| < T_d;
 * 0 when nothing qualifies). */
static uint32_t filter_okada(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    uint32_t P0 = sample(v, x, y, z);
    uint64_t s = 0, n = 0;
    for (int axis = -1; axis < 3; ++axis) {
        const int arm = axis < 0 ? 0 : r[axis];
        for (int t = -arm; t <= arm; ++t) {
            int64_t ox = 0, oy = 0, oz = 0;
            if (axis == -1) {            /* the centre itself, once */
                if (t != 0)
                    continue;
            } else {
                if (t == 0)
                    continue;
                if (axis == 0) ox = t;
                if (axis == 1) oy = t;
                if (axis == 2) oz = t;
            }
            uint32_t Pi = sample(v, x + ox, y + oy, z + oz);
            int64_t diff = (int64_t)P0 - (int64_t)Pi;
            if (diff < 0)
                diff = -diff;
            if (diff < p->okada_td) {
                s += Pi;
                n += 1;
            }
        }
    }
    if (n == 0)
        return 0;
    if (P0 < p->threshold || s < n * (uint64_t)p->threshold)
        return 0;
    return round_div(s, n);
}

/* Entropy filter, Eq. 7 (reading: p_i is the global probability of the grey
 * level of kernel voxel i; the criterion -sum p_i log2 p_i runs over the m =
 * M^3 cube voxels and is evaluated in the fixed point of the weight table). */
static uint32_t filter_entropy(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    uint64_t E = 0;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i)
                E += p->entropy_w[sample(v, x + i, y + j, z + k)];
    uint32_t P0 = sample(v, x, y, z);
    if (P0 < p->threshold)
        return 0;
    if ((int64_t)E > p->entropy_te)
        return P0;
    return 0;
}

/* Entropy filter with the cube's own grey-level probabilities ("Related Work":
 * the information entropy of the kernel, the average uncertainty of its
 * values).  Of the m = Mx My Mz cube voxels, c_g carry grey level g; the first
 * order entropy of the cube is
 *   H = -sum_g (c_g / m) log2 (c_g / m) = log2 m - (1/m) sum_g c_g log2 c_g,
 * so m 2^22 H = lt[m] - sum_g lt[c_g] in the fixed point of the table lt.
 * Each level is counted once, at its first tap in enumeration order.  The
 * voxel keeps P0 iff P0 >= T and m 2^22 H > m theta (strict, like Eq. 7). */
static uint32_t filter_entropy_local(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    uint32_t vals[ORACLE_MAX_CUBE];
    int64_t m = 0;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i)
                vals[m++] = sample(v, x + i, y + j, z + k);
    uint64_t K = 0;
    for (int64_t a = 0; a < m; ++a) {
        int first = 1;
        for (int64_t b = 0; b < a; ++b)
            if (vals[b] == vals[a]) {
                first = 0;
                break;
            }
        if (!first)
            continue;
        int64_t c = 0;
        for (int64_t b = a; b < m; ++b)
            c += vals[b] == vals[a];
        K += p->entropy_lt[c];
    }
    const int64_t crit = (int64_t)(p->entropy_lt[m] - K);
    const uint32_t P0 = sample(v, x, y, z);
    if (P0 < p->threshold)
        return 0;
    return crit > m * p->entropy_lte ? P0 : 0;
}

/* Cluster-layout variants of the paper's filter ("Our Method": the source
 * carries a commented-out S_0 that averages the centre and its six direct
 * neighbours, and the conclusion proposes analysing other cluster layouts).
 * The nine cluster centres are those of filter_ours; each cluster is
 *   id 5: the centre and the 6r voxels of its axis cross of arm r, averaged
 *         (r = 1 is the commented-out form: (1/7)(P0 + six neighbours));
 *   id 6: the M^3 cube around the centre, averaged;
 * and the voxel is replaced by the mean of the nine cluster averages, gated as
 * filter_ours. */
static uint32_t filter_ours_variant(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    int r[3], d[3];
    axis_extents(p, r, d);
    /* voxels per cluster: the centre and its arms, or the whole box */
    const uint64_t per = p->filter_id == 5 ? 1 + 2 * (uint64_t)(r[0] + r[1] + r[2])
                                           : (uint64_t)(2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1);
    uint64_t U = 0;
    for (int c = 0; c < 9; ++c) {
        int64_t cx = x, cy = y, cz = z;
        if (c > 0) {
            cx += ((c - 1) & 1) ? d[0] : -d[0];
            cy += ((c - 1) & 2) ? d[1] : -d[1];
            cz += ((c - 1) & 4) ? d[2] : -d[2];
        }
        if (p->filter_id == 5) {
            U += sample(v, cx, cy, cz);
            for (int t = 1; t <= r[0]; ++t)
                U += sample(v, cx - t, cy, cz) + sample(v, cx + t, cy, cz);
            for (int t = 1; t <= r[1]; ++t)
                U += sample(v, cx, cy - t, cz) + sample(v, cx, cy + t, cz);
            for (int t = 1; t <= r[2]; ++t)
                U += sample(v, cx, cy, cz - t) + sample(v, cx, cy, cz + t);
        } else {
            for (int k = -r[2]; k <= r[2]; ++k)
                for (int j = -r[1]; j <= r[1]; ++j)
                    for (int i = -r[0]; i <= r[0]; ++i)
                        U += sample(v, cx + i, cy + j, cz + k);
        }
    }
    const uint64_t den = 9 * per;
    if (sample(v, x, y, z) < p->threshold || U < den * p->threshold)
        return 0;
    return round_div(U, den);
}

static uint32_t filter_at(const vol_view *v, const oracle_params *p, int64_t x, int64_t y, int64_t z)
{
    switch (p->filter_id) {
    case 0: return filter_mean(v, p, x, y, z);
    case 1: return filter_sigma(v, p, x, y, z);
    case 2: return filter_entropy(v, p, x, y, z);
    case 3: return filter_okada(v, p, x, y, z);
    case 4: return filter_ours(v, p, x, y, z);
    case 5:
    case 6: return filter_ours_variant(v, p, x, y, z);
    case 7: return filter_sigma_local(v, p, x, y, z);
    case 8: return filter_entropy_local(v, p, x, y, z);
    default: return 0;
    }
}

/* Filter id and extents in range; the local entropy filter needs its table and
 * a cube of at most ORACLE_MAX_CUBE voxels. */
static int params_ok(const oracle_params *p)
{
    if (p->filter_id < 0 || p->filter_id > 8 || p->radius < 0)
        return 0;
    if (p->aniso)
        for (int a = 0; a < 3; ++a)
            if (p->rad[a] < 0 || p->off[a] < 0)
                return 0;
    if (p->filter_id == 8) {
        int r[3], d[3];
        axis_extents(p, r, d);
        if (!p->entropy_lt || (int64_t)(2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1) > ORACLE_MAX_CUBE)
            return 0;
    }
    return 1;
}

/* Filter the box [x0,x1) x [y0,y1) x [z0,z1) of the volume into `out`, which is
 * laid out x-fastest with dims (x1-x0, y1-y0, z1-z0) and the volume's dtype.
 * Returns 0 on success, -1 on bad arguments. */
int oracle_filter_box(const void *vol, int64_t nx, int64_t ny, int64_t nz, int dtype,
                      const oracle_params *p, void *out,
                      int64_t x0, int64_t x1, int64_t y0, int64_t y1, int64_t z0, int64_t z1)
{
    if (!vol || !p || !out || nx < 1 || ny < 1 || nz < 1 || (dtype != 0 && dtype != 1))
        return -1;
    if (x0 < 0 || y0 < 0 || z0 < 0 || x1 > nx || y1 > ny || z1 > nz || x1 < x0 || y1 < y0 || z1 < z0)
        return -1;
    if (!params_ok(p))
        return -1;
    vol_view v = {vol, nx, ny, nz, dtype};
    int64_t bx = x1 - x0, by = y1 - y0;
    for (int64_t z = z0; z < z1; ++z)
        for (int64_t y = y0; y < y1; ++y)
            for (int64_t x = x0; x < x1; ++x) {
                uint32_t f = filter_at(&v, p, x, y, z);
                int64_t o = ((z - z0) * by + (y - y0)) * bx + (x - x0);
                if (dtype == 0)
                    ((uint8_t *)out)[o] = (uint8_t)f;
                else
                    ((uint16_t *)out)[o] = (uint16_t)f;
            }
    return 0;
}

/* Evaluate the filter at npts points given as (x, y, z) triples. */
int oracle_filter_points(const void *vol, int64_t nx, int64_t ny, int64_t nz, int dtype,
                         const oracle_params *p, const int64_t *pts, int64_t npts, uint32_t *vals)
{
    if (!vol || !p || !pts || !vals || nx < 1 || ny < 1 || nz < 1 || (dtype != 0 && dtype != 1))
        return -1;
    if (!params_ok(p))
        return -1;
    vol_view v = {vol, nx, ny, nz, dtype};
    for (int64_t i = 0; i < npts; ++i) {
        int64_t x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz)
            return -1;
        vals[i] = filter_at(&v, p, x, y, z);
    }
    return 0;
}

/* Grey-level histogram (counts per value) and the moments S = sum P,
 * Q = sum P^2, min, max of the whole volume. */
int oracle_stats(const void *vol, int64_t n, int dtype, uint64_t *hist,
                 uint64_t *S, uint64_t *Q_lo, uint64_t *Q_hi, uint32_t *minv, uint32_t *maxv)
{
    if (!vol || n < 1 || (dtype != 0 && dtype != 1))
        return -1;
    int64_t L = dtype == 0 ? 256 : 65536;
    for (int64_t i = 0; i < L; ++i)
        hist[i] = 0;
    unsigned __int128 q = 0;
    uint64_t s = 0;
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t P = dtype == 0 ? ((const uint8_t *)vol)[i] : ((const uint16_t *)vol)[i];
        hist[P] += 1;
        s += P;
        q += (unsigned __int128)P * P;
        if (P < lo) lo = P;
        if (P > hi) hi = P;
    }
    *S = s;
    *Q_lo = (uint64_t)q;
    *Q_hi = (uint64_t)(q >> 64);
    *minv = lo;
    *maxv = hi;
    return 0;
}

/* ------------------------------------------------------------------ rendering
 *
 * The paper's use of its filter ("Introduction", "3D Spatial Noise Filters"):
 * a ray caster marches each pixel's ray through the volume; the first sample
 * at or above the threshold is a candidate surface point, where the filter
 * decides between structure and noise; a candidate the filter keeps (output
 * not 0) ends the ray and is shaded with a normal from a 3D Sobel operator and
 * Phong illumination; a rejected candidate is noise and the ray goes on.
 *
 * Readings (the paper fixes no camera, sampling or shading constants):
 *  - orthographic rays along one of the six axis directions (view 0..5 =
 *    +x, -x, +y, -y, +z, -z), one ray per voxel column, samples at the voxel
 *    centres, no interpolation;
 *  - image axes (u, w): views +-x -> (y, z), +-y -> (x, z), +-z -> (x, y);
 *    pixel index w * W + u;
 *  - Sobel: g_x = sum over the 3x3x3 neighbourhood (clamp-to-edge) of
 *    i * b(j) * b(k) * P(x+i, y+j, z+k) with b(-1) = b(1) = 1, b(0) = 2;
 *    g_y and g_z likewise;
 *  - headlight Phong: c = (g . d) / |g| with d the ray direction (c = 1 when
 *    g = 0); I = (0.1 + 0.7 max(c, 0)) + 0.2 s^16 with s = 2 c^2 - 1 when
 *    c > 0 and s > 0, else 0; pixel = min(255, floor(255 I + 1/2)); 0 where
 *    the ray finds no surface;
 *  - shading in IEEE double, the operations in the written order, no fused
 *    multiply-add (built with -ffp-contract=off).
 */
#include <math.h>

static int render_extent(int view, int64_t nx, int64_t ny, int64_t nz, int64_t *W, int64_t *H, int64_t *len)
{
    switch (view) {
    case 0: case 1: *W = ny; *H = nz; *len = nx; return 0;
    case 2: case 3: *W = nx; *H = nz; *len = ny; return 0;
    case 4: case 5: *W = nx; *H = ny; *len = nz; return 0;
    default: return -1;
    }
}

/* the voxel of ray (u, w) at step k */
static void render_voxel(int view, const vol_view *v, int64_t u, int64_t w, int64_t k,
                         int64_t *x, int64_t *y, int64_t *z)
{
    switch (view) {
    case 0: *x = k; *y = u; *z = w; break;
    case 1: *x = v->nx - 1 - k; *y = u; *z = w; break;
    case 2: *x = u; *y = k; *z = w; break;
    case 3: *x = u; *y = v->ny - 1 - k; *z = w; break;
    case 4: *x = u; *y = w; *z = k; break;
    default: *x = u; *y = w; *z = v->nz - 1 - k; break;
    }
}

static uint8_t shade(const vol_view *v, int view, int64_t x, int64_t y, int64_t z)
{
    static const int64_t b[3] = {1, 2, 1};
    int64_t gx = 0, gy = 0, gz = 0;
    for (int k = -1; k <= 1; ++k)
        for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
                const int64_t P = sample(v, x + i, y + j, z + k);
                gx += i * b[j + 1] * b[k + 1] * P;
                gy += j * b[i + 1] * b[k + 1] * P;
                gz += k * b[i + 1] * b[j + 1] * P;
            }
    const int64_t ga[3] = {gx, gy, gz};
    const int64_t along = ga[view / 2] * ((view & 1) ? -1 : 1);   /* g . d */
    const int64_t n2 = gx * gx + gy * gy + gz * gz;
    const double c = n2 > 0 ? (double)along / sqrt((double)n2) : 1.0;
    const double diff = c > 0.0 ? c : 0.0;
    double spec = 0.0;
    if (c > 0.0) {
        double s = 2.0 * (c * c) - 1.0;
        if (s > 0.0) {
            s = s * s;
            s = s * s;
            s = s * s;
            s = s * s;
            spec = s;
        }
    }
    const double I = (0.1 + 0.7 * diff) + 0.2 * spec;
    const double q = floor(255.0 * I + 0.5);
    return q >= 255.0 ? (uint8_t)255 : (uint8_t)q;
}

/* Render the volume along `view` with the filter of `p` deciding at each
 * candidate; image (W*H bytes), depth (W*H: step of the hit along the ray, or
 * -1) and value (W*H: the filter's output at the hit, or 0). */
int oracle_render(const void *vol, int64_t nx, int64_t ny, int64_t nz, int dtype, const oracle_params *p, int view,
                  uint8_t *image, int32_t *depth, uint32_t *value)
{
    if (!vol || !p || !image || !depth || !value || nx < 1 || ny < 1 || nz < 1 || (dtype != 0 && dtype != 1))
        return -1;
    if (!params_ok(p))
        return -1;
    int64_t W, H, len;
    if (render_extent(view, nx, ny, nz, &W, &H, &len) != 0)
        return -1;
    vol_view v = {vol, nx, ny, nz, dtype};
    for (int64_t w = 0; w < H; ++w)
        for (int64_t u = 0; u < W; ++u) {
            const int64_t o = w * W + u;
            image[o] = 0;
            depth[o] = -1;
            value[o] = 0;
            for (int64_t k = 0; k < len; ++k) {
                int64_t x, y, z;
                render_voxel(view, &v, u, w, k, &x, &y, &z);
                if (sample(&v, x, y, z) < p->threshold)
                    continue;   /* below the threshold: not a candidate */
                const uint32_t f = filter_at(&v, p, x, y, z);
                if (f == 0)
                    continue;   /* the filter calls it noise */
                image[o] = shade(&v, view, x, y, z);
                depth[o] = (int32_t)k;
                value[o] = f;
                break;
            }
        }
    return 0;
}
