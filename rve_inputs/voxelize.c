/*
 * voxelize.c -- seeded synthetic inputs: the octet-truss unit cell as a
 * per-voxel solid fraction phi in [0,1].
 *
 * Geometry (the paper's section 4.1 names the octet truss but does not define
 * it): the FCC nearest-neighbour truss.  Nodes at the four FCC lattice points
 * of the unit cell, struts along the 12 nearest-neighbour directions
 * (length L/sqrt(2)), each a capsule of radius r (cylinder plus spherical
 * caps), periodic.  24 distinct struts per cell.
 *
 * phi of a voxel is the fraction of its s^3 sub-cell centres that lie inside
 * the solid -- the "Voigt fine grid" volume fraction of section 3.3.  The
 * strut radius is chosen so that the mean of phi equals the requested
 * relative density to within one sub-sample, 1/(s^3 V) (section 4.3 measures
 * the model density as the mean of phi).
 *
 * This file holds geometry only; none of the homogenization arithmetic.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The 4 FCC lattice points and 6 of the 12 neighbour directions (one of each
 * +- pair), so that {node + t*dir, t in [0,1]} enumerates each strut once. */
static const double NODES[4][3] = {
    {0.0, 0.0, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};
static const double DIRS[6][3] = {
    {0.5, 0.5, 0.0}, {0.5, -0.5, 0.0}, {0.5, 0.0, 0.5},
    {0.5, 0.0, -0.5}, {0.0, 0.5, 0.5}, {0.0, 0.5, -0.5}};

static double wrap(double a) { return a - floor(a + 0.5); }  /* to [-1/2, 1/2) */

/* Distance from the point p (unit-cell coordinates) to the nearest strut
 * axis.  Exact whenever the result is below 1/2 - sqrt(2)/4 ~ 0.146 (the
 * wrapped midpoint offset then selects the nearest periodic image); larger
 * results are lower-bounded by that value, which is all the caller needs. */
static double octet_axis_distance(const double p[3]) {
    double best = 1e30;
    for (int a = 0; a < 4; ++a) {
        for (int d = 0; d < 6; ++d) {
            double h[3], r[3];
            for (int i = 0; i < 3; ++i) {
                h[i] = 0.5 * DIRS[d][i];
                r[i] = wrap(p[i] - (NODES[a][i] + h[i]));
            }
            double hh = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
            double t = (r[0] * h[0] + r[1] * h[1] + r[2] * h[2]) / hh;
            if (t > 1.0) t = 1.0;
            if (t < -1.0) t = -1.0;
            double e0 = r[0] - t * h[0], e1 = r[1] - t * h[1], e2 = r[2] - t * h[2];
            double dd = e0 * e0 + e1 * e1 + e2 * e2;
            if (dd < best) best = dd;
        }
    }
    return sqrt(best);
}

static int cmp_float(const void *a, const void *b) {
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* Distance of the point at grid position (i + u, j + v, k + w) / n, repeated
 * `cells` times per box edge. */
static double dist_at(const int n[3], int cells, double gi, double gj, double gk) {
    double p[3] = {cells * gi / n[0], cells * gj / n[1], cells * gk / n[2]};
    return octet_axis_distance(p);
}

/* Perturbation at grid position (gi, gj, gk): trilinear interpolation of the
 * per-voxel values p, which sit at the voxel centres (i + 1/2, ...); periodic. */
static double pert_at(const float *p, const int n[3], double gi, double gj, double gk) {
    const double g[3] = {gi - 0.5, gj - 0.5, gk - 0.5};
    int i0[3], i1[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double f = floor(g[a]);
        t[a] = g[a] - f;
        int b = (int)f % n[a];
        if (b < 0) b += n[a];
        i0[a] = b;
        i1[a] = (b + 1) % n[a];
    }
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
        const int x = (c & 4) ? i1[0] : i0[0], y = (c & 2) ? i1[1] : i0[1], z = (c & 1) ? i1[2] : i0[2];
        const double w = ((c & 4) ? t[0] : 1.0 - t[0]) * ((c & 2) ? t[1] : 1.0 - t[1]) *
                         ((c & 1) ? t[2] : 1.0 - t[2]);
        acc += w * p[((long)x * n[1] + y) * n[2] + z];
    }
    return acc;
}

/* Largest change of p between voxel v and any of its 26 periodic neighbours:
 * bounds how far the interpolated perturbation inside voxel v strays from its
 * centre value. */
static float pert_spread(const float *p, const int n[3], long v) {
    int i = (int)(v / ((long)n[1] * n[2])), j = (int)((v / n[2]) % n[1]), k = (int)(v % n[2]);
    float m = 0.f;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
                int x = (i + a + n[0]) % n[0], y = (j + b + n[1]) % n[1], z = (k + c + n[2]) % n[2];
                float d = fabsf(p[((long)x * n[1] + y) * n[2] + z] - p[v]);
                if (d > m) m = d;
            }
    return m;
}

/*
 * phi: output, V floats.  n: grid.  cells: unit cells per box edge.
 * rho: target relative density.  sub: sub-samples per voxel edge (4 for 4^3).
 * dist_perturb: optional V floats (unit-cell units, one per voxel centre),
 *   interpolated trilinearly to every sub-sample point and added to its axis
 *   distance; may be NULL (used for as-printed surfaces).
 * Returns the strut radius in unit-cell units (negative on failure).
 */
double octet_phi(float *phi, const int n[3], int cells, double rho, int sub,
                 const float *dist_perturb) {
    long V = (long)n[0] * n[1] * n[2];
    int S = sub * sub * sub;
    float *dc = (float *)malloc(sizeof(float) * V);
    float *sp = (float *)malloc(sizeof(float) * V);
    if (!dc || !sp) {
        free(dc);
        free(sp);
        return -1.0;
    }
    /* 1. axis distance at voxel centres, and how far the perturbation may
     *    move it inside the voxel (sub-point distances lie within
     *    dc +- (sp + delta), delta the geometric half diagonal below) */
#pragma omp parallel for schedule(static)
    for (long v = 0; v < V; ++v) {
        int i = (int)(v / ((long)n[1] * n[2])), j = (int)((v / n[2]) % n[1]), k = (int)(v % n[2]);
        double d = dist_at(n, cells, i + 0.5, j + 0.5, k + 0.5);
        if (dist_perturb) d += dist_perturb[v];
        dc[v] = (float)d;
        sp[v] = dist_perturb ? pert_spread(dist_perturb, n, v) : 0.f;
    }
    /* 2. plain-voxel estimate of the radius: quantile of the centre distances */
    float *sorted = (float *)malloc(sizeof(float) * V);
    memcpy(sorted, dc, sizeof(float) * V);
    qsort(sorted, V, sizeof(float), cmp_float);
    long kpv = (long)llround(rho * (double)V);
    if (kpv < 1) kpv = 1;
    if (kpv > V - 1) kpv = V - 1;
    double r0 = 0.5 * (sorted[kpv - 1] + sorted[kpv]);
    free(sorted);
    /* half diagonal of a voxel, in unit-cell units (1-Lipschitz bound) */
    double hx = cells / (double)n[0], hy = cells / (double)n[1], hz = cells / (double)n[2];
    double delta = 0.5 * sqrt(hx * hx + hy * hy + hz * hz);
    double band = 2.0 * delta;
    double radius = -1.0;
    long target = (long)llround(rho * (double)V * S);
    for (int attempt = 0; attempt < 12 && radius < 0; ++attempt, band *= 2.0) {
        double lo = r0 - band, hi = r0 + band;
        long n_inner = 0, n_band = 0;
        /* inner: every sub-point certainly below lo; band: sub-sampled */
        for (long v = 0; v < V; ++v) {
            if (dc[v] + sp[v] < lo) ++n_inner;
            else if (dc[v] - sp[v] <= hi) ++n_band;
        }
        float *bd = (float *)malloc(sizeof(float) * (size_t)n_band * S);
        long *bidx = (long *)malloc(sizeof(long) * (size_t)(n_band > 0 ? n_band : 1));
        long c = 0;
        for (long v = 0; v < V; ++v)
            if (dc[v] + sp[v] >= lo && dc[v] - sp[v] <= hi) bidx[c++] = v;
#pragma omp parallel for schedule(dynamic, 256)
        for (long b = 0; b < n_band; ++b) {
            long v = bidx[b];
            int i = (int)(v / ((long)n[1] * n[2])), j = (int)((v / n[2]) % n[1]), k = (int)(v % n[2]);
            int s = 0;
            for (int a = 0; a < sub; ++a)
                for (int bb = 0; bb < sub; ++bb)
                    for (int cc = 0; cc < sub; ++cc) {
                        const double gi = i + (a + 0.5) / sub, gj = j + (bb + 0.5) / sub,
                                     gk = k + (cc + 0.5) / sub;
                        double d = dist_at(n, cells, gi, gj, gk);
                        if (dist_perturb) d += pert_at(dist_perturb, n, gi, gj, gk);
                        bd[b * S + s++] = (float)d;
                    }
        }
        long kk = target - n_inner * S;       /* sub-points the band must supply */
        long nb = n_band * S;
        if (kk >= 1 && kk < nb) {
            float *sb = (float *)malloc(sizeof(float) * (size_t)nb);
            memcpy(sb, bd, sizeof(float) * (size_t)nb);
            qsort(sb, nb, sizeof(float), cmp_float);
            /* equal distances (the cell is symmetric) can make the exact
             * count unreachable: take the nearer end of the run of ties */
            long a = kk - 1, b = kk;
            while (a > 0 && sb[a - 1] == sb[kk - 1]) --a;        /* first tie */
            while (b < nb && sb[b] == sb[kk - 1]) ++b;           /* past ties */
            long cnt = (kk - a <= b - kk) ? a : b;               /* points below r */
            if (cnt < 1) cnt = b;
            if (cnt >= nb) cnt = a;
            double r = 0.5 * ((double)sb[cnt - 1] + (double)sb[cnt]);
            /* valid only if the voxels outside the band stay fully in/out */
            if (cnt >= 1 && cnt < nb && sb[cnt - 1] < sb[cnt] &&
                r >= lo + delta && r <= hi - delta) {
                radius = r;
                for (long v = 0; v < V; ++v) phi[v] = (dc[v] + sp[v] < lo) ? 1.0f : 0.0f;
#pragma omp parallel for schedule(static)
                for (long b = 0; b < n_band; ++b) {
                    int cnt = 0;
                    for (int s = 0; s < S; ++s) cnt += (bd[b * S + s] < r);
                    phi[bidx[b]] = (float)cnt / (float)S;
                }
            }
            free(sb);
        }
        free(bd);
        free(bidx);
    }
    free(dc);
    free(sp);
    return radius;
}

/* phi for a given radius by sub-sampling every voxel (no band shortcut);
 * used by tests of octet_phi. */
void octet_phi_at_radius(float *phi, const int n[3], int cells, double r, int sub, const float *dist_perturb) {
    long V = (long)n[0] * n[1] * n[2];
    int S = sub * sub * sub;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < V; ++v) {
        int i = (int)(v / ((long)n[1] * n[2])), j = (int)((v / n[2]) % n[1]), k = (int)(v % n[2]);
        int cnt = 0;
        for (int a = 0; a < sub; ++a)
            for (int bb = 0; bb < sub; ++bb)
                for (int cc = 0; cc < sub; ++cc) {
                    const double gi = i + (a + 0.5) / sub, gj = j + (bb + 0.5) / sub, gk = k + (cc + 0.5) / sub;
                    double d = dist_at(n, cells, gi, gj, gk);
                    if (dist_perturb) d += pert_at(dist_perturb, n, gi, gj, gk);
                    cnt += ((float)d < r);
                }
        phi[v] = (float)cnt / (float)S;
    }
}

/* Axis distances of every voxel's sub^3 sub-sample points: out[v * sub^3 + s]
 * (V sub^3 floats); a density family is then a threshold per radius. */
void octet_subpoint_distances(float *out, const int n[3], int cells, int sub) {
    long V = (long)n[0] * n[1] * n[2];
    int S = sub * sub * sub;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < V; ++v) {
        int i = (int)(v / ((long)n[1] * n[2])), j = (int)((v / n[2]) % n[1]), k = (int)(v % n[2]);
        int s = 0;
        for (int a = 0; a < sub; ++a)
            for (int bb = 0; bb < sub; ++bb)
                for (int cc = 0; cc < sub; ++cc)
                    out[v * S + s++] = (float)dist_at(n, cells, i + (a + 0.5) / sub, j + (bb + 0.5) / sub,
                                                      k + (cc + 0.5) / sub);
    }
}

/* Axis distance field at voxel centres (for tests of the geometry). */
void octet_center_distance(float *out, const int n[3], int cells) {
    long V = (long)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (long v = 0; v < V; ++v) {
        int i = (int)(v / ((long)n[1] * n[2])), j = (int)((v / n[2]) % n[1]), k = (int)(v % n[2]);
        out[v] = (float)dist_at(n, cells, i + 0.5, j + 0.5, k + 0.5);
    }
}
