/*
 * FP64 CPU oracle: scan geometry and the CT system matrix A (TEST
 * INFRASTRUCTURE ONLY -- used by the tests, the smoke check and the CPU
 * baseline of the benchmark; the product path never links it).
 *
 * The paper leaves A unspecified (Sec. IV, Eq. ct_recon names it only as the
 * scan's system matrix).  Reading taken here: a_ij is the exact length of ray i inside
 * pixel/voxel j (pixel basis, one ray per detector cell through the cell
 * centre), computed by Siddon's algorithm (R. L. Siddon, Med. Phys. 12, 1985):
 * parametrise the ray segment P(a) = P0 + a (P1 - P0), a in [0, 1]; collect the
 * parameters where it crosses the grid planes of every axis inside the image
 * box; merge them in increasing order; each pair of consecutive parameters
 * bounds one pixel, found from the midpoint, with length (a_{k+1}-a_k)|P1-P0|.
 * The back-projection is the transpose of the same A (scatter of the same
 * lengths).  Geometry convention:
 *   phi_v = pi tau_v, tau_v = angle_start/pi + v (angle_span/pi)/nviews,
 *   (cos phi, sin phi) by exact quarter-turn reduction of tau_v (views at
 *   multiples of 90 degrees are exactly axis-aligned), u=(cos phi, sin phi),
 *   e=(-sin phi, cos phi);
 *   parallel: line through s_c e along u, s_c=(c-(ns-1)/2+offset_s) ds;
 *   fan/arc : source -dso u, channel angle g_c = s_c/dsd, the ray ends on the
 *             arc of radius dsd around the source;
 *   cone/flat: source (-dso u, z_v), cell centre (dsd-dso) u + s_c e + (z_v+t_t) z,
 *             t_t=(t-(nt-1)/2+offset_t) dt; z_v = 0 on a circular orbit; on a
 *             helix (pitch > 0) source and detector rise by pitch nt dt per
 *             turn, z_v = pitch nt dt (phi_v - phi_mid)/(2 pi) with phi_mid the
 *             middle of the scanned angle range (a central voxel is then seen
 *             for dso/(pitch dsd) turns, as Sec. IV-B counts);
 *   pixels are half-open boxes [lo, hi): a ray lying exactly on the plane
 *   between two pixels belongs to the upper one (the midpoint rule below
 *   does this; an axis-parallel ray is inside when lo <= p < hi);
 *   pixel centre ((ix-(nx-1)/2) dx + offset_x, ...); images [z][y][x],
 *   sinograms [view][row][channel].
 * Parity unpinned: none (pinned by dense clipping, closed-form chords,
 * analytic ellipse integrals and the adjoint identity in the test suite).
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads of the projector loops (OpenMP).  The rays of a forward
 * projection are independent, so its result does not depend on the thread
 * count; a back-projection sums its views in a fixed number of view groups
 * (see oracle_backproject), so its result does not either. */
static int g_threads = 1;

int oracle_set_threads(int n)
{
    g_threads = n < 1 ? 1 : n;
    return g_threads;
}

int oracle_get_threads(void) { return g_threads; }

typedef struct {
    int kind; /* 0 parallel 2D, 1 fan 2D arc, 2 cone 3D flat */
    int nx, ny, nz;
    double dx, dy, dz;
    double offset_x, offset_y, offset_z;
    int nviews;
    double angle_start, angle_span;
    int ns, nt;
    double ds, dt;
    double offset_s, offset_t;
    double dso, dsd;
    double pitch;
} og_geom;

/* (cos(pi t), sin(pi t)) with exact quarter-turn reduction */
static void cos_sin_pi(double t, double *c, double *s)
{
    double n = floor(2.0 * t + 0.5);
    double r = t - 0.5 * n;
    double cr = cos(M_PI * r), sr = sin(M_PI * r);
    double q = fmod(n, 4.0);
    if (q < 0) q += 4.0;
    if (q == 0.0) { *c = cr; *s = sr; }
    else if (q == 1.0) { *c = -sr; *s = cr; }
    else if (q == 2.0) { *c = -cr; *s = -sr; }
    else { *c = sr; *s = -cr; }
}

/* ray i = (view, row t, channel c) as a segment P0 -> P1 */
static void ray_segment(const og_geom *g, int view, int t, int c, double P0[3], double P1[3])
{
    double tau = g->angle_start / M_PI + (double)view * (g->angle_span / M_PI) / (double)g->nviews;
    double ux, uy;
    cos_sin_pi(tau, &ux, &uy);
    double ex = -uy, ey = ux;
    double s = ((double)c - (g->ns - 1) / 2.0 + g->offset_s) * g->ds;
    if (g->kind == 0) {
        /* long enough to cover the whole image box from any angle */
        double half = 0.5 * sqrt((g->nx * g->dx) * (g->nx * g->dx) + (g->ny * g->dy) * (g->ny * g->dy))
                      + fabs(g->offset_x) + fabs(g->offset_y) + 1.0;
        double T = 2.0 * half + 10.0;
        P0[0] = s * ex - T * ux; P0[1] = s * ey - T * uy; P0[2] = 0.0;
        P1[0] = s * ex + T * ux; P1[1] = s * ey + T * uy; P1[2] = 0.0;
    } else if (g->kind == 1) {
        double gam = s / g->dsd;
        double dxr = cos(gam) * ux + sin(gam) * ex;
        double dyr = cos(gam) * uy + sin(gam) * ey;
        P0[0] = -g->dso * ux; P0[1] = -g->dso * uy; P0[2] = 0.0;
        P1[0] = P0[0] + g->dsd * dxr; P1[1] = P0[1] + g->dsd * dyr; P1[2] = 0.0;
    } else {
        double tt = ((double)t - (g->nt - 1) / 2.0 + g->offset_t) * g->dt;
        double dd = g->dsd - g->dso;
        double zv = 0.0;
        if (g->pitch != 0.0) {
            double dphi = (double)view * (g->angle_span / (double)g->nviews) - 0.5 * g->angle_span;
            zv = g->pitch * g->nt * g->dt * dphi / (2.0 * M_PI);
        }
        P0[0] = -g->dso * ux; P0[1] = -g->dso * uy; P0[2] = zv;
        P1[0] = dd * ux + s * ex; P1[1] = dd * uy + s * ey; P1[2] = zv + tt;
    }
}

typedef void (*visit_fn)(void *ctx, long pix, double len);

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Siddon's algorithm: call visit(pix, length) for every pixel the segment crosses. */
static void siddon(const og_geom *g, const double P0[3], const double P1[3], int three_d,
                   double *alphas, visit_fn visit, void *ctx)
{
    int n[3] = {g->nx, g->ny, three_d ? g->nz : 1};
    double d[3] = {g->dx, g->dy, three_d ? g->dz : 1.0};
    double off[3] = {g->offset_x, g->offset_y, three_d ? g->offset_z : 0.0};
    double lo[3], D[3];
    int naxes = three_d ? 3 : 2;
    double amin = 0.0, amax = 1.0;
    for (int k = 0; k < naxes; ++k) {
        lo[k] = off[k] - 0.5 * n[k] * d[k];
        D[k] = P1[k] - P0[k];
        double hi = lo[k] + n[k] * d[k];
        if (D[k] != 0.0) {
            double a0 = (lo[k] - P0[k]) / D[k];
            double a1 = (hi - P0[k]) / D[k];
            double mn = a0 < a1 ? a0 : a1, mx = a0 < a1 ? a1 : a0;
            if (mn > amin) amin = mn;
            if (mx < amax) amax = mx;
        } else if (P0[k] < lo[k] || P0[k] >= hi) {
            return; /* parallel to this axis and outside the slab */
        }
    }
    if (amax <= amin) return;
    double len = 0.0;
    for (int k = 0; k < naxes; ++k) len += D[k] * D[k];
    len = sqrt(len);
    /* gather crossing parameters of every plane strictly inside (amin, amax) */
    int cnt = 0;
    alphas[cnt++] = amin;
    for (int k = 0; k < naxes; ++k) {
        if (D[k] == 0.0) continue;
        for (int i = 0; i <= n[k]; ++i) {
            double a = (lo[k] + i * d[k] - P0[k]) / D[k];
            if (a > amin && a < amax) alphas[cnt++] = a;
        }
    }
    alphas[cnt++] = amax;
    qsort(alphas, (size_t)cnt, sizeof(double), cmp_double);
    for (int q = 0; q + 1 < cnt; ++q) {
        double a0 = alphas[q], a1 = alphas[q + 1];
        if (a1 <= a0) continue;
        double am = 0.5 * (a0 + a1);
        long idx[3] = {0, 0, 0};
        int inside = 1;
        for (int k = 0; k < naxes; ++k) {
            double p = P0[k] + am * D[k];
            long i = (long)floor((p - lo[k]) / d[k]);
            if (i < 0 || i >= n[k]) inside = 0;
            idx[k] = i;
        }
        if (!inside) continue;
        long pix = (idx[2] * (long)n[1] + idx[1]) * (long)n[0] + idx[0];
        visit(ctx, pix, (a1 - a0) * len);
    }
}

typedef struct { const double *x; double acc; } fp_ctx;
static void fp_visit(void *c, long pix, double len)
{
    fp_ctx *f = (fp_ctx *)c;
    f->acc += len * f->x[pix];
}

typedef struct { double *img; double val; } bp_ctx;
static void bp_visit(void *c, long pix, double len)
{
    bp_ctx *b = (bp_ctx *)c;
    b->img[pix] += len * b->val;
}

static int check_geom(const og_geom *g)
{
    if (!g) return -1;
    if (g->kind < 0 || g->kind > 2) return -1;
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->nviews <= 0 || g->ns <= 0 || g->nt <= 0) return -1;
    if (g->kind != 2 && (g->nz != 1 || g->nt != 1)) return -1;
    if (g->kind != 0 && !(g->dsd > g->dso && g->dso > 0)) return -1;
    return 0;
}

static long alpha_capacity(const og_geom *g)
{
    return (long)g->nx + g->ny + (g->kind == 2 ? g->nz : 1) + 8;
}

/* out[v][t][c] = sum_j a_ij x_j for the rays of the listed views. */
int oracle_project(const og_geom *g, const double *x, const int *views, int nv, double *out)
{
    if (check_geom(g)) return -1;
    for (int iv = 0; iv < nv; ++iv)
        if (views[iv] < 0 || views[iv] >= g->nviews) return -1;
    const int three_d = g->kind == 2;
    const long nrays = (long)nv * g->nt * g->ns;
    int err = 0;
#pragma omp parallel num_threads(g_threads)
    {
        double *alphas = (double *)malloc(sizeof(double) * (size_t)alpha_capacity(g));
        if (!alphas) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < nrays; ++i) {
            if (!alphas) continue;
            const int c = (int)(i % g->ns);
            const int t = (int)((i / g->ns) % g->nt);
            const int iv = (int)(i / ((long)g->ns * g->nt));
            double P0[3], P1[3];
            ray_segment(g, views[iv], t, c, P0, P1);
            fp_ctx f = {x, 0.0};
            siddon(g, P0, P1, three_d, alphas, fp_visit, &f);
            out[i] = f.acc;
        }
        free(alphas);
    }
    return err;
}

/* img_j = sum_i a_ij sino_i over the rays of the listed views (img overwritten).
 * The views are dealt to G groups (list position iv to group iv mod G, G
 * fixed by the sizes alone); each group scatters its rays, in list order,
 * into its own image, and the group images are added in group order. */
int oracle_backproject(const og_geom *g, const double *sino, const int *views, int nv, double *img)
{
    if (check_geom(g)) return -1;
    for (int iv = 0; iv < nv; ++iv)
        if (views[iv] < 0 || views[iv] >= g->nviews) return -1;
    const int three_d = g->kind == 2;
    const long npix = (long)g->nx * g->ny * g->nz;
    int G = nv < 32 ? nv : 32;
    while (G > 1 && (double)G * npix * sizeof(double) > 2.0e9) G /= 2;
    memset(img, 0, sizeof(double) * (size_t)npix);
    if (G < 1) return 0;
    double **part = (double **)calloc((size_t)G, sizeof(double *));
    if (!part) return -2;
    int err = 0;
    part[0] = img;
    for (int k = 1; k < G; ++k) {
        part[k] = (double *)calloc((size_t)npix, sizeof(double));
        if (!part[k]) err = -2;
    }
    if (!err) {
#pragma omp parallel num_threads(g_threads)
        {
            double *alphas = (double *)malloc(sizeof(double) * (size_t)alpha_capacity(g));
            if (!alphas) {
#pragma omp atomic write
                err = -2;
            }
#pragma omp for schedule(dynamic, 1)
            for (int k = 0; k < G; ++k) {
                if (!alphas) continue;
                for (int iv = k; iv < nv; iv += G)
                    for (int t = 0; t < g->nt; ++t)
                        for (int c = 0; c < g->ns; ++c) {
                            double P0[3], P1[3];
                            ray_segment(g, views[iv], t, c, P0, P1);
                            bp_ctx b = {part[k], sino[((long)iv * g->nt + t) * g->ns + c]};
                            if (b.val == 0.0) continue;
                            siddon(g, P0, P1, three_d, alphas, bp_visit, &b);
                        }
            }
            free(alphas);
        }
    }
    if (!err && G > 1) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (long j = 0; j < npix; ++j) {
            double acc = img[j];
            for (int k = 1; k < G; ++k) acc += part[k][j];
            img[j] = acc;
        }
    }
    for (int k = 1; k < G; ++k) free(part[k]);
    free(part);
    return err;
}

/* Segment end points of every ray of one view, [nt][ns][2][3] (for tests). */
int oracle_ray_segments(const og_geom *g, int view, double *out)
{
    if (check_geom(g)) return -1;
    for (int t = 0; t < g->nt; ++t)
        for (int c = 0; c < g->ns; ++c) {
            double *p = out + ((long)t * g->ns + c) * 6;
            ray_segment(g, view, t, c, p, p + 3);
        }
    return 0;
}
