// Geometry / system-model set-up, subset tables and the error model of the
// C ABI.  Host code, FP64; the per-ray tables it uploads are what the 2D
// projector pair reads (see common.cuh, Ray2).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "common.cuh"

namespace oslalm {

static thread_local char g_err[1024] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

bool is_3d(const oslalm_geom *g) { return g->d.kind == OSLALM_CONE3D_FLAT; }

// (cos(pi t), sin(pi t)) with the quarter turn taken out exactly, so that
// views at multiples of 90 degrees are exactly axis-aligned.
static void cos_sin_turns(double t, double *c, double *s) {
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

static double view_turns(const oslalm_geom_desc &d, int v) {
    return d.angle_start / M_PI + (double)v * (d.angle_span / M_PI) / (double)d.nviews;
}

// Parameters of the 2D line through P with unit direction (dx_, dy_).  If
// lo is given, it receives the FP32 rounding residues of f0 and kappa_lo
// (exact value minus the stored float), for callers that carry them.
static Ray2 make_ray2(const oslalm_geom_desc &d, double px, double py, double ux, double uy,
                      float *lo = nullptr) {
    const double xlo = d.offset_x - 0.5 * d.nx * d.dx;
    const double ylo = d.offset_y - 0.5 * d.ny * d.dy;
    const double ax = ux / d.dx, ay = uy / d.dy;  // direction in index units
    Ray2 r;
    int axis;
    double kappa, lrow, b0;
    if (fabs(ax) >= fabs(ay)) {  // x-major: b = y index along a = x index
        axis = 0;
        kappa = ay / ax;
        lrow = d.dx / fabs(ux);
        double yat = py + (xlo - px) * (uy / ux);
        b0 = (yat - ylo) / d.dy;
    } else {
        axis = 1;
        kappa = ax / ay;
        lrow = d.dy / fabs(uy);
        double xat = px + (ylo - py) * (ux / uy);
        b0 = (xat - xlo) / d.dx;
    }
    const int Na = axis ? d.ny : d.nx, Nb = axis ? d.nx : d.ny;
    int k = (int)nearbyint(kappa * 2048.0);
    if (k > 2048) k = 2048;
    if (k < -2048) k = -2048;
    double n0 = floor(b0 + 0.5);
    // a ray crosses the image only if b0 lies within [-Na, Nb + Na]; others get
    // zero length (and a representable n0)
    bool misses = !(b0 > -(double)Na - 2.0 && b0 < (double)(Nb + Na) + 2.0);
    if (misses) n0 = -(double)Na - 4.0;
    r.f0 = misses ? 0.f : (float)(b0 - n0);
    r.kappa_lo = (float)(kappa - k / 2048.0);
    r.lrow = misses ? 0.f : (float)lrow;
    r.packed = (int)((unsigned)k << 16) | (((int)n0 & 0x7fff) << 1) | axis;
    if (lo) {
        lo[0] = misses ? 0.f : (float)((b0 - n0) - (double)r.f0);
        lo[1] = (float)((kappa - k / 2048.0) - (double)r.kappa_lo);
    }
    return r;
}

// Device form of a 2D ray: integer fields as exact floats and the row
// half-width in float32 (fmaf is correctly rounded on every host).
static RayP make_rayp(const Ray2 &r) {
    RayP o;
    const int k = ray_k(r.packed);
    o.f0 = r.f0;
    o.kappa_lo = r.kappa_lo;
    o.lrow = r.lrow;
    o.kq = (float)k * 2.44140625e-4f;
    o.n0f = (float)ray_n0(r.packed);
    o.hw = fabsf(fmaf((float)k, 2.44140625e-4f, 0.5f * r.kappa_lo));
    o.axis = ray_axis(r.packed);
    o.lscale = o.hw > 0.f ? (float)((double)o.lrow / (2.0 * (double)o.hw)) : 0.f;
    return o;
}

// 2D ray parameters of every channel of view v (FP64 set-up).
static void ray_table_view(const oslalm_geom_desc &d, int v, Ray2 *out) {
    double cu, su;
    cos_sin_turns(view_turns(d, v), &cu, &su);
    const double ex = -su, ey = cu;
    for (int c = 0; c < d.ns; ++c) {
        double s = ((double)c - (d.ns - 1) / 2.0 + d.offset_s) * d.ds;
        double px, py, ux, uy;
        if (d.kind == OSLALM_PAR2D) {
            px = s * ex; py = s * ey; ux = cu; uy = su;
        } else {
            double gam = s / d.dsd;
            double cg = cos(gam), sg = sin(gam);
            px = -d.dso * cu; py = -d.dso * su;
            ux = cg * cu + sg * ex;
            uy = cg * su + sg * ey;
        }
        out[c] = make_ray2(d, px, py, ux, uy);
    }
}

// Cone-beam ray families of view v (FP64 set-up): transaxial line from the
// source through detector column c, and the height fraction alpha(a).
static void ray3_table_view(const oslalm_geom_desc &d, int v, Ray3 *out) {
    double cu, su;
    cos_sin_turns(view_turns(d, v), &cu, &su);
    const double ex = -su, ey = cu;
    const double sx = -d.dso * cu, sy = -d.dso * su;
    const double xlo = d.offset_x - 0.5 * d.nx * d.dx;
    const double ylo = d.offset_y - 0.5 * d.ny * d.dy;
    for (int c = 0; c < d.ns; ++c) {
        double s = ((double)c - (d.ns - 1) / 2.0 + d.offset_s) * d.ds;
        double dxv = d.dsd * cu + s * ex, dyv = d.dsd * su + s * ey;
        double ld = sqrt(dxv * dxv + dyv * dyv);
        double ux = dxv / ld, uy = dyv / ld;
        Ray3 r;
        float lo[2];
        r.xy = make_ray2(d, sx, sy, ux, uy, lo);
        r.f0l = lo[0];
        r.kll = lo[1];
        int axis = ray_axis(r.xy.packed);
        double u_a = axis ? uy : ux;
        double s_a = axis ? sy : sx;
        double a_lo = axis ? ylo : xlo;
        double da = axis ? d.dy : d.dx;
        double alpha0 = (a_lo - s_a) / (u_a * ld);
        double alpha1 = da / (u_a * ld);
        double Z0 = alpha0 * d.dt / (2.0 * d.dz);
        double W1 = alpha1 * d.dt / (4.0 * d.dz);  // Z1 / 2
        // z0h: Z0 rounded to 15 significant bits
        int e0;
        frexp(Z0, &e0);
        double z0h = Z0 == 0.0 ? 0.0 : ldexp(nearbyint(ldexp(Z0, 15 - e0)), e0 - 15);
        r.z0h = (float)z0h;
        r.z0l = (float)(Z0 - z0h);
        // kw / 2^sw: W1 with |kw| < 512
        int e1 = 0;
        if (W1 != 0.0) frexp(W1, &e1);
        int sw = 9 - e1;  // |W1| 2^sw in [256, 512)
        if (sw > 30) sw = 30;
        if (sw < 0) sw = 0;
        int kw = (int)nearbyint(ldexp(W1, sw));
        if (kw > 511) kw = 511;
        if (kw < -511) kw = -511;
        r.kw = kw;
        r.sw = sw;
        r.w1l = (float)(W1 - ldexp((double)kw, -sw));
        // offset of the bottom face: zb = (z - z_v)/dz + nz/2 - offset_z/dz + z_v/dz,
        // z_v the source height of this view (helix; 0 on a circular orbit)
        double zv = 0.0;
        if (d.pitch != 0.0) {
            const double dphi = (double)v * (d.angle_span / (double)d.nviews) - 0.5 * d.angle_span;
            zv = d.pitch * d.nt * d.dt * dphi / (2.0 * M_PI);
        }
        double oz = 0.5 * d.nz - d.offset_z / d.dz + zv / d.dz;
        double ozi = floor(oz);
        r.oz_i = (int)ozi;
        r.oz_f = (float)(oz - ozi);
        r.oz_fl = (float)((oz - ozi) - (double)r.oz_f);
        r.pad2 = 0.f;
        r.q = (float)(d.dt / (2.0 * ld));
        out[c] = r;
    }
}

static int validate(const oslalm_geom_desc *d) {
    if (!d) return fail(OSLALM_ERR_ARG, "geometry descriptor is NULL");
    if (d->kind < 0 || d->kind > 2) return fail(OSLALM_ERR_ARG, "unknown geometry kind %d", d->kind);
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || d->nviews <= 0 || d->ns <= 0 || d->nt <= 0)
        return fail(OSLALM_ERR_ARG, "sizes must be positive");
    if (!(d->pitch >= 0.0 && d->pitch < 1e6)) return fail(OSLALM_ERR_ARG, "pitch must be >= 0");
    if (d->pitch != 0.0 && d->kind != OSLALM_CONE3D_FLAT) return fail(OSLALM_ERR_ARG, "a helix needs the cone beam");
    if (d->kind != OSLALM_CONE3D_FLAT && (d->nz != 1 || d->nt != 1))
        return fail(OSLALM_ERR_ARG, "2D geometries need nz = nt = 1");
    if (!(d->dx > 0 && d->dy > 0 && d->dz > 0 && d->ds > 0 && d->dt > 0))
        return fail(OSLALM_ERR_ARG, "pixel and detector pitches must be positive");
    if ((long)d->nx * d->ny * d->nz > (1L << 31) - 1 || (long)d->nviews * d->ns * d->nt > (1L << 31) - 1)
        return fail(OSLALM_ERR_RANGE, "image or sinogram exceeds 2^31 elements");
    if (d->nx > 4096 || d->ny > 4096 || d->nviews > (1 << 24) || d->ns > (1 << 16))
        return fail(OSLALM_ERR_RANGE, "dimension too large (nx, ny <= 4096)");
    if (d->kind != OSLALM_PAR2D) {
        if (!(d->dso > 0 && d->dsd > d->dso)) return fail(OSLALM_ERR_ARG, "need 0 < dso < dsd");
        double hx = 0.5 * d->nx * d->dx + fabs(d->offset_x);
        double hy = 0.5 * d->ny * d->dy + fabs(d->offset_y);
        double r = sqrt(hx * hx + hy * hy);
        if (!(r < d->dso && r < d->dsd - d->dso))
            return fail(OSLALM_ERR_ARG, "image box (radius %.3f mm) must lie inside the source circle and before the detector", r);
        if (d->kind == OSLALM_CONE3D_FLAT) {
            if (fabs(2.0 * d->offset_t - nearbyint(2.0 * d->offset_t)) > 1e-12)
                return fail(OSLALM_ERR_ARG, "cone beam: offset_t must be a multiple of 1/2 row");
            if (d->nt > 256) return fail(OSLALM_ERR_RANGE, "cone beam: at most 256 detector rows");
            if (d->nz > 4096) return fail(OSLALM_ERR_RANGE, "cone beam: at most 4096 slices");
            // a ray rises by less than one slice per transaxial row (so a row
            // meets at most two slices): tan(cone angle) <= (nt/2 + |offset_t|)
            // dt / dsd, and a row is at most sqrt(2) max(dx, dy) long in the plane
            const double tan_cone = (0.5 * d->nt + fabs(d->offset_t)) * d->dt / d->dsd;
            if (tan_cone * sqrt(2.0) * fmax(d->dx, d->dy) >= d->dz)
                return fail(OSLALM_ERR_RANGE, "cone beam: cone angle too wide for the slice thickness (a ray "
                                              "must rise by less than one slice per pixel row)");
        }
        double gmax = fabs((0.5 * d->ns + fabs(d->offset_s)) * d->ds / d->dsd);
        if (d->kind == OSLALM_FAN2D_ARC && gmax >= 1.2)
            return fail(OSLALM_ERR_RANGE, "fan angle too wide");
    }
    return 0;
}

Geo2 geo2_of(const oslalm_geom *g);

}  // namespace oslalm

using namespace oslalm;

oslalm::Geo2 oslalm_geom::geo2() const {
    Geo2 o;
    o.kind = d.kind;
    o.nx = d.nx;
    o.ny = d.ny;
    o.ns = d.ns;
    o.nviews = d.nviews;
    o.dx = (float)d.dx;
    o.dy = (float)d.dy;
    o.xlo = (float)(d.offset_x - 0.5 * d.nx * d.dx);
    o.ylo = (float)(d.offset_y - 0.5 * d.ny * d.dy);
    o.inv_ds = (float)(1.0 / d.ds);
    o.c0 = (float)((d.ns - 1) / 2.0 - d.offset_s);
    o.dso = (float)d.dso;
    o.dsd = (float)d.dsd;
    o.half_diag = (float)(0.5 * sqrt(d.dx * d.dx + d.dy * d.dy));
    // |b| <= a at every pixel centre when the image's corners stay within
    // dso / sqrt(2) of the rotation centre
    double rc = 0.0;
    for (int cx = -1; cx <= 1; cx += 2)
        for (int cy = -1; cy <= 1; cy += 2) {
            double ex = d.offset_x + cx * 0.5 * d.nx * d.dx, ey = d.offset_y + cy * 0.5 * d.ny * d.dy;
            rc = fmax(rc, sqrt(ex * ex + ey * ey));
        }
    o.fast_atan = d.kind == OSLALM_FAN2D_ARC && rc < 0.99 * d.dso / sqrt(2.0);
    o.rays = d_rays;
    o.views = d_views;
    return o;
}

oslalm::Geo3 oslalm_geom::geo3() const {
    Geo3 o;
    o.nx = d.nx; o.ny = d.ny; o.nz = d.nz; o.ns = d.ns; o.nt = d.nt; o.nviews = d.nviews;
    o.dx = (float)d.dx; o.dy = (float)d.dy; o.dz = (float)d.dz;
    o.inv_dz = (float)(1.0 / d.dz);
    o.zlo = (float)(d.offset_z - 0.5 * d.nz * d.dz);
    o.xlo = (float)(d.offset_x - 0.5 * d.nx * d.dx);
    o.ylo = (float)(d.offset_y - 0.5 * d.ny * d.dy);
    o.dt = (float)d.dt;
    o.t0 = (float)((d.nt - 1) / 2.0 - d.offset_t);
    o.u0 = (int)nearbyint((d.nt - 1) - 2.0 * d.offset_t);
    o.inv_ds = (float)(1.0 / d.ds);
    o.c0 = (float)((d.ns - 1) / 2.0 - d.offset_s);
    o.dso = (float)d.dso; o.dsd = (float)d.dsd;
    o.half_diag = (float)(0.5 * sqrt(d.dx * d.dx + d.dy * d.dy));
    o.rays = d_rays3;
    o.views = d_views;
    return o;
}

extern "C" {

const char *oslalm_last_error(void) { return oslalm::g_err; }

int oslalm_version(void) { return 100; }

int oslalm_geom_create(const oslalm_geom_desc *desc, oslalm_geom **out) {
    clear_error();
    if (!out) return fail(OSLALM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (int rc = validate(desc)) return rc;
    const oslalm_geom_desc &d = *desc;
    oslalm_geom *g = new (std::nothrow) oslalm_geom();
    if (!g) return fail(OSLALM_ERR_ALLOC, "host allocation failed");
    g->d = d;
    cudaGetDevice(&g->device);
    std::vector<View2> views(d.nviews);
    std::vector<View3> views3(d.nviews);
    std::vector<int> allv(d.nviews);
    std::vector<RayP> rays;
    std::vector<Ray3> rays3;
    std::vector<Ray2> rview(d.ns);
    bool two_d = d.kind != OSLALM_CONE3D_FLAT;
    if (two_d) rays.resize((size_t)d.nviews * d.ns);
    else rays3.resize((size_t)d.nviews * d.ns);
    for (int v = 0; v < d.nviews; ++v) {
        double cu, su;
        cos_sin_turns(view_turns(d, v), &cu, &su);
        views[v] = View2{(float)cu, (float)su, d.ns, 0};
        views3[v] = View3{(float)cu, (float)su, (float)(-d.dso * cu), (float)(-d.dso * su)};
        allv[v] = v;
        if (two_d) {
            ray_table_view(d, v, rview.data());
            for (int c = 0; c < d.ns; ++c) rays[(size_t)v * d.ns + c] = make_rayp(rview[c]);
            // channels [0, split) share the orientation axis0, [split, ns) the other
            const int a0 = ray_axis(rview[0].packed);
            int split = 0;
            while (split < d.ns && ray_axis(rview[split].packed) == a0) ++split;
            for (int c = split; c < d.ns; ++c)
                if (ray_axis(rview[c].packed) == a0) {
                    delete g;
                    return fail(OSLALM_ERR_RANGE,
                                "view %d: rays switch orientation more than once (fan angle of 90 degrees or more)", v);
                }
            views[v].split = split;
            views[v].axis0 = a0;
        }
        else ray3_table_view(d, v, &rays3[(size_t)v * d.ns]);
    }
    auto cleanup = [&](int code, const char *what, cudaError_t e) {
        cudaFree(g->d_rays); cudaFree(g->d_rays3); cudaFree(g->d_views); cudaFree(g->d_views3); cudaFree(g->d_allviews);
        delete g;
        return fail(code, "%s: %s", what, cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&g->d_views, sizeof(View2) * d.nviews)) != cudaSuccess) return cleanup(OSLALM_ERR_ALLOC, "cudaMalloc views", e);
    if ((e = cudaMalloc(&g->d_views3, sizeof(View3) * d.nviews)) != cudaSuccess) return cleanup(OSLALM_ERR_ALLOC, "cudaMalloc views3", e);
    if ((e = cudaMalloc(&g->d_allviews, sizeof(int) * d.nviews)) != cudaSuccess) return cleanup(OSLALM_ERR_ALLOC, "cudaMalloc views", e);
    if (two_d && (e = cudaMalloc(&g->d_rays, sizeof(RayP) * rays.size())) != cudaSuccess) return cleanup(OSLALM_ERR_ALLOC, "cudaMalloc rays", e);
    if (!two_d && (e = cudaMalloc(&g->d_rays3, sizeof(Ray3) * rays3.size())) != cudaSuccess) return cleanup(OSLALM_ERR_ALLOC, "cudaMalloc rays3", e);
    if ((e = cudaMemcpy(g->d_views, views.data(), sizeof(View2) * d.nviews, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup(OSLALM_ERR_CUDA, "upload", e);
    if ((e = cudaMemcpy(g->d_views3, views3.data(), sizeof(View3) * d.nviews, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup(OSLALM_ERR_CUDA, "upload", e);
    if ((e = cudaMemcpy(g->d_allviews, allv.data(), sizeof(int) * d.nviews, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup(OSLALM_ERR_CUDA, "upload", e);
    if (two_d && (e = cudaMemcpy(g->d_rays, rays.data(), sizeof(RayP) * rays.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup(OSLALM_ERR_CUDA, "upload", e);
    if (!two_d && (e = cudaMemcpy(g->d_rays3, rays3.data(), sizeof(Ray3) * rays3.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup(OSLALM_ERR_CUDA, "upload", e);
    *out = g;
    return OSLALM_OK;
}

int oslalm_ray_table(const oslalm_geom_desc *desc, int view, float *f0, float *kappa_lo, float *lrow,
                     int *packed) {
    clear_error();
    if (int rc = validate(desc)) return rc;
    if (desc->kind == OSLALM_CONE3D_FLAT) return fail(OSLALM_ERR_ARG, "ray tables are 2D only");
    if (view < 0 || view >= desc->nviews || !f0 || !kappa_lo || !lrow || !packed)
        return fail(OSLALM_ERR_ARG, "bad ray table request");
    std::vector<Ray2> r(desc->ns);
    ray_table_view(*desc, view, r.data());
    for (int c = 0; c < desc->ns; ++c) {
        f0[c] = r[c].f0;
        kappa_lo[c] = r[c].kappa_lo;
        lrow[c] = r[c].lrow;
        packed[c] = r[c].packed;
    }
    return OSLALM_OK;
}

int oslalm_geom_destroy(oslalm_geom *g) {
    clear_error();
    if (!g) return OSLALM_OK;
    cudaFree(g->d_rays);
    cudaFree(g->d_rays3);
    cudaFree(g->d_views);
    cudaFree(g->d_views3);
    cudaFree(g->d_allviews);
    delete g;
    return OSLALM_OK;
}

int oslalm_max_subsets(const oslalm_geom_desc *d, double s, double *m_max) {
    clear_error();
    if (!d || !m_max) return fail(OSLALM_ERR_ARG, "NULL argument");
    if (!(s > 0.0)) return fail(OSLALM_ERR_ARG, "need s > 0");
    if (d->nviews <= 0 || !(d->angle_span > 0.0)) return fail(OSLALM_ERR_ARG, "need views over a positive angle");
    if (d->pitch == 0.0) {
        *m_max = (double)d->nviews / s;  // Eq. max_M_axial
    } else {
        if (!(d->dso > 0.0 && d->dsd > 0.0)) return fail(OSLALM_ERR_ARG, "helix needs dso, dsd > 0");
        const double per_turn = (double)d->nviews * (2.0 * M_PI / d->angle_span);
        *m_max = per_turn * d->dso / (d->pitch * s * d->dsd);  // Eq. max_M_helical
    }
    return OSLALM_OK;
}

int oslalm_subset_order(int M, int *order) {
    clear_error();
    if (M <= 0 || !order) return fail(OSLALM_ERR_ARG, "need M > 0 and an order buffer");
    int b = 0;
    while ((1 << b) < M) ++b;
    int k = 0;
    for (int i = 0; i < (1 << b); ++i) {
        int r = 0;
        for (int q = 0; q < b; ++q)
            if (i & (1 << q)) r |= 1 << (b - 1 - q);
        if (r < M) order[k++] = r;
    }
    return OSLALM_OK;
}

int oslalm_subset_views(const oslalm_geom *g, int M, int m, int *views, int *n) {
    clear_error();
    if (!g || M <= 0 || m < 0 || m >= M || !n) return fail(OSLALM_ERR_ARG, "bad subset request");
    int k = 0;
    for (int v = m; v < g->d.nviews; v += M) {
        if (views) views[k] = v;
        ++k;
    }
    *n = k;
    return OSLALM_OK;
}

}  // extern "C"
