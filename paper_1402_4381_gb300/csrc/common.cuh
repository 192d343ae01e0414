// Internal declarations shared by the liboslalm translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "../../include/oslalm.h"

namespace oslalm {

// ---------------------------------------------------------------- errors
int fail(int code, const char *fmt, ...);
void clear_error();

#define OSL_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::oslalm::fail(OSLALM_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,      \
                                  cudaGetErrorString(e_), __FILE__, __LINE__);          \
    } while (0)

#define OSL_LAUNCH_CHECK(what)                                                          \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return ::oslalm::fail(OSLALM_ERR_CUDA, "launch of %s failed: %s", what,      \
                                  cudaGetErrorString(e_));                              \
    } while (0)

// ---------------------------------------------------------------- geometry
// Per-ray parameters of a 2D ray in continuous pixel-index space.  The ray
// is written along its major axis a (the axis it advances fastest along, in
// index units) as  b(a) = n0 + f0 + a * kappa,  |kappa| <= 1,  where a, b are
// continuous index coordinates (pixel ia spans [ia, ia+1)).  The slope is
// split as kappa = k/2048 + kappa_lo with an integer k, so that a * k/2048
// is formed exactly in integer arithmetic and the float part of b stays
// below 3 in magnitude: positions keep ~1e-7 pixel precision anywhere in the
// image.  lrow is the ray length (mm) per unit of a.
// packed = (k << 16) | ((n0 & 0x7fff) << 1) | axis; axis 0: a = x, 1: a = y;
// n0 is the nearest integer to b(0), f0 in [-1/2, 1/2).
struct __align__(16) Ray2 {
    float f0;
    float kappa_lo;
    float lrow;
    int packed;
};

__host__ __device__ __forceinline__ int ray_axis(int packed) { return packed & 1; }
__host__ __device__ __forceinline__ int ray_n0(int packed) { return (int)((unsigned)packed << 16) >> 17; }
__host__ __device__ __forceinline__ int ray_k(int packed) { return packed >> 16; }

// Per-view parameters: beam direction u = (cu, su).  In a 2D view the rays
// of channels [0, split) advance along axis axis0 (0: x, 1: y) and those of
// [split, ns) along the other (a fan narrower than 90 degrees switches at
// most once).
struct __align__(16) View2 {
    float cu, su;
    int split, axis0;
};

// 3D cone-beam per-view parameters (FP32 copies of FP64 set-up values).
struct __align__(16) View3 {
    float cu, su;      // beam direction u
    float srcx, srcy;  // source position (z = 0)
};

// Cone beam, flat detector: all rays of channel c in view v lie in the plane
// through the source and detector column c, so every detector row shares the
// transaxial line xy (a Ray2).  The height law of the row-t ray in voxel
// units above the volume's bottom face is
//     zb(a) = u (Z0 + a Z1) + oz,   u = 2 (t - t0) (an integer),
// Z0 = alpha0 dt / (2 dz), Z1 = alpha1 dt / (2 dz) with alpha = alpha0 +
// a alpha1 the fraction of the transaxial way from the source to the detector
// at major index a.  For FP32 precision independent of the height, Z0 is split
// as z0h (15 significant bits, so u z0h is exact) + z0l, and Z1 / 2 as
// kw / 2^sw (integer kw, |kw| < 512, so u (2a+1) kw is an exact int32) + w1l;
// oz = oz_i + oz_f.  q = dt / (2 l_D) gives the 3D length per unit of a as
// lrow sqrt(1 + (u q)^2).
struct __align__(16) Ray3 {
    Ray2 xy;
    float z0h, z0l, w1l, q;
    int kw, sw, oz_i;
    float oz_f, oz_fl;  // oz - oz_i as a float pair
    // FP32 rounding residues of xy.f0 and xy.kappa_lo.  A ray within a few
    // hundredths of a degree of an axis (slope kappa ~ 1e-3) splits a row
    // between two voxels at a fraction whose error is the position error
    // divided by kappa, so the transaxial span carries these in its
    // compensated sum.
    float f0l, kll;
    float pad2;
};
struct Geo3 {  // kernel-side cone geometry (by value)
    int nx, ny, nz, ns, nt, nviews;
    float dx, dy, dz, inv_dz;
    float zlo;       // bottom face of the volume (mm)
    float xlo, ylo;
    float dt, t0;    // row pitch; row coordinate of t_t = 0: (nt-1)/2 - offset_t
    int u0;          // 2 t0 (an integer): u = 2 t - u0
    float inv_ds, c0, dso, dsd, half_diag;
    const Ray3 *rays;    // [nviews][ns]
    const View2 *views;  // [nviews]
};

// Device form of a 2D ray for the projector pair (32 bytes): the Ray2 line
// with its integer fields as exact floats and the per-ray constants of the
// length arithmetic precomputed once:
//   kq    = k / 4096                  (exact)
//   n0f   = n0                        (exact)
//   hw    = |k / 4096 + kappa_lo / 2| (half the minor-axis width of a row,
//                                      float32: |fma(k, 2^-12, 0.5 kappa_lo)|)
struct __align__(16) RayP {
    float f0, kappa_lo, lrow, kq;
    float n0f, hw;
    int axis;
    float lscale;  // lrow / (2 hw): length per unit of minor span (0 when hw = 0)
};

struct Geo2 {  // kernel-side 2D geometry (by value)
    int kind, nx, ny, ns, nviews;
    float dx, dy, xlo, ylo;  // pixel size, image lower corner (mm)
    float inv_ds;            // 1/ds
    float c0;                // channel coordinate of s = 0: (ns-1)/2 - offset_s
    float dso, dsd;
    float half_diag;         // pixel circumradius
    int fast_atan;           // fan beam: every pixel centre is within 45 degrees of the source's axis
    const RayP *rays;        // [nviews][ns]
    const View2 *views;      // [nviews]
};

}  // namespace oslalm

struct oslalm_geom {
    oslalm_geom_desc d;
    int device;
    oslalm::Ray3 *d_rays3;    // 3D: [nviews][ns]
    oslalm::RayP *d_rays;     // 2D: [nviews][ns]
    oslalm::View2 *d_views;   // [nviews]
    oslalm::View3 *d_views3;  // 3D: [nviews]
    int *d_allviews;          // 0..nviews-1
    oslalm::Geo2 geo2() const;
    oslalm::Geo3 geo3() const;
};

namespace oslalm {

bool is_3d(const oslalm_geom *g);

// ---------------------------------------------------------------- chords
// Length of a 2D ray inside the pixels of major row ia (a in [ia, ia+1]).
// The row is entered through the ray's minor position at the row centre,
// c = b(ia + 1/2), and the half-width hw = |kappa|/2: the row covers minor
// coordinates [c - hw, c + hw] (width |kappa| <= 1, so at most two pixels).
// A row inside one pixel gives it the full row length lrow; a row crossing
// the pixel boundary jl + 1 gives the first pixel the part of lrow in
// proportion to its overlap, (jl + 1 - lo) lrow / (2 hw), and the second the
// rest, so the two parts sum to lrow.  This is the exact intersection
// length of a straight ray with the pixels of the row.  The forward
// projector (marching along a) and the back-projectors call this same
// function, so both directions use bit-identical weights.
__device__ __forceinline__ float rcp_approx(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

struct RowW {
    float j;       // minor index of the first pixel touched (exact integer)
    float w0, w1;  // lengths in pixels j and j + 1
};

// ia2 = 2 ia + 1 and iah = ia + 1/2 as floats (exact)
__device__ __forceinline__ RowW row_weights(const RayP &r, float ia2, float iah) {
    const float pq = __fmul_rn(ia2, r.kq);  // (2 ia + 1) k / 4096: exact, |(2 ia + 1) k| < 2^24
    const float q = floorf(pq);
    const float fr = __fsub_rn(pq, q);      // exact fraction
    const float c = __fmaf_rn(iah, r.kappa_lo, __fadd_rn(r.f0, fr));  // relative to n0 + q
    const float lo = __fsub_rn(c, r.hw), hi = __fadd_rn(c, r.hw);
    const float jl = floorf(lo), jl1 = __fadd_rn(jl, 1.f);
    RowW w;
    w.j = __fadd_rn(__fadd_rn(r.n0f, q), jl);
    const float part = fminf(__fmul_rn(__fsub_rn(jl1, lo), r.lscale), r.lrow);
    w.w0 = hi > jl1 ? part : r.lrow;
    w.w1 = __fsub_rn(r.lrow, w.w0);
    return w;
}


// ---------------------------------------------------------------- projector launchers
enum FpMode { FP_PLAIN = 0, FP_RESID = 1 };
enum BpMode { BP_STORE = 0, BP_ACCUM = 1, BP_INIT = 2, BP_UPDATE = 3 };

struct WeightRef {  // statistical weights in a storage dtype, value = w[i] * (*scale)
    const void *ptr;
    int dtype;
    const float *scale;  // device scalar
};

// Continuation / split-gradient state on the device.
struct DevState {
    double rho;
    double xi;
    int l;
    int j;        // subset-iterations done
    unsigned int counter;
    int pad;
    double alpha;  // Barzilai-Borwein scale of the majorizer (1 without it)
    double bb_num, bb_den;  // sum s'y, sum s'Ds of the current iteration's secant pairs
    // FP32 factors of the current rho for the per-pixel kernels, formed once
    // where rho or alpha changes (FP64 arithmetic is scarce on this GPU):
    // rho_f = rho, rho_d_f = rho alpha, ga = rho/(rho+1), gb = 1/(rho+1)
    float rho_f, rho_d_f, ga, gb;
};

// Refresh the FP32 factors after rho or alpha changed (one thread).
__device__ __forceinline__ void refresh_rho_factors(DevState *st) {
    const double rho = st->rho;
    st->rho_f = (float)rho;
    st->rho_d_f = (float)(rho * st->alpha);
    st->ga = (float)(rho / (rho + 1.0));
    st->gb = (float)(1.0 / (rho + 1.0));
}

// The continuation's rho_l and its g-update weights for l = 0 .. n-1, formed
// on the host in FP64 with the same operations as rho_of_l and
// refresh_rho_factors (so the same bits): the last block of a
// subset-iteration looks them up instead of dividing in FP64.
struct RhoEnt {
    double rho;
    float ga, gb;  // (float)(rho/(rho+1)), (float)(1/(rho+1))
};

struct UpdateArgs {  // epilogue arguments of the fused back-projection
    float *zeta;
    float *g;
    DevState *state;
    double *partials;
    oslalm_stats *stats;
    int stats_cap;
    const signed char *replay;
    int replay_n;
    int rho_mode;
    double rho_min;
    double rho_fixed;
    int subset;
    // Barzilai-Borwein fit (bb != 0): subset `subset`'s gradient zeta+ is
    // taken at x_new; its previous gradient and iterate are in bbz, bbx
    // ([M][npix]) if bbhave[subset]; s = x_new - bbx, y = zeta+ - bbz; the
    // sums s'y and s'Ds go next to xi in the partials buffer (3 x blocks)
    int bb;
    int M;
    long npix;
    const float *x_new;
    float *bbx, *bbz;
    int *bbhave;
    const void *D;
    int d_dtype;
    const float *dscale;
    const RhoEnt *rho_tab;  // rho_l for l < rho_tab_n (continuation and replay modes), or null
    int rho_tab_n;
};

int launch_fp2d(const Geo2 &g, const float *x, float *out, const int *views, int nv,
                int mode, const float *y, WeightRef w, float gain, cudaStream_t st);
int launch_bp2d(const Geo2 &g, const float *r, float *out, const int *views, int nv,
                int mode, const UpdateArgs *ua, cudaStream_t st);
int launch_cost2d(const Geo2 &g, const float *x, const int *views, int nv, const float *y,
                  WeightRef w, double *partials, int *nparts, cudaStream_t st);
int bp2d_blocks(const Geo2 &g);

int launch_fp3d(const Geo3 &g, const float *x, float *out, const int *views, int nv,
                int mode, const float *y, WeightRef w, float gain, cudaStream_t st);
int launch_bp3d(const Geo3 &g, const float *r, float *out, const int *views, int nv,
                int mode, const UpdateArgs *ua, cudaStream_t st);
int launch_cost3d(const Geo3 &g, const float *x, const int *views, int nv, const float *y,
                  WeightRef w, double *partials, int *nparts, cudaStream_t st);
int bp3d_blocks(const Geo3 &g);
int launch_update3d(int nx, int ny, int nz, const float *x, float *xo, const float *zeta, const float *g,
                    const void *D, int d_dtype, const float *dscale, const DevState *st, float beta,
                    float inv_delta, int nbr, int curv_mode, cudaStream_t s);
// grad += gradient of the regularizer at x (2D images as one slice)
int launch_reg_grad_add(int nx, int ny, int nz, const float *x, float *grad, float beta, float inv_delta, int nbr,
                        cudaStream_t s);
int launch_reg_value3d(int nx, int ny, int nz, const float *x, double beta, double delta, int nbr,
                       double *partials, int *nparts, cudaStream_t s);
// inner FISTA step i >= 1: (v, x_k, u) -> u+, and v+ unless vo is null
int launch_fista2d(int nx, int ny, const float *v, const float *xk, const float *u, float *uo, float *vo,
                   const float *zeta, const float *g, const void *D, int d_dtype, const float *dscale,
                   const DevState *st, float beta, float inv_delta, int nbr, int curv_mode, float gamma,
                   cudaStream_t s);
int launch_fista3d(int nx, int ny, int nz, const float *v, const float *xk, const float *u, float *uo, float *vo,
                   const float *zeta, const float *g, const void *D, int d_dtype, const float *dscale,
                   const DevState *st, float beta, float inv_delta, int nbr, int curv_mode, float gamma,
                   cudaStream_t s);

}  // namespace oslalm
