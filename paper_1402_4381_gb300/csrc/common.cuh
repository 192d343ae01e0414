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

// Per-view parameters: beam direction u = (cu, su).
struct __align__(16) View2 {
    float cu, su, pad0, pad1;
};

// 3D cone-beam per-view parameters (FP32 copies of FP64 set-up values).
struct __align__(16) View3 {
    float cu, su;      // beam direction u
    float srcx, srcy;  // source position (z = 0)
};

struct Geo2 {  // kernel-side 2D geometry (by value)
    int kind, nx, ny, ns, nviews;
    float dx, dy, xlo, ylo;  // pixel size, image lower corner (mm)
    float inv_ds;            // 1/ds
    float c0;                // channel coordinate of s = 0: (ns-1)/2 - offset_s
    float dso, dsd;
    float half_diag;         // pixel circumradius
    const Ray2 *rays;        // [nviews][ns]
    const View2 *views;      // [nviews]
};

}  // namespace oslalm

struct oslalm_geom {
    oslalm_geom_desc d;
    int device;
    oslalm::Ray2 *d_rays;     // 2D: [nviews][ns]
    oslalm::View2 *d_views;   // [nviews]
    oslalm::View3 *d_views3;  // 3D: [nviews]
    int *d_allviews;          // 0..nviews-1
    oslalm::Geo2 geo2() const;
};

namespace oslalm {

bool is_3d(const oslalm_geom *g);

// ---------------------------------------------------------------- chords
// Length of a 2D ray inside pixel (ia, jb) given in the ray's (major, minor)
// index coordinates.  The forward projector (marching along a) and the
// gather back-projector call the same row/overlap arithmetic with explicit
// round-to-nearest intrinsics, so both directions use bit-identical weights.
struct RowSpan {
    int base;       // integer minor coordinate the span is measured from
    float lo, hi;   // minor-coordinate span of the ray inside row ia, relative to base
    float scale;    // lrow / (hi - lo), or 0 when hi == lo
};

__device__ __forceinline__ RowSpan row_span(const Ray2 &r, int ia) {
    const int k = ray_k(r.packed);
    const int p0 = ia * k, p1 = p0 + k;            // exact: |ia k| < 2^24
    const int q0 = p0 >> 11, q1 = p1 >> 11;        // floor(ia k / 2048)
    const float r0 = (float)(p0 & 2047) * 4.8828125e-4f;  // exact fractions
    const float r1 = (float)(p1 & 2047) * 4.8828125e-4f;
    float w0 = __fadd_rn(__fadd_rn(r.f0, r0), __fmul_rn((float)ia, r.kappa_lo));
    float w1 = __fadd_rn(__fadd_rn(r.f0, r1), __fmul_rn((float)(ia + 1), r.kappa_lo));
    w1 = __fadd_rn(w1, (float)(q1 - q0));
    RowSpan s;
    s.base = ray_n0(r.packed) + q0;
    s.lo = fminf(w0, w1);
    s.hi = fmaxf(w0, w1);
    float width = __fsub_rn(s.hi, s.lo);
    // widths below 1e-30 (never produced by a real geometry) count as zero
    s.scale = width > 1e-30f ? __fmul_rn(__frcp_rn(width), r.lrow) : 0.f;
    return s;
}

// chord of the row span inside minor pixel jj (relative to the span's base)
__device__ __forceinline__ float row_chord(const RowSpan &s, float lrow, float jj) {
    if (s.scale > 0.f) {
        float ov = __fsub_rn(fminf(s.hi, jj + 1.f), fmaxf(s.lo, jj));
        return ov > 0.f ? __fmul_rn(ov, s.scale) : 0.f;
    }
    return floorf(s.lo) == jj ? lrow : 0.f;
}

__device__ __forceinline__ float chord2(const Ray2 &r, int ix, int iy) {
    const int axis = ray_axis(r.packed);
    const int ia = axis ? iy : ix;
    const int jb = axis ? ix : iy;
    RowSpan s = row_span(r, ia);
    return row_chord(s, r.lrow, (float)(jb - s.base));
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
};

int launch_fp2d(const Geo2 &g, const float *x, float *out, const int *views, int nv,
                int mode, const float *y, WeightRef w, float gain, cudaStream_t st);
int launch_bp2d(const Geo2 &g, const float *r, float *out, const int *views, int nv,
                int mode, const UpdateArgs *ua, cudaStream_t st);
int launch_cost2d(const Geo2 &g, const float *x, const int *views, int nv, const float *y,
                  WeightRef w, double *partials, int *nparts, cudaStream_t st);
int bp2d_blocks(const Geo2 &g);

}  // namespace oslalm
