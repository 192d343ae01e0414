// 2D projector-pair and update building blocks shared by the single-problem
// kernels (kernels2d.cu) and the batched persistent kernels (batch.cu): the
// same device functions give bit-identical arithmetic in both.
#pragma once

#include "common.cuh"
#include "kernels_common.cuh"

namespace oslalm {

// Major-axis rows [ia0, ia1] whose minor span can meet [0, Nb) (conservative).
__device__ __forceinline__ void ray_rows(const Geo2 &g, const RayP &rp, int &ia0, int &ia1) {
    const int axis = rp.axis;
    const int Na = axis ? g.ny : g.nx;
    const int Nb = axis ? g.nx : g.ny;
    ia0 = 0;
    ia1 = Na - 1;
    if (rp.lrow == 0.f) {  // the ray misses the image
        ia1 = -1;
        return;
    }
    const float kap = __fadd_rn(__fadd_rn(rp.kq, rp.kq), rp.kappa_lo);
    if (kap != 0.f) {
        // b - n0 in [-1, Nb - n0 + 1] at the row ends, with a row of margin
        float t0 = (-rp.n0f - 1.f - rp.f0) / kap;
        float t1 = ((float)Nb - rp.n0f + 1.f - rp.f0) / kap;
        float tlo = fmaxf(fminf(t0, t1), -2.f), thi = fminf(fmaxf(t0, t1), (float)Na + 2.f);
        ia0 = max(0, (int)floorf(tlo) - 1);
        ia1 = min(Na - 1, (int)ceilf(thi) + 1);
    } else {
        int j = (int)rp.n0f + (int)floorf(rp.f0);
        if (j < 0 || j >= Nb) ia1 = -1;
    }
}

// Sum of length x pixel over rows first, first+stride, ... of the ray (each
// row adds its first pixel, then its second).
template <typename ACC>
__device__ __forceinline__ ACC march2(const Geo2 &g, const RayP &rp, const float *__restrict__ x, int first,
                                      int stride) {
    const int axis = rp.axis;
    const int Nb = axis ? g.nx : g.ny;
    const int sa = axis ? g.nx : 1;
    const int sb = axis ? 1 : g.nx;
    int ia0, ia1;
    ray_rows(g, rp, ia0, ia1);
    ACC acc = 0;
    int ia = ia0 + first;
    float ia2 = (float)(2 * ia + 1), iah = (float)ia + 0.5f;
    const float d2 = (float)(2 * stride), d1 = (float)stride;
#pragma unroll 2
    for (; ia <= ia1; ia += stride, ia2 += d2, iah += d1) {
        const RowW w = row_weights(rp, ia2, iah);
        const int j = (int)w.j;
        const int k = ia * sa + j * sb;  // 32-bit: images hold at most 4096^2 pixels
        const float x0 = (unsigned)j < (unsigned)Nb ? __ldg(x + k) : 0.f;
        const float x1 = (w.w1 != 0.f && (unsigned)(j + 1) < (unsigned)Nb) ? __ldg(x + k + sb) : 0.f;
        acc = fma((ACC)w.w0, (ACC)x0, acc);
        acc = fma((ACC)w.w1, (ACC)x1, acc);
    }
    return acc;
}

// atan(t) for |t| <= 1: t P(t^2), P of degree 5 fitted by least squares at
// Chebyshev nodes of [0, 1] (max error 1.9e-6 in float32 arithmetic)
__device__ __forceinline__ float atan_unit(float t) {
    const float s = t * t;
    float p = -1.146580931e-02f;
    p = fmaf(p, s, 5.195053294e-02f);
    p = fmaf(p, s, -1.157294437e-01f);
    p = fmaf(p, s, 1.932352930e-01f);
    p = fmaf(p, s, -3.325683177e-01f);
    p = fmaf(p, s, 9.999744892e-01f);
    return p * t;
}

// The back-projected value of a pixel is summed in a fixed order: the views
// are dealt to kBpGroups groups (list position lv goes to group lv mod
// kBpGroups); within a group the contributions of the x-major rays (views in
// list order, channels ascending) and of the y-major rays (same order) are
// summed separately, by fused multiply-adds, and added; the group totals are
// added in group order.  The single-problem and the batched kernels both run
// bp_tile_strips, so they give the same bits.
constexpr int kBpGroups = 8;

// ---------------------------------------------------------------- tiled back-projection
// A tile of kBpTile x kBpTile pixels is back-projected by 32 x kBpGroups
// threads: warp k takes view group k.  For the x-major rays lane l owns the
// vertical strip of column (l mod 16), rows 8 (l / 16) + [0, 8); for the
// y-major rays the horizontal strip of row (l mod 16), columns
// 8 (l / 16) + [0, 8).  Every pixel of a strip lies in the same major row of
// those rays, so one evaluation of a ray's row weights (first pixel j,
// lengths w0 and w1) serves both pixels it touches; the strip's candidate
// rays are the channel window of the whole strip.  Strip pixel d of lane l
// accumulates in word d * 32 + l of its group's (and orientation's) block,
// always in bank l: no shared-memory bank conflicts.
constexpr int kBpTile = 16;
constexpr int kBpStrip = 8;
constexpr int kBpThreads = 32 * kBpGroups;
static_assert(kBpTile * kBpTile == 32 * kBpStrip, "a warp's 32 strips cover the tile");

struct BpTileAcc {  // [view group][0: x-major, 1: y-major][strip pixel d][lane]
    float a[kBpGroups][2][kBpStrip][32];
};

// Channel window of a strip of pixels whose centres run from (pxa, pya) to
// (pxb, pyb), half_len apart from its middle: channels whose ray may cross
// any pixel of it.  The channel coordinate of a point is linear (parallel
// beam) or monotone (fan: the angle seen from the source) along a segment,
// so the end pixels span the centres; the half-width takes the smallest
// distance from the source that any point of the segment can have, and the
// circumradius of a pixel.  The window is widened by a margin far above the
// rounding of the ray tables and the error of the angle evaluation (fan:
// atan_unit, < 2.5e-6 rad, when every pixel centre is within 45 degrees of
// the source's axis), so that no channel with a non-zero length is missed.
__device__ __forceinline__ void strip_window(const Geo2 &g, const View2 &vw, float pxa, float pya, float pxb,
                                             float pyb, float half_len, int &c0, int &c1) {
    float ca, cb, hw;
    if (g.kind == OSLALM_PAR2D) {
        constexpr float kMargin = 0.02f;
        ca = (-pxa * vw.su + pya * vw.cu) * g.inv_ds + g.c0;
        cb = (-pxb * vw.su + pyb * vw.cu) * g.inv_ds + g.c0;
        hw = 0.5f * (g.dx * fabsf(vw.su) + g.dy * fabsf(vw.cu)) * g.inv_ds + kMargin;
    } else {
        const float aa = pxa * vw.cu + pya * vw.su + g.dso, ba = -pxa * vw.su + pya * vw.cu;
        const float ab = pxb * vw.cu + pyb * vw.su + g.dso, bb = -pxb * vw.su + pyb * vw.cu;
        const float ga = g.fast_atan ? atan_unit(__fdividef(ba, aa)) : atan2f(ba, aa);
        const float gb = g.fast_atan ? atan_unit(__fdividef(bb, ab)) : atan2f(bb, ab);
        const float kMargin = 0.02f + 2.5e-6f * g.dsd * g.inv_ds;
        const float dmin = fmaxf(sqrtf(fminf(fmaf(aa, aa, ba * ba), fmaf(ab, ab, bb * bb))) - half_len, 0.f);
        const float d2 = dmin * dmin - g.half_diag * g.half_diag;
        const float ang = g.half_diag * rsqrtf(fmaxf(d2, 1e-12f));  // >= angular radius of any strip pixel
        const float k = g.dsd * g.inv_ds;
        ca = ga * k + g.c0;
        cb = gb * k + g.c0;
        hw = ang * 1.0001f * k + kMargin;
    }
    c0 = max(0, (int)ceilf(fminf(ca, cb) - hw));
    c1 = min(g.ns - 1, (int)floorf(fmaxf(ca, cb) + hw));
}

// Adds one ray's row lengths times its residual to the strip pixels it
// touches: d = (first pixel j) - (first strip index), exact small integer.
__device__ __forceinline__ void strip_add(float *A, int d, const RowW &w, float val) {
    if ((unsigned)d < (unsigned)kBpStrip) A[d * 32] = fmaf(w.w0, val, A[d * 32]);
    if ((unsigned)(d + 1) < (unsigned)kBpStrip) A[(d + 1) * 32] = fmaf(w.w1, val, A[(d + 1) * 32]);
}

// The strip of lane `lane` for the rays of orientation ax (0: x-major,
// 1: y-major) in the tile with lower corner (tx0, ty0): its major row ia (as
// the exact floats 2 ia + 1 and ia + 1/2), its first minor index jb0, and the
// centres (mm) of its first and last pixel inside the image.
struct StripCtx {
    float ia2, iah, jbf;
    float pxa, pya, pxb, pyb, half_len;
    bool valid;
};

__device__ __forceinline__ StripCtx strip_ctx(const Geo2 &g, int ax, int tx0, int ty0, int lane) {
    StripCtx s;
    const int u = lane & (kBpTile - 1), s0 = (lane / kBpTile) * kBpStrip;
    const int ia = (ax ? ty0 : tx0) + u;   // major row of the rays
    const int jb0 = (ax ? tx0 : ty0) + s0;  // first minor index of the strip
    const int Na = ax ? g.ny : g.nx, Nb = ax ? g.nx : g.ny;
    s.valid = ia < Na && jb0 < Nb;
    const int jb1 = min(jb0 + kBpStrip, Nb) - 1;
    const float pa = ax ? g.dy : g.dx, pb = ax ? g.dx : g.dy;
    const float am = (ax ? g.ylo : g.xlo) + ((float)ia + 0.5f) * pa;  // major coordinate (mm)
    const float blo = (ax ? g.xlo : g.ylo) + ((float)jb0 + 0.5f) * pb;
    const float bhi = (ax ? g.xlo : g.ylo) + ((float)jb1 + 0.5f) * pb;
    s.pxa = ax ? blo : am;
    s.pya = ax ? am : blo;
    s.pxb = ax ? bhi : am;
    s.pyb = ax ? am : bhi;
    s.half_len = 0.5f * (float)(jb1 - jb0) * pb;
    s.ia2 = (float)(2 * ia + 1);
    s.iah = (float)ia + 0.5f;
    s.jbf = (float)jb0;
    return s;
}

// Candidate channels [c0, c1] of view vw for the strip (rays of orientation
// ax only); c0 > c1 when there are none.
__device__ __forceinline__ void strip_channels(const Geo2 &g, const View2 &vw, int ax, const StripCtx &s, int &c0,
                                               int &c1) {
    int k0 = 0, k1 = g.ns;  // channels of this view whose rays have this orientation
    if (vw.axis0 == ax) k1 = vw.split;
    else k0 = vw.split;
    if (k0 >= k1) {
        c0 = 0;
        c1 = -1;
        return;
    }
    strip_window(g, vw, s.pxa, s.pya, s.pxb, s.pyb, s.half_len, c0, c1);
    c0 = max(c0, k0);
    c1 = min(c1, k1 - 1);
}

// Back-projection of the tile with lower corner (tx0, ty0) over views
// [0, nv) into S (thread t in [0, kBpThreads)); the caller synchronises the
// block before reading S with bp_tile_total.
__device__ __forceinline__ void bp_tile_strips(const Geo2 &g, const float *__restrict__ r,
                                               const int *__restrict__ views, int nv, int tx0, int ty0, int t,
                                               BpTileAcc &S) {
    const int grp = t >> 5, lane = t & 31;
#pragma unroll 1
    for (int ax = 0; ax < 2; ++ax) {
        float *A = &S.a[grp][ax][0][lane];
#pragma unroll
        for (int d = 0; d < kBpStrip; ++d) A[d * 32] = 0.f;
        const StripCtx sc = strip_ctx(g, ax, tx0, ty0, lane);
        if (!sc.valid) continue;
        for (int lv = grp; lv < nv; lv += kBpGroups) {
            const int v = __ldg(views + lv);
            if ((unsigned)v >= (unsigned)g.nviews) continue;  // caller-supplied view out of range
            int c0, c1;
            strip_channels(g, g.views[v], ax, sc, c0, c1);
            const RayP *rr = g.rays + (size_t)v * g.ns;
            const float *rv = r + (size_t)lv * g.ns;
            for (int c = c0; c <= c1; ++c) {
                const RowW w = row_weights(rr[c], sc.ia2, sc.iah);
                strip_add(A, (int)__fsub_rn(w.j, sc.jbf), w, __ldg(rv + c));
            }
        }
    }
}

// A'r at tile pixel (px, py) from the accumulators, in the fixed order: the
// pixel is strip pixel py mod 8 of lane px + 16 (py / 8) for the x-major
// rays and strip pixel px mod 8 of lane py + 16 (px / 8) for the y-major rays.
__device__ __forceinline__ float bp_tile_total(const BpTileAcc &S, int px, int py) {
    const int lx = px + kBpTile * (py / kBpStrip), dx_ = py % kBpStrip;
    const int ly = py + kBpTile * (px / kBpStrip), dy_ = px % kBpStrip;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kBpGroups; ++k) acc += S.a[k][0][dx_][lx] + S.a[k][1][dy_][ly];
    return acc;
}

// Hyperbola-regularizer gradient and Huber (or maximum) curvature at pixel
// (tx, ty) of a shared-memory tile with a one-pixel halo (row width TX + 2):
// grad = sum_k w_k psi'(x_j - x_k), curv = sum_k w_k omega(x_j - x_k), both
// still to be scaled by beta and 2 beta.
template <int TX, int NBR>
__device__ __forceinline__ void stencil2d(const float *tile, int tx, int ty, int ix, int iy, int nx, int ny,
                                          float inv_delta, int curv_mode, float &grad, float &curv) {
    constexpr int W = TX + 2;
    const float xj = tile[(ty + 1) * W + tx + 1];
    grad = 0.f;
    curv = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int ox, oy;
        nbr2d(k, ox, oy);
        if (NBR == 4 && ox != 0 && oy != 0) continue;
        const int nxp = ix + ox, nyp = iy + oy;
        if (nxp < 0 || nxp >= nx || nyp < 0 || nyp >= ny) continue;
        const float wk = (ox != 0 && oy != 0) ? 0.70710678118654752f : 1.f;
        const float t = xj - tile[(ty + 1 + oy) * W + tx + 1 + ox];
        const float u = t * inv_delta;
        const float q = rsqrtf(fmaf(u, u, 1.f));
        grad = fmaf(wk * t, q, grad);
        curv += wk * (curv_mode == OSLALM_CURV_HUBER ? q : 1.f);
    }
}

// Cooperative load of a TX x TY tile of x with its one-pixel halo (zeros
// outside the image), then a barrier.
template <int TX, int TY>
__device__ __forceinline__ void load_tile_halo(float *tile, int ix0, int iy0, int tid, int nthreads, int nx, int ny,
                                               const float *__restrict__ x) {
    constexpr int W = TX + 2, H = TY + 2;
    for (int k = tid; k < W * H; k += nthreads) {
        const int yy = k / W, xx = k - yy * W;
        const int gx = ix0 + xx - 1, gy = iy0 + yy - 1;
        tile[k] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? __ldg(x + (size_t)gy * nx + gx) : 0.f;
    }
    __syncthreads();
}

// The n = 1 inner step on one TX x TY tile of pixels (Sec. IV-A):
// s = rho zeta + (1-rho) g; x+ = max(0, x - (s + grad R(x)) / (rho_d D + D_R(x))),
// rho_d = rho alpha (alpha = 1 without Barzilai-Borwein scaling),
// with the 4/8-neighbour hyperbola gradient and Huber curvature read from a
// shared-memory copy of the tile and its one-pixel halo.  (tx, ty): this
// thread's pixel in the tile; tid/nthreads: its rank for the cooperative load.
// This is also the first of n inner FISTA steps (from v = x).
template <int TX, int TY, typename DT, int NBR>
__device__ __forceinline__ void update_tile(float *tile, int ix0, int iy0, int tx, int ty, int tid, int nthreads,
                                            int nx, int ny, const float *__restrict__ x, float *__restrict__ xo,
                                            const float *__restrict__ zeta, const float *__restrict__ gs,
                                            const DT *__restrict__ D, const float *__restrict__ dscale, float rho,
                                            float rho_d, float beta, float inv_delta, int curv_mode) {
    const int ix = ix0 + tx, iy = iy0 + ty;
    const bool in = ix < nx && iy < ny;
    const size_t p = in ? (size_t)iy * nx + ix : 0;
    // this pixel's zeta, g and D are loaded before the tile's barrier, so
    // their latency overlaps the halo load
    float z = 0.f, g = 0.f, d = 0.f;
    if (in) {
        z = __ldg(zeta + p);
        g = __ldg(gs + p);
        d = load_w(D, p);
    }
    load_tile_halo<TX, TY>(tile, ix0, iy0, tid, nthreads, nx, ny, x);
    if (in) {
        const float xj = tile[(ty + 1) * (TX + 2) + tx + 1];
        float grad, curv;
        stencil2d<TX, NBR>(tile, tx, ty, ix, iy, nx, ny, inv_delta, curv_mode, grad, curv);
        grad *= beta;
        curv *= 2.f * beta;
        const float s = rho * z + (1.f - rho) * g;
        const float den = rho_d * (d * __ldg(dscale)) + curv;
        const float xn = den > 0.f ? xj - (s + grad) / den : xj;  // no curvature: unchanged
        xo[p] = fmaxf(xn, 0.f);
    }
}

// Inner FISTA step i >= 1 of the constrained denoising problem
//   min_{v >= 0} Phi(v) = R(v) + (rho/2) ||v - x_k + D^-1 s / rho||_D^2
// from the extrapolated point v (tile): u+ = max(0, v - grad Phi(v) / (rho D
// + D_R(v))), grad Phi(v) = grad R(v) + s + rho D (v - x_k); writes u+ and,
// unless vo is null, the next extrapolated point u+ + gamma (u+ - u).
template <int TX, int TY, typename DT, int NBR>
__device__ __forceinline__ void fista_tile(float *tile, int ix0, int iy0, int tx, int ty, int tid, int nthreads,
                                           int nx, int ny, const float *__restrict__ v, const float *__restrict__ xk,
                                           const float *__restrict__ u, float *__restrict__ uo, float *__restrict__ vo,
                                           const float *__restrict__ zeta, const float *__restrict__ gs,
                                           const DT *__restrict__ D, const float *__restrict__ dscale, float rho,
                                           float rho_d, float beta, float inv_delta, int curv_mode, float gamma) {
    load_tile_halo<TX, TY>(tile, ix0, iy0, tid, nthreads, nx, ny, v);
    const int ix = ix0 + tx, iy = iy0 + ty;
    if (ix < nx && iy < ny) {
        const float vj = tile[(ty + 1) * (TX + 2) + tx + 1];
        float grad, curv;
        stencil2d<TX, NBR>(tile, tx, ty, ix, iy, nx, ny, inv_delta, curv_mode, grad, curv);
        grad *= beta;
        curv *= 2.f * beta;
        const size_t p = (size_t)iy * nx + ix;
        const float s = rho * __ldg(zeta + p) + (1.f - rho) * __ldg(gs + p);
        const float rd = rho_d * (load_w(D, p) * __ldg(dscale));
        const float gphi = fmaf(rd, vj - __ldg(xk + p), s + grad);
        const float den = rd + curv;
        const float un = fmaxf(den > 0.f ? vj - gphi / den : vj, 0.f);
        uo[p] = un;
        if (vo) vo[p] = fmaf(gamma, un - __ldg(u + p), un);
    }
}

}  // namespace oslalm
