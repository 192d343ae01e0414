// 2D projector-pair and update building blocks shared by the single-problem
// kernels (kernels2d.cu) and the batched persistent kernels (batch.cu): the
// same device functions give bit-identical arithmetic in both.
#pragma once

#include "common.cuh"
#include "kernels_common.cuh"

namespace oslalm {

// Major-axis rows [ia0, ia1] whose minor span can meet [0, Nb) (conservative).
__device__ __forceinline__ void ray_rows(const Geo2 &g, const Ray2 &rp, int &ia0, int &ia1) {
    const int axis = ray_axis(rp.packed);
    const int n0 = ray_n0(rp.packed);
    const int Na = axis ? g.ny : g.nx;
    const int Nb = axis ? g.nx : g.ny;
    ia0 = 0;
    ia1 = Na - 1;
    if (rp.lrow == 0.f) {  // the ray misses the image
        ia1 = -1;
        return;
    }
    const float kap = (float)ray_k(rp.packed) * 4.8828125e-4f + rp.kappa_lo;
    if (kap != 0.f) {
        // b - n0 in [-1, Nb - n0 + 1] at the row ends, with a row of margin
        float t0 = ((float)(-n0) - 1.f - rp.f0) / kap;
        float t1 = ((float)(Nb - n0) + 1.f - rp.f0) / kap;
        float tlo = fmaxf(fminf(t0, t1), -2.f), thi = fminf(fmaxf(t0, t1), (float)Na + 2.f);
        ia0 = max(0, (int)floorf(tlo) - 1);
        ia1 = min(Na - 1, (int)ceilf(thi) + 1);
    } else {
        int j = n0 + (int)floorf(rp.f0);
        if (j < 0 || j >= Nb) ia1 = -1;
    }
}

// Sum of chord x pixel over rows first, first+stride, ... of the ray.
template <typename ACC>
__device__ __forceinline__ ACC march2(const Geo2 &g, const Ray2 &rp, const float *__restrict__ x, int first,
                                      int stride) {
    const int axis = ray_axis(rp.packed);
    const int Nb = axis ? g.nx : g.ny;
    const int sa = axis ? g.nx : 1;
    const int sb = axis ? 1 : g.nx;
    int ia0, ia1;
    ray_rows(g, rp, ia0, ia1);
    ACC acc = 0;
    for (int ia = ia0 + first; ia <= ia1; ia += stride) {
        const RowSpan s = row_span(rp, ia);
        const float jlo = floorf(s.lo), jhi = floorf(s.hi);
        if (jlo == jhi) {  // the row stays inside one pixel: full row length
            const int j = s.base + (int)jlo;
            if ((unsigned)j < (unsigned)Nb) acc += (ACC)rp.lrow * (ACC)__ldg(x + (size_t)ia * sa + (size_t)j * sb);
            continue;
        }
        for (float jj = jlo; jj <= jhi; jj += 1.f) {
            const int j = s.base + (int)jj;
            if ((unsigned)j < (unsigned)Nb) {
                const float ch = row_chord(s, rp.lrow, jj);
                acc += (ACC)ch * (ACC)__ldg(x + (size_t)ia * sa + (size_t)j * sb);
            }
        }
    }
    return acc;
}

// channel window of pixel centre (px, py) in view vw: channels whose ray may
// cross the pixel, widened by a margin far above the rounding of the ray
// tables so that no channel with a non-zero chord is missed.
__device__ __forceinline__ void channel_window(const Geo2 &g, const View2 &vw, float px, float py, int &c0,
                                               int &c1) {
    constexpr float kMargin = 0.02f;
    float cc, hw;
    if (g.kind == OSLALM_PAR2D) {
        float s = -px * vw.su + py * vw.cu;
        cc = s * g.inv_ds + g.c0;
        hw = 0.5f * (g.dx * fabsf(vw.su) + g.dy * fabsf(vw.cu)) * g.inv_ds;
    } else {
        float a = px * vw.cu + py * vw.su + g.dso;  // along u from the source
        float b = -px * vw.su + py * vw.cu;         // along e
        float gam = atan2f(b, a);
        float d2 = a * a + b * b - g.half_diag * g.half_diag;
        float ang = g.half_diag * rsqrtf(fmaxf(d2, 1e-12f));  // >= angular radius of the pixel
        cc = gam * g.dsd * g.inv_ds + g.c0;
        hw = ang * 1.0001f * g.dsd * g.inv_ds;
    }
    c0 = max(0, (int)ceilf(cc - hw - kMargin));
    c1 = min(g.ns - 1, (int)floorf(cc + hw + kMargin));
}

// Sum over the listed views of chord x r for the rays crossing pixel (ix, iy).
__device__ __forceinline__ float bp_pixel_sum(const Geo2 &g, const float *__restrict__ r,
                                              const int *__restrict__ views, int nv, int ix, int iy) {
    float acc = 0.f;
    const float px = g.xlo + ((float)ix + 0.5f) * g.dx;
    const float py = g.ylo + ((float)iy + 0.5f) * g.dy;
    for (int lv = 0; lv < nv; ++lv) {
        const int v = __ldg(views + lv);
        if ((unsigned)v >= (unsigned)g.nviews) continue;  // caller-supplied view out of range
        const View2 vw = g.views[v];
        int c0, c1;
        channel_window(g, vw, px, py, c0, c1);
        const Ray2 *rr = g.rays + (size_t)v * g.ns;
        const float *rv = r + (size_t)lv * g.ns;
        for (int c = c0; c <= c1; ++c) {
            const Ray2 rp = rr[c];
            acc = fmaf(chord2(rp, ix, iy), __ldg(rv + c), acc);
        }
    }
    return acc;
}

// The n = 1 inner step on one TX x TY tile of pixels (Sec. IV-A):
// s = rho zeta + (1-rho) g; x+ = max(0, x - (s + grad R(x)) / (rho D + D_R(x))),
// with the 4/8-neighbour hyperbola gradient and Huber curvature read from a
// shared-memory copy of the tile and its one-pixel halo.  (tx, ty): this
// thread's pixel in the tile; tid/nthreads: its rank for the cooperative load.
template <int TX, int TY, typename DT, int NBR>
__device__ __forceinline__ void update_tile(float *tile, int ix0, int iy0, int tx, int ty, int tid, int nthreads,
                                            int nx, int ny, const float *__restrict__ x, float *__restrict__ xo,
                                            const float *__restrict__ zeta, const float *__restrict__ gs,
                                            const DT *__restrict__ D, const float *__restrict__ dscale, float rho,
                                            float beta, float inv_delta, int curv_mode) {
    constexpr int W = TX + 2, H = TY + 2;
    for (int k = tid; k < W * H; k += nthreads) {
        const int yy = k / W, xx = k - yy * W;
        const int gx = ix0 + xx - 1, gy = iy0 + yy - 1;
        tile[k] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? __ldg(x + (size_t)gy * nx + gx) : 0.f;
    }
    __syncthreads();
    const int ix = ix0 + tx, iy = iy0 + ty;
    if (ix < nx && iy < ny) {
        const float xj = tile[(ty + 1) * W + tx + 1];
        float grad = 0.f, curv = 0.f;
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
        grad *= beta;
        curv *= 2.f * beta;
        const size_t p = (size_t)iy * nx + ix;
        const float s = rho * __ldg(zeta + p) + (1.f - rho) * __ldg(gs + p);
        const float den = rho * (load_w(D, p) * __ldg(dscale)) + curv;
        const float xn = xj - (s + grad) / den;
        xo[p] = fmaxf(xn, 0.f);
    }
}

}  // namespace oslalm
