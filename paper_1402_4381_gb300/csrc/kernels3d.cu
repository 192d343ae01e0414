// 3D circular cone-beam projector pair (flat detector) and the 3D update.
//
//  fp3d   : ray-driven forward projection, one thread per detector cell ray,
//           marching along the ray's transaxial major axis; per row the ray
//           crosses at most two minor columns and (cone angle < 45 deg in
//           index units) at most two z layers; exact ray/voxel lengths.
//  bp3d   : voxel-driven gather back-projection with the same per-(ray,
//           voxel) length arithmetic (exact transpose); a thread owns an
//           (x, y) column of KZ voxels and shares the transaxial part of every
//           ray family (view, channel) across the column.
//  update3d: the inner SQS step with the 6- or 26-neighbour hyperbola.
//
// Cone geometry: every ray of channel c in view v lies in the plane through
// the source and the detector column s_c, so all detector rows share the
// transaxial line of Ray2; the height law of each detector row is linear in
// the major index (see Ray3).  A row [ia, ia+1] of a ray covers a transaxial
// span and a height span; a row that stays in one voxel gives it the full row
// length, otherwise each voxel gets the row length times the overlap of the
// two fraction intervals.
#include <math.h>

#include "common.cuh"
#include "kernels_common.cuh"

namespace oslalm {


__device__ __forceinline__ float exp2_neg(int sw) { return __int_as_float((127 - sw) << 23); }  // 2^-sw, exact

// Error-free sum: s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// z part of the row-t ray family r (see Ray3): the height above the bottom
// face, in voxel units, of the row centres.  The fractional height is carried
// as a float pair so that the crossing fractions of nearly flat rays (small
// height change per row) keep their relative precision.
struct ZRow {
    int zi;         // integer part of the height offset of this detector row
    float kh, kl;   // its fractional part as a float pair
    int ukw;        // u * kw
    float uw1l;     // u * w1l
    float hwz;      // |u W1|: half the height change over one row
    bool inc;       // height grows with a
    float L;        // 3D ray length per unit of a
};

__device__ __forceinline__ ZRow zrow(const Ray3 &r, int u) {
    ZRow o;
    const float A = __fmul_rn((float)u, r.z0h);  // exact: 8 x 15 bits
    const float Ai = floorf(A);
    o.zi = (int)Ai + r.oz_i;
    float s, e;
    two_sum(__fsub_rn(A, Ai), r.oz_f, s, e);
    float t2, e2;
    two_sum(s, __fmul_rn((float)u, r.z0l), t2, e2);
    o.kh = t2;
    o.kl = __fadd_rn(__fadd_rn(e, e2), r.oz_fl);
    o.ukw = u * r.kw;
    o.uw1l = __fmul_rn((float)u, r.w1l);
    const float w = __fmaf_rn((float)o.ukw, exp2_neg(r.sw), o.uw1l);
    o.hwz = fabsf(w);
    o.inc = w > 0.f;
    const float qq = __fmul_rn((float)u, r.q);
    o.L = __fmul_rn(r.xy.lrow, __fsqrt_rn(__fmaf_rn(qq, qq, 1.f)));
    return o;
}

// Span of one coordinate over row ia: centre ch + cl relative to base (ch on a
// 2^-20 grid so that integer - ch is exact), half-width hw; lo/hi for the
// cell tests.
struct DSpan {
    int base;
    float ch, cl, hw, lo, hi;
};

__device__ __forceinline__ DSpan zspan(const Ray3 &r, const ZRow &z, int ia) {
    const int P = z.ukw * (2 * ia + 1);  // exact: < 2^31
    const int pi = P >> r.sw;
    const float pf = __fmul_rn((float)(P & ((1 << r.sw) - 1)), exp2_neg(r.sw));  // exact for sw <= 24
    float s, e, s2, e2;
    two_sum(z.kh, pf, s, e);
    two_sum(s, __fmul_rn((float)(2 * ia + 1), z.uw1l), s2, e2);
    const float lo_part = __fadd_rn(__fadd_rn(z.kl, e), e2);
    DSpan o;
    o.base = z.zi + pi;
    o.ch = __fmul_rn(rintf(__fmul_rn(s2, 1048576.f)), 9.5367431640625e-7f);
    o.cl = __fadd_rn(__fsub_rn(s2, o.ch), lo_part);
    o.hw = z.hwz;
    o.lo = __fadd_rn(__fsub_rn(o.ch, o.hw), o.cl);
    o.hi = __fadd_rn(__fadd_rn(o.ch, o.hw), o.cl);
    return o;
}

// fraction (in [0, 1] along increasing a) at which the coordinate equals v
__device__ __forceinline__ float span_tau(const DSpan &s, bool inc, float v, float rw) {
    const float d = __fsub_rn(v, s.ch);  // exact
    const float num = inc ? __fadd_rn(__fsub_rn(d, s.cl), s.hw) : __fadd_rn(__fadd_rn(-d, s.cl), s.hw);
    return __fmul_rn(num, rw);
}

// fraction interval of the row in which the coordinate lies in cell kk
// (the general form, for any cell)
__device__ __forceinline__ void dcell_frac(const DSpan &s, bool inc, float kk, float &flo, float &fhi) {
    const float jl = floorf(s.lo), jh = floorf(s.hi);
    if (jl == jh) {
        flo = kk == jl ? 0.f : 1.f;
        fhi = kk == jl ? 1.f : 0.f;
        return;
    }
    if (!(kk + 1.f > s.lo && kk < s.hi)) {
        flo = 1.f;
        fhi = 0.f;
        return;
    }
    const float rw = rcp_approx(__fadd_rn(s.hw, s.hw));
    const float t_lo = kk > s.lo ? span_tau(s, inc, kk, rw) : (inc ? 0.f : 1.f);
    const float t_hi = kk + 1.f < s.hi ? span_tau(s, inc, kk + 1.f, rw) : (inc ? 1.f : 0.f);
    flo = fmaxf(fminf(t_lo, t_hi), 0.f);
    fhi = fminf(fmaxf(t_lo, t_hi), 1.f);
}

// The same fraction intervals for the (at most two) cells of a span, with
// the one crossing evaluated once: a span is narrower than a cell, so it
// covers jl = floor(lo) and, when it crosses jl + 1, also jl + 1.  rw =
// rcp_approx(2 hw) of the span (a per-ray constant).  cell(0) / cell(1)
// give exactly what dcell_frac gives for cells jl / jl + 1.
struct SpanCells {
    float jl;      // first cell (relative to the span's base)
    bool two;      // floor(hi) > jl
    bool inc;
    bool cross;    // jl + 1 < hi: the second cell is entered
    float tau;     // fraction at which the coordinate passes jl + 1
    __device__ __forceinline__ void cell(int which, float &flo, float &fhi) const {
        const float e_lo = inc ? 0.f : 1.f, e_hi = inc ? 1.f : 0.f;
        if (!two) {
            flo = which == 0 ? 0.f : 1.f;
            fhi = which == 0 ? 1.f : 0.f;
            return;
        }
        float t_lo, t_hi;
        if (which == 0) {
            t_lo = e_lo;
            t_hi = cross ? tau : e_hi;
        } else {
            if (!cross) {
                flo = 1.f;
                fhi = 0.f;
                return;
            }
            t_lo = tau;
            t_hi = e_hi;
        }
        flo = fmaxf(fminf(t_lo, t_hi), 0.f);
        fhi = fminf(fmaxf(t_lo, t_hi), 1.f);
    }
};

__device__ __forceinline__ SpanCells span_cells(const DSpan &s, bool inc, float rw) {
    SpanCells o;
    o.jl = floorf(s.lo);
    o.two = floorf(s.hi) != o.jl;
    o.inc = inc;
    o.cross = __fadd_rn(o.jl, 1.f) < s.hi;
    o.tau = o.two && o.cross ? span_tau(s, inc, __fadd_rn(o.jl, 1.f), rw) : 0.f;
    return o;
}

// transaxial span of row ia, compensated like the height span: the centre
// b(ia + 1/2) = n0 + (2 ia + 1) k / 4096 + f0 + (ia + 1/2) kappa_lo, with the
// float residues of f0 and kappa_lo added to the low part
__device__ __forceinline__ DSpan bspan(const Ray3 &r, int ia) {
    const int k = ray_k(r.xy.packed);
    const int p = (2 * ia + 1) * k;  // exact: |p| < 2^24
    const float fr = __fmul_rn((float)(p & 4095), 2.44140625e-4f);  // exact
    const float ac = (float)ia + 0.5f;
    const float pr = __fmul_rn(ac, r.xy.kappa_lo);
    const float pe = __fmaf_rn(ac, r.xy.kappa_lo, -pr);  // exact product error
    float s, e, s2, e2;
    two_sum(r.xy.f0, fr, s, e);
    two_sum(s, pr, s2, e2);
    const float lo_part = __fadd_rn(__fadd_rn(__fadd_rn(e, e2), pe), __fmaf_rn(ac, r.kll, r.f0l));
    DSpan o;
    o.base = ray_n0(r.xy.packed) + (p >> 12);
    o.ch = __fmul_rn(rintf(__fmul_rn(s2, 1048576.f)), 9.5367431640625e-7f);
    o.cl = __fadd_rn(__fsub_rn(s2, o.ch), lo_part);
    o.hw = fabsf(__fmaf_rn((float)k, 2.44140625e-4f, __fmul_rn(0.5f, r.xy.kappa_lo)));
    o.lo = __fadd_rn(__fsub_rn(o.ch, o.hw), o.cl);
    o.hi = __fadd_rn(__fadd_rn(o.ch, o.hw), o.cl);
    return o;
}

__device__ __forceinline__ float pair_len(float blo, float bhi, float zlo, float zhi, float L) {
    const float ov = __fsub_rn(fminf(bhi, zhi), fmaxf(blo, zlo));
    return ov > 0.f ? __fmul_rn(ov, L) : 0.f;
}

__device__ __forceinline__ bool b_increasing(const Ray3 &r) {
    return ((float)ray_k(r.xy.packed) * 4.8828125e-4f + r.xy.kappa_lo) > 0.f;
}


// transaxial rows [ia0, ia1] that can meet the volume, also clipped in z
__device__ __forceinline__ void ray_rows3(const Geo3 &g, const Ray3 &rp, const ZRow &z, int &ia0, int &ia1) {
    const int axis = ray_axis(rp.xy.packed);
    const int n0 = ray_n0(rp.xy.packed);
    const int Na = axis ? g.ny : g.nx;
    const int Nb = axis ? g.nx : g.ny;
    ia0 = 0;
    ia1 = Na - 1;
    if (rp.xy.lrow == 0.f) {
        ia1 = -1;
        return;
    }
    const float kap = (float)ray_k(rp.xy.packed) * 4.8828125e-4f + rp.xy.kappa_lo;
    if (kap != 0.f) {
        float t0 = ((float)(-n0) - 1.f - rp.xy.f0) / kap;
        float t1 = ((float)(Nb - n0) + 1.f - rp.xy.f0) / kap;
        float tlo = fmaxf(fminf(t0, t1), -2.f), thi = fminf(fmaxf(t0, t1), (float)Na + 2.f);
        ia0 = max(ia0, (int)floorf(tlo) - 1);
        ia1 = min(ia1, (int)ceilf(thi) + 1);
    } else {
        int j = n0 + (int)floorf(rp.xy.f0);
        if (j < 0 || j >= Nb) {
            ia1 = -1;
            return;
        }
    }
    // z: zb(a) = Az + a Bz must stay within [-1, nz + 1]
    const float Bz = 2.f * __fmaf_rn((float)z.ukw, exp2_neg(rp.sw), z.uw1l);
    const float Az = (float)z.zi + z.kh;
    if (Bz != 0.f) {
        float a0 = (-1.f - Az) / Bz, a1 = ((float)g.nz + 1.f - Az) / Bz;
        float lo = fmaxf(fminf(a0, a1), -2.f), hi = fminf(fmaxf(a0, a1), (float)Na + 2.f);
        ia0 = max(ia0, (int)floorf(lo) - 1);
        ia1 = min(ia1, (int)ceilf(hi) + 1);
    } else if (Az < -1.f || Az > (float)g.nz + 1.f) {
        ia1 = -1;
    }
}

template <typename ACC>
__device__ __forceinline__ ACC march3(const Geo3 &g, const Ray3 &rp, int u, const float *__restrict__ x) {
    const int axis = ray_axis(rp.xy.packed);
    const int Nb = axis ? g.nx : g.ny;
    const size_t sa = axis ? (size_t)g.nx : 1, sb = axis ? 1 : (size_t)g.nx;
    const size_t sz = (size_t)g.nx * g.ny;
    const ZRow z = zrow(rp, u);
    int ia0, ia1;
    ray_rows3(g, rp, z, ia0, ia1);
    const bool binc = b_increasing(rp), zinc = z.inc;
    // per-ray reciprocals of the two span widths (the spans' half-widths are
    // the same in every row)
    const float rwb = rcp_approx(__fadd_rn(bspan(rp, 0).hw, bspan(rp, 0).hw));
    const float rwz = rcp_approx(__fadd_rn(z.hwz, z.hwz));
    ACC acc = 0;
    for (int ia = ia0; ia <= ia1; ++ia) {
        const DSpan sb_ = bspan(rp, ia);
        const DSpan sz_ = zspan(rp, z, ia);
        const SpanCells cb = span_cells(sb_, binc, rwb);
        const SpanCells cz = span_cells(sz_, zinc, rwz);
        if (!cb.two && !cz.two) {  // the row stays inside one voxel
            const int j = sb_.base + (int)cb.jl, kz = sz_.base + (int)cz.jl;
            if ((unsigned)j < (unsigned)Nb && (unsigned)kz < (unsigned)g.nz)
                acc += (ACC)z.L * (ACC)__ldg(x + (size_t)ia * sa + (size_t)j * sb + (size_t)kz * sz);
            continue;
        }
#pragma unroll
        for (int bj = 0; bj < 2; ++bj) {
            if (bj == 1 && !cb.two) break;
            const int j = sb_.base + (int)cb.jl + bj;
            if ((unsigned)j >= (unsigned)Nb) continue;
            float blo, bhi;
            cb.cell(bj, blo, bhi);
            if (!(bhi > blo)) continue;
#pragma unroll
            for (int bk = 0; bk < 2; ++bk) {
                if (bk == 1 && !cz.two) break;
                const int kz = sz_.base + (int)cz.jl + bk;
                if ((unsigned)kz >= (unsigned)g.nz) continue;
                float zlo_, zhi_;
                cz.cell(bk, zlo_, zhi_);
                const float ch = pair_len(blo, bhi, zlo_, zhi_, z.L);
                if (ch > 0.f) acc += (ACC)ch * (ACC)__ldg(x + (size_t)ia * sa + (size_t)j * sb + (size_t)kz * sz);
            }
        }
    }
    return acc;
}

template <int MODE, typename WT>
__global__ void __launch_bounds__(128) fp3d_kernel(Geo3 g, const float *__restrict__ x, float *__restrict__ out,
                                                   const int *__restrict__ views, int nv,
                                                   const float *__restrict__ y, const WT *__restrict__ w,
                                                   const float *__restrict__ wscale, float gain) {
    const long ray = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nrays = (long)nv * g.nt * g.ns;
    if (ray >= nrays) return;
    const int c = (int)(ray % g.ns);
    const long lt = ray / g.ns;
    const int t = (int)(lt % g.nt);
    const int lv = (int)(lt / g.nt);
    const int v = __ldg(views + lv);
    if ((unsigned)v >= (unsigned)g.nviews) {
        out[ray] = __int_as_float(0x7fc00000);
        return;
    }
    const Ray3 rp = g.rays[(size_t)v * g.ns + c];
    const float acc = march3<float>(g, rp, 2 * t - g.u0, x);
    if (MODE == FP_PLAIN) {
        out[ray] = acc;
    } else {
        const float wv = load_w(w, ray) * __ldg(wscale);
        out[ray] = gain * wv * (acc - __ldg(y + ray));
    }
}

template <typename WT>
__global__ void __launch_bounds__(128) cost3d_kernel(Geo3 g, const float *__restrict__ x,
                                                     const int *__restrict__ views, int nv,
                                                     const float *__restrict__ y, const WT *__restrict__ w,
                                                     const float *__restrict__ wscale, double *__restrict__ partials) {
    const long ray = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nrays = (long)nv * g.nt * g.ns;
    double val = 0.0;
    if (ray < nrays) {
        const int c = (int)(ray % g.ns);
        const long lt = ray / g.ns;
        const int t = (int)(lt % g.nt);
        const int lv = (int)(lt / g.nt);
        const int v = __ldg(views + lv);
        double acc = 0.0;
        if ((unsigned)v < (unsigned)g.nviews) acc = march3<double>(g, g.rays[(size_t)v * g.ns + c], 2 * t - g.u0, x);
        const double res = (double)__ldg(y + ray) - acc;
        val = 0.5 * (double)load_w(w, ray) * (double)__ldg(wscale) * res * res;
    }
    val = block_sum<128>(val);
    if (threadIdx.x == 0) partials[blockIdx.x] = val;
}

// ---------------------------------------------------------------- back-projection
constexpr int KZ = 32;  // voxels per thread along z

template <int MODE>
__global__ void __launch_bounds__(256) bp3d_kernel(Geo3 g, const float *__restrict__ r, float *__restrict__ out,
                                                   const int *__restrict__ views, int nv, UpdateArgs ua) {
    const int ix = blockIdx.x * 32 + threadIdx.x;
    const int iy = blockIdx.y * 8 + threadIdx.y;
    const int kz0 = blockIdx.z * KZ;
    const bool valid = ix < g.nx && iy < g.ny;
    // the column's KZ accumulators in shared memory, word q * 256 + thread
    // (bank = thread mod 32: conflict free), so that a detector row adds to
    // only the one or two voxels it crosses
    __shared__ float accs[KZ * 256];
    float *acc = accs + threadIdx.y * 32 + threadIdx.x;
#pragma unroll
    for (int q = 0; q < KZ; ++q) acc[q * 256] = 0.f;
    if (valid) {
        const float px = g.xlo + ((float)ix + 0.5f) * g.dx;
        const float py = g.ylo + ((float)iy + 0.5f) * g.dy;
        // height (voxel units above the bottom face) covered by this thread's voxels
        const float zc_lo = (float)kz0, zc_hi = (float)min(kz0 + KZ, g.nz);
        const float rpix = g.half_diag;
        for (int lv = 0; lv < nv; ++lv) {
            const int v = __ldg(views + lv);
            if ((unsigned)v >= (unsigned)g.nviews) continue;
            const View2 vw = g.views[v];
            const Ray3 *rr = g.rays + (size_t)v * g.ns;
            const float U = px * vw.cu + py * vw.su + g.dso;
            const float Bq = -px * vw.su + py * vw.cu;
            // flat-detector channel window of the pixel's circumscribed disk
            const float T = Bq / U;
            const float td = rpix * rsqrtf(fmaxf(U * U + Bq * Bq - rpix * rpix, 1e-12f)) * 1.0001f;
            const float slo = g.dsd * (T - td) / (1.f + T * td);
            const float shi = g.dsd * (T + td) / fmaxf(1.f - T * td, 1e-6f);
            const int c0i = max(0, (int)ceilf(slo * g.inv_ds + g.c0 - 0.02f));
            const int c1i = min(g.ns - 1, (int)floorf(shi * g.inv_ds + g.c0 + 0.02f));
            const float *rv = r + (size_t)lv * g.nt * g.ns;
            for (int c = c0i; c <= c1i; ++c) {
                const Ray3 rp = rr[c];
                const int axis = ray_axis(rp.xy.packed);
                const int ia = axis ? iy : ix;
                const int jb = axis ? ix : iy;
                const DSpan sb_ = bspan(rp, ia);
                const SpanCells cb = span_cells(sb_, b_increasing(rp), rcp_approx(__fadd_rn(sb_.hw, sb_.hw)));
                const int jrel = jb - sb_.base - (int)cb.jl;  // 0 or 1 when the ray meets this column
                if (jrel != 0 && jrel != 1) continue;
                float blo, bhi;
                cb.cell(jrel, blo, bhi);
                if (!(bhi > blo)) continue;
                // rows t whose height within row ia can meet [zc_lo, zc_hi]:
                // zb(a) = u (Z0 + a Z1) + oz, a in [ia, ia+1], solved for u
                const float s0 = (float)rp.z0h + rp.z0l;
                const float s1 = 2.f * ((float)rp.kw * exp2_neg(rp.sw) + rp.w1l);
                const float ga = __fmaf_rn((float)ia, s1, s0), gb = __fmaf_rn((float)(ia + 1), s1, s0);
                const float smin = fmaxf(fminf(ga, gb), 1e-9f), smax = fmaxf(ga, gb);
                const float oz = (float)rp.oz_i + rp.oz_f;
                const float a_lo = zc_lo - oz - 1e-3f, a_hi = zc_hi - oz + 1e-3f;
                const float u_lo = fminf(a_lo / smin, a_lo / smax);
                const float u_hi = fmaxf(a_hi / smin, a_hi / smax);
                // u = 2 t - u0
                const int t_lo = max(0, (int)ceilf(0.5f * (u_lo + (float)g.u0) - 0.02f));
                const int t_hi = min(g.nt - 1, (int)floorf(0.5f * (u_hi + (float)g.u0) + 0.02f));
                for (int t = t_lo; t <= t_hi; ++t) {
                    const ZRow z = zrow(rp, 2 * t - g.u0);
                    const DSpan sz_ = zspan(rp, z, ia);
                    const SpanCells cz = span_cells(sz_, z.inc, rcp_approx(__fadd_rn(z.hwz, z.hwz)));
                    const int k0 = sz_.base + (int)cz.jl;  // first slice the row meets
                    const int nk = cz.two ? 2 : 1;
                    if (k0 + nk - 1 < kz0 || k0 >= kz0 + KZ) continue;
                    const float val = __ldg(rv + (size_t)t * g.ns + c);
#pragma unroll
                    for (int bk = 0; bk < 2; ++bk) {
                        if (bk == nk) break;
                        const int q = k0 + bk - kz0;
                        if ((unsigned)q >= (unsigned)KZ || k0 + bk >= g.nz) continue;
                        float zlo_, zhi_;
                        cz.cell(bk, zlo_, zhi_);
                        acc[q * 256] = fmaf(pair_len(blo, bhi, zlo_, zhi_, z.L), val, acc[q * 256]);
                    }
                }
            }
        }
    }
    const size_t sz = (size_t)g.nx * g.ny;
    const size_t p0 = (size_t)iy * g.nx + ix;
    if (MODE == BP_STORE || MODE == BP_ACCUM || MODE == BP_INIT) {
        if (!valid) return;
#pragma unroll
        for (int q = 0; q < KZ; ++q) {
            const int kz = kz0 + q;
            if (kz >= g.nz) break;
            const size_t p = (size_t)kz * sz + p0;
            if (MODE == BP_STORE) out[p] = acc[q * 256];
            else if (MODE == BP_ACCUM) out[p] += acc[q * 256];
            else {
                ua.zeta[p] = acc[q * 256];
                ua.g[p] = acc[q * 256];
            }
        }
    } else {
        IterSums sums{0.0, 0.0, 0.0};
        if (valid) {
            const float a = ua.state->ga, b = ua.state->gb;
#pragma unroll
            for (int q = 0; q < KZ; ++q) {
                const int kz = kz0 + q;
                if (kz >= g.nz) break;
                const size_t p = (size_t)kz * sz + p0;
                const float z_old = ua.zeta[p];
                const float g_old = ua.g[p];
                ua.zeta[p] = acc[q * 256];
                ua.g[p] = a * acc[q * 256] + b * g_old;
                add_iter_terms(ua, p, g_old, z_old, acc[q * 256], sums);
            }
        }
        subset_iteration_epilogue(ua, sums);
    }
}


// ---------------------------------------------------------------- update (3D)
// neighbour k (0..25) of the 3x3x3 cube without the centre
__device__ __forceinline__ void nbr3d(int k, int &ox, int &oy, int &oz) {
    const int idx = k < 13 ? k : k + 1;
    ox = idx % 3 - 1;
    oy = (idx / 3) % 3 - 1;
    oz = idx / 9 - 1;
}

// Hyperbola-regularizer gradient and Huber (or maximum) curvature at voxel
// (ix, iy, iz) of x over the 6- or 26-neighbourhood, before the beta and
// 2 beta scaling.
template <int NBR>
__device__ __forceinline__ void stencil3d(const float *__restrict__ x, int nx, int ny, int nz, int ix, int iy, int iz,
                                          float xj, float inv_delta, int curv_mode, float &grad, float &curv) {
    const size_t sxy = (size_t)nx * ny;
    grad = 0.f;
    curv = 0.f;
#pragma unroll
    for (int k = 0; k < 26; ++k) {
        int ox, oy, oz;
        nbr3d(k, ox, oy, oz);
        const int nn = (ox != 0) + (oy != 0) + (oz != 0);
        if (NBR == 6 && nn != 1) continue;
        const int qx = ix + ox, qy = iy + oy, qz = iz + oz;
        if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
        const float wk = nn == 1 ? 1.f : (nn == 2 ? 0.70710678118654752f : 0.57735026918962576f);
        const float t = xj - __ldg(x + (size_t)qz * sxy + (size_t)qy * nx + qx);
        const float u = t * inv_delta;
        const float q = rsqrtf(fmaf(u, u, 1.f));
        grad = fmaf(wk * t, q, grad);
        curv += wk * (curv_mode == OSLALM_CURV_HUBER ? q : 1.f);
    }
}

template <typename DT, int NBR>
__global__ void __launch_bounds__(256) update3d_kernel(int nx, int ny, int nz, const float *__restrict__ x,
                                                       float *__restrict__ xo, const float *__restrict__ zeta,
                                                       const float *__restrict__ gs, const DT *__restrict__ D,
                                                       const float *__restrict__ dscale,
                                                       const DevState *__restrict__ st, float beta,
                                                       float inv_delta, int curv_mode) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y, iz = blockIdx.z;
    if (ix >= nx || iy >= ny) return;
    const size_t p = (size_t)iz * nx * ny + (size_t)iy * nx + ix;
    const float xj = __ldg(x + p);
    float grad, curv;
    stencil3d<NBR>(x, nx, ny, nz, ix, iy, iz, xj, inv_delta, curv_mode, grad, curv);
    grad *= beta;
    curv *= 2.f * beta;
    const float rho = st->rho_f, rho_d = st->rho_d_f;  // rho_d = rho alpha, alpha: Barzilai-Borwein scale
    const float s = rho * __ldg(zeta + p) + (1.f - rho) * __ldg(gs + p);
    const float den = rho_d * (load_w(D, p) * __ldg(dscale)) + curv;
    const float xn = den > 0.f ? xj - (s + grad) / den : xj;  // no curvature: unchanged
    xo[p] = fmaxf(xn, 0.f);
}

// inner FISTA step i >= 1 (see fista_tile in proj2d.cuh), 3D stencil
template <typename DT, int NBR>
__global__ void __launch_bounds__(256) fista3d_kernel(int nx, int ny, int nz, const float *__restrict__ v,
                                                      const float *__restrict__ xk, const float *__restrict__ u,
                                                      float *__restrict__ uo, float *__restrict__ vo,
                                                      const float *__restrict__ zeta, const float *__restrict__ gs,
                                                      const DT *__restrict__ D, const float *__restrict__ dscale,
                                                      const DevState *__restrict__ st, float beta, float inv_delta,
                                                      int curv_mode, float gamma) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y, iz = blockIdx.z;
    if (ix >= nx || iy >= ny) return;
    const size_t p = (size_t)iz * nx * ny + (size_t)iy * nx + ix;
    const float vj = __ldg(v + p);
    float grad, curv;
    stencil3d<NBR>(v, nx, ny, nz, ix, iy, iz, vj, inv_delta, curv_mode, grad, curv);
    grad *= beta;
    curv *= 2.f * beta;
    const float rho = st->rho_f, rho_d = st->rho_d_f;
    const float s = rho * __ldg(zeta + p) + (1.f - rho) * __ldg(gs + p);
    const float rd = rho_d * (load_w(D, p) * __ldg(dscale));
    const float gphi = fmaf(rd, vj - __ldg(xk + p), s + grad);
    const float den = rd + curv;
    const float un = fmaxf(den > 0.f ? vj - gphi / den : vj, 0.f);
    uo[p] = un;
    if (vo) vo[p] = fmaf(gamma, un - __ldg(u + p), un);
}

template <int NBR>
__global__ void __launch_bounds__(256) reg_value3d_kernel(int nx, int ny, int nz, const float *__restrict__ x,
                                                          double beta, double delta, double *__restrict__ partials) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y, iz = blockIdx.z;
    double v = 0.0;
    if (ix < nx && iy < ny) {
        const size_t sxy = (size_t)nx * ny;
        const double xj = x[(size_t)iz * sxy + (size_t)iy * nx + ix];
        // forward half of the neighbourhood (each unordered pair once): k >= 13
        for (int k = 13; k < 26; ++k) {
            int ox, oy, oz;
            nbr3d(k, ox, oy, oz);
            const int nn = (ox != 0) + (oy != 0) + (oz != 0);
            if (NBR == 6 && nn != 1) continue;
            const int qx = ix + ox, qy = iy + oy, qz = iz + oz;
            if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || qz < 0 || qz >= nz) continue;
            const double wk = nn == 1 ? 1.0 : (nn == 2 ? 0.70710678118654752440 : 0.57735026918962576451);
            const double t = xj - (double)x[(size_t)qz * sxy + (size_t)qy * nx + qx];
            v += wk * hyperbola(t, delta);
        }
        v *= beta;
    }
    __shared__ double red[32];
    v = block_sum2d(v, red);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = v;
}

// ---------------------------------------------------------------- launchers
int bp3d_blocks(const Geo3 &g) { return ((g.nx + 31) / 32) * ((g.ny + 7) / 8) * ((g.nz + KZ - 1) / KZ); }

template <int MODE>
static int launch_fp3d_t(const Geo3 &g, const float *x, float *out, const int *views, int nv, const float *y,
                         WeightRef w, float gain, cudaStream_t st) {
    const long n = (long)nv * g.nt * g.ns;
    const unsigned grid = (unsigned)((n + 127) / 128);
    if (MODE == FP_PLAIN || w.dtype == OSLALM_F32)
        fp3d_kernel<MODE, float><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const float *)w.ptr, w.scale, gain);
    else if (w.dtype == OSLALM_F16)
        fp3d_kernel<MODE, __half><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const __half *)w.ptr, w.scale, gain);
    else
        fp3d_kernel<MODE, __nv_bfloat16><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const __nv_bfloat16 *)w.ptr,
                                                               w.scale, gain);
    OSL_LAUNCH_CHECK("fp3d_kernel");
    return OSLALM_OK;
}

int launch_fp3d(const Geo3 &g, const float *x, float *out, const int *views, int nv, int mode, const float *y,
                WeightRef w, float gain, cudaStream_t st) {
    if (nv <= 0) return OSLALM_OK;
    if (mode == FP_PLAIN) return launch_fp3d_t<FP_PLAIN>(g, x, out, views, nv, y, w, gain, st);
    return launch_fp3d_t<FP_RESID>(g, x, out, views, nv, y, w, gain, st);
}

int launch_bp3d(const Geo3 &g, const float *r, float *out, const int *views, int nv, int mode, const UpdateArgs *ua,
                cudaStream_t st) {
    dim3 block(32, 8), grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + KZ - 1) / KZ);
    UpdateArgs a{};
    if (ua) a = *ua;
    switch (mode) {
        case BP_STORE: bp3d_kernel<BP_STORE><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
        case BP_ACCUM: bp3d_kernel<BP_ACCUM><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
        case BP_INIT: bp3d_kernel<BP_INIT><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
        default: bp3d_kernel<BP_UPDATE><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
    }
    OSL_LAUNCH_CHECK("bp3d_kernel");
    return OSLALM_OK;
}

int launch_cost3d(const Geo3 &g, const float *x, const int *views, int nv, const float *y, WeightRef w,
                  double *partials, int *nparts, cudaStream_t st) {
    const long n = (long)nv * g.nt * g.ns;
    const int grid = (int)((n + 127) / 128);
    *nparts = grid;
    if (grid == 0) return OSLALM_OK;
    if (w.dtype == OSLALM_F32)
        cost3d_kernel<float><<<grid, 128, 0, st>>>(g, x, views, nv, y, (const float *)w.ptr, w.scale, partials);
    else if (w.dtype == OSLALM_F16)
        cost3d_kernel<__half><<<grid, 128, 0, st>>>(g, x, views, nv, y, (const __half *)w.ptr, w.scale, partials);
    else
        cost3d_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(g, x, views, nv, y, (const __nv_bfloat16 *)w.ptr, w.scale,
                                                           partials);
    OSL_LAUNCH_CHECK("cost3d_kernel");
    return OSLALM_OK;
}

int launch_update3d(int nx, int ny, int nz, const float *x, float *xo, const float *zeta, const float *g,
                    const void *D, int d_dtype, const float *dscale, const DevState *st, float beta, float inv_delta,
                    int nbr, int curv_mode, cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8, nz);
#define OSL_UPD3(DT, N)                                                                                           \
    update3d_kernel<DT, N><<<grid, block, 0, s>>>(nx, ny, nz, x, xo, zeta, g, (const DT *)D, dscale, st, beta, \
                                                  inv_delta, curv_mode)
    if (nbr == 26) {
        if (d_dtype == OSLALM_F32) OSL_UPD3(float, 26);
        else if (d_dtype == OSLALM_F16) OSL_UPD3(__half, 26);
        else OSL_UPD3(__nv_bfloat16, 26);
    } else {
        if (d_dtype == OSLALM_F32) OSL_UPD3(float, 6);
        else if (d_dtype == OSLALM_F16) OSL_UPD3(__half, 6);
        else OSL_UPD3(__nv_bfloat16, 6);
    }
#undef OSL_UPD3
    OSL_LAUNCH_CHECK("update3d_kernel");
    return OSLALM_OK;
}

int launch_fista3d(int nx, int ny, int nz, const float *v, const float *xk, const float *u, float *uo, float *vo,
                   const float *zeta, const float *g, const void *D, int d_dtype, const float *dscale,
                   const DevState *st, float beta, float inv_delta, int nbr, int curv_mode, float gamma,
                   cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8, nz);
#define OSL_FIS3(DT, N)                                                                                         \
    fista3d_kernel<DT, N><<<grid, block, 0, s>>>(nx, ny, nz, v, xk, u, uo, vo, zeta, g, (const DT *)D, dscale, st, \
                                                 beta, inv_delta, curv_mode, gamma)
    if (nbr == 26) {
        if (d_dtype == OSLALM_F32) OSL_FIS3(float, 26);
        else if (d_dtype == OSLALM_F16) OSL_FIS3(__half, 26);
        else OSL_FIS3(__nv_bfloat16, 26);
    } else {
        if (d_dtype == OSLALM_F32) OSL_FIS3(float, 6);
        else if (d_dtype == OSLALM_F16) OSL_FIS3(__half, 6);
        else OSL_FIS3(__nv_bfloat16, 6);
    }
#undef OSL_FIS3
    OSL_LAUNCH_CHECK("fista3d_kernel");
    return OSLALM_OK;
}

// grad += beta sum_k w_jk psi'(x_j - x_k): the regularizer's gradient
// (Sec. IV, R of Eq. ct_recon), added to a data-term gradient.  One slice
// (nz = 1) gives the 2D neighbourhoods: 26 -> the 8 in-plane neighbours,
// 6 -> the 4 in-plane neighbours.
template <int NBR>
__global__ void __launch_bounds__(256) reg_grad_add_kernel(int nx, int ny, int nz, const float *__restrict__ x,
                                                           float *__restrict__ grad, float beta, float inv_delta) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y, iz = blockIdx.z;
    if (ix >= nx || iy >= ny) return;
    const size_t p = (size_t)iz * nx * ny + (size_t)iy * nx + ix;
    float gr, curv;
    stencil3d<NBR>(x, nx, ny, nz, ix, iy, iz, __ldg(x + p), inv_delta, OSLALM_CURV_HUBER, gr, curv);
    grad[p] += beta * gr;
}

int launch_reg_grad_add(int nx, int ny, int nz, const float *x, float *grad, float beta, float inv_delta, int nbr,
                        cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8, nz);
    if (nbr == 26 || nbr == 8) reg_grad_add_kernel<26><<<grid, block, 0, s>>>(nx, ny, nz, x, grad, beta, inv_delta);
    else reg_grad_add_kernel<6><<<grid, block, 0, s>>>(nx, ny, nz, x, grad, beta, inv_delta);
    OSL_LAUNCH_CHECK("reg_grad_add_kernel");
    return OSLALM_OK;
}

int launch_reg_value3d(int nx, int ny, int nz, const float *x, double beta, double delta, int nbr, double *partials,
                       int *nparts, cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8, nz);
    *nparts = grid.x * grid.y * grid.z;
    if (nbr == 26) reg_value3d_kernel<26><<<grid, block, 0, s>>>(nx, ny, nz, x, beta, delta, partials);
    else reg_value3d_kernel<6><<<grid, block, 0, s>>>(nx, ny, nz, x, beta, delta, partials);
    OSL_LAUNCH_CHECK("reg_value3d_kernel");
    return OSLALM_OK;
}

}  // namespace oslalm
