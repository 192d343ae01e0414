// 2D projector pair and the fused OS-LALM kernels (sm_103a).
//
//  fp2d   : ray-driven forward projection A_m x (Sec. IV system matrix, exact
//           ray/pixel lengths), one thread per ray marching along its major
//           axis; epilogue writes either A_m x or the weighted residual
//           M W_m (A_m x - y_m) of Eq. os_lalm_iterates.
//  bp2d   : pixel-driven gather back-projection A_m' r with the same
//           per-(ray,pixel) weights (exact transpose, no atomics); epilogues
//           store / accumulate, initialise zeta = g, or apply the split-
//           gradient update g+ = (rho zeta+ + g)/(rho+1), the restart
//           indicator xi = (g - zeta+)'(zeta+ - zeta) (Eq. period_indicator_qp,
//           FP64 sum) and the continuation rho_l (Eq. rho_l_formula_qp).
//  update2d: the n = 1 inner step of the constrained denoising problem
//           (Sec. IV-A): s = rho zeta + (1-rho) g,
//           x+ = max(0, x - (s + grad R(x)) / (rho D + D_R(x))).
#include <math.h>

#include "common.cuh"
#include "kernels_common.cuh"

namespace oslalm {

// ---------------------------------------------------------------- forward
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

// One warp = 8 rays (adjacent channels) x 4 lanes; lane q of a ray takes
// rows ia0+q, ia0+q+4, ...; the 4 partial sums are combined by shuffles in a
// fixed order.
template <int MODE, typename WT>
__global__ void __launch_bounds__(128) fp2d_kernel(Geo2 g, const float *__restrict__ x, float *__restrict__ out,
                                                   const int *__restrict__ views, int nv,
                                                   const float *__restrict__ y, const WT *__restrict__ w,
                                                   const float *__restrict__ wscale, float gain) {
    const int lane = threadIdx.x & 31;
    const int q = lane >> 3;
    const int ray = (blockIdx.x * 4 + (threadIdx.x >> 5)) * 8 + (lane & 7);
    const bool valid = ray < nv * g.ns;
    float acc = 0.f;
    int lv = 0, c = 0, v = -1;
    if (valid) {
        lv = ray / g.ns;
        c = ray - lv * g.ns;
        v = __ldg(views + lv);
        if ((unsigned)v < (unsigned)g.nviews) {
            const Ray2 rp = g.rays[(size_t)v * g.ns + c];
            acc = march2<float>(g, rp, x, q, 4);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (!valid || q != 0) return;
    if ((unsigned)v >= (unsigned)g.nviews) {  // caller-supplied view out of range
        out[ray] = __int_as_float(0x7fc00000);
        return;
    }
    if (MODE == FP_PLAIN) {
        out[ray] = acc;
    } else {
        const float wv = load_w(w, ray) * __ldg(wscale);
        out[ray] = gain * wv * (acc - __ldg(y + ray));
    }
}

template <typename WT>
__global__ void __launch_bounds__(128) cost2d_kernel(Geo2 g, const float *__restrict__ x,
                                                     const int *__restrict__ views, int nv,
                                                     const float *__restrict__ y, const WT *__restrict__ w,
                                                     const float *__restrict__ wscale, double *__restrict__ partials) {
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    if (ray < nv * g.ns) {
        const int lv = ray / g.ns;
        const int c = ray - lv * g.ns;
        const int v = __ldg(views + lv);
        double acc = 0.0;
        if ((unsigned)v < (unsigned)g.nviews) acc = march2<double>(g, g.rays[(size_t)v * g.ns + c], x, 0, 1);
        double res = (double)__ldg(y + ray) - acc;
        val = 0.5 * (double)load_w(w, ray) * (double)__ldg(wscale) * res * res;
    }
    val = block_sum<128>(val);
    if (threadIdx.x == 0) partials[blockIdx.x] = val;
}

// ---------------------------------------------------------------- back-projection
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

template <int MODE>
__global__ void __launch_bounds__(256) bp2d_kernel(Geo2 g, const float *__restrict__ r, float *__restrict__ out,
                                                   const int *__restrict__ views, int nv, UpdateArgs ua) {
    const int ix = blockIdx.x * 32 + threadIdx.x;
    const int iy = blockIdx.y * 8 + threadIdx.y;
    const bool valid = ix < g.nx && iy < g.ny;
    float acc = 0.f;
    if (valid) {
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
    }
    const size_t p = (size_t)iy * g.nx + ix;
    if (MODE == BP_STORE) {
        if (valid) out[p] = acc;
    } else if (MODE == BP_ACCUM) {
        if (valid) out[p] += acc;
    } else if (MODE == BP_INIT) {
        if (valid) {
            ua.zeta[p] = acc;
            ua.g[p] = acc;
        }
    } else {
        // split-gradient update and restart indicator (old g, old zeta)
        double xi_local = 0.0;
        if (valid) {
            const double rho = ua.state->rho;
            const float a = (float)(rho / (rho + 1.0));
            const float b = (float)(1.0 / (rho + 1.0));
            const float z_old = ua.zeta[p];
            const float g_old = ua.g[p];
            ua.zeta[p] = acc;
            ua.g[p] = a * acc + b * g_old;
            xi_local = (double)(g_old - acc) * (double)(acc - z_old);
        }
        subset_iteration_epilogue(ua, xi_local);
    }
}

// ---------------------------------------------------------------- update
template <typename DT, int NBR>
__global__ void __launch_bounds__(256) update2d_kernel(int nx, int ny, const float *__restrict__ x,
                                                       float *__restrict__ xo, const float *__restrict__ zeta,
                                                       const float *__restrict__ gs, const DT *__restrict__ D,
                                                       const float *__restrict__ dscale,
                                                       const DevState *__restrict__ st, float beta,
                                                       float inv_delta, int curv_mode) {
    __shared__ float tile[10][34];
    const int ix0 = blockIdx.x * 32, iy0 = blockIdx.y * 8;
    for (int k = threadIdx.y * 32 + threadIdx.x; k < 10 * 34; k += 256) {
        int ty = k / 34, tx = k - ty * 34;
        int gx = ix0 + tx - 1, gy = iy0 + ty - 1;
        tile[ty][tx] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? __ldg(x + (size_t)gy * nx + gx) : 0.f;
    }
    __syncthreads();
    const int ix = ix0 + threadIdx.x, iy = iy0 + threadIdx.y;
    if (ix >= nx || iy >= ny) return;
    const float xj = tile[threadIdx.y + 1][threadIdx.x + 1];
    float grad = 0.f, curv = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int ox, oy;
        nbr2d(k, ox, oy);
        if (NBR == 4 && ox != 0 && oy != 0) continue;
        const int nxp = ix + ox, nyp = iy + oy;
        if (nxp < 0 || nxp >= nx || nyp < 0 || nyp >= ny) continue;
        const float wk = (ox != 0 && oy != 0) ? 0.70710678118654752f : 1.f;
        const float t = xj - tile[threadIdx.y + 1 + oy][threadIdx.x + 1 + ox];
        const float u = t * inv_delta;
        const float q = rsqrtf(fmaf(u, u, 1.f));
        grad = fmaf(wk * t, q, grad);
        curv += wk * (curv_mode == OSLALM_CURV_HUBER ? q : 1.f);
    }
    grad *= beta;
    curv *= 2.f * beta;
    const size_t p = (size_t)iy * nx + ix;
    const float rho = (float)st->rho;
    const float s = rho * __ldg(zeta + p) + (1.f - rho) * __ldg(gs + p);
    const float den = rho * (load_w(D, p) * __ldg(dscale)) + curv;
    float xn = xj - (s + grad) / den;
    xo[p] = fmaxf(xn, 0.f);
}

template <int NBR>
__global__ void __launch_bounds__(256) reg_value2d_kernel(int nx, int ny, const float *__restrict__ x, double beta,
                                                          double delta, double *__restrict__ partials) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
    double v = 0.0;
    if (ix < nx && iy < ny) {
        const double xj = x[(size_t)iy * nx + ix];
        // forward half-neighbourhood: (1,0), (0,1), (1,1), (-1,1)
        const int hx[4] = {1, 0, 1, -1}, hy[4] = {0, 1, 1, 1};
        for (int k = 0; k < (NBR == 8 ? 4 : 2); ++k) {
            int qx = ix + hx[k], qy = iy + hy[k];
            if (qx < 0 || qx >= nx || qy >= ny) continue;
            double t = xj - (double)x[(size_t)qy * nx + qx];
            double wk = (k >= 2) ? 0.70710678118654752440 : 1.0;
            v += wk * hyperbola(t, delta);
        }
        v *= beta;
    }
    __shared__ double red[32];
    v = block_sum2d(v, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// ---------------------------------------------------------------- launchers
int bp2d_blocks(const Geo2 &g) { return ((g.nx + 31) / 32) * ((g.ny + 7) / 8); }

template <int MODE>
static int launch_fp2d_t(const Geo2 &g, const float *x, float *out, const int *views, int nv, const float *y,
                         WeightRef w, float gain, cudaStream_t st) {
    const int n = nv * g.ns;
    const int grid = (n + 31) / 32;  // 32 rays per 128-thread block
    if (MODE == FP_PLAIN || w.dtype == OSLALM_F32)
        fp2d_kernel<MODE, float><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const float *)w.ptr, w.scale, gain);
    else if (w.dtype == OSLALM_F16)
        fp2d_kernel<MODE, __half><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const __half *)w.ptr, w.scale, gain);
    else
        fp2d_kernel<MODE, __nv_bfloat16><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const __nv_bfloat16 *)w.ptr,
                                                               w.scale, gain);
    OSL_LAUNCH_CHECK("fp2d_kernel");
    return OSLALM_OK;
}

int launch_fp2d(const Geo2 &g, const float *x, float *out, const int *views, int nv, int mode, const float *y,
                WeightRef w, float gain, cudaStream_t st) {
    if (nv <= 0) return OSLALM_OK;
    if (mode == FP_PLAIN) return launch_fp2d_t<FP_PLAIN>(g, x, out, views, nv, y, w, gain, st);
    return launch_fp2d_t<FP_RESID>(g, x, out, views, nv, y, w, gain, st);
}

int launch_bp2d(const Geo2 &g, const float *r, float *out, const int *views, int nv, int mode, const UpdateArgs *ua,
                cudaStream_t st) {
    dim3 block(32, 8), grid((g.nx + 31) / 32, (g.ny + 7) / 8);
    UpdateArgs a{};
    if (ua) a = *ua;
    switch (mode) {
        case BP_STORE: bp2d_kernel<BP_STORE><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
        case BP_ACCUM: bp2d_kernel<BP_ACCUM><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
        case BP_INIT: bp2d_kernel<BP_INIT><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
        default: bp2d_kernel<BP_UPDATE><<<grid, block, 0, st>>>(g, r, out, views, nv, a); break;
    }
    OSL_LAUNCH_CHECK("bp2d_kernel");
    return OSLALM_OK;
}

int launch_cost2d(const Geo2 &g, const float *x, const int *views, int nv, const float *y, WeightRef w,
                  double *partials, int *nparts, cudaStream_t st) {
    const int n = nv * g.ns;
    const int grid = (n + 127) / 128;
    *nparts = grid;
    if (grid == 0) return OSLALM_OK;
    if (w.dtype == OSLALM_F32)
        cost2d_kernel<float><<<grid, 128, 0, st>>>(g, x, views, nv, y, (const float *)w.ptr, w.scale, partials);
    else if (w.dtype == OSLALM_F16)
        cost2d_kernel<__half><<<grid, 128, 0, st>>>(g, x, views, nv, y, (const __half *)w.ptr, w.scale, partials);
    else
        cost2d_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(g, x, views, nv, y, (const __nv_bfloat16 *)w.ptr, w.scale,
                                                           partials);
    OSL_LAUNCH_CHECK("cost2d_kernel");
    return OSLALM_OK;
}

int launch_update2d(int nx, int ny, const float *x, float *xo, const float *zeta, const float *g, const void *D,
                    int d_dtype, const float *dscale, const DevState *st, float beta, float inv_delta, int nbr,
                    int curv_mode, cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
#define OSL_UPD(DT, N) \
    update2d_kernel<DT, N><<<grid, block, 0, s>>>(nx, ny, x, xo, zeta, g, (const DT *)D, dscale, st, beta, inv_delta, curv_mode)
    if (nbr == 8) {
        if (d_dtype == OSLALM_F32) OSL_UPD(float, 8);
        else if (d_dtype == OSLALM_F16) OSL_UPD(__half, 8);
        else OSL_UPD(__nv_bfloat16, 8);
    } else {
        if (d_dtype == OSLALM_F32) OSL_UPD(float, 4);
        else if (d_dtype == OSLALM_F16) OSL_UPD(__half, 4);
        else OSL_UPD(__nv_bfloat16, 4);
    }
#undef OSL_UPD
    OSL_LAUNCH_CHECK("update2d_kernel");
    return OSLALM_OK;
}

int launch_reg_value2d(int nx, int ny, const float *x, double beta, double delta, int nbr, double *partials,
                       int *nparts, cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
    *nparts = grid.x * grid.y;
    if (nbr == 8) reg_value2d_kernel<8><<<grid, block, 0, s>>>(nx, ny, x, beta, delta, partials);
    else reg_value2d_kernel<4><<<grid, block, 0, s>>>(nx, ny, x, beta, delta, partials);
    OSL_LAUNCH_CHECK("reg_value2d_kernel");
    return OSLALM_OK;
}

}  // namespace oslalm
