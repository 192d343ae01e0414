// 2D projector pair and the fused OS-LALM kernels (sm_103a).
//
//  fp2d   : ray-driven forward projection A_m x (Sec. IV system matrix, exact
//           ray/pixel lengths), one thread per ray marching along its major
//           axis; epilogue writes either A_m x or the weighted residual
//           M W_m (A_m x - y_m) of Eq. os_lalm_iterates.
//  bp2d   : gather back-projection A_m' r over pixel tiles with the same
//           per-(ray,pixel) weights (exact transpose, no atomics): each
//           thread owns a strip of pixels along a major row of the rays, so
//           one evaluation of a ray's row weights serves both pixels it
//           touches; epilogues
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
#include "proj2d.cuh"

namespace oslalm {

// ---------------------------------------------------------------- forward
// One warp = 4 rays (adjacent channels) x 8 lanes; lane q of a ray takes
// rows ia0+q, ia0+q+8, ...; the 8 partial sums are combined by shuffles in a
// fixed order.  Warp k of block b takes the rays of group b + k gridDim.x
// (groups of 4 rays in list order): a block's four groups lie a quarter of
// the list apart, at different places in the fan, so that long central and
// short edge rays mix in every block and the SMs, which receive the whole
// grid at once, get equal work.
template <int MODE, typename WT>
__global__ void __launch_bounds__(128) fp2d_kernel(Geo2 g, const float *__restrict__ x, float *__restrict__ out,
                                                   const int *__restrict__ views, int nv,
                                                   const float *__restrict__ y, const WT *__restrict__ w,
                                                   const float *__restrict__ wscale, float gain) {
    const int lane = threadIdx.x & 31;
    const int q = lane >> 2;
    const int ray = (blockIdx.x + (threadIdx.x >> 5) * gridDim.x) * 4 + (lane & 3);
    const bool valid = ray < nv * g.ns;
    float acc = 0.f;
    int lv = 0, c = 0, v = -1;
    if (valid) {
        lv = ray / g.ns;
        c = ray - lv * g.ns;
        v = __ldg(views + lv);
        if ((unsigned)v < (unsigned)g.nviews) {
            const RayP rp = g.rays[(size_t)v * g.ns + c];
            acc = march2<float>(g, rp, x, q, 8);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
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
// One block of kBpThreads threads per kBpTile^2 pixel tile (bp_tile_strips);
// then each thread finishes two pixels of the tile.
template <int MODE>
__device__ __forceinline__ void bp2d_epilogue(const UpdateArgs &ua, float *out, size_t p, float acc, IterSums &sums) {
    if (MODE == BP_STORE) {
        out[p] = acc;
    } else if (MODE == BP_ACCUM) {
        out[p] += acc;
    } else if (MODE == BP_INIT) {
        ua.zeta[p] = acc;
        ua.g[p] = acc;
    } else {
        // split-gradient update and restart indicator (old g, old zeta)
        const float a = ua.state->ga, b = ua.state->gb;
        const float z_old = ua.zeta[p];
        const float g_old = ua.g[p];
        ua.zeta[p] = acc;
        ua.g[p] = a * acc + b * g_old;
        add_iter_terms(ua, p, g_old, z_old, acc, sums);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kBpThreads, 8) bp2d_kernel(Geo2 g, const float *__restrict__ r,
                                                             float *__restrict__ out, const int *__restrict__ views,
                                                             int nv, UpdateArgs ua) {
    __shared__ BpTileAcc S;
    const int tx0 = blockIdx.x * kBpTile, ty0 = blockIdx.y * kBpTile;
    bp_tile_strips(g, r, views, nv, tx0, ty0, threadIdx.x, S);
    __syncthreads();
    IterSums sums{0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < kBpTile * kBpTile / kBpThreads; ++k) {
        const int i = threadIdx.x + k * kBpThreads;
        const int px = i % kBpTile, py = i / kBpTile;
        const int ix = tx0 + px, iy = ty0 + py;
        if (ix < g.nx && iy < g.ny)
            bp2d_epilogue<MODE>(ua, out, (size_t)iy * g.nx + ix, bp_tile_total(S, px, py), sums);
    }
    if (MODE == BP_UPDATE) subset_iteration_epilogue(ua, sums);
}

// ---------------------------------------------------------------- update
template <typename DT, int NBR>
__global__ void __launch_bounds__(256) update2d_kernel(int nx, int ny, const float *__restrict__ x,
                                                       float *__restrict__ xo, const float *__restrict__ zeta,
                                                       const float *__restrict__ gs, const DT *__restrict__ D,
                                                       const float *__restrict__ dscale,
                                                       const DevState *__restrict__ st, float beta,
                                                       float inv_delta, int curv_mode) {
    __shared__ float tile[10 * 34];
    update_tile<32, 8, DT, NBR>(tile, blockIdx.x * 32, blockIdx.y * 8, threadIdx.x, threadIdx.y,
                                threadIdx.y * 32 + threadIdx.x, 256, nx, ny, x, xo, zeta, gs, D, dscale,
                                st->rho_f, st->rho_d_f, beta, inv_delta, curv_mode);
}

template <typename DT, int NBR>
__global__ void __launch_bounds__(256) fista2d_kernel(int nx, int ny, const float *__restrict__ v,
                                                      const float *__restrict__ xk, const float *__restrict__ u,
                                                      float *__restrict__ uo, float *__restrict__ vo,
                                                      const float *__restrict__ zeta, const float *__restrict__ gs,
                                                      const DT *__restrict__ D, const float *__restrict__ dscale,
                                                      const DevState *__restrict__ st, float beta, float inv_delta,
                                                      int curv_mode, float gamma) {
    __shared__ float tile[10 * 34];
    fista_tile<32, 8, DT, NBR>(tile, blockIdx.x * 32, blockIdx.y * 8, threadIdx.x, threadIdx.y,
                               threadIdx.y * 32 + threadIdx.x, 256, nx, ny, v, xk, u, uo, vo, zeta, gs, D, dscale,
                               st->rho_f, st->rho_d_f, beta, inv_delta, curv_mode, gamma);
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
int bp2d_blocks(const Geo2 &g) { return ((g.nx + kBpTile - 1) / kBpTile) * ((g.ny + kBpTile - 1) / kBpTile); }

template <int MODE, typename WT>
static void launch_fp2d_w(const Geo2 &g, const float *x, float *out, const int *views, int nv, const float *y,
                          const void *w, const float *wscale, float gain, cudaStream_t st) {
    const int n = nv * g.ns;
    const int grid = (n + 15) / 16;  // 16 rays per 128-thread block
    fp2d_kernel<MODE, WT><<<grid, 128, 0, st>>>(g, x, out, views, nv, y, (const WT *)w, wscale, gain);
}

template <int MODE>
static int launch_fp2d_t(const Geo2 &g, const float *x, float *out, const int *views, int nv, const float *y,
                         WeightRef w, float gain, cudaStream_t st) {
    if (MODE == FP_PLAIN || w.dtype == OSLALM_F32)
        launch_fp2d_w<MODE, float>(g, x, out, views, nv, y, w.ptr, w.scale, gain, st);
    else if (w.dtype == OSLALM_F16)
        launch_fp2d_w<MODE, __half>(g, x, out, views, nv, y, w.ptr, w.scale, gain, st);
    else
        launch_fp2d_w<MODE, __nv_bfloat16>(g, x, out, views, nv, y, w.ptr, w.scale, gain, st);
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
    dim3 block(kBpThreads), grid((g.nx + kBpTile - 1) / kBpTile, (g.ny + kBpTile - 1) / kBpTile);
    UpdateArgs a{};
    if (ua) a = *ua;
#define OSL_BP(MODE) bp2d_kernel<MODE><<<grid, block, 0, st>>>(g, r, out, views, nv, a)
    switch (mode) {
        case BP_STORE: OSL_BP(BP_STORE); break;
        case BP_ACCUM: OSL_BP(BP_ACCUM); break;
        case BP_INIT: OSL_BP(BP_INIT); break;
        default: OSL_BP(BP_UPDATE); break;
    }
#undef OSL_BP
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

int launch_fista2d(int nx, int ny, const float *v, const float *xk, const float *u, float *uo, float *vo,
                   const float *zeta, const float *g, const void *D, int d_dtype, const float *dscale,
                   const DevState *st, float beta, float inv_delta, int nbr, int curv_mode, float gamma,
                   cudaStream_t s) {
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8);
#define OSL_FIS(DT, N)                                                                                            \
    fista2d_kernel<DT, N><<<grid, block, 0, s>>>(nx, ny, v, xk, u, uo, vo, zeta, g, (const DT *)D, dscale, st, beta, \
                                                 inv_delta, curv_mode, gamma)
    if (nbr == 8) {
        if (d_dtype == OSLALM_F32) OSL_FIS(float, 8);
        else if (d_dtype == OSLALM_F16) OSL_FIS(__half, 8);
        else OSL_FIS(__nv_bfloat16, 8);
    } else {
        if (d_dtype == OSLALM_F32) OSL_FIS(float, 4);
        else if (d_dtype == OSLALM_F16) OSL_FIS(__half, 4);
        else OSL_FIS(__nv_bfloat16, 4);
    }
#undef OSL_FIS
    OSL_LAUNCH_CHECK("fista2d_kernel");
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
