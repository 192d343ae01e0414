// PWLS problem state and the OS-LALM driver of the C ABI.
//
// Per subset-iteration three kernels run on the caller's stream (Eq.
// os_lalm_iterates with n = 1 inner step, Sec. IV-A):
//   1. update      x+ = max(0, x - (rho zeta + (1-rho) g + grad R(x)) / (rho D + D_R(x)))
//   2. forward     r  = M W_m' (A_m' x+ - y_m')            (next subset m')
//   3. back-proj.  zeta+ = A_m'^T r;  g+ = (rho zeta+ + g)/(rho+1);
//                  xi = (g - zeta+)'(zeta+ - zeta) (FP64);  l, rho_l  (Sec. III-B)
// rho and l live on the device, so whole iterations replay from a CUDA graph
// without host round trips.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"
#include "kernels_common.cuh"
#include "problem.cuh"

namespace oslalm {

int launch_update2d(int nx, int ny, const float *x, float *xo, const float *zeta, const float *g, const void *D,
                    int d_dtype, const float *dscale, const DevState *st, float beta, float inv_delta, int nbr,
                    int curv_mode, cudaStream_t s);
int launch_reg_value2d(int nx, int ny, const float *x, double beta, double delta, int nbr, double *partials,
                       int *nparts, cudaStream_t s);

// ---------------------------------------------------------------- small kernels
__global__ void gather_views_kernel(const float *__restrict__ src, float *__restrict__ dst,
                                    const int *__restrict__ perm, int nviews, int per_view) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)nviews * per_view;
    if (i >= n) return;
    size_t k = i / per_view, c = i - k * per_view;
    dst[i] = src[(size_t)perm[k] * per_view + c];
}

__global__ void absmax_kernel(const float *__restrict__ a, size_t n, unsigned int *__restrict__ out) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Per-array power-of-two scale s = 2^k, k the smallest integer with
// max <= 32768 * 2^k (s = 1 for an all-zero array), so that stored values
// stay below 32768 and the division by s is exact.
__global__ void pow2_scale_kernel(const unsigned int *__restrict__ maxbits, float *__restrict__ scale, int dtype) {
    float mx = __uint_as_float(*maxbits);
    float s = 1.f;
    if (dtype != OSLALM_F32 && mx > 0.f) {
        int e;
        float m = frexpf(mx, &e);
        int k = (m == 0.5f) ? e - 16 : e - 15;
        s = ldexpf(1.f, k);
    }
    *scale = s;
}

template <typename T>
__device__ __forceinline__ T to_store(float v);
template <>
__device__ __forceinline__ float to_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__global__ void quantize_kernel(const float *__restrict__ src, T *__restrict__ dst, size_t n,
                                const float *__restrict__ scale) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = to_store<T>(src[i] / *scale);
}

template <typename T>
__global__ void dequantize_kernel(const T *__restrict__ src, float *__restrict__ dst, size_t n,
                                  const float *__restrict__ scale) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = load_w(src, i) * *scale;
}

template <typename T>
__global__ void mul_weight_kernel(float *__restrict__ r, const T *__restrict__ w, const float *__restrict__ scale,
                                  size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] *= load_w(w, i) * *scale;
}

__global__ void fill_kernel(float *__restrict__ a, size_t n, float v) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void set_state_kernel(DevState *st, double rho, int l, int j, double alpha) {
    st->rho = rho;
    st->alpha = alpha;
    st->bb_num = 0.0;
    st->bb_den = 0.0;
    st->xi = 0.0;
    st->l = l;
    st->j = j;
    st->counter = 0;
    refresh_rho_factors(st);
}

__global__ void rmsd_kernel(const float *__restrict__ x, const float *__restrict__ xr, const uint8_t *__restrict__ m,
                            long n, double *__restrict__ partials) {
    double s = 0.0, c = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (m[i]) {
            double d = (double)x[i] - (double)xr[i];
            s += d * d;
            c += 1.0;
        }
    }
    s = block_sum<256>(s);
    c = block_sum<256>(c);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s;
        partials[2 * blockIdx.x + 1] = c;
    }
}

static inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

static size_t dtype_size(int dt) { return dt == OSLALM_F32 ? 4 : 2; }

}  // namespace oslalm

using namespace oslalm;


namespace {

// geometry-generic projector / update launches
int launch_fp_any(const oslalm_geom *g, const float *x, float *out, const int *views, int nv, int mode,
                  const float *y, WeightRef w, float gain, cudaStream_t st) {
    if (is_3d(g)) return launch_fp3d(g->geo3(), x, out, views, nv, mode, y, w, gain, st);
    return launch_fp2d(g->geo2(), x, out, views, nv, mode, y, w, gain, st);
}

int launch_bp_any(const oslalm_geom *g, const float *r, float *out, const int *views, int nv, int mode,
                  const UpdateArgs *ua, cudaStream_t st) {
    if (is_3d(g)) return launch_bp3d(g->geo3(), r, out, views, nv, mode, ua, st);
    return launch_bp2d(g->geo2(), r, out, views, nv, mode, ua, st);
}

int bp_blocks_any(const oslalm_geom *g) { return is_3d(g) ? bp3d_blocks(g->geo3()) : bp2d_blocks(g->geo2()); }

int check_problem(const oslalm_problem *p) {
    if (!p) return fail(OSLALM_ERR_ARG, "problem handle is NULL");
    return OSLALM_OK;
}

WeightRef wref(const oslalm_problem *p, int m) {
    WeightRef w;
    w.ptr = (const char *)p->d_w + (size_t)p->off[m] * p->per_view * dtype_size(p->p.w_dtype);
    w.dtype = p->p.w_dtype;
    w.scale = p->d_wscale;
    return w;
}

int fp_subset(oslalm_problem *p, const float *x, int m, int mode, float gain, cudaStream_t st) {
    const float *y = p->d_y + (size_t)p->off[m] * p->per_view;
    return launch_fp_any(p->g, x, p->d_r, p->d_views + p->off[m], p->cnt[m], mode, y, wref(p, m), gain, st);
}

UpdateArgs update_args(oslalm_problem *p, int subset) {
    UpdateArgs a{};
    a.zeta = p->d_zeta;
    a.g = p->d_g;
    a.state = p->d_state;
    a.partials = p->d_partials;
    a.stats = p->d_stats;
    a.stats_cap = p->stats_cap;
    a.replay = p->d_replay;
    a.replay_n = p->replay_n;
    a.rho_mode = p->p.rho_mode;
    a.rho_min = p->p.rho_min;
    a.rho_fixed = p->p.rho_fixed;
    a.subset = subset;
    a.bb = p->p.bb;
    a.M = p->p.M;
    a.npix = p->npix;
    a.bbx = p->d_bbx;
    a.bbz = p->d_bbz;
    a.bbhave = p->d_bbhave;
    a.D = p->d_D;
    a.d_dtype = p->p.d_dtype;
    a.dscale = p->d_dscale;
    a.rho_tab = p->d_rho_tab;
    a.rho_tab_n = p->rho_tab_n;
    return a;
}

// quantize a full float array into storage dtype with a pow2 scale (device side)
int store_scaled(oslalm_problem *p, const float *src, void *dst, int dtype, float *scale, size_t n, cudaStream_t st) {
    OSL_CUDA_TRY(cudaMemsetAsync(p->d_maxbits, 0, sizeof(unsigned int), st));
    absmax_kernel<<<std::min<unsigned>(nblk(n, 256), 4096), 256, 0, st>>>(src, n, p->d_maxbits);
    pow2_scale_kernel<<<1, 1, 0, st>>>(p->d_maxbits, scale, dtype);
    if (dtype == OSLALM_F32) quantize_kernel<float><<<nblk(n, 256), 256, 0, st>>>(src, (float *)dst, n, scale);
    else if (dtype == OSLALM_F16) quantize_kernel<__half><<<nblk(n, 256), 256, 0, st>>>(src, (__half *)dst, n, scale);
    else quantize_kernel<__nv_bfloat16><<<nblk(n, 256), 256, 0, st>>>(src, (__nv_bfloat16 *)dst, n, scale);
    OSL_LAUNCH_CHECK("quantize");
    return OSLALM_OK;
}

int load_data(oslalm_problem *p, const float *y, const float *w, cudaStream_t st) {
    const oslalm_geom_desc &d = p->g->d;
    size_t n = (size_t)d.nviews * p->per_view;
    gather_views_kernel<<<nblk(n, 256), 256, 0, st>>>(y, p->d_y, p->d_views, d.nviews, p->per_view);
    gather_views_kernel<<<nblk(n, 256), 256, 0, st>>>(w, p->d_tmp, p->d_views, d.nviews, p->per_view);
    OSL_LAUNCH_CHECK("gather_views");
    if (int rc = store_scaled(p, p->d_tmp, p->d_w, p->p.w_dtype, p->d_wscale, n, st)) return rc;
    p->d_valid = false;
    return OSLALM_OK;
}

int compute_denominator(oslalm_problem *p, cudaStream_t st) {
    // D = A' W A 1 (Sec. IV-A), accumulated subset by subset into d_g (scratch)
    const size_t npix = p->npix;
    fill_kernel<<<nblk(npix, 256), 256, 0, st>>>(p->d_xalt, npix, 1.f);
    OSL_CUDA_TRY(cudaMemsetAsync(p->d_g, 0, npix * sizeof(float), st));
    for (int m = 0; m < p->p.M; ++m) {
        if (p->cnt[m] == 0) continue;
        if (int rc = fp_subset(p, p->d_xalt, m, FP_PLAIN, 1.f, st)) return rc;
        size_t nr = (size_t)p->cnt[m] * p->per_view;
        WeightRef w = wref(p, m);
        if (w.dtype == OSLALM_F32) mul_weight_kernel<float><<<nblk(nr, 256), 256, 0, st>>>(p->d_r, (const float *)w.ptr, w.scale, nr);
        else if (w.dtype == OSLALM_F16) mul_weight_kernel<__half><<<nblk(nr, 256), 256, 0, st>>>(p->d_r, (const __half *)w.ptr, w.scale, nr);
        else mul_weight_kernel<__nv_bfloat16><<<nblk(nr, 256), 256, 0, st>>>(p->d_r, (const __nv_bfloat16 *)w.ptr, w.scale, nr);
        OSL_LAUNCH_CHECK("mul_weight");
        if (int rc = launch_bp_any(p->g, p->d_r, p->d_g, p->d_views + p->off[m], p->cnt[m], BP_ACCUM, nullptr, st))
            return rc;
    }
    if (int rc = store_scaled(p, p->d_g, p->d_D, p->p.d_dtype, p->d_dscale, npix, st)) return rc;
    p->d_valid = true;
    return OSLALM_OK;
}

// The x-update: the constrained denoising problem of Sec. IV-A by n inner
// FISTA steps from x_in.  Step 0 is the projected SQS step from x_in (the
// whole update when n = 1); step i >= 1 starts from the extrapolated point
// v_i with the previous u_i; the last step writes x_out.  Buffers: u in
// d_fu[0], d_fu[1] alternately, v in d_fv[0], d_fv[1] (never read and
// written by one launch).
int update_step(oslalm_problem *p, const float *x_in, float *x_out, cudaStream_t st) {
    const oslalm_geom_desc &d = p->g->d;
    const int n = p->p.n_inner;
    const float beta = (float)p->p.beta, inv_delta = (float)(1.0 / p->p.delta);
    float *u0 = n == 1 ? x_out : p->d_fu[0];
    int rc = is_3d(p->g)
                 ? launch_update3d(d.nx, d.ny, d.nz, x_in, u0, p->d_zeta, p->d_g, p->d_D, p->p.d_dtype, p->d_dscale,
                                   p->d_state, beta, inv_delta, p->p.nbr, p->p.curvature, st)
                 : launch_update2d(d.nx, d.ny, x_in, u0, p->d_zeta, p->d_g, p->d_D, p->p.d_dtype, p->d_dscale,
                                   p->d_state, beta, inv_delta, p->p.nbr, p->p.curvature, st);
    if (rc || n == 1) return rc;
    // after step 0: u_1 = v_1 (gamma_0 = 0), both in d_fu[0]
    const float *v = p->d_fu[0], *u = p->d_fu[0];
    for (int i = 1; i < n; ++i) {
        const bool last = i == n - 1;
        float *uo = last ? x_out : p->d_fu[i & 1];
        float *vo = last ? nullptr : p->d_fv[(i - 1) & 1];
        const float gm = p->fista_gamma[i];
        rc = is_3d(p->g) ? launch_fista3d(d.nx, d.ny, d.nz, v, x_in, u, uo, vo, p->d_zeta, p->d_g, p->d_D,
                                          p->p.d_dtype, p->d_dscale, p->d_state, beta, inv_delta, p->p.nbr,
                                          p->p.curvature, gm, st)
                         : launch_fista2d(d.nx, d.ny, v, x_in, u, uo, vo, p->d_zeta, p->d_g, p->d_D, p->p.d_dtype,
                                          p->d_dscale, p->d_state, beta, inv_delta, p->p.nbr, p->p.curvature, gm, st);
        if (rc) return rc;
        v = vo;
        u = uo;
    }
    return OSLALM_OK;
}

// back-projection with the split-gradient update; x_new is the iterate at
// which subset `next`'s gradient is taken (Barzilai-Borwein secant pairs)
int bp_update(oslalm_problem *p, int next, const float *x_new, cudaStream_t st) {
    UpdateArgs ua = update_args(p, next);
    ua.x_new = x_new;
    return launch_bp_any(p->g, p->d_r, nullptr, p->d_views + p->off[next], p->cnt[next], BP_UPDATE, &ua, st);
}

// one subset-iteration: x_in -> x_out, gradient of subset `next`
int subset_iteration(oslalm_problem *p, const float *x_in, float *x_out, int next, cudaStream_t st) {
    if (int rc = update_step(p, x_in, x_out, st)) return rc;
    if (int rc = fp_subset(p, x_out, next, FP_RESID, (float)p->p.M, st)) return rc;
    return bp_update(p, next, x_out, st);
}

// `iters` whole iterations starting at subset-iteration j0 (a multiple of M)
int run_iterations(oslalm_problem *p, float *x, int iters, cudaStream_t st) {
    const int M = p->p.M;
    float *cur = x, *nxt = p->d_xalt;
    for (int it = 0; it < iters; ++it) {
        for (int q = 0; q < M; ++q) {
            int next = p->order[(q + 1) % M];
            if (int rc = subset_iteration(p, cur, nxt, next, st)) return rc;
            std::swap(cur, nxt);
        }
    }
    if (cur != x) OSL_CUDA_TRY(cudaMemcpyAsync(x, cur, p->npix * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return OSLALM_OK;
}

void drop_graph(oslalm_problem *p) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->g_x = nullptr;
}

int build_graph(oslalm_problem *p, float *x, cudaStream_t st) {
    drop_graph(p);
    const int iters = (p->p.M % 2) ? 2 : 1;  // return x to the caller's buffer
    cudaStream_t cs;
    OSL_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(OSLALM_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    int rc = run_iterations(p, x, iters, cs);
    e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(OSLALM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&p->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        p->gexec = nullptr;
        return fail(OSLALM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    p->g_x = x;
    p->g_iters = iters;
    p->g_stats_ptr = p->d_stats;
    (void)st;
    return OSLALM_OK;
}

int ensure_stats(oslalm_problem *p, long n) {
    if (n <= p->stats_cap) return OSLALM_OK;
    int cap = (int)std::max<long>(n, 4096);
    oslalm_stats *s = nullptr;
    OSL_CUDA_TRY(cudaMalloc(&s, sizeof(oslalm_stats) * cap));
    cudaFree(p->d_stats);
    p->d_stats = s;
    p->stats_cap = cap;
    drop_graph(p);  // the graph bakes the stats pointer
    return OSLALM_OK;
}

void free_problem(oslalm_problem *p) {
    drop_graph(p);
    cudaFree(p->d_views); cudaFree(p->d_y); cudaFree(p->d_w); cudaFree(p->d_wscale); cudaFree(p->d_D);
    cudaFree(p->d_dscale); cudaFree(p->d_maxbits); cudaFree(p->d_g); cudaFree(p->d_zeta); cudaFree(p->d_xalt);
    cudaFree(p->d_r); cudaFree(p->d_tmp); cudaFree(p->d_state); cudaFree(p->d_partials); cudaFree(p->d_stats);
    cudaFree(p->d_replay);
    cudaFree(p->d_fu[0]); cudaFree(p->d_fu[1]); cudaFree(p->d_fv[0]); cudaFree(p->d_fv[1]);
    cudaFree(p->d_bbx); cudaFree(p->d_bbz); cudaFree(p->d_bbhave); cudaFree(p->d_rho_tab);
    delete p;
}

}  // namespace

extern "C" {

int oslalm_project(const oslalm_geom *g, const float *x, float *sino, const int *views, int nv, void *stream) {
    clear_error();
    if (!g || nv < 0 || (nv > 0 && (!x || !sino || !views))) return fail(OSLALM_ERR_ARG, "bad project arguments");
    WeightRef w{nullptr, OSLALM_F32, nullptr};
    return launch_fp_any(g, x, sino, views, nv, FP_PLAIN, nullptr, w, 1.f, (cudaStream_t)stream);
}

int oslalm_backproject(const oslalm_geom *g, const float *sino, float *x, const int *views, int nv, int accumulate,
                       void *stream) {
    clear_error();
    if (!g || nv < 0 || !x || (nv > 0 && (!sino || !views))) return fail(OSLALM_ERR_ARG, "bad backproject arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (nv == 0) {
        if (!accumulate) OSL_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(float) * g->d.nx * g->d.ny * g->d.nz, st));
        return OSLALM_OK;
    }
    return launch_bp_any(g, sino, x, views, nv, accumulate ? BP_ACCUM : BP_STORE, nullptr, st);
}

int oslalm_problem_create(const oslalm_geom *g, const float *y, const float *w, const oslalm_params *prm,
                          oslalm_problem **out) {
    clear_error();
    if (!out) return fail(OSLALM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !y || !w || !prm) return fail(OSLALM_ERR_ARG, "NULL argument");
    const oslalm_params &pp = *prm;
    if (pp.M <= 0 || pp.M > g->d.nviews) return fail(OSLALM_ERR_ARG, "need 0 < M <= nviews (M=%d)", pp.M);
    if (!(pp.beta >= 0) || !(pp.delta > 0)) return fail(OSLALM_ERR_ARG, "need beta >= 0 and delta > 0");
    if (!is_3d(g) && pp.nbr != 4 && pp.nbr != 8) return fail(OSLALM_ERR_ARG, "2D neighbourhood must be 4 or 8");
    if (is_3d(g) && pp.nbr != 6 && pp.nbr != 26) return fail(OSLALM_ERR_ARG, "3D neighbourhood must be 6 or 26");
    if (pp.n_inner < 1 || pp.n_inner > 64) return fail(OSLALM_ERR_RANGE, "need 1 <= n_inner <= 64");
    if (pp.rho_mode < 0 || pp.rho_mode > 2) return fail(OSLALM_ERR_ARG, "bad rho_mode");
    if (pp.rho_mode == OSLALM_RHO_FIXED && !(pp.rho_fixed > 0)) return fail(OSLALM_ERR_ARG, "rho_fixed must be > 0");
    if (pp.rho_mode != OSLALM_RHO_FIXED && !(pp.rho_min > 0 && pp.rho_min <= 1)) return fail(OSLALM_ERR_ARG, "need 0 < rho_min <= 1");
    if (pp.w_dtype < 0 || pp.w_dtype > 2 || pp.d_dtype < 0 || pp.d_dtype > 2) return fail(OSLALM_ERR_ARG, "bad dtype");
    if (pp.curvature != OSLALM_CURV_HUBER && pp.curvature != OSLALM_CURV_MAX) return fail(OSLALM_ERR_ARG, "bad curvature");
    if (pp.bb != 0 && pp.bb != 1) return fail(OSLALM_ERR_ARG, "bb must be 0 or 1");
    int p_n_partials_tmp = 0;
    oslalm_problem *p = new (std::nothrow) oslalm_problem();
    if (!p) return fail(OSLALM_ERR_ALLOC, "host allocation failed");
    p->g = g;
    p->p = pp;
    {  // FISTA momentum gamma_i = (tau_i - 1) / tau_{i+1}, tau_0 = 1 (Beck & Teboulle)
        double tau = 1.0;
        for (int i = 0; i < pp.n_inner; ++i) {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tau * tau));
            p->fista_gamma.push_back((float)((tau - 1.0) / tn));
            tau = tn;
        }
    }
    const oslalm_geom_desc &d = g->d;
    p->npix = (long)d.nx * d.ny * d.nz;
    p->per_view = d.nt * d.ns;
    p->order.resize(pp.M);
    oslalm_subset_order(pp.M, p->order.data());
    std::vector<int> perm;
    p->max_cnt = 0;
    for (int m = 0; m < pp.M; ++m) {
        p->off.push_back((int)perm.size());
        for (int v = m; v < d.nviews; v += pp.M) perm.push_back(v);
        p->cnt.push_back((int)perm.size() - p->off.back());
        p->max_cnt = std::max(p->max_cnt, p->cnt.back());
    }
    size_t nsino = (size_t)d.nviews * p->per_view;
    size_t nr = (size_t)std::max(p->max_cnt, 1) * p->per_view;
    // cost: one partial per 128 rays of every subset plus the regularizer blocks
    {
        const oslalm_geom_desc &dd = g->d;
        long reg_blocks = (long)((dd.nx + 31) / 32) * ((dd.ny + 7) / 8) * dd.nz;
        long np = (long)nblk(nsino, 128) + pp.M + std::max<long>(reg_blocks, bp_blocks_any(g)) + 64;
        np = std::max<long>(np, 3L * bp_blocks_any(g) + 64);  // xi, s'y, s'Ds per back-projection block
        if (np > (1L << 30)) {
            delete p;
            return fail(OSLALM_ERR_RANGE, "problem too large");
        }
        p_n_partials_tmp = (int)np;
    }
    p->n_partials = p_n_partials_tmp;
    cudaError_t e = cudaSuccess;
#define OSL_ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
    OSL_ALLOC(p->d_views, sizeof(int) * d.nviews);
    OSL_ALLOC(p->d_y, sizeof(float) * nsino);
    OSL_ALLOC(p->d_w, dtype_size(pp.w_dtype) * nsino);
    OSL_ALLOC(p->d_tmp, sizeof(float) * nsino);
    OSL_ALLOC(p->d_wscale, sizeof(float));
    OSL_ALLOC(p->d_D, dtype_size(pp.d_dtype) * p->npix);
    OSL_ALLOC(p->d_dscale, sizeof(float));
    OSL_ALLOC(p->d_maxbits, sizeof(unsigned int));
    OSL_ALLOC(p->d_g, sizeof(float) * p->npix);
    OSL_ALLOC(p->d_zeta, sizeof(float) * p->npix);
    OSL_ALLOC(p->d_xalt, sizeof(float) * p->npix);
    OSL_ALLOC(p->d_r, sizeof(float) * nr);
    OSL_ALLOC(p->d_state, sizeof(DevState));
    OSL_ALLOC(p->d_partials, sizeof(double) * p->n_partials);
    if (pp.n_inner > 1) {
        for (int k = 0; k < 2; ++k) {
            OSL_ALLOC(p->d_fu[k], sizeof(float) * p->npix);
            OSL_ALLOC(p->d_fv[k], sizeof(float) * p->npix);
        }
    }
    if (pp.bb) {
        OSL_ALLOC(p->d_bbx, sizeof(float) * p->npix * pp.M);
        OSL_ALLOC(p->d_bbz, sizeof(float) * p->npix * pp.M);
        OSL_ALLOC(p->d_bbhave, sizeof(int) * pp.M);
    }
#undef OSL_ALLOC
    if (e != cudaSuccess) {
        free_problem(p);
        return fail(OSLALM_ERR_ALLOC, "device allocation failed: %s", cudaGetErrorString(e));
    }
    if (pp.rho_mode != OSLALM_RHO_FIXED) {
        // rho_l of the continuation (Eq. rho_l_formula_qp) up to the first l at
        // which it reaches rho_min (at most 65536 entries), with the weights of
        // the g-update, in the operations of the device's rho_of_l
        std::vector<RhoEnt> tab;
        for (int l = 0; l < 65536; ++l) {
            double rho = 1.0;
            if (l > 0) {
                const double pi = 3.14159265358979323846;
                const double a = pi / (double)(l + 1), b = pi / (double)(2 * l + 2);
                const double v = a * sqrt(1.0 - b * b);
                rho = v > pp.rho_min ? v : pp.rho_min;
            }
            tab.push_back(RhoEnt{rho, (float)(rho / (rho + 1.0)), (float)(1.0 / (rho + 1.0))});
            if (l > 0 && rho == pp.rho_min) break;
        }
        if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_rho_tab, sizeof(RhoEnt) * tab.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->d_rho_tab, tab.data(), sizeof(RhoEnt) * tab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_problem(p);
            return fail(OSLALM_ERR_ALLOC, "continuation table: %s", cudaGetErrorString(e));
        }
        // past the last entry rho stays at rho_min; the device reads the table
        // only for l + 1 < rho_tab_n and otherwise forms rho_l itself
        p->rho_tab_n = (int)tab.size();
    }
    if ((e = cudaMemcpy(p->d_views, perm.data(), sizeof(int) * d.nviews, cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_problem(p);
        return fail(OSLALM_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }
    int rc = load_data(p, y, w, nullptr);
    if (!rc && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = fail(OSLALM_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (rc) {
        free_problem(p);
        return rc;
    }
    *out = p;
    return OSLALM_OK;
}

int oslalm_problem_destroy(oslalm_problem *p) {
    clear_error();
    if (!p) return OSLALM_OK;
    free_problem(p);
    return OSLALM_OK;
}

int oslalm_problem_set_data(oslalm_problem *p, const float *y, const float *w, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!y || !w) return fail(OSLALM_ERR_ARG, "NULL data");
    return load_data(p, y, w, (cudaStream_t)stream);
}

int oslalm_init(oslalm_problem *p, const float *x, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!x) return fail(OSLALM_ERR_ARG, "x is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (!p->d_valid)
        if (int rc = compute_denominator(p, st)) return rc;
    const int m0 = p->order[0];
    if (int rc = fp_subset(p, x, m0, FP_RESID, (float)p->p.M, st)) return rc;
    UpdateArgs ua = update_args(p, m0);
    if (int rc = launch_bp_any(p->g, p->d_r, nullptr, p->d_views + p->off[m0], p->cnt[m0], BP_INIT, &ua, st))
        return rc;
    const double rho0 = p->p.rho_mode == OSLALM_RHO_FIXED ? p->p.rho_fixed : 1.0;
    set_state_kernel<<<1, 1, 0, st>>>(p->d_state, rho0, 0, 0, 1.0);
    OSL_LAUNCH_CHECK("set_state");
    if (p->p.bb) {  // the first gradient (subset sigma(0) at x0) opens its secant history
        const size_t nb = sizeof(float) * p->npix;
        OSL_CUDA_TRY(cudaMemsetAsync(p->d_bbhave, 0, sizeof(int) * p->p.M, st));
        OSL_CUDA_TRY(cudaMemcpyAsync(p->d_bbx + (size_t)m0 * p->npix, x, nb, cudaMemcpyDeviceToDevice, st));
        OSL_CUDA_TRY(cudaMemcpyAsync(p->d_bbz + (size_t)m0 * p->npix, p->d_zeta, nb, cudaMemcpyDeviceToDevice, st));
        const int one = 1;
        OSL_CUDA_TRY(cudaMemcpyAsync(p->d_bbhave + m0, &one, sizeof(int), cudaMemcpyHostToDevice, st));
        OSL_CUDA_TRY(cudaStreamSynchronize(st));  // `one` lives on this stack frame
    }
    p->j_host = 0;
    p->initialized = true;
    return OSLALM_OK;
}

int oslalm_iterate(oslalm_problem *p, float *x, int n_iter, oslalm_stats *stats, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!p->initialized) return fail(OSLALM_ERR_STATE, "oslalm_iterate before oslalm_init");
    if (!x || n_iter < 0) return fail(OSLALM_ERR_ARG, "bad iterate arguments");
    if (n_iter == 0) return OSLALM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const long nsub = (long)n_iter * p->p.M;
    const long j0 = p->j_host;
    if (stats)
        if (int rc = ensure_stats(p, nsub)) return rc;
    int done = 0;
    if (p->p.use_graph) {
        if (!p->gexec || p->g_x != x || p->g_stats_ptr != p->d_stats)
            if (int rc = build_graph(p, x, st)) return rc;
        while (n_iter - done >= p->g_iters) {
            OSL_CUDA_TRY(cudaGraphLaunch(p->gexec, st));
            done += p->g_iters;
        }
    }
    if (done < n_iter)
        if (int rc = run_iterations(p, x, n_iter - done, st)) return rc;
    p->j_host += nsub;
    if (stats) {
        OSL_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<oslalm_stats> ring(p->stats_cap);
        OSL_CUDA_TRY(cudaMemcpy(ring.data(), p->d_stats, sizeof(oslalm_stats) * p->stats_cap, cudaMemcpyDeviceToHost));
        for (long k = 0; k < nsub; ++k) stats[k] = ring[(size_t)((j0 + k) % p->stats_cap)];
    }
    return OSLALM_OK;
}

int oslalm_profile_iterate(oslalm_problem *p, float *x, int n_iter, double *ms_out, int *launches_out,
                           void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!p->initialized) return fail(OSLALM_ERR_STATE, "oslalm_profile_iterate before oslalm_init");
    if (!x || n_iter < 0 || !ms_out || !launches_out) return fail(OSLALM_ERR_ARG, "bad profile arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int M = p->p.M;
    const long nsub = (long)n_iter * M;
    std::vector<cudaEvent_t> ev(6 * nsub);
    for (auto &e : ev) OSL_CUDA_TRY(cudaEventCreate(&e));
    float *cur = x, *nxt = p->d_xalt;
    int rc = OSLALM_OK;
    long k = 0;
    for (int it = 0; it < n_iter && !rc; ++it) {
        for (int q = 0; q < M && !rc; ++q, ++k) {
            int next = p->order[(q + 1) % M];
            cudaEventRecord(ev[6 * k + 0], st);
            rc = update_step(p, cur, nxt, st);
            cudaEventRecord(ev[6 * k + 1], st);
            cudaEventRecord(ev[6 * k + 2], st);
            if (!rc) rc = fp_subset(p, nxt, next, FP_RESID, (float)M, st);
            cudaEventRecord(ev[6 * k + 3], st);
            cudaEventRecord(ev[6 * k + 4], st);
            if (!rc) rc = bp_update(p, next, nxt, st);
            cudaEventRecord(ev[6 * k + 5], st);
            std::swap(cur, nxt);
        }
    }
    if (!rc && cur != x) {
        cudaError_t e = cudaMemcpyAsync(x, cur, p->npix * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = fail(OSLALM_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(OSLALM_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    if (!rc) {
        for (int kind = 0; kind < 3; ++kind) {
            ms_out[kind] = 0.0;
            launches_out[kind] = (int)k;
        }
        for (long i = 0; i < k; ++i)
            for (int kind = 0; kind < 3; ++kind) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[6 * i + 2 * kind], ev[6 * i + 2 * kind + 1]);
                ms_out[kind] += ms;
            }
        p->j_host += nsub;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

int oslalm_set_replay(oslalm_problem *p, const int *restarts, int n) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (n < 0 || (n > 0 && !restarts)) return fail(OSLALM_ERR_ARG, "bad replay list");
    std::vector<signed char> h(n);
    for (int i = 0; i < n; ++i) h[i] = restarts[i] ? 1 : 0;
    OSL_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(p->d_replay);
    p->d_replay = nullptr;
    p->replay_n = 0;
    if (n > 0) {
        OSL_CUDA_TRY(cudaMalloc(&p->d_replay, n));
        OSL_CUDA_TRY(cudaMemcpy(p->d_replay, h.data(), n, cudaMemcpyHostToDevice));
    }
    p->replay_n = n;
    drop_graph(p);
    return OSLALM_OK;
}

int oslalm_cost(oslalm_problem *p, const float *x, double *out, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!x || !out) return fail(OSLALM_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int used = 0;
    for (int m = 0; m < p->p.M; ++m) {
        int np = 0;
        const float *y = p->d_y + (size_t)p->off[m] * p->per_view;
        if (used + (int)nblk((size_t)p->cnt[m] * p->per_view, 128) > p->n_partials)
            return fail(OSLALM_ERR_RANGE, "cost partial buffer too small");
        int rc = is_3d(p->g) ? launch_cost3d(p->g->geo3(), x, p->d_views + p->off[m], p->cnt[m], y, wref(p, m),
                                             p->d_partials + used, &np, st)
                             : launch_cost2d(p->g->geo2(), x, p->d_views + p->off[m], p->cnt[m], y, wref(p, m),
                                             p->d_partials + used, &np, st);
        if (rc) return rc;
        used += np;
    }
    const oslalm_geom_desc &d = p->g->d;
    if (used + (long)((d.nx + 31) / 32) * ((d.ny + 7) / 8) * d.nz > p->n_partials)
        return fail(OSLALM_ERR_RANGE, "cost partial buffer too small");
    int np = 0;
    int rcr = is_3d(p->g) ? launch_reg_value3d(d.nx, d.ny, d.nz, x, p->p.beta, p->p.delta, p->p.nbr,
                                               p->d_partials + used, &np, st)
                          : launch_reg_value2d(d.nx, d.ny, x, p->p.beta, p->p.delta, p->p.nbr, p->d_partials + used,
                                               &np, st);
    if (rcr) return rcr;
    used += np;
    std::vector<double> h(used);
    OSL_CUDA_TRY(cudaMemcpyAsync(h.data(), p->d_partials, sizeof(double) * used, cudaMemcpyDeviceToHost, st));
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int i = 0; i < used; ++i) s += h[i];
    *out = s;
    return OSLALM_OK;
}

int oslalm_gradient(oslalm_problem *p, const float *x, float *grad, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!x || !grad) return fail(OSLALM_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    OSL_CUDA_TRY(cudaMemsetAsync(grad, 0, p->npix * sizeof(float), st));
    for (int m = 0; m < p->p.M; ++m) {  // A_m' W_m (A_m x - y_m), subset by subset
        if (p->cnt[m] == 0) continue;
        if (int rc = fp_subset(p, x, m, FP_RESID, 1.f, st)) return rc;
        if (int rc = launch_bp_any(p->g, p->d_r, grad, p->d_views + p->off[m], p->cnt[m], BP_ACCUM, nullptr, st))
            return rc;
    }
    const oslalm_geom_desc &d = p->g->d;
    return launch_reg_grad_add(d.nx, d.ny, d.nz, x, grad, (float)p->p.beta, (float)(1.0 / p->p.delta), p->p.nbr, st);
}

int oslalm_get_state(oslalm_problem *p, float *g, float *zeta, double *rho_l_j, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!p->initialized) return fail(OSLALM_ERR_STATE, "no state before oslalm_init");
    cudaStream_t st = (cudaStream_t)stream;
    if (g) OSL_CUDA_TRY(cudaMemcpyAsync(g, p->d_g, p->npix * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (zeta) OSL_CUDA_TRY(cudaMemcpyAsync(zeta, p->d_zeta, p->npix * sizeof(float), cudaMemcpyDeviceToDevice, st));
    DevState h;
    OSL_CUDA_TRY(cudaMemcpyAsync(&h, p->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    if (rho_l_j) {
        rho_l_j[0] = h.rho;
        rho_l_j[1] = h.l;
        rho_l_j[2] = h.j;
        rho_l_j[3] = h.alpha;
    }
    return OSLALM_OK;
}

int oslalm_set_state(oslalm_problem *p, const float *g, const float *zeta, const double *rho_l_j, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!p->initialized) return fail(OSLALM_ERR_STATE, "oslalm_set_state before oslalm_init");
    if (!g || !zeta || !rho_l_j) return fail(OSLALM_ERR_ARG, "NULL argument");
    long j = (long)rho_l_j[2];
    if (j < 0 || j % p->p.M != 0) return fail(OSLALM_ERR_ARG, "resume point must be a whole iteration");
    cudaStream_t st = (cudaStream_t)stream;
    OSL_CUDA_TRY(cudaMemcpyAsync(p->d_g, g, p->npix * sizeof(float), cudaMemcpyDeviceToDevice, st));
    OSL_CUDA_TRY(cudaMemcpyAsync(p->d_zeta, zeta, p->npix * sizeof(float), cudaMemcpyDeviceToDevice, st));
    set_state_kernel<<<1, 1, 0, st>>>(p->d_state, rho_l_j[0], (int)rho_l_j[1], (int)j, rho_l_j[3]);
    OSL_LAUNCH_CHECK("set_state");
    if (p->p.bb) OSL_CUDA_TRY(cudaMemsetAsync(p->d_bbhave, 0, sizeof(int) * p->p.M, st));  // secant history restarts
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    p->j_host = j;
    return OSLALM_OK;
}

int oslalm_get_denominator(oslalm_problem *p, float *dout, void *stream) {
    clear_error();
    if (int rc = check_problem(p)) return rc;
    if (!p->d_valid) return fail(OSLALM_ERR_STATE, "denominator not computed (call oslalm_init)");
    if (!dout) return fail(OSLALM_ERR_ARG, "NULL output");
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = p->npix;
    if (p->p.d_dtype == OSLALM_F32) dequantize_kernel<float><<<nblk(n, 256), 256, 0, st>>>((const float *)p->d_D, dout, n, p->d_dscale);
    else if (p->p.d_dtype == OSLALM_F16) dequantize_kernel<__half><<<nblk(n, 256), 256, 0, st>>>((const __half *)p->d_D, dout, n, p->d_dscale);
    else dequantize_kernel<__nv_bfloat16><<<nblk(n, 256), 256, 0, st>>>((const __nv_bfloat16 *)p->d_D, dout, n, p->d_dscale);
    OSL_LAUNCH_CHECK("dequantize");
    return OSLALM_OK;
}

int oslalm_rmsd(const float *x, const float *xref, const uint8_t *mask, long n, double *out, void *stream) {
    clear_error();
    if (!x || !xref || !mask || !out || n <= 0) return fail(OSLALM_ERR_ARG, "bad rmsd arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::min<long>((n + 255) / 256, 1024);
    double *part = nullptr;
    OSL_CUDA_TRY(cudaMallocAsync((void **)&part, sizeof(double) * 2 * blocks, st));
    rmsd_kernel<<<blocks, 256, 0, st>>>(x, xref, mask, n, part);
    OSL_LAUNCH_CHECK("rmsd");
    std::vector<double> h(2 * blocks);
    OSL_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, st));
    OSL_CUDA_TRY(cudaFreeAsync(part, st));
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0, c = 0.0;
    for (int i = 0; i < blocks; ++i) {
        s += h[2 * i];
        c += h[2 * i + 1];
    }
    *out = c > 0 ? sqrt(s / c) : 0.0;
    return OSLALM_OK;
}

}  // extern "C"
