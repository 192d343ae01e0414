// Small device helpers shared by the kernel translation units.
#pragma once

#include "common.cuh"

namespace oslalm {

__device__ __forceinline__ float load_w(const float *p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_w(const __half *p, size_t i) { return __half2float(p[i]); }
__device__ __forceinline__ float load_w(const __nv_bfloat16 *p, size_t i) { return __bfloat162float(p[i]); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a 1D block of NT threads; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[NT / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < NT / 32 ? red[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Sum over a 2D block (any shape up to 1024 threads) using caller scratch;
// result valid in thread (0, 0).  Fixed order: deterministic.
__device__ __forceinline__ double block_sum2d(double v, double *red) {
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (tid < 32) {
        t = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Sum of FP64 values over a block in FP32 double-float arithmetic (each value
// split into hi + lo floats, pairs added with Knuth's error-free two-sum and
// renormalised), for the per-subset-iteration reductions: FP64 throughput is
// scarce on this GPU, and the pair keeps about 2^-44 relative accuracy.  Fixed
// order: deterministic.  Result valid in thread (0, 0) of the block; red holds
// 2 x 32 floats of caller scratch.
__device__ __forceinline__ void df_add(float &hi, float &lo, float h2, float l2) {
    const float s = __fadd_rn(hi, h2);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
    const float t = __fadd_rn(__fadd_rn(lo, l2), e);
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

__device__ __forceinline__ double block_sum_df(double v, float *red) {
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        df_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
    if ((tid & 31) == 0) {
        red[tid >> 5] = hi;
        red[32 + (tid >> 5)] = lo;
    }
    __syncthreads();
    double t = 0.0;
    if (tid < 32) {
        const bool in = tid < (nt + 31) / 32;
        hi = in ? red[tid] : 0.f;
        lo = in ? red[32 + tid] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            df_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
        t = (double)hi + (double)lo;
    }
    __syncthreads();
    return t;
}

// hyperbola potential psi(t) = delta^2 (sqrt(1 + (t/delta)^2) - 1), written
// without the cancellation of the difference
__device__ __forceinline__ double hyperbola(double t, double delta) {
    double u = t / delta;
    return t * t / (sqrt(1.0 + u * u) + 1.0);
}

// neighbour k (0..7) of the 3x3 square without the centre
__device__ __forceinline__ void nbr2d(int k, int &ox, int &oy) {
    const int idx = k < 4 ? k : k + 1;
    ox = idx % 3 - 1;
    oy = idx / 3 - 1;
}

// rho_l of the deterministic downward continuation (Eq. rho_l_formula_qp)
__device__ __forceinline__ double rho_of_l(int l, double rho_min) {
    if (l == 0) return 1.0;
    const double pi = 3.14159265358979323846;
    double a = pi / (double)(l + 1);
    double b = pi / (double)(2 * l + 2);
    double v = a * sqrt(1.0 - b * b);
    return v > rho_min ? v : rho_min;
}

// D at pixel p (dequantized) for the Barzilai-Borwein sum s'Ds.
__device__ __forceinline__ double bb_dval(const UpdateArgs &ua, size_t p) {
    float v;
    if (ua.d_dtype == OSLALM_F32) v = load_w((const float *)ua.D, p);
    else if (ua.d_dtype == OSLALM_F16) v = load_w((const __half *)ua.D, p);
    else v = load_w((const __nv_bfloat16 *)ua.D, p);
    return (double)v * (double)__ldg(ua.dscale);
}

// Per-pixel terms of the subset-iteration's reductions: the restart
// indicator xi += (g - zeta+)(zeta+ - zeta) (old g, old zeta) and, with the
// Barzilai-Borwein fit, the secant pair of this subset over the last
// iteration (supplement Eq. scale_factor_alpha_k): s'y += s (zeta+ - zeta_m)
// and s'Ds += D s^2, s = x_new - x_m, where (x_m, zeta_m) is where and what
// this subset's gradient was last time; then (x_new, zeta+) replace them.
struct IterSums {
    double xi, sy, sds;
};

__device__ __forceinline__ void add_iter_terms(const UpdateArgs &ua, size_t p, float g_old, float z_old, float zn,
                                               IterSums &acc) {
    acc.xi += (double)(g_old - zn) * (double)(zn - z_old);
    if (ua.bb) {
        const size_t q = (size_t)ua.subset * (size_t)ua.npix + p;
        const float xn = __ldg(ua.x_new + p);
        if (ua.bbhave[ua.subset]) {
            const double s = (double)xn - (double)ua.bbx[q];
            acc.sy += s * ((double)zn - (double)ua.bbz[q]);
            acc.sds += bb_dval(ua, p) * s * s;
        }
        ua.bbx[q] = xn;
        ua.bbz[q] = zn;
    }
}

// Last block of a grid: reduce the per-block partials in a fixed order and
// advance the continuation state (Sec. III-B): restart (l = 0) when xi > 0,
// else l + 1; rho = rho_l; with Barzilai-Borwein scaling, the secant sums
// are added up over the iteration and at its end alpha = min(s'y / s'Ds, 1),
// or 1 when s'y <= 0 or s'Ds = 0.  One thread writes the state.
__device__ __forceinline__ void finish_subset_iteration(const UpdateArgs &ua, int nblocks) {
    __shared__ double red_last[32];
    __shared__ float red_df[64];
    double v = 0.0, vy = 0.0, vd = 0.0;
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    DevState *st = ua.state;
    // thread 0 fetches the state and the two continuation-table entries the
    // update may need (l + 1, or 0 after a restart) before the partials, so
    // their latency overlaps the reduction
    double rho_used = 0.0, alpha = 1.0;
    int j = 0, l = 0;
    bool tab = false;
    RhoEnt e0{}, e1{};
    if (tid == 0) {
        rho_used = __ldcg(&st->rho);
        alpha = __ldcg(&st->alpha);
        j = __ldcg(&st->j);
        l = __ldcg(&st->l);
        tab = ua.rho_mode != OSLALM_RHO_FIXED && ua.rho_tab && l + 1 < ua.rho_tab_n;
        if (tab) {
            e0 = ua.rho_tab[0];
            e1 = ua.rho_tab[l + 1];
        }
    }
    for (int i = tid; i < nblocks; i += nt) {
        v += __ldcg(ua.partials + i);
        if (ua.bb) {
            vy += __ldcg(ua.partials + nblocks + i);
            vd += __ldcg(ua.partials + 2 * nblocks + i);
        }
    }
    v = block_sum_df(v, red_df);
    if (ua.bb) {
        vy = block_sum2d(vy, red_last);
        vd = block_sum2d(vd, red_last);
    }
    if (tid == 0) {
        const double xi = v;
        int restart = 0;
        double rho = rho_used;
        if (ua.rho_mode == OSLALM_RHO_CONTINUATION) {
            restart = xi > 0.0;
        } else if (ua.rho_mode == OSLALM_RHO_REPLAY) {
            restart = (ua.replay && j < ua.replay_n) ? (ua.replay[j] != 0) : 0;
        }
        if (ua.rho_mode != OSLALM_RHO_FIXED) {
            l = restart ? 0 : l + 1;
            rho = tab ? (restart ? e0.rho : e1.rho) : rho_of_l(l, ua.rho_min);
        }
        if (ua.bb) {  // refit H = alpha D at the end of every iteration
            st->bb_num += vy;
            st->bb_den += vd;
            ua.bbhave[ua.subset] = 1;
            if ((j + 1) % ua.M == 0) {
                const double num = st->bb_num, den = st->bb_den;
                alpha = (den > 0.0 && num > 0.0) ? fmin(num / den, 1.0) : 1.0;
                st->alpha = alpha;
                st->bb_num = 0.0;
                st->bb_den = 0.0;
            }
        }
        st->xi = xi;
        st->l = l;
        st->rho = rho;
        if (tab) {  // the same values refresh_rho_factors forms, from the host's table
            const RhoEnt &e = restart ? e0 : e1;
            st->rho_f = (float)rho;
            st->rho_d_f = alpha == 1.0 ? (float)rho : (float)(rho * alpha);
            st->ga = e.ga;
            st->gb = e.gb;
        } else if (ua.rho_mode != OSLALM_RHO_FIXED || ua.bb) {
            refresh_rho_factors(st);
        }
        if (ua.stats && ua.stats_cap > 0) {
            oslalm_stats rec;
            rec.xi = xi;
            rec.rho_used = rho_used;
            rec.l = l;
            rec.restart = restart;
            rec.subset = ua.subset;
            rec.pad = 0;
            rec.alpha = alpha;
            ua.stats[j % ua.stats_cap] = rec;
        }
        st->j = j + 1;
        st->counter = 0;  // read by the next launch (kernel boundaries order it)
    }
}

// Block sums of the threads' terms into the partials buffer; the last block
// to arrive finishes the subset-iteration.  Called by every thread.
__device__ __forceinline__ void subset_iteration_epilogue(const UpdateArgs &ua, const IterSums &loc) {
    __shared__ double red[32];
    __shared__ float red_df[64];
    __shared__ int is_last;
    const double bs = block_sum_df(loc.xi, red_df);
    double by = 0.0, bd = 0.0;
    if (ua.bb) {
        by = block_sum2d(loc.sy, red);
        bd = block_sum2d(loc.sds, red);
    }
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int tid = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    if (tid == 0) {
        const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        ua.partials[bid] = bs;
        if (ua.bb) {
            ua.partials[nblocks + bid] = by;
            ua.partials[2 * nblocks + bid] = bd;
        }
        __threadfence();
        unsigned t = atomicAdd(&ua.state->counter, 1u);
        is_last = (t == (unsigned)(nblocks - 1));
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        finish_subset_iteration(ua, nblocks);
    }
}

}  // namespace oslalm
