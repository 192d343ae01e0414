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
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
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

}  // namespace oslalm
