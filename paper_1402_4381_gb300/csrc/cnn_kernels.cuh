// BF16 tensor-core kernels of the warm-start network (FP32 accumulation).
//
// Activations are NHWC BF16 with channel counts that are multiples of 32; a
// tensor may be a channel slice of a wider buffer (leading dimension `ld`,
// channel offset `coff`), which makes the U-Net's concatenations free.
//
// conv3x3_kernel: implicit GEMM  out[p][co] = sum_{tap, ci} in[p + shift(tap)][ci] w[co][tap][ci]
//   block tile 128 pixels x 32 output channels, K step = one tap x 32 input
//   channels, double-buffered cp.async staging, ldmatrix + mma.sync
//   m16n8k16 (bf16 x bf16 -> f32).  With transposed, tap-flipped weights the
//   same kernel computes the data gradient.
// wgrad3x3_kernel: dW[co][tap][ci] = sum_p dz[p][co] x[p + shift(tap)][ci],
//   split over pixel ranges, partial tiles added with FP32 atomics.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace oslalm {
namespace cnn {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;  // zero-fill when the source is out of bounds
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma16816(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct ConvArgs {
    const __nv_bfloat16 *in;  // NHWC, channel slice [coff_in, coff_in + cin) of ld_in channels
    int ld_in, coff_in, cin;
    const __nv_bfloat16 *w;   // [cout][9][cin]
    const float *bias;        // [cout] or null
    __nv_bfloat16 *out;       // NHWC slice [coff_out, coff_out + cout) of ld_out channels
    int ld_out, coff_out, cout;
    int n, h, wd;             // images, height, width
    int relu;
};

constexpr int kBM = 128, kBN = 32, kBK = 32, kStride = 40;  // smem row stride (elements): conflict-free ldmatrix

__global__ void __launch_bounds__(128) conv3x3_kernel(ConvArgs a) {
    __shared__ __align__(16) __nv_bfloat16 sA[2][kBM * kStride];
    __shared__ __align__(16) __nv_bfloat16 sB[2][kBN * kStride];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long P = (long)a.n * a.h * a.wd;
    const long p0 = (long)blockIdx.x * kBM;
    const int co0 = blockIdx.y * kBN;
    const int nk = 9 * (a.cin / kBK);  // K steps
    // per-thread A rows: 4 chunks of 16 B -> (row, chunk)
    auto load_stage = [&](int ks, int buf) {
        const int tap = ks / (a.cin / kBK), ci0 = (ks % (a.cin / kBK)) * kBK;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + q * 128;  // 0..511
            const int row = idx >> 2, ch = idx & 3;
            const long p = p0 + row;
            bool ok = p < P;
            long src = 0;
            if (ok) {
                const int x = (int)(p % a.wd);
                const long t = p / a.wd;
                const int y = (int)(t % a.h);
                const int yy = y + dy, xx = x + dx;
                ok = yy >= 0 && yy < a.h && xx >= 0 && xx < a.wd;
                src = p + (long)dy * a.wd + dx;
            }
            const __nv_bfloat16 *g = a.in + (ok ? src : 0) * a.ld_in + a.coff_in + ci0 + ch * 8;
            cp_async16(&sA[buf][row * kStride + ch * 8], g, ok);
        }
        {
            const int row = tid >> 2, ch = tid & 3;  // 32 rows (co) x 4 chunks
            const __nv_bfloat16 *g = a.w + ((long)(co0 + row) * 9 + tap) * a.cin + ci0 + ch * 8;
            cp_async16(&sB[buf][row * kStride + ch * 8], g, co0 + row < a.cout);
        }
        cp_async_commit();
    };
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    load_stage(0, 0);
    for (int ks = 0; ks < nk; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < nk) {
            load_stage(ks + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = warp * 32 + mi * 16 + (lane & 15);
                ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], &sA[buf][r * kStride + kk + (lane >> 4) * 8]);
            }
            uint32_t bf[4][2];
#pragma unroll
            for (int nj = 0; nj < 4; nj += 2) {
                // two n8 tiles: matrices (n rows 0-7, k0), (n 0-7, k0+8), (n 8-15, k0), (n 8-15, k0+8)
                const int r = nj * 8 + (lane & 7) + ((lane >> 4) << 3);
                const int c = kk + ((lane >> 3) & 1) * 8;
                ldsm_x4(bf[nj][0], bf[nj][1], bf[nj + 1][0], bf[nj + 1][1], &sB[buf][r * kStride + c]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int nj = 0; nj < 4; ++nj) mma16816(acc[mi][nj], af[mi], bf[nj][0], bf[nj][1]);
        }
        __syncthreads();
    }
    // epilogue: bias, ReLU, BF16 store of pairs of channels
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj)
#pragma unroll
            for (int hrow = 0; hrow < 2; ++hrow) {
                const long p = p0 + warp * 32 + mi * 16 + (lane >> 2) + hrow * 8;
                const int co = co0 + nj * 8 + (lane & 3) * 2;
                if (p >= P || co >= a.cout) continue;
                float v0 = acc[mi][nj][hrow * 2 + 0], v1 = acc[mi][nj][hrow * 2 + 1];
                if (a.bias) {
                    v0 += a.bias[co];
                    v1 += a.bias[co + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162 *>(a.out + p * a.ld_out + a.coff_out + co) = __floats2bfloat162_rn(v0, v1);
            }
}

struct WgradArgs {
    const __nv_bfloat16 *dz;  // [P][cout] (ld_dz, coff_dz)
    int ld_dz, coff_dz, cout;
    const __nv_bfloat16 *x;   // [P][cin] slice (ld_x, coff_x)
    int ld_x, coff_x, cin;
    float *dw;                // [cout][9][cin], accumulated with atomics
    int n, h, wd;
    int pix_per_block;
};

// block: 64 output channels x 32 input channels of one tap, over a pixel range
__global__ void __launch_bounds__(128) wgrad3x3_kernel(WgradArgs a) {
    constexpr int BM = 64, BN = 32, BK = 32;
    __shared__ __align__(16) __nv_bfloat16 sA[2][BK * 72];  // [p][co], row stride 72 (64 + 8)
    __shared__ __align__(16) __nv_bfloat16 sB[2][BK * 40];  // [p][ci], row stride 40
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long P = (long)a.n * a.h * a.wd;
    const int co0 = blockIdx.x * BM;
    const int tap = blockIdx.y / (a.cin / BN);
    const int ci0 = (blockIdx.y % (a.cin / BN)) * BN;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long pbeg = (long)blockIdx.z * a.pix_per_block;
    const long pend = pbeg + a.pix_per_block < P ? pbeg + a.pix_per_block : P;
    const int nk = (int)((pend - pbeg + BK - 1) / BK);
    auto load_stage = [&](int ks, int buf) {
        const long pb = pbeg + (long)ks * BK;
        // A: 32 pixels x 64 channels of dz = 256 chunks -> 2 per thread
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int idx = tid + q * 128;
            const int row = idx >> 3, ch = idx & 7;
            const long p = pb + row;
            const bool ok = p < pend && co0 + ch * 8 < a.cout;
            const __nv_bfloat16 *g = a.dz + (ok ? p : 0) * a.ld_dz + a.coff_dz + (ok ? co0 + ch * 8 : 0);
            cp_async16(&sA[buf][row * 72 + ch * 8], g, ok);
        }
        // B: 32 pixels x 32 channels of x at the tap shift = 128 chunks -> 1 per thread
        {
            const int row = tid >> 2, ch = tid & 3;
            const long p = pb + row;
            bool ok = p < pend;
            long src = 0;
            if (ok) {
                const int xq = (int)(p % a.wd);
                const int yq = (int)((p / a.wd) % a.h);
                ok = yq + dy >= 0 && yq + dy < a.h && xq + dx >= 0 && xq + dx < a.wd;
                src = p + (long)dy * a.wd + dx;
            }
            const __nv_bfloat16 *g = a.x + (ok ? src : 0) * a.ld_x + a.coff_x + ci0 + ch * 8;
            cp_async16(&sB[buf][row * 40 + ch * 8], g, ok);
        }
        cp_async_commit();
    };
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[j][k] = 0.f;
    if (nk > 0) load_stage(0, 0);
    for (int ks = 0; ks < nk; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < nk) {
            load_stage(ks + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            // A fragment (16 co x 16 p) from sA[p][co] by transposed loads
            uint32_t af[4];
            {
                const int prow = kk + (lane & 7) + ((lane >> 4) << 3);
                const int col = warp * 16 + ((lane >> 3) & 1) * 8;
                ldsm_x4_t(af[0], af[1], af[2], af[3], &sA[buf][prow * 72 + col]);
            }
            uint32_t bf[4][2];
#pragma unroll
            for (int nj = 0; nj < 4; nj += 2) {
                const int prow = kk + (lane & 7) + (((lane >> 3) & 1) << 3);
                const int col = nj * 8 + ((lane >> 4) << 3);
                ldsm_x4_t(bf[nj][0], bf[nj][1], bf[nj + 1][0], bf[nj + 1][1], &sB[buf][prow * 40 + col]);
            }
#pragma unroll
            for (int nj = 0; nj < 4; ++nj) mma16816(acc[nj], af, bf[nj][0], bf[nj][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int nj = 0; nj < 4; ++nj)
#pragma unroll
        for (int hrow = 0; hrow < 2; ++hrow) {
            const int co = co0 + warp * 16 + (lane >> 2) + hrow * 8;
            const int ci = ci0 + nj * 8 + (lane & 3) * 2;
            if (co >= a.cout) continue;
            float *d = a.dw + ((long)co * 9 + tap) * a.cin + ci;
            atomicAdd(d, acc[nj][hrow * 2 + 0]);
            atomicAdd(d + 1, acc[nj][hrow * 2 + 1]);
        }
}

}  // namespace cnn
}  // namespace oslalm
