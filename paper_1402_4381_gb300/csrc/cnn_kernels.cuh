// BF16 tensor-core kernels of the warm-start network (FP32 accumulation).
//
// Activations are NHWC BF16 with channel counts that are multiples of 32; a
// tensor may be a channel slice of a wider buffer (leading dimension `ld`,
// channel offset `coff`), which makes the U-Net's concatenations free.
//
// conv3x3_kernel: implicit GEMM  out[p][co] = sum_{tap, ci} in[p + shift(tap)][ci] w[co][tap][ci]
//   on the tcgen05 tensor cores: block tile 128 pixels x BN output channels
//   (BN = 32..256) accumulated in tensor memory, K step = one tap x 32 input
//   channels, double-buffered cp.async staging into the core-matrix layout,
//   MMAs issued by one thread and tracked by mbarriers.  With transposed,
//   tap-flipped weights the same kernel computes the data gradient.
// wgrad3x3_tc_kernel: dW[co][tap][ci] = sum_p dz[p][co] x[p + shift(tap)][ci]
//   on the tcgen05 tensor cores with both operands MN-major (pixel-major
//   activations staged as they are), split over pixel ranges, partial tiles
//   added with FP32 atomics.
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

// ---------------------------------------------------------------- tcgen05 (5th-generation tensor cores)
// Shared-memory operand tiles in the canonical K-major layout without
// swizzle: 8 x 8 "core matrices" of 8 rows x 16 bytes stored contiguously
// (128 bytes); the core matrices of one 8-row group follow each other along K
// (leading byte offset 128), the 8-row groups follow at the stride byte offset.
namespace tc {

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded: each try suspends for a bounded time, the loop ends in well under a second
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// tensor-memory columns for the accumulator (one warp; a power of two >= 32)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D[tmem] (+)= A[smem] x B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier completes once every MMA issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 8 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc

constexpr int kBM = 128, kBK = 32;  // pixels per block; input channels (one tap) per K step

// dynamic shared memory of conv3x3_kernel<BN>: two stages of A (128 x 32) and
// B (BN x 32) tiles, then two mbarriers and the tensor-memory address
__host__ __device__ constexpr int conv_smem_bytes(int bn) { return 2 * (kBM + bn) * kBK * 2 + 32; }

// One block: 128 pixels x BN output channels.  Every K step (one tap x 32 input
// channels) is staged by all threads with cp.async into the core-matrix
// layout (zero rows outside the image), then one thread issues two
// 128 x BN x 16 tcgen05 MMAs into the tensor-memory accumulator and commits
// them to the stage's mbarrier, which the stage's next loads wait for.  The
// epilogue reads the accumulator row by row (thread = pixel), adds the bias,
// applies ReLU and stores BF16.  err: set when a wait runs out (the block then
// stops issuing work, leaves its outputs unwritten and exits after a bounded
// wait for its own MMAs, instead of hanging).
template <int BN>
__global__ void __launch_bounds__(128) conv3x3_kernel(ConvArgs a, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2;
    unsigned char *sA = sm, *sB = sm + 2 * A_BYTES;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * (A_BYTES + B_BYTES));
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long P = (long)a.n * a.h * a.wd;
    const long p0 = (long)blockIdx.x * kBM;
    const int co0 = blockIdx.y * BN;
    const int csteps = a.cin / kBK;
    const int nk = 9 * csteps;
    if (warp == 0) tc::tmem_alloc(s_taddr, BN);
    if (tid < 2) tc::mbar_init(&bar[tid], 1);
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    auto load_stage = [&](int ks, int buf) {
        const int tap = ks / csteps, ci0 = (ks % csteps) * kBK;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        unsigned char *A = sA + buf * A_BYTES;
        unsigned char *B = sB + buf * B_BYTES;
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 128 rows x 4 chunks of 8 channels
            const int idx = tid + q * 128;
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
            cp_async16(A + (row >> 3) * 512 + ch * 128 + (row & 7) * 16, g, ok);
        }
#pragma unroll
        for (int q = 0; q < BN / 32; ++q) {  // BN rows x 4 chunks
            const int idx = tid + q * 128;
            const int row = idx >> 2, ch = idx & 3;
            const __nv_bfloat16 *g = a.w + ((long)(co0 + row) * 9 + tap) * a.cin + ci0 + ch * 8;
            cp_async16(B + (row >> 3) * 512 + ch * 128 + (row & 7) * 16, g, true);
        }
        cp_async_commit();
    };
    bool ok = true;
    int last = -1;  // last K step whose MMAs were committed
    load_stage(0, 0);
    for (int ks = 0; ks < nk; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < nk) {
            // stage buf ^ 1 was read by the MMAs of step ks - 1
            if (ks >= 1) ok = tc::mbar_wait(&bar[buf ^ 1], ((ks - 1) >> 1) & 1);
            // one decision for the whole block: after a wait that ran out, no
            // thread may overwrite a stage the tensor cores could still read
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            load_stage(ks + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        tc::fence_proxy_async();  // this thread's staged tiles -> visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const unsigned char *A = sA + buf * A_BYTES, *B = sB + buf * B_BYTES;
#pragma unroll
            for (int kh = 0; kh < kBK / 16; ++kh)
                tc::mma_bf16(taddr, tc::smem_desc(A + kh * 256, 128, 512), tc::smem_desc(B + kh * 256, 128, 512),
                             tc::idesc_bf16(kBM, BN), (ks > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&bar[buf]);
        }
        last = ks;
    }
    if (ok) ok = tc::mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1);
    if (!__syncthreads_and(ok)) {
        // A wait ran out: flag the network, skip the epilogue, let the copies
        // in flight land, give the MMAs committed so far one more bounded wait
        // (their last commit), then release the tensor memory and return.
        // The total wait of the block is bounded by three wait limits.
        if (tid == 0) atomicOr(err, 1);
        cp_async_wait<0>();
        if (last >= 0) tc::mbar_wait(&bar[last & 1], (last >> 1) & 1);
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, BN);
        return;
    }
    tc::fence_after_sync();
    const long p = p0 + warp * 32 + lane;  // this thread's accumulator row (tensor-memory lane)
#pragma unroll 1
    for (int c = 0; c < BN; c += 8) {
        float v[8];
        tc::tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        if (p < P) {
            const int co = co0 + c;
            __align__(16) __nv_bfloat162 o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v0 = v[2 * i], v1 = v[2 * i + 1];
                if (a.bias) {
                    v0 += a.bias[co + 2 * i];
                    v1 += a.bias[co + 2 * i + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                o[i] = __floats2bfloat162_rn(v0, v1);
            }
            *reinterpret_cast<uint4 *>(a.out + p * a.ld_out + a.coff_out + co) = *reinterpret_cast<const uint4 *>(o);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, BN);
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

// Weight gradient on the tcgen05 tensor cores: for one tap and a slice of
// 128 output channels (M, padded with zero rows) x BN input channels (N), a
// block adds up dW[co][tap][ci] = sum_p dz[p][co] x[p + shift][ci] over a pixel
// range (K) into a tensor-memory accumulator, then adds it to dw with FP32
// atomics.  Both operands are stored pixel-major (channels contiguous), which
// is the MN-major canonical layout without swizzle: a core matrix is 8 pixels
// (K) x 16 bytes (8 channels, MN) = 128 contiguous bytes, so every 16-byte
// chunk (8 channels of one pixel) is staged by cp.async straight into place:
// K groups of 8 pixels 128 bytes apart (leading byte offset), MN groups of 8
// channels 512 bytes apart (stride byte offset), 32 pixels per stage.  The
// instruction descriptor marks A and B as MN-major.  Waits are bounded as in
// conv3x3_kernel.
__host__ __device__ constexpr int wgrad_tc_smem_bytes(int bn) { return 2 * (128 + bn) * 32 * 2 + 32; }

template <int BN>
__global__ void __launch_bounds__(128) wgrad3x3_tc_kernel(WgradArgs a, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int BM = 128, BK = 32;
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    unsigned char *sA = sm, *sB = sm + 2 * A_BYTES;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * (A_BYTES + B_BYTES));
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long P = (long)a.n * a.h * a.wd;
    const int co0 = blockIdx.x * BM;
    const int tap = blockIdx.y / (a.cin / BN);
    const int ci0 = (blockIdx.y % (a.cin / BN)) * BN;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long pbeg = (long)blockIdx.z * a.pix_per_block;
    const long pend = pbeg + a.pix_per_block < P ? pbeg + a.pix_per_block : P;
    const int nk = (int)((pend - pbeg + BK - 1) / BK);
    if (warp == 0) tc::tmem_alloc(s_taddr, BN);
    if (tid < 2) tc::mbar_init(&bar[tid], 1);
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    auto load_stage = [&](int ks, int buf) {
        const long pb = pbeg + (long)ks * BK;
        unsigned char *A = sA + buf * A_BYTES;
        unsigned char *B = sB + buf * B_BYTES;
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // A: 32 pixels x 16 groups of 8 output channels
            const int idx = tid + q * 128;
            const int px = idx >> 4, cg = idx & 15;
            const long p = pb + px;
            const bool ok = p < pend && co0 + cg * 8 < a.cout;
            const __nv_bfloat16 *g = a.dz + (ok ? p : 0) * a.ld_dz + a.coff_dz + (ok ? co0 + cg * 8 : 0);
            cp_async16(A + cg * 512 + (px >> 3) * 128 + (px & 7) * 16, g, ok);
        }
#pragma unroll
        for (int q = 0; q < BN / 32; ++q) {  // B: 32 pixels x BN/8 groups of 8 input channels
            const int idx = tid + q * 128;
            const int px = idx / (BN / 8), cg = idx % (BN / 8);
            const long p = pb + px;
            bool ok = p < pend;
            long src = 0;
            if (ok) {
                const int xq = (int)(p % a.wd);
                const int yq = (int)((p / a.wd) % a.h);
                ok = yq + dy >= 0 && yq + dy < a.h && xq + dx >= 0 && xq + dx < a.wd;
                src = p + (long)dy * a.wd + dx;
            }
            const __nv_bfloat16 *g = a.x + (ok ? src : 0) * a.ld_x + a.coff_x + ci0 + cg * 8;
            cp_async16(B + cg * 512 + (px >> 3) * 128 + (px & 7) * 16, g, ok);
        }
        cp_async_commit();
    };
    constexpr uint32_t idesc = tc::idesc_bf16(BM, BN) | (1u << 15) | (1u << 16);  // A and B MN-major
    bool ok = true;
    int last = -1;  // last K step whose MMAs were committed
    if (nk > 0) load_stage(0, 0);
    for (int ks = 0; ks < nk; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < nk) {
            if (ks >= 1) ok = tc::mbar_wait(&bar[buf ^ 1], ((ks - 1) >> 1) & 1);
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            load_stage(ks + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const unsigned char *A = sA + buf * A_BYTES, *B = sB + buf * B_BYTES;
#pragma unroll
            for (int kh = 0; kh < BK / 16; ++kh)  // 16 pixels (two K groups) per MMA
                tc::mma_bf16(taddr, tc::smem_desc(A + kh * 256, 128, 512), tc::smem_desc(B + kh * 256, 128, 512),
                             idesc, (ks > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&bar[buf]);
        }
        last = ks;
    }
    if (ok && nk > 0) ok = tc::mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1);
    if (!__syncthreads_and(ok)) {
        // a wait ran out: flag, let the copies land, one more bounded wait for
        // the committed MMAs, release the tensor memory, add nothing
        if (tid == 0) atomicOr(err, 1);
        cp_async_wait<0>();
        if (last >= 0) tc::mbar_wait(&bar[last & 1], (last >> 1) & 1);
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, BN);
        return;
    }
    tc::fence_after_sync();
    if (nk > 0) {
        const int co = co0 + warp * 32 + lane;  // this thread's accumulator row (tensor-memory lane)
#pragma unroll 1
        for (int c = 0; c < BN; c += 8) {
            float v[8];
            tc::tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (co < a.cout) {
                float *d = a.dw + ((long)co * 9 + tap) * a.cin + ci0 + c;
#pragma unroll
                for (int i = 0; i < 8; ++i) atomicAdd(d + i, v[i]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, BN);
}

}  // namespace cnn
}  // namespace oslalm
