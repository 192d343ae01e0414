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
// conv3x3_tma_kernel / conv3x3_halo_kernel: the same with the tiles brought
//   in by TMA as 64-byte swizzled rows (whole-row blocks); the halo form loads
//   each input row once with a one-pixel halo for its three horizontal taps.
//   All three take the K steps in one order (tap row, channel step, tap
//   column), so they give the same bits.
// wgrad3x3_tc_kernel: dW[co][tap][ci] = sum_p dz[p][co] x[p + shift(tap)][ci]
//   on the tcgen05 tensor cores with both operands MN-major (pixel-major
//   activations staged as they are), split over pixel ranges, partial tiles
//   added with FP32 atomics.
// wgrad3x3_tma_kernel / wgrad3x3_halo_kernel: the same by TMA; the halo form
//   computes the three horizontal taps of a tap row per block, with dz and a
//   66-pixel input row loaded once and three tensor-memory accumulators.
#pragma once

#include <cuda.h>
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
// the same, but a thread whose phase is not complete sleeps until it completes
// or for at most `ns` nanoseconds, instead of coming back at once
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, unsigned parity, unsigned ns) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: false after half a second of the global timer (or 2^24 tries,
// should the timer not advance), so a block can never hang on a phase that
// does not complete; waiting threads sleep rather than spin, leaving the
// issue slots to the other blocks on the SM
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < (1 << 24); ++i) {
        if (mbar_try_wait_sleep(bar, parity, 2000)) return true;
        if (global_ns() - t0 > 500000000ull) return false;
    }
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
// descriptor of a K-major tile in the 64-byte swizzled layout (rows of 32
// BF16 = 64 bytes, 8-row atoms of 512 bytes, 16-byte chunks exchanged by
// the TMA's 64-byte swizzle): stride byte offset 512 between 8-row groups,
// leading byte offset unused (16), layout type 4 (64-byte swizzle); a K step
// of 16 elements inside the row advances the start address by 32 bytes
__device__ __forceinline__ uint64_t smem_desc_sw64(const void *p) {
    return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46) | (4ull << 61);
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

// Epilogue of a 128-pixel x BN tile: thread = pixel (tensor-memory lane),
// bias, ReLU, BF16 stores of 8 channels at a time.
template <int BN>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, uint32_t taddr, long p0, int co0, long P) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
}

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
    const int tid = threadIdx.x, warp = tid >> 5;
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
    // this thread's 4 pixel rows (row = tid / 4 + 32 q, chunk tid % 4) are the
    // same in every K step: their image coordinates are found once
    const int ch = tid & 3;
    int px[4], py[4];
    const __nv_bfloat16 *pin[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long p = p0 + (tid >> 2) + 32 * q;
        const bool in = p < P;
        px[q] = in ? (int)(p % a.wd) : -4;  // -4: outside the image for every tap
        py[q] = in ? (int)((p / a.wd) % a.h) : 0;
        pin[q] = a.in + (in ? p : 0) * a.ld_in + a.coff_in + ch * 8;
    }
    auto load_stage = [&](int ks, int buf) {
        // K order: tap row dy, then channel step, then dx (the order of the
        // halo kernel, which reads a row's three taps from one load)
        const int dyi = ks / (3 * csteps), rem = ks - dyi * 3 * csteps;
        const int cs = rem / 3, tap = dyi * 3 + (rem - cs * 3), ci0 = cs * kBK;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const long shift = ((long)dy * a.wd + dx) * a.ld_in + ci0;
        unsigned char *A = sA + buf * A_BYTES;
        unsigned char *B = sB + buf * B_BYTES;
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 128 rows x 4 chunks of 8 channels
            const int row = (tid >> 2) + 32 * q;
            const bool ok = (unsigned)(py[q] + dy) < (unsigned)a.h && (unsigned)(px[q] + dx) < (unsigned)a.wd;
            cp_async16(A + (row >> 3) * 512 + ch * 128 + (row & 7) * 16, ok ? pin[q] + shift : a.in, ok);
        }
#pragma unroll
        for (int q = 0; q < BN / 32; ++q) {  // BN rows x 4 chunks
            const int idx = tid + q * 128;
            const int row = idx >> 2, cb = idx & 3;
            const __nv_bfloat16 *g = a.w + ((long)(co0 + row) * 9 + tap) * a.cin + ci0 + cb * 8;
            cp_async16(B + (row >> 3) * 512 + cb * 128 + (row & 7) * 16, g, true);
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
    conv_epilogue<BN>(a, taddr, p0, co0, P);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, BN);
}

// ---------------------------------------------------------------- TMA (tensor memory accelerator)
namespace tma {
__device__ __forceinline__ void prefetch_map(const CUtensorMap *m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}
// one arrival on `bar` that also expects `bytes` of TMA transfers in this phase
__device__ __forceinline__ void arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// box of a rank-4 / rank-2 tensor map at the given element coordinates (the
// innermost first) into shared memory; elements outside the tensor read as zero
__device__ __forceinline__ void load_4d(void *dst, const CUtensorMap *m, int c0, int c1, int c2, int c3,
                                        uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *m, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
}  // namespace tma

constexpr int kConvTmaStages = 4;
// barriers + tensor-memory address in the first 1 KB, then the stages (1 KB
// aligned for the swizzle): A (128 pixels x 32 channels) and B (BN output
// channels x 32 channels), 64 bytes per row
__host__ __device__ constexpr int conv_tma_smem_bytes(int bn) { return 1024 + kConvTmaStages * (kBM + bn) * kBK * 2; }

// The convolution with its operand tiles brought in by TMA, for images whose
// 128-pixel blocks are whole rows or row segments (width a multiple of 128,
// or 128 / width rows with the height a multiple of that).  The activations
// are a rank-4 tensor map (channel, column, row, image) over the input
// slice: the tile of tap (dy, dx) is the box of 32 channels x bw columns x
// bh rows at (ci, x0 + dx, y0 + dy, image), and the map's zero fill outside
// the image is the convolution's zero padding.  Each box lands as 128 rows
// (pixels) of 64 bytes in the 64-byte swizzled K-major layout, which the MMA
// descriptors read directly; the weights [cout][9 cin] are a rank-2 map read
// the same way.  One thread runs the whole loop: it keeps all four stages in
// flight, waits for a stage's bytes on its `full` mbarrier, issues the two
// MMAs, commits them to the stage's `empty` mbarrier and refills the stage
// used one step earlier once those MMAs are done.  The other threads wait
// for the epilogue.  Waits are bounded; after one runs out the block lets its
// transfers land and its MMAs finish (bounded), flags err, releases the
// tensor memory and returns.
template <int BN>
__global__ void __launch_bounds__(128) conv3x3_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, ConvArgs a,
                                                          int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int NS = kConvTmaStages;
    constexpr int A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2, S_BYTES = A_BYTES + B_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);
    uint64_t *empty = full + NS;
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(empty + NS);
    unsigned char *stages = sm + 1024;
    const int tid = threadIdx.x, warp = tid >> 5;
    // the swizzled tiles need 1 KB aligned buffers: if the runtime ever placed
    // the dynamic shared memory otherwise, flag and stop before any transfer
    if (smem_u32(stages) & 1023u) {
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    const long P = (long)a.n * a.h * a.wd;
    const long p0 = (long)blockIdx.x * kBM;
    const int co0 = blockIdx.y * BN;
    const int csteps = a.cin / kBK;
    const int nk = 9 * csteps;
    if (warp == 0) tc::tmem_alloc(s_taddr, BN);
    if (tid < 2 * NS) tc::mbar_init(&full[tid], 1);  // full[0..NS) and empty[0..NS)
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    bool ok = true;
    if (tid == 0) {
        tma::prefetch_map(&tmA);
        tma::prefetch_map(&tmB);
        const long hw = (long)a.h * a.wd;
        const int img = (int)(p0 / hw);
        const int rem = (int)(p0 - (long)img * hw);
        const int y0 = rem / a.wd, x0 = rem - (rem / a.wd) * a.wd;
        int issued = 0, done = 0;
        // K order: tap row dy, then channel step, then dx (as in conv3x3_kernel)
        int dy_i = 0, cs_i = 0, dx_i = 0;  // of the next stage to issue
        auto issue = [&]() {
            const int s = issued++;
            unsigned char *A = stages + (s % NS) * S_BYTES, *B = A + A_BYTES;
            uint64_t *fb = &full[s % NS];
            const int tap = dy_i * 3 + dx_i, dy = dy_i - 1, dx = dx_i - 1, ci0 = cs_i * kBK;
            tma::arrive_expect_tx(fb, (uint32_t)S_BYTES);
            tma::load_4d(A, &tmA, ci0, x0 + dx, y0 + dy, img, fb);
            tma::load_2d(B, &tmB, tap * a.cin + ci0, co0, fb);
            if (++dx_i == 3) {
                dx_i = 0;
                if (++cs_i == csteps) {
                    cs_i = 0;
                    ++dy_i;
                }
            }
        };
        while (issued < NS && issued < nk) issue();
        for (int ks = 0; ks < nk; ++ks) {
            const int buf = ks % NS;
            if (!tc::mbar_wait(&full[buf], (ks / NS) & 1)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const unsigned char *A = stages + buf * S_BYTES, *B = A + A_BYTES;
#pragma unroll
            for (int kh = 0; kh < kBK / 16; ++kh)  // 16 channels (32 bytes of the row) per MMA
                tc::mma_bf16(taddr, tc::smem_desc_sw64(A + kh * 32), tc::smem_desc_sw64(B + kh * 32),
                             tc::idesc_bf16(kBM, BN), (ks > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&empty[buf]);
            done = ks + 1;
            // refill the stage of step ks - 1: its MMAs precede this step's in
            // the tensor pipe, so they are normally done
            if (ks >= 1 && issued < nk) {
                if (!tc::mbar_wait(&empty[(ks - 1) % NS], ((ks - 1) / NS) & 1)) {
                    ok = false;
                    break;
                }
                issue();
            }
        }
        if (ok && nk > 0) ok = tc::mbar_wait(&empty[(nk - 1) % NS], ((nk - 1) / NS) & 1);
        if (!ok) {
            // let the issued transfers land and the committed MMAs finish
            // (each wait bounded) before the block's memory is released
            atomicOr(err, 1);
            for (int s = done; s < issued; ++s) tc::mbar_wait(&full[s % NS], (s / NS) & 1);
            if (done > 0) tc::mbar_wait(&empty[(done - 1) % NS], ((done - 1) / NS) & 1);
        }
    }
    if (!__syncthreads_and(ok)) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, BN);
        return;
    }
    tc::fence_after_sync();
    conv_epilogue<BN>(a, taddr, p0, co0, P);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, BN);
}

// The convolution on a level whose width is a multiple of 128, with each
// input row read once for its three horizontal taps.  A stage is one tap row
// dy and one 32-channel step: the box of 32 channels x 130 pixels x 1 row at
// (ci, x0 - 1, y0 + dy, image) (the map's zero fill is the padding at both
// ends) lands as 130 rows of 64 bytes in the 64-byte swizzle, and the MMAs of
// taps dx = -1, 0, +1 read it from 0, 64 and 128 bytes on (one pixel per 64
// bytes; the tensor cores apply the swizzle from the shared-memory address,
// as the TMA wrote it), with the stage's three weight tiles.  Three stages in
// flight, refilled as in conv3x3_tma_kernel; the MMAs run in the K order of
// the other convolution kernels (dy, channel step, dx), so the results are
// the same bits.
constexpr int kHaloSlot = 9216;  // 130 x 64 bytes, rounded up to 1 KB
constexpr int kHaloStages = 3;
__host__ __device__ constexpr int conv_halo_smem_bytes(int bn) {
    return 1024 + kHaloStages * (kHaloSlot + 3 * bn * 64);
}

template <int BN>
__global__ void __launch_bounds__(128) conv3x3_halo_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, ConvArgs a,
                                                           int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int NS = kHaloStages, B_TAP = BN * 64, S_BYTES = kHaloSlot + 3 * B_TAP;
    constexpr uint32_t TX = 130 * 64 + 3 * B_TAP;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);
    uint64_t *empty = full + NS;
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(empty + NS);
    unsigned char *stages = sm + 1024;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (smem_u32(stages) & 1023u) {  // the swizzled rows need 1 KB aligned buffers
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    const long P = (long)a.n * a.h * a.wd;
    const long p0 = (long)blockIdx.x * kBM;
    const int co0 = blockIdx.y * BN;
    const int csteps = a.cin / kBK;
    const int nk = 3 * csteps;
    if (warp == 0) tc::tmem_alloc(s_taddr, BN);
    if (tid < 2 * NS) tc::mbar_init(&full[tid], 1);  // full[0..NS) and empty[0..NS)
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    bool ok = true;
    if (tid == 0) {
        tma::prefetch_map(&tmA);
        tma::prefetch_map(&tmB);
        const long hw = (long)a.h * a.wd;
        const int img = (int)(p0 / hw);
        const int rem = (int)(p0 - (long)img * hw);
        const int y0 = rem / a.wd, x0 = rem - (rem / a.wd) * a.wd;
        int issued = 0, done = 0;
        int dy_i = 0, cs_i = 0;  // tap row and channel step of the next stage to issue
        auto issue = [&]() {
            const int s = issued++;
            unsigned char *A = stages + (s % NS) * S_BYTES, *B = A + kHaloSlot;
            uint64_t *fb = &full[s % NS];
            const int ci0 = cs_i * kBK;
            tma::arrive_expect_tx(fb, TX);
            tma::load_4d(A, &tmA, ci0, x0 - 1, y0 + dy_i - 1, img, fb);
#pragma unroll
            for (int d = 0; d < 3; ++d) tma::load_2d(B + d * B_TAP, &tmB, (3 * dy_i + d) * a.cin + ci0, co0, fb);
            if (++cs_i == csteps) {
                cs_i = 0;
                ++dy_i;
            }
        };
        while (issued < NS && issued < nk) issue();
        for (int ks = 0; ks < nk; ++ks) {
            const int buf = ks % NS;
            if (!tc::mbar_wait(&full[buf], (ks / NS) & 1)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const unsigned char *A = stages + buf * S_BYTES, *B = A + kHaloSlot;
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int kh = 0; kh < kBK / 16; ++kh)
                    tc::mma_bf16(taddr, tc::smem_desc_sw64(A + d * 64 + kh * 32),
                                 tc::smem_desc_sw64(B + d * B_TAP + kh * 32), tc::idesc_bf16(kBM, BN),
                                 (ks > 0 || d > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&empty[buf]);
            done = ks + 1;
            // refill the stage of step ks - 1: its MMAs precede this step's
            if (ks >= 1 && issued < nk) {
                if (!tc::mbar_wait(&empty[(ks - 1) % NS], ((ks - 1) / NS) & 1)) {
                    ok = false;
                    break;
                }
                issue();
            }
        }
        if (ok && nk > 0) ok = tc::mbar_wait(&empty[(nk - 1) % NS], ((nk - 1) / NS) & 1);
        if (!ok) {
            // let the issued transfers land and the committed MMAs finish
            // (each wait bounded) before the block's memory is released
            atomicOr(err, 1);
            for (int s = done; s < issued; ++s) tc::mbar_wait(&full[s % NS], (s / NS) & 1);
            if (done > 0) tc::mbar_wait(&empty[(done - 1) % NS], ((done - 1) / NS) & 1);
        }
    }
    if (!__syncthreads_and(ok)) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, BN);
        return;
    }
    tc::fence_after_sync();
    conv_epilogue<BN>(a, taddr, p0, co0, P);
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

// Weight gradient on the tcgen05 tensor cores: for one tap and a slice of
// 128 output channels (M) x BN input channels (N), a block adds up
// dW[co][tap][ci] = sum_p dz[p][co] x[p + shift][ci] over a pixel range (K)
// into a tensor-memory accumulator, then adds it to dw with FP32 atomics.
// Both operands are stored pixel-major (channels contiguous), which is the
// MN-major canonical layout without swizzle: a core matrix is 8 pixels (K) x
// 16 bytes (8 channels, MN) = 128 contiguous bytes, so every 16-byte chunk (8
// channels of one pixel) is staged by cp.async straight into place.  Within
// a group of 8 channels the 64 pixels of a stage are contiguous (K groups 128
// bytes apart: the leading byte offset); the groups are 1024 bytes apart (the
// stride byte offset).  The instruction descriptor marks A and B as MN-major.
//
// Only the GA = min(16, cout / 8) channel groups of dz that exist are staged
// (4 for 32 output channels): the MMA's other A rows read whatever lies
// beyond the stage (later stages, the B tiles, a pad at the end of shared
// memory) and only make accumulator rows that are never stored, so the small
// layers take a quarter of the shared memory and fit more blocks per SM.
// Every thread stages the same channel group of fixed pixels of each stage,
// so its source pointers advance by constants; which of a stage's 64 pixels
// exist (ragged tail) and have the tap's neighbour inside the image is one
// 64-bit mask per stage, built by every warp with two ballots.  The loads run
// NS - 2 stages ahead of the MMAs and refill the buffer whose MMAs were
// issued two steps before; one block barrier per step, which also carries
// the decision after a wait that ran out (waits are bounded as in
// conv3x3_kernel).
constexpr int kWgBK = 64;  // pixels per stage
__host__ __device__ constexpr int wgrad_groups(int cout) { return cout / 8 < 16 ? cout / 8 : 16; }
__host__ __device__ constexpr int wgrad_b_bytes(int bn) { return bn * kWgBK * 2; }
__host__ __device__ constexpr int wgrad_stage_bytes(int bn, int ga) { return ga * kWgBK * 16 + wgrad_b_bytes(bn); }
// stages: 6 when six fit in 100 KB of shared memory (two or more blocks per SM), else 4
__host__ __device__ constexpr int wgrad_stages(int bn, int ga) { return 6 * wgrad_stage_bytes(bn, ga) <= 100 * 1024 ? 6 : 4; }
// mbarriers and the tensor-memory address (128 bytes), the stages, then the
// pad that the last A stage's unstaged rows may reach into
__host__ __device__ constexpr int wgrad_tc_smem_bytes(int bn, int ga) {
    return 128 + wgrad_stages(bn, ga) * wgrad_stage_bytes(bn, ga) +
           ((16 - ga) * kWgBK * 16 > wgrad_stages(bn, ga) * wgrad_b_bytes(bn)
                ? (16 - ga) * kWgBK * 16 - wgrad_stages(bn, ga) * wgrad_b_bytes(bn)
                : 0);
}

template <int BN, int GA>
__global__ void __launch_bounds__(128) wgrad3x3_tc_kernel(WgradArgs a, int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int BM = 128, BK = kWgBK, NS = wgrad_stages(BN, GA);
    constexpr int A_BYTES = GA * BK * 16, B_BYTES = wgrad_b_bytes(BN);
    constexpr int BG = BN / 8;             // channel groups of x
    constexpr int QA = GA * BK / 128;      // A chunks per thread and stage
    constexpr int QB = BG * BK / 128;      // B chunks per thread and stage
    static_assert(GA >= 2 && GA <= 16 && 128 % GA == 0 && 128 % BG == 0, "channel groups");
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(sm + 8 * NS);
    unsigned char *sA = sm + 128, *sB = sA + NS * A_BYTES;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long P = (long)a.n * a.h * a.wd;
    const int co0 = blockIdx.x * BM;
    const int tap = blockIdx.y / (a.cin / BN);
    const int ci0 = (blockIdx.y % (a.cin / BN)) * BN;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long pbeg = (long)blockIdx.z * a.pix_per_block;
    const long pend = pbeg + a.pix_per_block < P ? pbeg + a.pix_per_block : P;
    const int nk = pend > pbeg ? (int)((pend - pbeg + BK - 1) / BK) : 0;
    if (warp == 0) tc::tmem_alloc(s_taddr, BN);
    if (tid < NS) tc::mbar_init(&bar[tid], 1);
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    // A: this thread stages group tid % GA of pixels tid / GA + q 128 / GA;
    // B: group tid % BG of pixels tid / BG + q 128 / BG (consecutive threads
    // read consecutive 16 bytes of a pixel's channels)
    const int cga = tid % GA, pxa = tid / GA, cgb = tid % BG, pxb = tid / BG;
    const bool a_real = co0 + cga * 8 < a.cout;  // channel group inside dz
    const long stepA = (long)(128 / GA) * a.ld_dz, stepB = (long)(128 / BG) * a.ld_x;
    const __nv_bfloat16 *srcA = a.dz + (pbeg + pxa) * a.ld_dz + a.coff_dz + co0 + cga * 8;
    const __nv_bfloat16 *srcB = a.x + (pbeg + pxb + (long)dy * a.wd + dx) * a.ld_x + a.coff_x + ci0 + cgb * 8;
    const uint32_t dstA = smem_u32(sA) + cga * (BK * 16) + pxa * 16;
    const uint32_t dstB = smem_u32(sB) + cgb * (BK * 16) + pxb * 16;
    // image coordinates (column, row) of the first pixel of the next stage to load
    int sx = (int)(pbeg % a.wd), sy = (int)((pbeg / a.wd) % a.h);
    auto load_stage = [&](int ks, int buf) {
        const long pb = pbeg + (long)ks * BK;
        // bit i: pixel pb + i exists (tail) / and its tap neighbour is in the image
        bool e0, e1, v0, v1;
        {
            const int i0 = lane, i1 = lane + 32;
            e0 = pb + i0 < pend;
            e1 = pb + i1 < pend;
            int x = sx + i0, y = sy;
            while (x >= a.wd) {
                x -= a.wd;
                ++y;
            }
            while (y >= a.h) y -= a.h;
            v0 = e0 && (unsigned)(y + dy) < (unsigned)a.h && (unsigned)(x + dx) < (unsigned)a.wd;
            x = sx + i1;
            y = sy;
            while (x >= a.wd) {
                x -= a.wd;
                ++y;
            }
            while (y >= a.h) y -= a.h;
            v1 = e1 && (unsigned)(y + dy) < (unsigned)a.h && (unsigned)(x + dx) < (unsigned)a.wd;
        }
        const uint64_t em = (uint64_t)__ballot_sync(0xffffffffu, e0) | ((uint64_t)__ballot_sync(0xffffffffu, e1) << 32);
        const uint64_t vm = (uint64_t)__ballot_sync(0xffffffffu, v0) | ((uint64_t)__ballot_sync(0xffffffffu, v1) << 32);
        const long off = (long)ks * BK;
        const __nv_bfloat16 *gA = srcA + off * a.ld_dz;
        const __nv_bfloat16 *gB = srcB + off * a.ld_x;
#pragma unroll
        for (int q = 0; q < QA; ++q) {
            const bool ok = a_real && ((em >> (pxa + q * (128 / GA))) & 1);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dstA + buf * A_BYTES +
                                                                              q * (128 / GA) * 16),
                         "l"(ok ? gA + q * stepA : a.dz), "r"(ok ? 16 : 0));
        }
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            const bool ok = (vm >> (pxb + q * (128 / BG))) & 1;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dstB + buf * B_BYTES +
                                                                              q * (128 / BG) * 16),
                         "l"(ok ? gB + q * stepB : a.x), "r"(ok ? 16 : 0));
        }
        cp_async_commit();
        sx += BK;
        while (sx >= a.wd) {
            sx -= a.wd;
            ++sy;
        }
        while (sy >= a.h) sy -= a.h;
    };
    constexpr uint32_t idesc = tc::idesc_bf16(BM, BN) | (1u << 15) | (1u << 16);  // A and B MN-major
    // stage ks lives in buffer ks % NS; the n-th use of a buffer (n = ks / NS)
    // completes its mbarrier's phase n, of parity n & 1
    bool ok = true;
    int last = -1;  // last K step whose MMAs were committed
    for (int s = 0; s < NS - 2; ++s) {  // prologue: NS - 2 stages in flight (empty groups past the end)
        if (s < nk) load_stage(s, s);
        else cp_async_commit();
    }
    for (int ks = 0; ks < nk; ++ks) {
        const int buf = ks % NS;
        cp_async_wait<NS - 3>();  // stage ks has landed (this thread's copies)
        tc::fence_proxy_async();
        // one decision for the whole block: after a wait that ran out, no
        // thread issues MMAs or overwrites a stage the tensor cores could read
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            tc::fence_after_sync();
            const unsigned char *A = sA + buf * A_BYTES, *B = sB + buf * B_BYTES;
#pragma unroll
            for (int kh = 0; kh < BK / 16; ++kh)  // 16 pixels (two K groups) per MMA
                tc::mma_bf16(taddr, tc::smem_desc(A + kh * 256, 128, BK * 16),
                             tc::smem_desc(B + kh * 256, 128, BK * 16), idesc, (ks > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&bar[buf]);
        }
        last = ks;
        // refill the buffer of stage ks - 2 with stage ks + NS - 2 once its MMAs
        // are done (issued two steps earlier, so the wait is normally over)
        const int nxt = ks + NS - 2;
        if (nxt < nk && ks >= 2) ok = tc::mbar_wait(&bar[(ks - 2) % NS], ((ks - 2) / NS) & 1);
        if (nxt < nk && ok) load_stage(nxt, nxt % NS);
        else cp_async_commit();  // keep one group per step for the wait count
    }
    if (ok && nk > 0) ok = tc::mbar_wait(&bar[(nk - 1) % NS], ((nk - 1) / NS) & 1);
    if (!__syncthreads_and(ok)) {
        // a wait ran out: flag, let the copies land, one more bounded wait for
        // the committed MMAs, release the tensor memory, add nothing
        if (tid == 0) atomicOr(err, 1);
        cp_async_wait<0>();
        if (last >= 0) tc::mbar_wait(&bar[last % NS], (last / NS) & 1);
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, BN);
        return;
    }
    tc::fence_after_sync();
    if (nk > 0 && co0 + warp * 32 < a.cout) {  // warps whose rows are all padding skip the epilogue
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

// ---------------------------------------------------------------- weight gradient by TMA
// descriptor of an MN-major tile in the 64-byte swizzled layout: rows are K
// (pixels) of 64 bytes = 32 channels of MN, 8-row groups 512 bytes apart
// (stride byte offset), 32-channel atoms `lbo` bytes apart (leading byte
// offset), layout type 4 (64-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc_mn_sw64(const void *p, uint32_t lbo) {
    return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

constexpr int kWgTmaStages = 4;
constexpr int kWgTmaAtom = kWgBK * 64;  // one 32-channel atom of a stage: 64 pixels x 64 bytes
// barriers (1 KB), the stages (ga32 atoms of dz, bn / 32 atoms of x each),
// then a pad of 4 atoms that the unstaged A rows of the last stage may reach
__host__ __device__ constexpr int wgrad_tma_smem_bytes(int bn, int ga32) {
    return 1024 + kWgTmaStages * (ga32 + bn / 32) * kWgTmaAtom + 4 * kWgTmaAtom;
}

// The weight gradient with both operands brought in by TMA, for images whose
// 64-pixel stages are row segments or whole rows (width a multiple of 64, or
// 64 / width rows with the height a multiple of that): dz as a rank-2 map
// (channel, pixel) with boxes of 32 channels x 64 pixels, x as a rank-4 map
// (channel, column, row, image) with boxes of 32 channels x bw x bh at the
// tap's shift, whose zero fill outside the image drops the pixels the tap
// does not reach.  Each box is 64 rows (pixels, K) of 64 bytes (32 channels,
// MN) in the 64-byte swizzle, which the MMA reads as an MN-major operand.
// GA32 = min(4, cout / 32) atoms of dz are staged; as in wgrad3x3_tc_kernel
// the other A rows read past the stage and only make accumulator rows that
// are never stored.  One thread runs the loop over the block's stages (four
// in flight, full / empty mbarriers, bounded waits), as in
// conv3x3_tma_kernel; the epilogue adds the accumulator to dw with atomics.
template <int BN, int GA32>
__global__ void __launch_bounds__(128) wgrad3x3_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, WgradArgs a,
                                                           int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int NS = kWgTmaStages, BM = 128, BK = kWgBK;
    constexpr int A_BYTES = GA32 * kWgTmaAtom, B_BYTES = (BN / 32) * kWgTmaAtom, S_BYTES = A_BYTES + B_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);
    uint64_t *empty = full + NS;
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(empty + NS);
    unsigned char *stages = sm + 1024;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (smem_u32(stages) & 1023u) {  // the swizzle needs 1 KB aligned buffers
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    const long P = (long)a.n * a.h * a.wd;
    const int co0 = blockIdx.x * BM;
    const int tap = blockIdx.y / (a.cin / BN);
    const int ci0 = (blockIdx.y % (a.cin / BN)) * BN;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long pbeg = (long)blockIdx.z * a.pix_per_block;
    const long pend = pbeg + a.pix_per_block < P ? pbeg + a.pix_per_block : P;
    const int nk = pend > pbeg ? (int)((pend - pbeg) / BK) : 0;  // whole stages (P, pix_per_block: multiples of 64)
    if (warp == 0) tc::tmem_alloc(s_taddr, BN);
    if (tid < 2 * NS) tc::mbar_init(&full[tid], 1);
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    bool ok = true;
    if (tid == 0) {
        tma::prefetch_map(&tmA);
        tma::prefetch_map(&tmB);
        const long hw = (long)a.h * a.wd;
        int issued = 0, done = 0;
        auto issue = [&]() {
            const int s = issued++;
            const long pb = pbeg + (long)s * BK;
            const int img = (int)(pb / hw);
            const int rem = (int)(pb - (long)img * hw);
            const int y0 = rem / a.wd, x0 = rem - (rem / a.wd) * a.wd;
            unsigned char *A = stages + (s % NS) * S_BYTES, *B = A + A_BYTES;
            uint64_t *fb = &full[s % NS];
            tma::arrive_expect_tx(fb, (uint32_t)S_BYTES);
#pragma unroll
            for (int g = 0; g < GA32; ++g) tma::load_2d(A + g * kWgTmaAtom, &tmA, co0 + 32 * g, (int)pb, fb);
#pragma unroll
            for (int g = 0; g < BN / 32; ++g)
                tma::load_4d(B + g * kWgTmaAtom, &tmB, ci0 + 32 * g, x0 + dx, y0 + dy, img, fb);
        };
        while (issued < NS && issued < nk) issue();
        constexpr uint32_t idesc = tc::idesc_bf16(BM, BN) | (1u << 15) | (1u << 16);  // A and B MN-major
        for (int ks = 0; ks < nk; ++ks) {
            const int buf = ks % NS;
            if (!tc::mbar_wait(&full[buf], (ks / NS) & 1)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const unsigned char *A = stages + buf * S_BYTES, *B = A + A_BYTES;
#pragma unroll
            for (int kh = 0; kh < BK / 16; ++kh)  // 16 pixels (two 8-row groups) per MMA
                tc::mma_bf16(taddr, smem_desc_mn_sw64(A + kh * 1024, kWgTmaAtom),
                             smem_desc_mn_sw64(B + kh * 1024, kWgTmaAtom), idesc, (ks > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&empty[buf]);
            done = ks + 1;
            if (ks >= 1 && issued < nk) {
                if (!tc::mbar_wait(&empty[(ks - 1) % NS], ((ks - 1) / NS) & 1)) {
                    ok = false;
                    break;
                }
                issue();
            }
        }
        if (ok && nk > 0) ok = tc::mbar_wait(&empty[(nk - 1) % NS], ((nk - 1) / NS) & 1);
        if (!ok) {
            atomicOr(err, 1);
            for (int s = done; s < issued; ++s) tc::mbar_wait(&full[s % NS], (s / NS) & 1);
            if (done > 0) tc::mbar_wait(&empty[(done - 1) % NS], ((done - 1) / NS) & 1);
        }
    }
    if (!__syncthreads_and(ok)) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, BN);
        return;
    }
    tc::fence_after_sync();
    if (nk > 0 && co0 + warp * 32 < a.cout) {
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

// The weight gradient of the three horizontal taps of one tap row at once, on
// levels whose width is a multiple of 64: a stage is 64 pixels of one image
// row; dz as in wgrad3x3_tma_kernel, the input as a halo row of 66 pixels
// (x0 - 1 .. x0 + 64 of row y0 + dy, zero outside the image) per 32-channel
// atom, so that the tap dx reads it from (dx + 1) x 64 bytes on (one pixel per
// 64-byte row of the swizzled tile).  Three accumulators of BN columns in
// tensor memory, one per tap; both operands are loaded once for the three.
constexpr int kWgHaloAtom = 5120;  // 66 x 64 bytes, rounded up to 1 KB
__host__ __device__ constexpr int wgrad_halo_stage_bytes(int bn, int ga32) {
    return ga32 * kWgTmaAtom + (bn / 32) * kWgHaloAtom;
}
__host__ __device__ constexpr int wgrad_halo_smem_bytes(int bn, int ga32) {
    return 1024 + kWgTmaStages * wgrad_halo_stage_bytes(bn, ga32) + 4 * kWgTmaAtom;
}
__host__ __device__ constexpr int wgrad_halo_tmem_cols(int bn) { return bn <= 32 ? 128 : (bn <= 64 ? 256 : 512); }

template <int BN, int GA32>
__global__ void __launch_bounds__(128) wgrad3x3_halo_kernel(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB, WgradArgs a,
                                                            int *err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int NS = kWgTmaStages, BM = 128, BK = kWgBK, TC = wgrad_halo_tmem_cols(BN);
    constexpr int A_BYTES = GA32 * kWgTmaAtom, S_BYTES = wgrad_halo_stage_bytes(BN, GA32);
    constexpr uint32_t TX = A_BYTES + (BN / 32) * 66 * 64;
    static_assert(3 * BN <= 512, "three accumulators");
    uint64_t *full = reinterpret_cast<uint64_t *>(sm);
    uint64_t *empty = full + NS;
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(empty + NS);
    unsigned char *stages = sm + 1024;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (smem_u32(stages) & 1023u) {
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    const long P = (long)a.n * a.h * a.wd;
    const int co0 = blockIdx.x * BM;
    const int dyi = blockIdx.y / (a.cin / BN);
    const int ci0 = (blockIdx.y % (a.cin / BN)) * BN;
    const long pbeg = (long)blockIdx.z * a.pix_per_block;
    const long pend = pbeg + a.pix_per_block < P ? pbeg + a.pix_per_block : P;
    const int nk = pend > pbeg ? (int)((pend - pbeg) / BK) : 0;
    if (warp == 0) tc::tmem_alloc(s_taddr, TC);
    if (tid < 2 * NS) tc::mbar_init(&full[tid], 1);
    tc::fence_barrier_init();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    bool ok = true;
    if (tid == 0) {
        tma::prefetch_map(&tmA);
        tma::prefetch_map(&tmB);
        const long hw = (long)a.h * a.wd;
        int issued = 0, done = 0;
        auto issue = [&]() {
            const int s = issued++;
            const long pb = pbeg + (long)s * BK;
            const int img = (int)(pb / hw);
            const int rem = (int)(pb - (long)img * hw);
            const int y0 = rem / a.wd, x0 = rem - (rem / a.wd) * a.wd;
            unsigned char *A = stages + (s % NS) * S_BYTES, *B = A + A_BYTES;
            uint64_t *fb = &full[s % NS];
            tma::arrive_expect_tx(fb, TX);
#pragma unroll
            for (int g = 0; g < GA32; ++g) tma::load_2d(A + g * kWgTmaAtom, &tmA, co0 + 32 * g, (int)pb, fb);
#pragma unroll
            for (int g = 0; g < BN / 32; ++g)
                tma::load_4d(B + g * kWgHaloAtom, &tmB, ci0 + 32 * g, x0 - 1, y0 + dyi - 1, img, fb);
        };
        while (issued < NS && issued < nk) issue();
        constexpr uint32_t idesc = tc::idesc_bf16(BM, BN) | (1u << 15) | (1u << 16);  // A and B MN-major
        for (int ks = 0; ks < nk; ++ks) {
            const int buf = ks % NS;
            if (!tc::mbar_wait(&full[buf], (ks / NS) & 1)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const unsigned char *A = stages + buf * S_BYTES, *B = A + A_BYTES;
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int kh = 0; kh < BK / 16; ++kh)  // 16 pixels (two 8-row groups) per MMA
                    tc::mma_bf16(taddr + (uint32_t)(d * BN), smem_desc_mn_sw64(A + kh * 1024, kWgTmaAtom),
                                 smem_desc_mn_sw64(B + d * 64 + kh * 1024, kWgHaloAtom), idesc,
                                 (ks > 0 || kh > 0) ? 1u : 0u);
            tc::mma_commit(&empty[buf]);
            done = ks + 1;
            if (ks >= 1 && issued < nk) {
                if (!tc::mbar_wait(&empty[(ks - 1) % NS], ((ks - 1) / NS) & 1)) {
                    ok = false;
                    break;
                }
                issue();
            }
        }
        if (ok && nk > 0) ok = tc::mbar_wait(&empty[(nk - 1) % NS], ((nk - 1) / NS) & 1);
        if (!ok) {
            atomicOr(err, 1);
            for (int s = done; s < issued; ++s) tc::mbar_wait(&full[s % NS], (s / NS) & 1);
            if (done > 0) tc::mbar_wait(&empty[(done - 1) % NS], ((done - 1) / NS) & 1);
        }
    }
    if (!__syncthreads_and(ok)) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(taddr, TC);
        return;
    }
    tc::fence_after_sync();
    if (nk > 0 && co0 + warp * 32 < a.cout) {
        const int co = co0 + warp * 32 + lane;  // this thread's accumulator row (tensor-memory lane)
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const int tap = dyi * 3 + d;
#pragma unroll 1
            for (int c = 0; c < BN; c += 8) {
                float v[8];
                tc::tmem_ld8(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * BN + c), v);
                if (co < a.cout) {
                    float *dd = a.dw + ((long)co * 9 + tap) * a.cin + ci0 + c;
#pragma unroll
                    for (int i = 0; i < 8; ++i) atomicAdd(dd + i, v[i]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, TC);
}

}  // namespace cnn
}  // namespace oslalm
