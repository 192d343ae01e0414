// Warm-start network: a 4-level U-Net (32/64/128/256 channels, 3x3 convs,
// ReLU, 2x2 average pooling, nearest 2x upsampling, skip concatenation,
// 1x1 output conv plus the input as a residual) that maps the FBP image to
// an estimate of the converged PWLS image; training and inference run on the
// BF16 tensor-core kernels of cnn_kernels.cuh with FP32 accumulation, FP32
// master weights and Adam.
#include <math.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "cnn_kernels.cuh"
#include "common.cuh"
#include "kernels_common.cuh"

namespace oslalm {
namespace cnn {

struct LayerSpec {
    const char *name;
    int cin_real, cin, cout;
};
// cin padded to a multiple of 32 (the 1-channel input is stored with 32 channels)
static const LayerSpec kLayers[14] = {
    {"e0a", 1, 32, 32},    {"e0b", 32, 32, 32},   {"e1a", 32, 32, 64},    {"e1b", 64, 64, 64},
    {"e2a", 64, 64, 128},  {"e2b", 128, 128, 128}, {"b3a", 128, 128, 256}, {"b3b", 256, 256, 256},
    {"d2a", 384, 384, 128}, {"d2b", 128, 128, 128}, {"d1a", 192, 192, 64}, {"d1b", 64, 64, 64},
    {"d0a", 96, 96, 32},   {"d0b", 32, 32, 32},
};
enum { E0A, E0B, E1A, E1B, E2A, E2B, B3A, B3B, D2A, D2B, D1A, D1B, D0A, D0B, NL };

// ---------------------------------------------------------------- elementwise kernels
// One thread moves 8 channels (16 bytes) of one pixel; C / 8 = 2^lc8 chunks
// per pixel (channel counts 32, 64, 128, 256), pixel indices below 2^31
// (checked when the network is created).  Every output element is computed
// with the same FP32 operations in the same order as an element-wise loop.
__device__ __forceinline__ uint4 ld16(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint4 *>(p); }
__device__ __forceinline__ void st16(__nv_bfloat16 *p, const uint4 &v) { *reinterpret_cast<uint4 *>(p) = v; }
__device__ __forceinline__ void unpack8(const uint4 &u, float *f) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __bfloat1622float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float *f) {
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    return u;
}

// input image x * s in channel 0 of 32 (the others zero)
__global__ void pack_input_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ out, long P, float s) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // chunk: pixel i / 4, channels 8 (i % 4)
    if (i >= P * 4) return;
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if ((i & 3) == 0) f[0] = x[i >> 2] * s;
    st16(out + i * 8, pack8(f));
}

// y = x (scaled) + b + sum_c w[c] h[p][c]; optional loss against t (scaled):
// dy = 2 (y - t) / count, loss partial sums in double
__global__ void output_kernel(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ w, const float *__restrict__ b,
                              const float *__restrict__ x, const float *__restrict__ t, float s, long P,
                              float *__restrict__ y_out, float *__restrict__ dy, double *__restrict__ loss,
                              float inv_count) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (p < P) {
        float acc = b[0];
        const __nv_bfloat162 *hp = reinterpret_cast<const __nv_bfloat162 *>(h + p * 32);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float2 v = __bfloat1622float2(hp[c]);
            acc = fmaf(w[2 * c], v.x, acc);
            acc = fmaf(w[2 * c + 1], v.y, acc);
        }
        const float yn = x[p] * s + acc;
        if (y_out) y_out[p] = yn / s;
        if (t) {
            const float r = yn - t[p] * s;
            dy[p] = 2.f * r * inv_count;
            l = (double)r * (double)r;
        }
    }
    if (t) {
        l = block_sum<256>(l);
        if (threadIdx.x == 0) atomicAdd(loss, l);
    }
}

// dh[p][c] = dy[p] w[c]; dw[c] += sum_p dy[p] h[p][c]; db += sum_p dy[p]
__global__ void output_bwd_kernel(const float *__restrict__ dy, const __nv_bfloat16 *__restrict__ h,
                                  const float *__restrict__ w, long P, __nv_bfloat16 *__restrict__ dh,
                                  float *__restrict__ dw, float *__restrict__ db) {
    __shared__ float sw[33];
    const int tid = threadIdx.x;
    if (tid < 33) sw[tid] = 0.f;
    __syncthreads();
    float part[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) part[c] = 0.f;
    float pb = 0.f;
    float wr[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) wr[c] = w[c];
    for (long p = (long)blockIdx.x * blockDim.x + tid; p < P; p += (long)gridDim.x * blockDim.x) {
        const float g = dy[p];
        pb += g;
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 8 channels (16 bytes) at a time
            float hv[8], o[8];
            unpack8(ld16(h + p * 32 + 8 * q), hv);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                o[k] = g * wr[8 * q + k];
                part[8 * q + k] = fmaf(g, hv[k], part[8 * q + k]);
            }
            st16(dh + p * 32 + 8 * q, pack8(o));
        }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        float v = part[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) atomicAdd(&sw[c], v);
    }
    for (int o = 16; o > 0; o >>= 1) pb += __shfl_xor_sync(0xffffffffu, pb, o);
    if ((tid & 31) == 0) atomicAdd(&sw[32], pb);
    __syncthreads();
    if (tid < 32) atomicAdd(&dw[tid], sw[tid]);
    if (tid == 32) atomicAdd(db, sw[32]);
}

// dz[p][c] = y[p][c] > 0 ? dy[p][c] : 0 (compact output), and the bias
// gradient db[c] += sum_p dz[p][c] of the stored BF16 values: the block sums
// its pixels per channel in shared memory, one atomic per channel and block
// (256 threads)
__global__ void __launch_bounds__(256) relu_bwd_kernel(const __nv_bfloat16 *__restrict__ y, int ld_y, int coff_y,
                                                       const __nv_bfloat16 *__restrict__ dy, int ld_dy, int coff_dy,
                                                       int lc8, long P, __nv_bfloat16 *__restrict__ dz,
                                                       float *__restrict__ db) {
    __shared__ float part[256][9];  // [thread][8 channels of its chunk] (+1: no bank conflicts)
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < (P << lc8)) {
        const long p = i >> lc8;
        const int c = (int)(i & ((1 << lc8) - 1)) * 8;
        const uint4 yv = ld16(y + p * ld_y + coff_y + c), gv = ld16(dy + p * ld_dy + coff_dy + c);
        const __nv_bfloat16 *ys = reinterpret_cast<const __nv_bfloat16 *>(&yv);
        const __nv_bfloat16 *gs = reinterpret_cast<const __nv_bfloat16 *>(&gv);
        uint4 o;
        __nv_bfloat16 *os = reinterpret_cast<__nv_bfloat16 *>(&o);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            os[k] = __bfloat162float(ys[k]) > 0.f ? gs[k] : __float2bfloat16_rn(0.f);
            f[k] = __bfloat162float(os[k]);
        }
        st16(dz + i * 8, o);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[threadIdx.x][k] = f[k];
    __syncthreads();
    // channel ch lives in chunk c8 = ch / 8 of every pixel, i.e. in the rows of
    // threads c8, c8 + C / 8, ... (the block starts at a pixel).  Thread t sums
    // channel t % C over every (256 / C)-th of those rows, 8 values; then
    // thread ch < C adds the 256 / C slices and makes the block's one atomic.
    __shared__ float slice[256];
    const int C8 = 1 << lc8, C = 8 * C8, S = 256 / C;
    {
        const int ch = threadIdx.x % C, sl = threadIdx.x / C;
        const int c8 = ch >> 3, k = ch & 7;
        float acc = 0.f;
        for (int j = sl; j < 256 / C8; j += S) acc += part[c8 + j * C8][k];
        slice[threadIdx.x] = acc;  // = slice[sl * C + ch]
    }
    __syncthreads();
    if ((int)threadIdx.x < C) {
        float acc = 0.f;
        for (int sl = 0; sl < S; ++sl) acc += slice[sl * C + threadIdx.x];
        atomicAdd(db + threadIdx.x, acc);
    }
}

// 2x2 average pooling of an NHWC slice
__global__ void pool_kernel(const __nv_bfloat16 *__restrict__ in, int ld_in, int coff_in, int lc8, int n, int h, int w,
                            __nv_bfloat16 *__restrict__ out) {
    const int h2 = h / 2, w2 = w / 2;
    const long total = ((long)n * h2 * w2) << lc8;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i & ((1 << lc8) - 1)) * 8;
    const unsigned q = (unsigned)(i >> lc8);
    const unsigned x = q % w2, t = q / w2, y = t % h2, img = t / h2;
    const long p00 = ((long)img * h + 2 * y) * w + 2 * x;
    const long src[4] = {p00, p00 + 1, p00 + w, p00 + w + 1};
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        unpack8(ld16(in + src[j] * ld_in + coff_in + c), v);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += v[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = 0.25f * s[k];
    st16(out + i * 8, pack8(s));
}

// gradient of pooling plus a skip gradient slice: out[p][c] = dpool[p/2][c] / 4 + add[p][c]
__global__ void pool_bwd_kernel(const __nv_bfloat16 *__restrict__ dpool, const __nv_bfloat16 *__restrict__ add,
                                int ld_add, int coff_add, int lc8, int n, int h, int w, __nv_bfloat16 *__restrict__ out) {
    const long total = ((long)n * h * w) << lc8;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i & ((1 << lc8) - 1)) * 8;
    const unsigned p = (unsigned)(i >> lc8);
    const unsigned x = p % w, q = p / w, y = q % h, img = q / h;
    const long pp = ((long)img * (h / 2) + y / 2) * (w / 2) + x / 2;
    float d[8], a[8];
    unpack8(ld16(dpool + (pp << (lc8 + 3)) + c), d);
    unpack8(ld16(add + (long)p * ld_add + coff_add + c), a);
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = 0.25f * d[k] + a[k];
    st16(out + i * 8, pack8(d));
}

// nearest 2x upsampling of [n][h][w][C] into a slice of a [n][2h][2w][ld] buffer
// (one thread per low-resolution chunk, written to its 2x2 block)
__global__ void up_kernel(const __nv_bfloat16 *__restrict__ in, int lc8, int n, int h, int w,
                          __nv_bfloat16 *__restrict__ out, int ld_out, int coff_out) {
    const long total = ((long)n * h * w) << lc8;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i & ((1 << lc8) - 1)) * 8;
    const unsigned q = (unsigned)(i >> lc8);
    const unsigned x = q % w, t = q / w, y = t % h, img = t / h;
    const uint4 v = ld16(in + i * 8);
    const long W2 = 2L * w;
    const long p00 = ((long)img * 2 * h + 2 * y) * W2 + 2 * x;
    st16(out + p00 * ld_out + coff_out + c, v);
    st16(out + (p00 + 1) * ld_out + coff_out + c, v);
    st16(out + (p00 + W2) * ld_out + coff_out + c, v);
    st16(out + (p00 + W2 + 1) * ld_out + coff_out + c, v);
}

// gradient of upsampling: out[p][c] = sum of the 2x2 block of a gradient slice
__global__ void up_bwd_kernel(const __nv_bfloat16 *__restrict__ g, int ld_g, int coff_g, int lc8, int n, int h, int w,
                              __nv_bfloat16 *__restrict__ out) {
    const long total = ((long)n * h * w) << lc8;  // h, w: the low-resolution size
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int c = (int)(i & ((1 << lc8) - 1)) * 8;
    const unsigned q = (unsigned)(i >> lc8);
    const unsigned x = q % w, t = q / w, y = t % h, img = t / h;
    const long W2 = 2L * w;
    const long p00 = ((long)img * 2 * h + 2 * y) * W2 + 2 * x;
    const long src[4] = {p00, p00 + 1, p00 + W2, p00 + W2 + 1};
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        unpack8(ld16(g + src[j] * ld_g + coff_g + c), v);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += v[k];
    }
    st16(out + i * 8, pack8(s));
}

// BF16 working copies of one layer: w [co][tap][ci] and the transposed,
// tap-flipped wt [ci][8 - tap][co] used for the data gradient
__global__ void convert_weights_kernel(const float *__restrict__ w32, int cin, int cout, __nv_bfloat16 *__restrict__ w,
                                       __nv_bfloat16 *__restrict__ wt) {
    const long total = (long)cout * 9 * cin;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int ci = (int)(i % cin);
    const int tap = (int)((i / cin) % 9);
    const int co = (int)(i / (9L * cin));
    const __nv_bfloat16 v = __float2bfloat16_rn(w32[i]);
    w[i] = v;
    wt[((long)ci * 9 + (8 - tap)) * cout + co] = v;
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

static inline unsigned nb(long n, int t) { return (unsigned)((n + t - 1) / t); }
// kernel launches issued by the network functions (all networks of the process)
static std::atomic<long> g_launches{0};
static inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
// log2 of C / 8 for the 16-byte elementwise kernels (C = 32, 64, 128 or 256)
static inline int lc8(int C) {
    int l = 0;
    while ((8 << l) < C) ++l;
    return l;
}

}  // namespace cnn
}  // namespace oslalm

using namespace oslalm;
using namespace oslalm::cnn;

struct oslalm_cnn {
    int batch, H, W;
    long P[4];  // pixels per level (all images)
    // parameters: FP32 master (padded layout), gradients, Adam moments
    long off_w[NL], off_b[NL], off_ow, off_ob, nparam;
    float *w32 = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb[NL] = {}, *wt[NL] = {};
    long step = 0;
    int use_tma = 1;  // convolutions whose blocks are whole rows take their tiles by TMA
    // activations (BF16 NHWC)
    __nv_bfloat16 *in0 = nullptr, *e0a = nullptr, *cat0 = nullptr, *p0 = nullptr, *e1a = nullptr, *cat1 = nullptr,
                  *p1 = nullptr, *e2a = nullptr, *cat2 = nullptr, *p2 = nullptr, *b3a = nullptr, *b3b = nullptr,
                  *d2a = nullptr, *d2b = nullptr, *d1a = nullptr, *d1b = nullptr, *d0a = nullptr, *d0b = nullptr;
    // gradients
    __nv_bfloat16 *g_cat0 = nullptr, *g_cat1 = nullptr, *g_cat2 = nullptr, *ga = nullptr, *gb = nullptr,
                  *dz = nullptr;
    float *dy = nullptr;
    double *loss = nullptr;
    int *err = nullptr;  // set by a convolution whose tensor-core wait ran out
    std::vector<void *> allocs;
};

namespace {

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime
// (null if the driver does not provide it)
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor maps of the TMA convolution: the input slice as (channel, column,
// row, image) with boxes of 32 channels x bw x bh, the weights [cout][9 cin]
// with boxes of 32 x bn, both in the 64-byte swizzle.  False if the geometry or the alignment does not allow it.
bool conv_tensor_maps(const __nv_bfloat16 *in, int ld_in, int coff_in, int cin, const __nv_bfloat16 *w, int cout,
                      int n, int h, int wd, int bn, CUtensorMap *ta, CUtensorMap *tb) {
    int bw = 0, bh = 0;  // a block's 128 pixels: a row segment, or 128 / wd whole rows
    if (wd % kBM == 0) {
        bw = kBM;
        bh = 1;
    } else if (kBM % wd == 0 && h % (kBM / wd) == 0) {
        bw = wd;
        bh = kBM / wd;
    } else {
        return false;
    }
    const __nv_bfloat16 *base = in + coff_in;
    if (reinterpret_cast<uintptr_t>(base) % 16 || reinterpret_cast<uintptr_t>(w) % 16 || ld_in % 8 || cin % kBK)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t es = 2;  // bytes per BF16
    const cuuint64_t gdA[4] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t gsA[3] = {ld_in * es, (cuuint64_t)wd * ld_in * es, (cuuint64_t)h * wd * ld_in * es};
    const cuuint32_t boxA[4] = {(cuuint32_t)kBK, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(base), gdA, gsA, boxA, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t gdB[2] = {(cuuint64_t)9 * cin, (cuuint64_t)cout};
    const cuuint64_t gsB[1] = {(cuuint64_t)9 * cin * es};
    const cuuint32_t boxB[2] = {(cuuint32_t)kBK, (cuuint32_t)bn};
    return enc(tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(w), gdB, gsB, boxB, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the halo convolution (width a multiple of 128): the input as
// (channel, column, row, image) with boxes of 32 channels x 130 pixels x 1
// row, the weights as for conv_tensor_maps.
bool conv_halo_maps(const __nv_bfloat16 *in, int ld_in, int coff_in, int cin, const __nv_bfloat16 *w, int cout,
                    int n, int h, int wd, int bn, CUtensorMap *ta, CUtensorMap *tb) {
    if (cin % kBK || wd % kBM) return false;
    // the weights' map and the alignment checks are those of the row-tile path
    if (!conv_tensor_maps(in, ld_in, coff_in, cin, w, cout, n, h, wd, bn, ta, tb)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    const cuuint64_t es = 2;
    const cuuint64_t gdA[4] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t gsA[3] = {ld_in * es, (cuuint64_t)wd * ld_in * es, (cuuint64_t)h * wd * ld_in * es};
    const cuuint32_t boxA[4] = {(cuuint32_t)kBK, (cuuint32_t)(kBM + 2), 1, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    return enc(ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(in + coff_in), gdA, gsA, boxA,
               one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int conv(const oslalm_cnn *c, const __nv_bfloat16 *in, int ld_in, int coff_in, int cin, const __nv_bfloat16 *w,
         const float *bias, __nv_bfloat16 *out, int ld_out, int coff_out, int cout, int n, int h, int wd, int relu,
         cudaStream_t st) {
    ConvArgs a;
    a.in = in; a.ld_in = ld_in; a.coff_in = coff_in; a.cin = cin;
    a.w = w; a.bias = bias;
    a.out = out; a.ld_out = ld_out; a.coff_out = coff_out; a.cout = cout;
    a.n = n; a.h = h; a.wd = wd; a.relu = relu;
    const long P = (long)n * h * wd;
    // output channels per block: the largest power of two <= 256 dividing cout
    // (tensor-memory columns come in powers of two)
    int bn = 256;
    while (cout % bn) bn >>= 1;
    if (bn < 32 || cin % kBK) return fail(OSLALM_ERR_ARG, "convolution needs channel counts that are multiples of 32");
    dim3 grid(nb(P, kBM), cout / bn);
    CUtensorMap ta, tb;
    if (c->use_tma && conv_halo_maps(in, ld_in, coff_in, cin, w, cout, n, h, wd, bn, &ta, &tb)) {
#define OSL_CONV_HALO(BN)                                                                                  \
    do {                                                                                                   \
        static bool opted = false;                                                                         \
        if (!opted) {                                                                                      \
            OSL_CUDA_TRY(cudaFuncSetAttribute(conv3x3_halo_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              conv_halo_smem_bytes(BN)));                                  \
            opted = true;                                                                                  \
        }                                                                                                  \
        conv3x3_halo_kernel<BN><<<grid, 128, conv_halo_smem_bytes(BN), st>>>(ta, tb, a, c->err);          \
        note_launch();                                                                                     \
    } while (0)
        switch (bn) {
            case 32: OSL_CONV_HALO(32); break;
            case 64: OSL_CONV_HALO(64); break;
            case 128: OSL_CONV_HALO(128); break;
            default: OSL_CONV_HALO(256); break;
        }
#undef OSL_CONV_HALO
        OSL_LAUNCH_CHECK("conv3x3_halo_kernel");
        return OSLALM_OK;
    }
    if (c->use_tma && conv_tensor_maps(in, ld_in, coff_in, cin, w, cout, n, h, wd, bn, &ta, &tb)) {
#define OSL_CONV_TMA(BN)                                                                                   \
    do {                                                                                                   \
        static bool opted = false;                                                                         \
        if (!opted) {                                                                                      \
            OSL_CUDA_TRY(cudaFuncSetAttribute(conv3x3_tma_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              conv_tma_smem_bytes(BN)));                                   \
            opted = true;                                                                                  \
        }                                                                                                  \
        conv3x3_tma_kernel<BN><<<grid, 128, conv_tma_smem_bytes(BN), st>>>(ta, tb, a, c->err);            \
        note_launch();                                                                                    \
    } while (0)
        switch (bn) {
            case 32: OSL_CONV_TMA(32); break;
            case 64: OSL_CONV_TMA(64); break;
            case 128: OSL_CONV_TMA(128); break;
            default: OSL_CONV_TMA(256); break;
        }
#undef OSL_CONV_TMA
        OSL_LAUNCH_CHECK("conv3x3_tma_kernel");
        return OSLALM_OK;
    }
#define OSL_CONV(BN)                                                                                       \
    do {                                                                                                   \
        static bool opted = false; /* dynamic shared memory above 48 KB, once */                          \
        if (!opted) {                                                                                      \
            OSL_CUDA_TRY(cudaFuncSetAttribute(conv3x3_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              conv_smem_bytes(BN)));                                       \
            opted = true;                                                                                  \
        }                                                                                                  \
        conv3x3_kernel<BN><<<grid, 128, conv_smem_bytes(BN), st>>>(a, c->err);                            \
        note_launch();                                                                                    \
    } while (0)
    switch (bn) {
        case 32: OSL_CONV(32); break;
        case 64: OSL_CONV(64); break;
        case 128: OSL_CONV(128); break;
        default: OSL_CONV(256); break;
    }
#undef OSL_CONV
    OSL_LAUNCH_CHECK("conv3x3_kernel");
    return OSLALM_OK;
}

// Tensor maps of the TMA weight gradient: dz [P][cout] (slice of ld_dz
// channels at coff_dz) as (channel, pixel) with boxes of 32 x 64, the x slice
// as (channel, column, row, image) with boxes of 32 channels x bw x bh (64
// pixels), both in the 64-byte swizzle.  False if the geometry or the
// alignment does not allow it.
bool wgrad_tensor_maps(const __nv_bfloat16 *dz, int ld_dz, int coff_dz, int cout, const __nv_bfloat16 *x, int ld_x,
                       int coff_x, int cin, int n, int h, int wd, CUtensorMap *ta, CUtensorMap *tb) {
    int bw = 0, bh = 0;  // a 64-pixel stage: a row segment, or 64 / wd whole rows
    if (wd % kWgBK == 0) {
        bw = kWgBK;
        bh = 1;
    } else if (kWgBK % wd == 0 && h % (kWgBK / wd) == 0) {
        bw = wd;
        bh = kWgBK / wd;
    } else {
        return false;
    }
    const __nv_bfloat16 *a0 = dz + coff_dz, *b0 = x + coff_x;
    if (reinterpret_cast<uintptr_t>(a0) % 16 || reinterpret_cast<uintptr_t>(b0) % 16 || ld_dz % 8 || ld_x % 8 ||
        cin % 32 || cout % 32)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t es = 2;
    const long P = (long)n * h * wd;
    const cuuint64_t gdA[2] = {(cuuint64_t)cout, (cuuint64_t)P};
    const cuuint64_t gsA[1] = {(cuuint64_t)ld_dz * es};
    const cuuint32_t boxA[2] = {32, (cuuint32_t)kWgBK};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    if (enc(ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(a0), gdA, gsA, boxA, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t gdB[4] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t gsB[3] = {ld_x * es, (cuuint64_t)wd * ld_x * es, (cuuint64_t)h * wd * ld_x * es};
    const cuuint32_t boxB[4] = {32, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    return enc(tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(b0), gdB, gsB, boxB, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the three-tap weight gradient (width a multiple of 64): dz as
// for wgrad_tensor_maps, the input slice with boxes of 32 channels x 66 pixels
// x 1 row (the halo row of a 64-pixel stage).
bool wgrad_halo_maps(const __nv_bfloat16 *dz, int ld_dz, int coff_dz, int cout, const __nv_bfloat16 *x, int ld_x,
                     int coff_x, int cin, int n, int h, int wd, CUtensorMap *ta, CUtensorMap *tb) {
    if (wd % kWgBK) return false;
    if (!wgrad_tensor_maps(dz, ld_dz, coff_dz, cout, x, ld_x, coff_x, cin, n, h, wd, ta, tb)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    const cuuint64_t es = 2;
    const cuuint64_t gdB[4] = {(cuuint64_t)cin, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)n};
    const cuuint64_t gsB[3] = {ld_x * es, (cuuint64_t)wd * ld_x * es, (cuuint64_t)h * wd * ld_x * es};
    const cuuint32_t boxB[4] = {32, (cuuint32_t)(kWgBK + 2), 1, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    return enc(tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(x + coff_x), gdB, gsB, boxB, one,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int wgrad(const oslalm_cnn *c, const __nv_bfloat16 *dz, int cout, const __nv_bfloat16 *x, int ld_x, int coff_x,
          int cin, float *dw, int n, int h, int wd, cudaStream_t st) {
    WgradArgs a;
    a.dz = dz; a.ld_dz = cout; a.coff_dz = 0; a.cout = cout;
    a.x = x; a.ld_x = ld_x; a.coff_x = coff_x; a.cin = cin;
    a.dw = dw; a.n = n; a.h = h; a.wd = wd;
    const long P = (long)n * h * wd;
    // input channels per block: the largest power of two <= 256 dividing cin
    int bn = 256;
    while (cin % bn) bn >>= 1;
    if (bn < 32 || cout % 8) return fail(OSLALM_ERR_ARG, "weight gradient needs channel counts that are multiples of 32");
    int dev = 0, sms = 0, smem_sm = 0;
    OSL_CUDA_TRY(cudaGetDevice(&dev));
    OSL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    OSL_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    // one wave of blocks (blocks per SM from shared memory and tensor-memory
    // columns), the pixels split evenly in multiples of the 64-pixel stage
    auto split = [&](int smem, long tiles) {
        int occ = std::min(smem_sm / (smem + 1024), std::min(512 / bn, 16));
        if (occ < 1) occ = 1;
        long splits = ((long)sms * occ) / tiles;
        if (splits < 1) splits = 1;
        long per = (P + splits - 1) / splits;
        per = ((per + kWgBK - 1) / kWgBK) * kWgBK;
        a.pix_per_block = (int)per;
        return dim3((cout + 127) / 128, 9 * (cin / bn), (unsigned)((P + per - 1) / per));
    };
    CUtensorMap ta, tb;
    const int ga32 = std::min(4, cout / 32);
    if (c->use_tma && cout % 32 == 0 && ga32 != 3 && bn <= 128 &&
        wgrad_halo_maps(dz, cout, 0, cout, x, ld_x, coff_x, cin, n, h, wd, &ta, &tb)) {
        // the three horizontal taps of a tap row per block
        const int smem = wgrad_halo_smem_bytes(bn, ga32);
        int occ = std::min(smem_sm / (smem + 1024), std::min(512 / wgrad_halo_tmem_cols(bn), 16));
        if (occ < 1) occ = 1;
        const long tiles = (long)((cout + 127) / 128) * 3 * (cin / bn);
        long splits = ((long)sms * occ) / tiles;
        if (splits < 1) splits = 1;
        long per = (P + splits - 1) / splits;
        per = ((per + kWgBK - 1) / kWgBK) * kWgBK;
        a.pix_per_block = (int)per;
        const dim3 grid((cout + 127) / 128, 3 * (cin / bn), (unsigned)((P + per - 1) / per));
#define OSL_WGH(BN, GA)                                                                                      \
    do {                                                                                                     \
        static bool opted = false;                                                                           \
        if (!opted) {                                                                                        \
            OSL_CUDA_TRY(cudaFuncSetAttribute(wgrad3x3_halo_kernel<BN, GA>,                                  \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                              wgrad_halo_smem_bytes(BN, GA)));                               \
            opted = true;                                                                                    \
        }                                                                                                    \
        wgrad3x3_halo_kernel<BN, GA><<<grid, 128, wgrad_halo_smem_bytes(BN, GA), st>>>(ta, tb, a, c->err);  \
        note_launch();                                                                                       \
    } while (0)
        switch (bn * 10 + ga32) {
            case 321: OSL_WGH(32, 1); break;
            case 322: OSL_WGH(32, 2); break;
            case 324: OSL_WGH(32, 4); break;
            case 641: OSL_WGH(64, 1); break;
            case 642: OSL_WGH(64, 2); break;
            case 644: OSL_WGH(64, 4); break;
            case 1281: OSL_WGH(128, 1); break;
            case 1282: OSL_WGH(128, 2); break;
            default: OSL_WGH(128, 4); break;
        }
#undef OSL_WGH
        OSL_LAUNCH_CHECK("wgrad3x3_halo_kernel");
        return OSLALM_OK;
    }
    if (c->use_tma && cout % 32 == 0 && ga32 != 3 &&
        wgrad_tensor_maps(dz, cout, 0, cout, x, ld_x, coff_x, cin, n, h, wd, &ta, &tb)) {
        const int smem = wgrad_tma_smem_bytes(bn, ga32);
        const dim3 grid = split(smem, (long)((cout + 127) / 128) * 9 * (cin / bn));
#define OSL_WGT(BN, GA)                                                                                      \
    do {                                                                                                     \
        static bool opted = false;                                                                           \
        if (!opted) {                                                                                        \
            OSL_CUDA_TRY(cudaFuncSetAttribute(wgrad3x3_tma_kernel<BN, GA>,                                   \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                              wgrad_tma_smem_bytes(BN, GA)));                                \
            opted = true;                                                                                    \
        }                                                                                                    \
        wgrad3x3_tma_kernel<BN, GA><<<grid, 128, wgrad_tma_smem_bytes(BN, GA), st>>>(ta, tb, a, c->err);    \
        note_launch();                                                                                      \
    } while (0)
        switch (bn * 10 + ga32) {
            case 321: OSL_WGT(32, 1); break;
            case 322: OSL_WGT(32, 2); break;
            case 324: OSL_WGT(32, 4); break;
            case 641: OSL_WGT(64, 1); break;
            case 642: OSL_WGT(64, 2); break;
            case 644: OSL_WGT(64, 4); break;
            case 1281: OSL_WGT(128, 1); break;
            case 1282: OSL_WGT(128, 2); break;
            case 1284: OSL_WGT(128, 4); break;
            case 2561: OSL_WGT(256, 1); break;
            case 2562: OSL_WGT(256, 2); break;
            default: OSL_WGT(256, 4); break;
        }
#undef OSL_WGT
        OSL_LAUNCH_CHECK("wgrad3x3_tma_kernel");
        return OSLALM_OK;
    }
    // dz channel groups staged per block: 4, 8 or 16 (output channel counts
    // of 32, 64 or a multiple of 128 ... any multiple of 8 from 128 on)
    const int ga = wgrad_groups(cout);
    if (ga != 4 && ga != 8 && ga != 16)
        return fail(OSLALM_ERR_ARG, "weight gradient needs 32, 64 or at least 128 output channels");
    const dim3 grid = split(wgrad_tc_smem_bytes(bn, ga), (long)((cout + 127) / 128) * 9 * (cin / bn));
#define OSL_WG(BN, GA)                                                                                       \
    do {                                                                                                     \
        static bool opted = false; /* dynamic shared memory above 48 KB, once */                            \
        if (!opted) {                                                                                        \
            OSL_CUDA_TRY(cudaFuncSetAttribute(wgrad3x3_tc_kernel<BN, GA>,                                    \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                              wgrad_tc_smem_bytes(BN, GA)));                                 \
            opted = true;                                                                                    \
        }                                                                                                    \
        wgrad3x3_tc_kernel<BN, GA><<<grid, 128, wgrad_tc_smem_bytes(BN, GA), st>>>(a, c->err);              \
        note_launch();                                                                                      \
    } while (0)
    switch (bn * 100 + ga) {
        case 3204: OSL_WG(32, 4); break;
        case 3208: OSL_WG(32, 8); break;
        case 3216: OSL_WG(32, 16); break;
        case 6404: OSL_WG(64, 4); break;
        case 6408: OSL_WG(64, 8); break;
        case 6416: OSL_WG(64, 16); break;
        case 12804: OSL_WG(128, 4); break;
        case 12808: OSL_WG(128, 8); break;
        case 12816: OSL_WG(128, 16); break;
        case 25604: OSL_WG(256, 4); break;
        case 25608: OSL_WG(256, 8); break;
        default: OSL_WG(256, 16); break;
    }
#undef OSL_WG
    OSL_LAUNCH_CHECK("wgrad3x3_tc_kernel");
    return OSLALM_OK;
}

// backward of layer L with input slice (x, ld_x, coff_x) and output slice
// (y, ld_y, coff_y) given the output gradient slice (gy, ld_gy, coff_gy);
// writes the input gradient into (gx, ld_gx, coff_gx) unless gx is null
int layer_bwd(oslalm_cnn *c, int L, int lvl, const __nv_bfloat16 *x, int ld_x, int coff_x, const __nv_bfloat16 *y,
              int ld_y, int coff_y, const __nv_bfloat16 *gy, int ld_gy, int coff_gy, __nv_bfloat16 *gx, int ld_gx,
              int coff_gx, cudaStream_t st) {
    const LayerSpec &s = kLayers[L];
    const int h = c->H >> lvl, w = c->W >> lvl;
    const long P = c->P[lvl];
    relu_bwd_kernel<<<nb(P * s.cout / 8, 256), 256, 0, st>>>(y, ld_y, coff_y, gy, ld_gy, coff_gy, lc8(s.cout), P, c->dz,
                                                             c->grad + c->off_b[L]);
    note_launch();
    OSL_LAUNCH_CHECK("relu_bwd_kernel");
    if (int rc = wgrad(c, c->dz, s.cout, x, ld_x, coff_x, s.cin, c->grad + c->off_w[L], c->batch, h, w, st)) return rc;
    if (gx)
        return conv(c, c->dz, s.cout, 0, s.cout, c->wt[L], nullptr, gx, ld_gx, coff_gx, s.cin, c->batch, h, w, 0, st);
    return OSLALM_OK;
}

int forward_net(oslalm_cnn *c, cudaStream_t st) {
    const int n = c->batch, H = c->H, W = c->W;
    auto L = [&](int id) { return c->wb[id]; };
    auto B = [&](int id) { return c->w32 + c->off_b[id]; };
    int rc = 0;
#define C3(in, ldi, ci0, cin, id, out, ldo, co0, cout, lvl)                                                       \
    if ((rc = conv(c, in, ldi, ci0, cin, L(id), B(id), out, ldo, co0, cout, n, H >> (lvl), W >> (lvl), 1, st))) \
        return rc;
    C3(c->in0, 32, 0, 32, E0A, c->e0a, 32, 0, 32, 0);
    C3(c->e0a, 32, 0, 32, E0B, c->cat0, 96, 64, 32, 0);
    pool_kernel<<<nb(c->P[1] * 32 / 8, 256), 256, 0, st>>>(c->cat0, 96, 64, lc8(32), n, H, W, c->p0);
    note_launch();
    C3(c->p0, 32, 0, 32, E1A, c->e1a, 64, 0, 64, 1);
    C3(c->e1a, 64, 0, 64, E1B, c->cat1, 192, 128, 64, 1);
    pool_kernel<<<nb(c->P[2] * 64 / 8, 256), 256, 0, st>>>(c->cat1, 192, 128, lc8(64), n, H / 2, W / 2, c->p1);
    note_launch();
    C3(c->p1, 64, 0, 64, E2A, c->e2a, 128, 0, 128, 2);
    C3(c->e2a, 128, 0, 128, E2B, c->cat2, 384, 256, 128, 2);
    pool_kernel<<<nb(c->P[3] * 128 / 8, 256), 256, 0, st>>>(c->cat2, 384, 256, lc8(128), n, H / 4, W / 4, c->p2);
    note_launch();
    C3(c->p2, 128, 0, 128, B3A, c->b3a, 256, 0, 256, 3);
    C3(c->b3a, 256, 0, 256, B3B, c->b3b, 256, 0, 256, 3);
    up_kernel<<<nb(c->P[3] * 256 / 8, 256), 256, 0, st>>>(c->b3b, lc8(256), n, H / 8, W / 8, c->cat2, 384, 0);
    note_launch();
    C3(c->cat2, 384, 0, 384, D2A, c->d2a, 128, 0, 128, 2);
    C3(c->d2a, 128, 0, 128, D2B, c->d2b, 128, 0, 128, 2);
    up_kernel<<<nb(c->P[2] * 128 / 8, 256), 256, 0, st>>>(c->d2b, lc8(128), n, H / 4, W / 4, c->cat1, 192, 0);
    note_launch();
    C3(c->cat1, 192, 0, 192, D1A, c->d1a, 64, 0, 64, 1);
    C3(c->d1a, 64, 0, 64, D1B, c->d1b, 64, 0, 64, 1);
    up_kernel<<<nb(c->P[1] * 64 / 8, 256), 256, 0, st>>>(c->d1b, lc8(64), n, H / 2, W / 2, c->cat0, 96, 0);
    note_launch();
    C3(c->cat0, 96, 0, 96, D0A, c->d0a, 32, 0, 32, 0);
    C3(c->d0a, 32, 0, 32, D0B, c->d0b, 32, 0, 32, 0);
#undef C3
    OSL_LAUNCH_CHECK("forward");
    return OSLALM_OK;
}

int backward_net(oslalm_cnn *c, cudaStream_t st) {
    const int n = c->batch, H = c->H, W = c->W;
    const long P0 = c->P[0];
    int rc;
    OSL_CUDA_TRY(cudaMemsetAsync(c->grad, 0, sizeof(float) * c->nparam, st));
    output_bwd_kernel<<<std::min<long>(nb(P0, 256), 1024), 256, 0, st>>>(c->dy, c->d0b, c->w32 + c->off_ow, P0, c->ga,
                                                                         c->grad + c->off_ow, c->grad + c->off_ob);
    note_launch();
    OSL_LAUNCH_CHECK("output_bwd_kernel");
    // decoder level 0: ga = d(d0b) -> gb = d(d0a) -> g_cat0
    if ((rc = layer_bwd(c, D0B, 0, c->d0a, 32, 0, c->d0b, 32, 0, c->ga, 32, 0, c->gb, 32, 0, st))) return rc;
    if ((rc = layer_bwd(c, D0A, 0, c->cat0, 96, 0, c->d0a, 32, 0, c->gb, 32, 0, c->g_cat0, 96, 0, st))) return rc;
    up_bwd_kernel<<<nb(c->P[1] * 64 / 8, 256), 256, 0, st>>>(c->g_cat0, 96, 0, lc8(64), n, H / 2, W / 2, c->ga);  // d(d1b)
    note_launch();
    if ((rc = layer_bwd(c, D1B, 1, c->d1a, 64, 0, c->d1b, 64, 0, c->ga, 64, 0, c->gb, 64, 0, st))) return rc;
    if ((rc = layer_bwd(c, D1A, 1, c->cat1, 192, 0, c->d1a, 64, 0, c->gb, 64, 0, c->g_cat1, 192, 0, st))) return rc;
    up_bwd_kernel<<<nb(c->P[2] * 128 / 8, 256), 256, 0, st>>>(c->g_cat1, 192, 0, lc8(128), n, H / 4, W / 4, c->ga);  // d(d2b)
    note_launch();
    if ((rc = layer_bwd(c, D2B, 2, c->d2a, 128, 0, c->d2b, 128, 0, c->ga, 128, 0, c->gb, 128, 0, st))) return rc;
    if ((rc = layer_bwd(c, D2A, 2, c->cat2, 384, 0, c->d2a, 128, 0, c->gb, 128, 0, c->g_cat2, 384, 0, st))) return rc;
    up_bwd_kernel<<<nb(c->P[3] * 256 / 8, 256), 256, 0, st>>>(c->g_cat2, 384, 0, lc8(256), n, H / 8, W / 8, c->ga);  // d(b3b)
    note_launch();
    if ((rc = layer_bwd(c, B3B, 3, c->b3a, 256, 0, c->b3b, 256, 0, c->ga, 256, 0, c->gb, 256, 0, st))) return rc;
    if ((rc = layer_bwd(c, B3A, 3, c->p2, 128, 0, c->b3a, 256, 0, c->gb, 256, 0, c->ga, 128, 0, st))) return rc;
    // pool 2 backward + skip gradient -> d(e2b) in gb
    pool_bwd_kernel<<<nb(c->P[2] * 128 / 8, 256), 256, 0, st>>>(c->ga, c->g_cat2, 384, 256, lc8(128), n, H / 4, W / 4, c->gb);
    note_launch();
    if ((rc = layer_bwd(c, E2B, 2, c->e2a, 128, 0, c->cat2, 384, 256, c->gb, 128, 0, c->ga, 128, 0, st))) return rc;
    if ((rc = layer_bwd(c, E2A, 2, c->p1, 64, 0, c->e2a, 128, 0, c->ga, 128, 0, c->gb, 64, 0, st))) return rc;
    pool_bwd_kernel<<<nb(c->P[1] * 64 / 8, 256), 256, 0, st>>>(c->gb, c->g_cat1, 192, 128, lc8(64), n, H / 2, W / 2, c->ga);
    note_launch();
    if ((rc = layer_bwd(c, E1B, 1, c->e1a, 64, 0, c->cat1, 192, 128, c->ga, 64, 0, c->gb, 64, 0, st))) return rc;
    if ((rc = layer_bwd(c, E1A, 1, c->p0, 32, 0, c->e1a, 64, 0, c->gb, 64, 0, c->ga, 32, 0, st))) return rc;
    pool_bwd_kernel<<<nb(c->P[0] * 32 / 8, 256), 256, 0, st>>>(c->ga, c->g_cat0, 96, 64, lc8(32), n, H, W, c->gb);
    note_launch();
    if ((rc = layer_bwd(c, E0B, 0, c->e0a, 32, 0, c->cat0, 96, 64, c->gb, 32, 0, c->ga, 32, 0, st))) return rc;
    if ((rc = layer_bwd(c, E0A, 0, c->in0, 32, 0, c->e0a, 32, 0, c->ga, 32, 0, nullptr, 0, 0, st))) return rc;
    OSL_LAUNCH_CHECK("backward");
    return OSLALM_OK;
}

int refresh_weights(oslalm_cnn *c, cudaStream_t st) {
    for (int L = 0; L < NL; ++L) {
        const LayerSpec &s = kLayers[L];
        const long n = (long)s.cout * 9 * s.cin;
        convert_weights_kernel<<<nb(n, 256), 256, 0, st>>>(c->w32 + c->off_w[L], s.cin, s.cout, c->wb[L], c->wt[L]);
        note_launch();
    }
    OSL_LAUNCH_CHECK("convert_weights_kernel");
    return OSLALM_OK;
}

int check_n(const oslalm_cnn *c, int n) {
    if (!c) return fail(OSLALM_ERR_ARG, "network handle is NULL");
    if (n != c->batch) return fail(OSLALM_ERR_ARG, "the network was created for batches of %d images", c->batch);
    return OSLALM_OK;
}

// After a synchronisation: report (and clear) a tensor-core wait of an
// earlier convolution that ran out of iterations.
int check_waits(oslalm_cnn *c) {
    int flag = 0;
    OSL_CUDA_TRY(cudaMemcpy(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return OSLALM_OK;
    OSL_CUDA_TRY(cudaMemset(c->err, 0, sizeof(int)));
    if (flag & 2) return fail(OSLALM_ERR_CUDA, "TMA convolution found its shared memory misaligned; output invalid");
    return fail(OSLALM_ERR_TIMEOUT, "a convolution's tensor-core wait ran out; its output is invalid");
}

int run_forward(oslalm_cnn *c, const float *x, const float *t, float s, float *y, cudaStream_t st) {
    const long P0 = c->P[0];
    pack_input_kernel<<<nb(P0 * 4, 256), 256, 0, st>>>(x, c->in0, P0, s);
    note_launch();
    OSL_LAUNCH_CHECK("pack_input_kernel");
    if (int rc = forward_net(c, st)) return rc;
    if (t) OSL_CUDA_TRY(cudaMemsetAsync(c->loss, 0, sizeof(double), st));
    output_kernel<<<nb(P0, 256), 256, 0, st>>>(c->d0b, c->w32 + c->off_ow, c->w32 + c->off_ob, x, t, s, P0, y, c->dy,
                                               c->loss, 1.f / (float)P0);
    note_launch();
    OSL_LAUNCH_CHECK("output_kernel");
    return OSLALM_OK;
}

// reference parameter order: per layer w [co][3][3][ci_real] then b; out.w, out.b
void copy_params(oslalm_cnn *c, std::vector<float> &dev_layout, float *ref, bool to_ref) {
    long k = 0;
    for (int L = 0; L < NL; ++L) {
        const LayerSpec &s = kLayers[L];
        for (int co = 0; co < s.cout; ++co)
            for (int tap = 0; tap < 9; ++tap)
                for (int ci = 0; ci < s.cin_real; ++ci) {
                    float &d = dev_layout[c->off_w[L] + ((long)co * 9 + tap) * s.cin + ci];
                    if (to_ref) ref[k++] = d;
                    else d = ref[k++];
                }
        for (int co = 0; co < s.cout; ++co) {
            float &d = dev_layout[c->off_b[L] + co];
            if (to_ref) ref[k++] = d;
            else d = ref[k++];
        }
    }
    for (int cc = 0; cc < 32; ++cc) {
        float &d = dev_layout[c->off_ow + cc];
        if (to_ref) ref[k++] = d;
        else d = ref[k++];
    }
    float &d = dev_layout[c->off_ob];
    if (to_ref) ref[k++] = d;
    else d = ref[k++];
}

long ref_param_count() {
    long k = 0;
    for (int L = 0; L < NL; ++L) k += (long)kLayers[L].cout * 9 * kLayers[L].cin_real + kLayers[L].cout;
    return k + 33;
}

}  // namespace

extern "C" {

long oslalm_cnn_param_count(void) { return ref_param_count(); }

int oslalm_cnn_create(int batch, int height, int width, unsigned long long seed, oslalm_cnn **out) {
    clear_error();
    if (!out) return fail(OSLALM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (batch <= 0 || height <= 0 || width <= 0 || height % 8 || width % 8)
        return fail(OSLALM_ERR_ARG, "need batch > 0 and height, width positive multiples of 8");
    if ((long)batch * height * width >= (1L << 31)) return fail(OSLALM_ERR_ARG, "need batch x height x width < 2^31");
    oslalm_cnn *c = new (std::nothrow) oslalm_cnn();
    if (!c) return fail(OSLALM_ERR_ALLOC, "host allocation failed");
    c->batch = batch;
    c->H = height;
    c->W = width;
    for (int l = 0; l < 4; ++l) c->P[l] = (long)batch * (height >> l) * (width >> l);
    long o = 0;
    for (int L = 0; L < NL; ++L) {
        c->off_w[L] = o;
        o += (long)kLayers[L].cout * 9 * kLayers[L].cin;
        c->off_b[L] = o;
        o += kLayers[L].cout;
    }
    c->off_ow = o;
    o += 32;
    c->off_ob = o;
    o += 1;
    c->nparam = o;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) c->allocs.push_back(*p);
    };
    const size_t bf = sizeof(__nv_bfloat16);
    A((void **)&c->err, sizeof(int));
    A((void **)&c->w32, sizeof(float) * o);
    A((void **)&c->grad, sizeof(float) * o);
    A((void **)&c->m, sizeof(float) * o);
    A((void **)&c->v, sizeof(float) * o);
    for (int L = 0; L < NL; ++L) {
        const size_t n = (size_t)kLayers[L].cout * 9 * kLayers[L].cin;
        A((void **)&c->wb[L], bf * n);
        A((void **)&c->wt[L], bf * n);
    }
    const long *P = c->P;
    A((void **)&c->in0, bf * P[0] * 32);
    A((void **)&c->e0a, bf * P[0] * 32);
    A((void **)&c->cat0, bf * P[0] * 96);
    A((void **)&c->p0, bf * P[1] * 32);
    A((void **)&c->e1a, bf * P[1] * 64);
    A((void **)&c->cat1, bf * P[1] * 192);
    A((void **)&c->p1, bf * P[2] * 64);
    A((void **)&c->e2a, bf * P[2] * 128);
    A((void **)&c->cat2, bf * P[2] * 384);
    A((void **)&c->p2, bf * P[3] * 128);
    A((void **)&c->b3a, bf * P[3] * 256);
    A((void **)&c->b3b, bf * P[3] * 256);
    A((void **)&c->d2a, bf * P[2] * 128);
    A((void **)&c->d2b, bf * P[2] * 128);
    A((void **)&c->d1a, bf * P[1] * 64);
    A((void **)&c->d1b, bf * P[1] * 64);
    A((void **)&c->d0a, bf * P[0] * 32);
    A((void **)&c->d0b, bf * P[0] * 32);
    A((void **)&c->g_cat0, bf * P[0] * 96);
    A((void **)&c->g_cat1, bf * P[1] * 192);
    A((void **)&c->g_cat2, bf * P[2] * 384);
    const long gmax = std::max(std::max(P[0] * 32, P[1] * 64), std::max(P[2] * 128, P[3] * 256));
    A((void **)&c->ga, bf * gmax);
    A((void **)&c->gb, bf * gmax);
    A((void **)&c->dz, bf * gmax);
    A((void **)&c->dy, sizeof(float) * P[0]);
    A((void **)&c->loss, sizeof(double));
    if (e != cudaSuccess) {
        for (void *p : c->allocs) cudaFree(p);
        delete c;
        return fail(OSLALM_ERR_ALLOC, "network allocation failed: %s", cudaGetErrorString(e));
    }
    // He-normal initialisation from a seeded splitmix64 / Box-Muller stream
    std::vector<float> h(o, 0.f);
    unsigned long long state = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
        unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    auto normal = [&]() { return sqrt(-2.0 * log(next())) * cos(6.283185307179586 * next()); };
    for (int L = 0; L < NL; ++L) {
        const LayerSpec &s = kLayers[L];
        const double sd = sqrt(2.0 / (9.0 * s.cin_real));
        for (int co = 0; co < s.cout; ++co)
            for (int tap = 0; tap < 9; ++tap)
                for (int ci = 0; ci < s.cin_real; ++ci)
                    h[c->off_w[L] + ((long)co * 9 + tap) * s.cin + ci] = (float)(sd * normal());
    }
    for (int cc = 0; cc < 32; ++cc) h[c->off_ow + cc] = (float)(0.01 * normal());
    e = cudaMemcpy(c->w32, h.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->m, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->v, 0, sizeof(float) * o);
    int rc = e == cudaSuccess ? refresh_weights(c, nullptr) : fail(OSLALM_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (!rc && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = fail(OSLALM_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (rc) {
        for (void *p : c->allocs) cudaFree(p);
        delete c;
        return rc;
    }
    *out = c;
    return OSLALM_OK;
}

int oslalm_cnn_destroy(oslalm_cnn *c) {
    clear_error();
    if (!c) return OSLALM_OK;
    for (void *p : c->allocs) cudaFree(p);
    delete c;
    return OSLALM_OK;
}

long oslalm_cnn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int oslalm_cnn_set_tma(oslalm_cnn *c, int enable) {
    clear_error();
    if (!c) return fail(OSLALM_ERR_ARG, "network handle is NULL");
    c->use_tma = enable != 0;
    return OSLALM_OK;
}

int oslalm_cnn_mark_timeout(oslalm_cnn *c) {
    clear_error();
    if (!c) return fail(OSLALM_ERR_ARG, "network handle is NULL");
    const int one = 1;
    OSL_CUDA_TRY(cudaMemcpy(c->err, &one, sizeof(int), cudaMemcpyHostToDevice));
    return OSLALM_OK;
}

int oslalm_cnn_get_params(oslalm_cnn *c, float *host) {
    clear_error();
    if (!c || !host) return fail(OSLALM_ERR_ARG, "NULL argument");
    std::vector<float> h(c->nparam);
    OSL_CUDA_TRY(cudaMemcpy(h.data(), c->w32, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost));
    if (int rc = check_waits(c)) return rc;
    copy_params(c, h, host, true);
    return OSLALM_OK;
}

int oslalm_cnn_set_params(oslalm_cnn *c, const float *host) {
    clear_error();
    if (!c || !host) return fail(OSLALM_ERR_ARG, "NULL argument");
    std::vector<float> h(c->nparam, 0.f);
    copy_params(c, h, const_cast<float *>(host), false);
    OSL_CUDA_TRY(cudaMemcpy(c->w32, h.data(), sizeof(float) * c->nparam, cudaMemcpyHostToDevice));
    OSL_CUDA_TRY(cudaMemset(c->m, 0, sizeof(float) * c->nparam));
    OSL_CUDA_TRY(cudaMemset(c->v, 0, sizeof(float) * c->nparam));
    c->step = 0;
    if (int rc = refresh_weights(c, nullptr)) return rc;
    OSL_CUDA_TRY(cudaDeviceSynchronize());
    return OSLALM_OK;
}

int oslalm_cnn_forward(oslalm_cnn *c, const float *x, float *y, int n, float scale, void *stream) {
    clear_error();
    if (int rc = check_n(c, n)) return rc;
    if (!x || !y || !(scale > 0)) return fail(OSLALM_ERR_ARG, "bad forward arguments");
    return run_forward(c, x, nullptr, scale, y, (cudaStream_t)stream);
}

int oslalm_cnn_gradients(oslalm_cnn *c, const float *x, const float *t, int n, float scale, float *grad_host,
                         double *loss, void *stream) {
    clear_error();
    if (int rc = check_n(c, n)) return rc;
    if (!x || !t || !(scale > 0)) return fail(OSLALM_ERR_ARG, "bad gradient arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = run_forward(c, x, t, scale, nullptr, st)) return rc;
    if (int rc = backward_net(c, st)) return rc;
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    if (int rc = check_waits(c)) return rc;
    if (loss) {
        double l;
        OSL_CUDA_TRY(cudaMemcpy(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost));
        *loss = l / (double)c->P[0];
    }
    if (grad_host) {
        std::vector<float> h(c->nparam);
        OSL_CUDA_TRY(cudaMemcpy(h.data(), c->grad, sizeof(float) * c->nparam, cudaMemcpyDeviceToHost));
        copy_params(c, h, grad_host, true);
    }
    return OSLALM_OK;
}

int oslalm_cnn_train_step(oslalm_cnn *c, const float *x, const float *t, int n, float scale, float lr, double *loss,
                          void *stream) {
    clear_error();
    if (int rc = check_n(c, n)) return rc;
    if (!x || !t || !(scale > 0) || !(lr > 0)) return fail(OSLALM_ERR_ARG, "bad train arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = run_forward(c, x, t, scale, nullptr, st)) return rc;
    if (int rc = backward_net(c, st)) return rc;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)c->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)c->step)));
    adam_kernel<<<nb(c->nparam, 256), 256, 0, st>>>(c->w32, c->grad, c->m, c->v, c->nparam, lr, b1, b2, 1e-8f, c1, c2);
    note_launch();
    OSL_LAUNCH_CHECK("adam_kernel");
    if (int rc = refresh_weights(c, st)) return rc;
    if (loss) {
        double l;
        OSL_CUDA_TRY(cudaMemcpyAsync(&l, c->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        OSL_CUDA_TRY(cudaStreamSynchronize(st));
        if (int rc = check_waits(c)) return rc;
        *loss = l / (double)c->P[0];
    }
    return OSLALM_OK;
}

double oslalm_cnn_flops_per_image(int height, int width) {
    double f = 0.0;
    const int lvl[NL] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
    for (int L = 0; L < NL; ++L)
        f += 2.0 * 9.0 * kLayers[L].cin_real * kLayers[L].cout * (double)(height >> lvl[L]) * (width >> lvl[L]);
    return f + 2.0 * 32.0 * height * width;
}

}  // extern "C"
