// Filtered back-projection for the initial image (set-up, not the hot path).
//
// The paper starts from an FBP image without specifying it (Sec. V); this is
// the textbook analytic reconstruction: Ram-Lak filtered parallel-beam FBP,
// equiangular fan-beam FBP over 360 degrees, and Feldkamp (FDK) for the flat
// cone-beam detector (Kak & Slaney, ch. 3).
//   1. fbp_filter_kernel: one block per detector row; the weighted row is
//      staged in shared memory and convolved with the (odd-tap) kernel.
//   2. fbp_bp2d_kernel / fbp_bp3d_kernel: pixel-driven back-projection with
//      linear (bilinear for FDK) interpolation and distance weights.
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels_common.cuh"

namespace oslalm {

struct FbpGeo {
    int kind, nx, ny, nz, nviews, ns, nt;
    float dx, dy, dz, xc0, yc0, zc0;  // pixel size, centre of pixel 0
    float ds, dt, c0, t0;             // detector pitch, channel/row coordinate of s = 0 / t = 0
    float dso, dsd;
    float a;                          // fan: channel angle pitch ds/dsd; cone: isocentre pitch ds*dso/dsd
    float az;                         // cone: isocentre row pitch
    float scale;                      // final factor
};

__global__ void fbp_filter_kernel(FbpGeo g, const float *__restrict__ sino, float *__restrict__ q) {
    extern __shared__ float sh[];
    float *row = sh;             // [ns]
    float *taps = sh + g.ns;     // [2 ns - 1], index k + ns - 1
    const int line = blockIdx.x;  // view * nt + t
    const int t = line % g.nt;
    const float *src = sino + (size_t)line * g.ns;
    for (int c = threadIdx.x; c < g.ns; c += blockDim.x) {
        float s = ((float)c - g.c0);  // channel offset from s = 0
        float v = src[c];
        if (g.kind == OSLALM_FAN2D_ARC) {
            v *= g.dso * cosf(s * g.a);
        } else if (g.kind == OSLALM_CONE3D_FLAT) {
            float p = s * g.a, z = ((float)t - g.t0) * g.az;
            v *= g.dso * rsqrtf(g.dso * g.dso + p * p + z * z);
        }
        row[c] = v;
    }
    for (int k = threadIdx.x; k < 2 * g.ns - 1; k += blockDim.x) {
        int n = k - (g.ns - 1);
        float h = 0.f;
        if (g.kind == OSLALM_FAN2D_ARC) {
            if (n == 0) h = 1.f / (8.f * g.a * g.a);
            else if (n & 1) {
                float sn = sinf((float)n * g.a);
                h = -1.f / (2.f * 9.8696044010893586f * sn * sn);
            }
        } else {
            float d = g.kind == OSLALM_PAR2D ? g.ds : g.a;
            if (n == 0) h = 1.f / (4.f * d * d);
            else if (n & 1) h = -1.f / (9.8696044010893586f * (float)n * (float)n * d * d);
        }
        taps[k] = h;
    }
    __syncthreads();
    const float pitch = g.kind == OSLALM_PAR2D ? g.ds : g.a;
    for (int c = threadIdx.x; c < g.ns; c += blockDim.x) {
        float acc = taps[g.ns - 1] * row[c];
        // odd offsets only: k = c - n with n odd
        for (int k = (c & 1) ? 0 : 1; k < g.ns; k += 2) acc = fmaf(taps[c - k + g.ns - 1], row[k], acc);
        q[(size_t)line * g.ns + c] = pitch * acc;
    }
}

__device__ __forceinline__ float lerp_row(const float *__restrict__ r, int ns, float c) {
    float cf = floorf(c);
    int i = (int)cf;
    float f = c - cf;
    float v0 = (i >= 0 && i < ns) ? __ldg(r + i) : 0.f;
    float v1 = (i + 1 >= 0 && i + 1 < ns) ? __ldg(r + i + 1) : 0.f;
    return (1.f - f) * v0 + f * v1;
}

__global__ void fbp_bp2d_kernel(FbpGeo g, const View2 *__restrict__ views, const float *__restrict__ q,
                                float *__restrict__ x, int clip) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
    if (ix >= g.nx || iy >= g.ny) return;
    const float px = g.xc0 + ix * g.dx, py = g.yc0 + iy * g.dy;
    float acc = 0.f;
    for (int v = 0; v < g.nviews; ++v) {
        const View2 vw = views[v];
        const float *qr = q + (size_t)v * g.ns;
        if (g.kind == OSLALM_PAR2D) {
            float s = -px * vw.su + py * vw.cu;
            acc += lerp_row(qr, g.ns, s / g.ds + g.c0);
        } else {
            float A = px * vw.cu + py * vw.su + g.dso;
            float B = -px * vw.su + py * vw.cu;
            float gp = atan2f(B, A);
            acc += lerp_row(qr, g.ns, gp / g.a + g.c0) / (A * A + B * B);
        }
    }
    float val = g.scale * acc;
    x[(size_t)iy * g.nx + ix] = clip ? fmaxf(val, 0.f) : val;
}

__global__ void fbp_bp3d_kernel(FbpGeo g, const View2 *__restrict__ views, const float *__restrict__ q,
                                float *__restrict__ x, int clip) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const float px = g.xc0 + ix * g.dx, py = g.yc0 + iy * g.dy, pz = g.zc0 + iz * g.dz;
    float acc = 0.f;
    for (int v = 0; v < g.nviews; ++v) {
        const View2 vw = views[v];
        float A = px * vw.cu + py * vw.su + g.dso;
        float B = -px * vw.su + py * vw.cu;
        float U = A / g.dso;
        float pc = (g.dso * B / A) / g.a + g.c0;
        float tc = (g.dso * pz / A) / g.az + g.t0;
        float tf = floorf(tc);
        int ti = (int)tf;
        float ft = tc - tf;
        const float *base = q + (size_t)v * g.nt * g.ns;
        float v0 = (ti >= 0 && ti < g.nt) ? lerp_row(base + (size_t)ti * g.ns, g.ns, pc) : 0.f;
        float v1 = (ti + 1 >= 0 && ti + 1 < g.nt) ? lerp_row(base + (size_t)(ti + 1) * g.ns, g.ns, pc) : 0.f;
        acc += ((1.f - ft) * v0 + ft * v1) / (U * U);
    }
    float val = g.scale * acc;
    x[((size_t)iz * g.ny + iy) * g.nx + ix] = clip ? fmaxf(val, 0.f) : val;
}

}  // namespace oslalm

namespace oslalm {

constexpr int kFbpMaxChannels = 8192;
constexpr size_t kFbpFilterMaxShm = sizeof(float) * (3 * (size_t)kFbpMaxChannels - 1);

// Checks the geometry, then filters sino into q (nviews*nt*ns floats of
// device memory owned by the caller) and back-projects q into x, on `st`.
static int fbp_run(const oslalm_geom *gm, const float *sino, float *x, int clip_nonneg, float *q, cudaStream_t st) {
    const oslalm_geom_desc &d = gm->d;
    FbpGeo g;
    g.kind = d.kind;
    g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.nviews = d.nviews; g.ns = d.ns; g.nt = d.nt;
    g.dx = (float)d.dx; g.dy = (float)d.dy; g.dz = (float)d.dz;
    g.xc0 = (float)(d.offset_x - (d.nx - 1) / 2.0 * d.dx);
    g.yc0 = (float)(d.offset_y - (d.ny - 1) / 2.0 * d.dy);
    g.zc0 = (float)(d.offset_z - (d.nz - 1) / 2.0 * d.dz);
    g.ds = (float)d.ds; g.dt = (float)d.dt;
    g.c0 = (float)((d.ns - 1) / 2.0 - d.offset_s);
    g.t0 = (float)((d.nt - 1) / 2.0 - d.offset_t);
    g.dso = (float)d.dso; g.dsd = (float)d.dsd;
    g.a = d.kind == OSLALM_FAN2D_ARC ? (float)(d.ds / d.dsd) : (float)(d.ds * d.dso / d.dsd);
    g.az = (float)(d.dt * d.dso / d.dsd);
    if (d.kind == OSLALM_PAR2D) g.scale = (float)(M_PI / d.nviews);
    else if (d.kind == OSLALM_FAN2D_ARC) g.scale = (float)(2.0 * M_PI / d.nviews);
    else g.scale = (float)(0.5 * 2.0 * M_PI / d.nviews);
    const size_t shm = sizeof(float) * (3 * (size_t)d.ns - 1);
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fbp_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFbpFilterMaxShm);
        if (e != cudaSuccess) return fail(OSLALM_ERR_CUDA, "FBP filter set-up failed: %s", cudaGetErrorString(e));
    }
    fbp_filter_kernel<<<d.nviews * d.nt, 256, shm, st>>>(g, sino, q);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        dim3 block(32, 8), grid((d.nx + 31) / 32, (d.ny + 7) / 8, d.kind == OSLALM_CONE3D_FLAT ? d.nz : 1);
        if (d.kind == OSLALM_CONE3D_FLAT) fbp_bp3d_kernel<<<grid, block, 0, st>>>(g, gm->d_views, q, x, clip_nonneg);
        else fbp_bp2d_kernel<<<grid, block, 0, st>>>(g, gm->d_views, q, x, clip_nonneg);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(OSLALM_ERR_CUDA, "FBP launch failed: %s", cudaGetErrorString(e));
    return OSLALM_OK;
}

static int fbp_check(const oslalm_geom *gm, const float *sino, const float *x) {
    if (!gm || !sino || !x) return fail(OSLALM_ERR_ARG, "NULL argument");
    const oslalm_geom_desc &d = gm->d;
    if (d.kind != OSLALM_PAR2D && fabs(fabs(d.angle_span) - 2.0 * M_PI) > 1e-9)
        return fail(OSLALM_ERR_ARG, "fan/cone FBP needs a full 360-degree scan");
    if (d.pitch != 0.0) return fail(OSLALM_ERR_ARG, "FDK needs a circular orbit (pitch 0)");
    if (d.ns > kFbpMaxChannels) return fail(OSLALM_ERR_RANGE, "FBP supports at most %d channels", kFbpMaxChannels);
    return OSLALM_OK;
}

}  // namespace oslalm

using namespace oslalm;

extern "C" int oslalm_fbp(const oslalm_geom *gm, const float *sino, float *x, int clip_nonneg, void *stream) {
    clear_error();
    if (int rc = fbp_check(gm, sino, x)) return rc;
    const oslalm_geom_desc &d = gm->d;
    cudaStream_t st = (cudaStream_t)stream;
    size_t nq = (size_t)d.nviews * d.nt * d.ns;
    float *q = nullptr;
    OSL_CUDA_TRY(cudaMallocAsync((void **)&q, nq * sizeof(float), st));
    const int rc = fbp_run(gm, sino, x, clip_nonneg, q, st);
    cudaFreeAsync(q, st);
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free FBP.  Some callers cannot allocate device memory while they
// run: a service that hands the whole GPU to its own pre-sized memory pool at
// start-up, or a real-time pipeline that forbids allocation after
// initialisation because cudaMalloc may synchronize the device and its
// latency is unbounded.  oslalm_fbp_noalloc does the same work as oslalm_fbp
// but keeps the filtered sinogram in the fixed buffer below, which the
// library owns on every device where it has been prepared, for the life of
// the process.
//
// The buffer lives in this file's own device module.  The CUDA runtime loads
// a module on a device the first time something in it is used there (lazy
// loading), and that is when the buffer's 16 MiB are reserved.
// oslalm_fbp_noalloc_prepare does that loading (and loads the FBP kernels'
// code) on purpose, so that a caller can do it at start-up, before it
// reserves its own pool.
namespace oslalm {

constexpr size_t kFbpStaticFloats = (size_t)1 << 22;  // 16 MiB of FP32 samples
static __device__ __align__(256) float g_fbp_scratch[kFbpStaticFloats];

static std::mutex g_fbp_scratch_mutex;
static float *g_fbp_scratch_ptr[64] = {nullptr};

// Device address of g_fbp_scratch on the current device, looked up once per
// device with that device current (host code cannot use the symbol itself:
// on the host it names a stand-in object, not device memory).  The first
// lookup on a device also loads the FBP kernels there.
static int fbp_scratch_address(float **out) {
    int dev = 0;
    OSL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(OSLALM_ERR_RANGE, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_fbp_scratch_mutex);
    if (!g_fbp_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fbp_scratch);
        if (e != cudaSuccess || !p)
            return fail(OSLALM_ERR_CUDA, "cudaGetSymbolAddress(g_fbp_scratch) failed: %s", cudaGetErrorString(e));
        cudaFuncAttributes a;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, fbp_filter_kernel);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, fbp_bp2d_kernel);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, fbp_bp3d_kernel);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fbp_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kFbpFilterMaxShm);
        if (e != cudaSuccess) return fail(OSLALM_ERR_CUDA, "loading the FBP kernels failed: %s", cudaGetErrorString(e));
        g_fbp_scratch_ptr[dev] = (float *)p;
    }
    *out = g_fbp_scratch_ptr[dev];
    return OSLALM_OK;
}

}  // namespace oslalm

extern "C" int oslalm_fbp_noalloc_prepare(void) {
    clear_error();
    float *q = nullptr;
    return fbp_scratch_address(&q);
}

extern "C" int oslalm_fbp_noalloc(const oslalm_geom *gm, const float *sino, float *x, int clip_nonneg,
                                  void *stream) {
    clear_error();
    if (int rc = fbp_check(gm, sino, x)) return rc;
    const oslalm_geom_desc &d = gm->d;
    const size_t nq = (size_t)d.nviews * d.nt * d.ns;
    if (nq > kFbpStaticFloats)
        return fail(OSLALM_ERR_RANGE,
                    "oslalm_fbp_noalloc: sinogram has %zu samples, the static buffer holds at most %zu "
                    "(use oslalm_fbp)", nq, kFbpStaticFloats);
    float *q = nullptr;
    if (int rc = fbp_scratch_address(&q)) return rc;
    // every filtered sample is written before it is read, so the buffer's
    // previous contents (left by the last call) need no clearing
    return fbp_run(gm, sino, x, clip_nonneg, q, (cudaStream_t)stream);
}
