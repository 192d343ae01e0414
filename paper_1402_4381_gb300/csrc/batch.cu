// Batched OS-LALM: many independent 2D scans (uneven image sizes, view counts
// and subset counts) advanced together.  Every subset-iteration step is four
// persistent launches, each a grid of resident blocks that walks a work list
// covering all scans still running:
//   1. update   (tiles of every scan's image)      x+ = SQS step (Sec. IV-A)
//   2. forward  (groups of rays of every scan's next subset)  r = M W (A x+ - y)
//   3. back-proj(16x16 tiles)  zeta+ = A' r, g+, per-tile restart-indicator partials
//   4. finish   (one block per scan)  xi, l, rho_l (Sec. III-B), in a fixed order
// The per-scan arithmetic is the single-problem code (proj2d.cuh), so with
// the default launch shape a batched scan is bit-identical to the same scan
// iterated alone.  Whole calls are captured into a CUDA graph.  The launch
// shape (image tile, lanes per ray, blocks per SM) is picked by a timing
// autotuner.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels_common.cuh"
#include "proj2d.cuh"
#include "problem.cuh"

namespace oslalm {

constexpr int kMaxSlices = 1024;

struct SliceDesc {
    Geo2 geo;
    float *x, *xalt, *r;
    const void *D;
    const float *dscale;
    int d_dtype;
    const float *y;
    const void *w;
    const float *wscale;
    int w_dtype;
    const int *views, *off, *cnt, *order;
    int M, nsteps, nbr, curv;
    float beta, inv_delta, gain;
    UpdateArgs ua;
};

struct BatchShape {
    int tx, ty, lanes;
};
static const BatchShape kShapes[] = {{32, 8, 8}, {16, 16, 4}, {32, 8, 4}, {16, 16, 8}, {64, 4, 2}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

__device__ __forceinline__ bool slice_active(const SliceDesc &d, int step) { return step < d.nsteps; }

template <int TX, int TY>
__device__ __forceinline__ int slice_tiles(const SliceDesc &d) {
    return ((d.geo.nx + TX - 1) / TX) * ((d.geo.ny + TY - 1) / TY);
}

// prefix sums of per-scan item counts into shared memory (one thread; n is small)
template <typename F>
__device__ __forceinline__ int work_prefix(const SliceDesc *S, int n, int step, F count, int *pre) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int s = 0; s < n; ++s) {
            pre[s] = acc;
            acc += slice_active(S[s], step) ? count(S[s]) : 0;
        }
        pre[n] = acc;
    }
    __syncthreads();
    return pre[n];
}

__device__ __forceinline__ int find_slice(const int *pre, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {  // largest s with pre[s] <= item
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int TX, int TY>
__global__ void __launch_bounds__(256) batch_update_kernel(const SliceDesc *__restrict__ S, int n, int step) {
    __shared__ int pre[kMaxSlices + 1];
    __shared__ float tile[(TX + 2) * (TY + 2)];
    const int total = work_prefix(S, n, step, [](const SliceDesc &d) { return slice_tiles<TX, TY>(d); }, pre);
    const int tid = threadIdx.x;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int s = find_slice(pre, n, item);
        const SliceDesc &d = S[s];
        const int t = item - pre[s];
        const int ntx = (d.geo.nx + TX - 1) / TX;
        const int ix0 = (t % ntx) * TX, iy0 = (t / ntx) * TY;
        const float *xin = (step & 1) ? d.xalt : d.x;
        float *xout = (step & 1) ? d.x : d.xalt;
        const float rho = d.ua.state->rho_f;
        const float rho_d = d.ua.state->rho_d_f;
#define OSL_BUPD(DT, N)                                                                                          \
    update_tile<TX, TY, DT, N>(tile, ix0, iy0, tid % TX, tid / TX, tid, 256, d.geo.nx, d.geo.ny, xin, xout,     \
                               d.ua.zeta, d.ua.g, (const DT *)d.D, d.dscale, rho, rho_d, d.beta, d.inv_delta, d.curv)
        if (d.nbr == 8) {
            if (d.d_dtype == OSLALM_F32) OSL_BUPD(float, 8);
            else if (d.d_dtype == OSLALM_F16) OSL_BUPD(__half, 8);
            else OSL_BUPD(__nv_bfloat16, 8);
        } else {
            if (d.d_dtype == OSLALM_F32) OSL_BUPD(float, 4);
            else if (d.d_dtype == OSLALM_F16) OSL_BUPD(__half, 4);
            else OSL_BUPD(__nv_bfloat16, 4);
        }
#undef OSL_BUPD
        __syncthreads();  // the tile buffer is reused by the next item
    }
}

template <int LANES>
__global__ void __launch_bounds__(256) batch_forward_kernel(const SliceDesc *__restrict__ S, int n, int step) {
    constexpr int RPB = 256 / LANES;  // rays per block
    constexpr int RPW = 32 / LANES;   // rays per warp
    __shared__ int pre[kMaxSlices + 1];
    const int total = work_prefix(
        S, n, step,
        [step](const SliceDesc &d) {
            const int next = d.order[(step + 1) % d.M];
            return (d.cnt[next] * d.geo.ns + RPB - 1) / RPB;
        },
        pre);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane / RPW;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int s = find_slice(pre, n, item);
        const SliceDesc &d = S[s];
        const int next = d.order[(step + 1) % d.M];
        const int nv = d.cnt[next];
        const int ray = (item - pre[s]) * RPB + warp * RPW + lane % RPW;
        const bool valid = ray < nv * d.geo.ns;
        const float *xcur = (step & 1) ? d.x : d.xalt;  // the updated image
        float acc = 0.f;
        if (valid) {
            const int lv = ray / d.geo.ns, c = ray - lv * d.geo.ns;
            const int v = __ldg(d.views + d.off[next] + lv);
            const RayP rp = d.geo.rays[(size_t)v * d.geo.ns + c];
            acc = march2<float>(d.geo, rp, xcur, q, LANES);
        }
#pragma unroll
        for (int o = RPW; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (valid && q == 0) {
            const size_t base = (size_t)d.off[next] * d.geo.ns;
            float wv;
            if (d.w_dtype == OSLALM_F32) wv = load_w((const float *)d.w, base + ray);
            else if (d.w_dtype == OSLALM_F16) wv = load_w((const __half *)d.w, base + ray);
            else wv = load_w((const __nv_bfloat16 *)d.w, base + ray);
            wv *= __ldg(d.wscale);
            d.r[ray] = d.gain * wv * (acc - __ldg(d.y + base + ray));
        }
    }
}

// Back-projection tiles of every scan: the single-problem tile code
// (bp_tile_strips, same tiles and summation order), then the split-gradient
// update and the tile's restart-indicator partial.
__global__ void __launch_bounds__(kBpThreads, 8) batch_backproject_kernel(const SliceDesc *__restrict__ S, int n,
                                                                       int step) {
    __shared__ int pre[kMaxSlices + 1];
    __shared__ float red[64];
    __shared__ BpTileAcc acc;
    const int total =
        work_prefix(S, n, step, [](const SliceDesc &d) { return slice_tiles<kBpTile, kBpTile>(d); }, pre);
    const int tid = threadIdx.x;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int s = find_slice(pre, n, item);
        const SliceDesc &d = S[s];
        const int t = item - pre[s];
        const int ntx = (d.geo.nx + kBpTile - 1) / kBpTile;
        const int tx0 = (t % ntx) * kBpTile, ty0 = (t / ntx) * kBpTile;
        const int next = d.order[(step + 1) % d.M];
        bp_tile_strips(d.geo, d.r, d.views + d.off[next], d.cnt[next], tx0, ty0, tid, acc);
        __syncthreads();
        const int px = tid % kBpTile, py = tid / kBpTile;
        const int ix = tx0 + px, iy = ty0 + py;
        double xi_local = 0.0;
        if (ix < d.geo.nx && iy < d.geo.ny) {
            const float v = bp_tile_total(acc, px, py);
            const size_t p = (size_t)iy * d.geo.nx + ix;
            const float a = d.ua.state->ga, b = d.ua.state->gb;
            const float z_old = d.ua.zeta[p];
            const float g_old = d.ua.g[p];
            d.ua.zeta[p] = v;
            d.ua.g[p] = a * v + b * g_old;
            xi_local = (double)(g_old - v) * (double)(v - z_old);
        }
        const double bs = block_sum_df(xi_local, red);  // ends with a barrier: acc is free again
        if (tid == 0) d.ua.partials[t] = bs;
    }
}

// One block per scan: the restart test and the continuation (Sec. III-B).
template <int TX, int TY>
__global__ void __launch_bounds__(256) batch_finish_kernel(const SliceDesc *__restrict__ S, int n, int step) {
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const SliceDesc &d = S[s];
        if (!slice_active(d, step)) continue;
        UpdateArgs ua = d.ua;
        ua.subset = d.order[(step + 1) % d.M];
        finish_subset_iteration(ua, slice_tiles<kBpTile, kBpTile>(d));
        __syncthreads();
    }
}

}  // namespace oslalm

using namespace oslalm;

struct oslalm_batch {
    int n = 0;
    std::vector<oslalm_problem *> probs;
    std::vector<SliceDesc> h;
    SliceDesc *d = nullptr;
    int *d_ints = nullptr;  // off / cnt / order of every scan
    int shape = 0;          // index into kShapes
    int blocks_per_sm = 0;  // 0: occupancy maximum
    int num_sms = 0;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const float *> g_x;
    int g_iters = -1, g_shape = -1, g_bps = -1;
};

namespace {

template <int TX, int TY, int LANES>
int launch_step(const oslalm_batch *b, int step, int grid_upd, int grid_fp, int grid_bp, cudaStream_t st) {
    batch_update_kernel<TX, TY><<<grid_upd, 256, 0, st>>>(b->d, b->n, step);
    batch_forward_kernel<LANES><<<grid_fp, 256, 0, st>>>(b->d, b->n, step);
    batch_backproject_kernel<<<grid_bp, kBpThreads, 0, st>>>(b->d, b->n, step);
    batch_finish_kernel<TX, TY><<<std::min(b->n, 4096), 256, 0, st>>>(b->d, b->n, step);
    OSL_LAUNCH_CHECK("batch step");
    return OSLALM_OK;
}

template <int TX, int TY, int LANES>
int grid_sizes(const oslalm_batch *b, int &gu, int &gf, int &gb) {
    int ou = 0, of = 0, ob = 0;
    OSL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ou, batch_update_kernel<TX, TY>, 256, 0));
    OSL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, batch_forward_kernel<LANES>, 256, 0));
    OSL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, batch_backproject_kernel, kBpThreads, 0));
    auto pick = [&](int occ) {
        int per = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, std::max(occ, 1)) : std::max(occ, 1);
        return b->num_sms * per;
    };
    gu = pick(ou);
    gf = pick(of);
    gb = pick(ob);
    return OSLALM_OK;
}

int run_step(const oslalm_batch *b, int shape, int step, cudaStream_t st) {
    int gu, gf, gb, rc;
    switch (shape) {
        case 0: if ((rc = grid_sizes<32, 8, 8>(b, gu, gf, gb))) return rc; return launch_step<32, 8, 8>(b, step, gu, gf, gb, st);
        case 1: if ((rc = grid_sizes<16, 16, 4>(b, gu, gf, gb))) return rc; return launch_step<16, 16, 4>(b, step, gu, gf, gb, st);
        case 2: if ((rc = grid_sizes<32, 8, 4>(b, gu, gf, gb))) return rc; return launch_step<32, 8, 4>(b, step, gu, gf, gb, st);
        case 3: if ((rc = grid_sizes<16, 16, 8>(b, gu, gf, gb))) return rc; return launch_step<16, 16, 8>(b, step, gu, gf, gb, st);
        default: if ((rc = grid_sizes<64, 4, 2>(b, gu, gf, gb))) return rc; return launch_step<64, 4, 2>(b, step, gu, gf, gb, st);
    }
}

// refresh the per-scan descriptors (caller's x, steps of this call, the
// problems' current stats / replay buffers) and upload them on `st`
int upload_desc(oslalm_batch *b, float *const *x, int n_iter, cudaStream_t st, int *max_steps_out) {
    int max_steps = 0;
    for (int s = 0; s < b->n; ++s) {
        SliceDesc &h = b->h[s];
        const oslalm_problem *p = b->probs[s];
        h.x = x[s];
        h.nsteps = n_iter * h.M;
        h.ua.stats = p->d_stats;
        h.ua.stats_cap = p->stats_cap;
        h.ua.replay = p->d_replay;
        h.ua.replay_n = p->replay_n;
        max_steps = std::max(max_steps, h.nsteps);
    }
    OSL_CUDA_TRY(cudaMemcpyAsync(b->d, b->h.data(), sizeof(SliceDesc) * b->n, cudaMemcpyHostToDevice, st));
    *max_steps_out = max_steps;
    return OSLALM_OK;
}

// the steps of one call (capturable: kernel launches and device copies only)
int launch_steps(const oslalm_batch *b, int max_steps, cudaStream_t st) {
    for (int step = 0; step < max_steps; ++step)
        if (int rc = run_step(b, b->shape, step, st)) return rc;
    for (int s = 0; s < b->n; ++s) {
        const SliceDesc &h = b->h[s];
        if (h.nsteps & 1)
            OSL_CUDA_TRY(cudaMemcpyAsync(h.x, h.xalt, sizeof(float) * h.geo.nx * h.geo.ny, cudaMemcpyDeviceToDevice, st));
    }
    return OSLALM_OK;
}

int run_batch(oslalm_batch *b, float *const *x, int n_iter, cudaStream_t st) {
    int max_steps = 0;
    if (int rc = upload_desc(b, x, n_iter, st, &max_steps)) return rc;
    return launch_steps(b, max_steps, st);
}

void drop_graph(oslalm_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->g_iters = -1;
}

}  // namespace

extern "C" {

int oslalm_batch_create(oslalm_problem *const *probs, int n, oslalm_batch **out) {
    clear_error();
    if (!out) return fail(OSLALM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!probs || n <= 0 || n > kMaxSlices) return fail(OSLALM_ERR_ARG, "need 1..%d problems", kMaxSlices);
    for (int s = 0; s < n; ++s) {
        const oslalm_problem *p = probs[s];
        if (!p) return fail(OSLALM_ERR_ARG, "problem %d is NULL", s);
        if (is_3d(p->g)) return fail(OSLALM_ERR_ARG, "batches hold 2D problems only (problem %d)", s);
        if (!p->initialized) return fail(OSLALM_ERR_STATE, "problem %d: call oslalm_init first", s);
        if (p->p.n_inner != 1) return fail(OSLALM_ERR_ARG, "problem %d: batches run n_inner = 1", s);
        if (p->p.bb) return fail(OSLALM_ERR_ARG, "problem %d: batches run without Barzilai-Borwein scaling", s);
        if (p->j_host % p->p.M) return fail(OSLALM_ERR_STATE, "problem %d is not at a whole iteration", s);
    }
    oslalm_batch *b = new (std::nothrow) oslalm_batch();
    if (!b) return fail(OSLALM_ERR_ALLOC, "host allocation failed");
    b->n = n;
    b->probs.assign(probs, probs + n);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<int> ints;
    std::vector<size_t> at(n);
    for (int s = 0; s < n; ++s) {
        const oslalm_problem *p = probs[s];
        at[s] = ints.size();
        ints.insert(ints.end(), p->off.begin(), p->off.end());
        ints.insert(ints.end(), p->cnt.begin(), p->cnt.end());
        ints.insert(ints.end(), p->order.begin(), p->order.end());
    }
    cudaError_t e = cudaMalloc(&b->d_ints, sizeof(int) * ints.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d, sizeof(SliceDesc) * n);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->d_ints);
        cudaFree(b->d);
        delete b;
        return fail(OSLALM_ERR_ALLOC, "batch allocation failed: %s", cudaGetErrorString(e));
    }
    b->h.resize(n);
    for (int s = 0; s < n; ++s) {
        oslalm_problem *p = probs[s];
        SliceDesc &h = b->h[s];
        memset(&h, 0, sizeof(h));
        h.geo = p->g->geo2();
        h.xalt = p->d_xalt;
        h.r = p->d_r;
        h.D = p->d_D;
        h.dscale = p->d_dscale;
        h.d_dtype = p->p.d_dtype;
        h.y = p->d_y;
        h.w = p->d_w;
        h.wscale = p->d_wscale;
        h.w_dtype = p->p.w_dtype;
        h.views = p->d_views;
        const int M = p->p.M;
        h.off = b->d_ints + at[s];
        h.cnt = b->d_ints + at[s] + M;
        h.order = b->d_ints + at[s] + 2 * M;
        h.M = M;
        h.nbr = p->p.nbr;
        h.curv = p->p.curvature;
        h.beta = (float)p->p.beta;
        h.inv_delta = (float)(1.0 / p->p.delta);
        h.gain = (float)M;
        UpdateArgs &a = h.ua;
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
        a.rho_tab = p->d_rho_tab;
        a.rho_tab_n = p->rho_tab_n;
    }
    *out = b;
    return OSLALM_OK;
}

int oslalm_batch_destroy(oslalm_batch *b) {
    clear_error();
    if (!b) return OSLALM_OK;
    drop_graph(b);
    cudaFree(b->d);
    cudaFree(b->d_ints);
    delete b;
    return OSLALM_OK;
}

int oslalm_batch_iterate(oslalm_batch *b, float *const *x, int n_iter, int use_graph, void *stream) {
    clear_error();
    if (!b || !x || n_iter < 0) return fail(OSLALM_ERR_ARG, "bad batch iterate arguments");
    if (n_iter == 0) return OSLALM_OK;
    for (int s = 0; s < b->n; ++s)
        if (!x[s]) return fail(OSLALM_ERR_ARG, "x[%d] is NULL", s);
    cudaStream_t st = (cudaStream_t)stream;
    int max_steps = 0;
    if (int rc = upload_desc(b, x, n_iter, st, &max_steps)) return rc;
    if (use_graph) {
        bool same = b->gexec && b->g_iters == n_iter && b->g_shape == b->shape && b->g_bps == b->blocks_per_sm &&
                    (int)b->g_x.size() == b->n && std::equal(b->g_x.begin(), b->g_x.end(), x);
        if (!same) {
            drop_graph(b);
            cudaStream_t cs;
            OSL_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t graph;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaStreamDestroy(cs);
                return fail(OSLALM_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
            }
            int rc = launch_steps(b, max_steps, cs);
            e = cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            if (rc) return rc;
            if (e != cudaSuccess) return fail(OSLALM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->gexec = nullptr;
                return fail(OSLALM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
            b->g_x.assign(x, x + b->n);
            b->g_iters = n_iter;
            b->g_shape = b->shape;
            b->g_bps = b->blocks_per_sm;
        }
        OSL_CUDA_TRY(cudaGraphLaunch(b->gexec, st));
    } else {
        if (int rc = launch_steps(b, max_steps, st)) return rc;
    }
    for (int s = 0; s < b->n; ++s) b->probs[s]->j_host += (long)n_iter * b->probs[s]->p.M;
    return OSLALM_OK;
}

int oslalm_batch_set_shape(oslalm_batch *b, int shape, int blocks_per_sm) {
    clear_error();
    if (!b || shape < 0 || shape >= kNumShapes || blocks_per_sm < 0) return fail(OSLALM_ERR_ARG, "bad shape");
    b->shape = shape;
    b->blocks_per_sm = blocks_per_sm;
    return OSLALM_OK;
}

int oslalm_batch_shape_count(void) { return kNumShapes; }

int oslalm_batch_shape_info(int shape, int *tile_x, int *tile_y, int *lanes) {
    clear_error();
    if (shape < 0 || shape >= kNumShapes || !tile_x || !tile_y || !lanes) return fail(OSLALM_ERR_ARG, "bad shape");
    *tile_x = kShapes[shape].tx;
    *tile_y = kShapes[shape].ty;
    *lanes = kShapes[shape].lanes;
    return OSLALM_OK;
}

int oslalm_batch_autotune(oslalm_batch *b, float *const *x, int probe_iters, double *ms_out, void *stream) {
    clear_error();
    if (!b || !x || probe_iters <= 0) return fail(OSLALM_ERR_ARG, "bad autotune arguments");
    cudaStream_t st = (cudaStream_t)stream;
    // save the state of every scan, try every launch shape, restore
    std::vector<float *> save(b->n * 4, nullptr);
    std::vector<DevState> st_save(b->n);
    auto cleanup = [&]() {
        for (float *q : save) cudaFree(q);
    };
    for (int s = 0; s < b->n; ++s) {
        oslalm_problem *p = b->probs[s];
        size_t bytes = sizeof(float) * p->npix;
        const float *src[4] = {x[s], p->d_xalt, p->d_zeta, p->d_g};
        for (int k = 0; k < 4; ++k) {
            cudaError_t e = cudaMalloc(&save[4 * s + k], bytes);
            if (e == cudaSuccess) e = cudaMemcpyAsync(save[4 * s + k], src[k], bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) {
                cleanup();
                return fail(OSLALM_ERR_ALLOC, "autotune backup: %s", cudaGetErrorString(e));
            }
        }
        cudaMemcpyAsync(&st_save[s], p->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, st);
    }
    cudaStreamSynchronize(st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int old_shape = b->shape, old_bps = b->blocks_per_sm;
    double best = 1e300;
    int best_shape = old_shape, best_bps = old_bps;
    int rc = OSLALM_OK;
    const int bps_options[2] = {0, 2};
    for (int sh = 0; sh < kNumShapes && !rc; ++sh) {
        for (int bi = 0; bi < 2 && !rc; ++bi) {
            b->shape = sh;
            b->blocks_per_sm = bps_options[bi];
            rc = run_batch(b, x, 1, st);  // warm-up
            cudaEventRecord(e0, st);
            if (!rc) rc = run_batch(b, x, probe_iters, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms_out) ms_out[sh * 2 + bi] = ms;
            if (!rc && ms < best) {
                best = ms;
                best_shape = sh;
                best_bps = bps_options[bi];
            }
            // restore
            for (int s = 0; s < b->n; ++s) {
                oslalm_problem *p = b->probs[s];
                size_t bytes = sizeof(float) * p->npix;
                float *dst[4] = {x[s], p->d_xalt, p->d_zeta, p->d_g};
                for (int k = 0; k < 4; ++k) cudaMemcpyAsync(dst[k], save[4 * s + k], bytes, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(p->d_state, &st_save[s], sizeof(DevState), cudaMemcpyHostToDevice, st);
            }
            cudaStreamSynchronize(st);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    b->shape = rc ? old_shape : best_shape;
    b->blocks_per_sm = rc ? old_bps : best_bps;
    drop_graph(b);
    cudaError_t e = cudaGetLastError();
    if (!rc && e != cudaSuccess) rc = fail(OSLALM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    return rc;
}

int oslalm_batch_get_shape(const oslalm_batch *b, int *shape, int *blocks_per_sm) {
    clear_error();
    if (!b || !shape || !blocks_per_sm) return fail(OSLALM_ERR_ARG, "NULL argument");
    *shape = b->shape;
    *blocks_per_sm = b->blocks_per_sm;
    return OSLALM_OK;
}

}  // extern "C"
