// System matrix of a 2D geometry held in device memory.
//
// The projector pair evaluates every (ray, major row) length pair from the
// ray tables (row_weights).  For a 2D scan the whole matrix fits in HBM many
// times over (the 512^2 fan scan with 984 x 888 rays: ~4.7e8 row pairs,
// ~8 GB in the two layouts below), so it can be evaluated once, by the same
// device functions, and streamed afterwards:
//
//  forward layout  : ray-major, one 8-byte entry per row of the ray's row
//                    range (ray_rows), the first pixel of each row rebuilt
//                    from two step bits;
//  back-projection : per (view, ray orientation, 16x16 tile) an ELL block of
//                    32 lanes (the strips of bp_tile_strips), each lane's
//                    entries the rays that touch its strip, in channel order,
//                    with the first strip pixel rebuilt from two step bits.
//
// The table-driven kernels add the same products in the same order as the
// evaluating kernels, so both give the same bits (tested).  Layout details
// are in the Geo2 comment (common.cuh).
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "kernels_common.cuh"
#include "proj2d.cuh"

namespace oslalm {

namespace {

// ---------------------------------------------------------------- forward layout
__global__ void mat_fp_count_kernel(Geo2 g, unsigned *__restrict__ nrows) {
    const long ray = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long)g.nviews * g.ns) return;
    int ia0, ia1;
    ray_rows(g, g.rays[ray], ia0, ia1);
    nrows[ray] = ia1 >= ia0 ? (unsigned)(ia1 - ia0 + 1) : 0u;
}

__global__ void mat_fp_fill_kernel(Geo2 g, const unsigned *__restrict__ first, uint4 *__restrict__ hdr,
                                   uint2 *__restrict__ ent, int *__restrict__ err) {
    const long ray = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long)g.nviews * g.ns) return;
    const RayP rp = g.rays[ray];
    int ia0, ia1;
    ray_rows(g, rp, ia0, ia1);
    if (ia1 < ia0) {
        hdr[ray] = make_uint4(0u, 0u, 0u, (unsigned)rp.axis << 1);
        return;
    }
    const unsigned f = first[ray];
    const int ja = (int)row_weights(rp, (float)(2 * ia0 + 1), (float)ia0 + 0.5f).j;
    const int jz = (int)row_weights(rp, (float)(2 * ia1 + 1), (float)ia1 + 0.5f).j;
    const int dir = jz >= ja ? 1 : -1;
    int jprev = ja;
    bool bad = false;
    for (int ia = ia0; ia <= ia1; ++ia) {
        const RowW w = row_weights(rp, (float)(2 * ia + 1), (float)ia + 0.5f);
        const int j = (int)w.j;
        // 0 or 1 per row; 2 only where rounding meets an exactly 45-degree ray
        const int step = ia == ia0 ? 0 : (j - jprev) * dir;
        const unsigned b0 = __float_as_uint(w.w0), b1 = __float_as_uint(w.w1);
        bad |= step < 0 || step > 3 || (b0 >> 31) || (b1 >> 31);
        ent[(size_t)f + (ia - ia0)] = make_uint2(b0 | ((unsigned)(step & 1) << 31), b1 | ((unsigned)(step >> 1) << 31));
        jprev = j;
    }
    if (bad) atomicOr(err, 1);
    hdr[ray] = make_uint4(f, (unsigned)ia0 | ((unsigned)(ia1 - ia0 + 1) << 16), (unsigned)ja,
                          (dir < 0 ? 1u : 0u) | ((unsigned)rp.axis << 1));
}

// ---------------------------------------------------------------- back-projection layout
// One block per (tile, view), 64 threads: orientation = thread / 32, lane =
// thread mod 32 (the strip of bp_tile_strips).  Pass 0 counts each lane's
// touching rays (its first channel, first strip pixel and direction go to the
// lane header, the block's longest count to bp_blk.y); pass 1 writes them.
template <int PASS>
__global__ void __launch_bounds__(64) mat_bp_kernel(Geo2 g, unsigned *__restrict__ hdr, uint2 *__restrict__ blk,
                                                    uint2 *__restrict__ ent, int *__restrict__ err) {
    const int tile = blockIdx.x, v = blockIdx.y;
    const int ax = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntx = (g.nx + kBpTile - 1) / kBpTile;
    const size_t ntiles = (size_t)ntx * ((g.ny + kBpTile - 1) / kBpTile);
    const int tx0 = (tile % ntx) * kBpTile, ty0 = (tile / ntx) * kBpTile;
    const size_t b = ((size_t)v * 2 + ax) * ntiles + tile;
    const StripCtx sc = strip_ctx(g, ax, tx0, ty0, lane);
    int c0 = 0, c1 = -1;
    if (sc.valid) strip_channels(g, g.views[v], ax, sc, c0, c1);
    const RayP *rr = g.rays + (size_t)v * g.ns;
    if (PASS == 0) {
        int cnt = 0, cfirst = 0, dfirst = 0, dprev = 0, state = 0, dir = 0;
        bool bad = false;
        for (int c = c0; c <= c1; ++c) {
            const RowW w = row_weights(rr[c], sc.ia2, sc.iah);
            const int d = (int)__fsub_rn(w.j, sc.jbf);
            if (d >= -1 && d < kBpStrip) {  // the ray adds to strip pixel d or d + 1
                if (state == 2) bad = true;  // touching rays must be consecutive channels
                if (state == 0) {
                    cfirst = c;
                    dfirst = d;
                    state = 1;
                } else {
                    const int st = d - dprev;
                    if (st != 0) {
                        const int sd = st > 0 ? 1 : -1;
                        if (dir != 0 && sd != dir) bad = true;
                        dir = sd;
                    }
                    if (st > 3 || st < -3) bad = true;
                }
                bad |= (__float_as_uint(w.w0) >> 31) || (__float_as_uint(w.w1) >> 31);
                dprev = d;
                ++cnt;
            } else if (state == 1) {
                state = 2;
            }
        }
        if (cnt > 255) bad = true;
        if (bad) atomicOr(err, 2);
        hdr[b * 32 + lane] = (unsigned)cfirst | ((unsigned)(dfirst + 1) << 16) | ((dir < 0 ? 1u : 0u) << 20) |
                             ((unsigned)min(cnt, 255) << 24);
        int m = cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) blk[b] = make_uint2(0u, (unsigned)min(m, 255));
    } else {
        const unsigned h = hdr[b * 32 + lane];
        const int cnt = (int)(h >> 24);
        if (cnt == 0) return;
        const int cfirst = (int)(h & 0xffffu);
        const int dir = (h >> 20) & 1u ? -1 : 1;
        int dprev = (int)((h >> 16) & 15u) - 1;
        uint2 *E = ent + (size_t)blk[b].x * 32 + lane;
        for (int i = 0; i < cnt; ++i) {
            const RowW w = row_weights(rr[cfirst + i], sc.ia2, sc.iah);
            const int d = (int)__fsub_rn(w.j, sc.jbf);
            const unsigned s = i == 0 ? 0u : (unsigned)((d - dprev) * dir);
            E[(size_t)i * 32] = make_uint2(__float_as_uint(w.w0) | ((s & 1u) << 31),
                                           __float_as_uint(w.w1) | ((s >> 1) << 31));
            dprev = d;
        }
    }
}

struct DevBuf {  // cudaFree on scope exit unless released
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
    void *release() {
        void *q = p;
        p = nullptr;
        return q;
    }
};

}  // namespace

void free_matrix2d(oslalm_geom *g) {
    cudaFree(g->d_fp_hdr);
    cudaFree(g->d_fp_ent);
    cudaFree(g->d_bp_blk);
    cudaFree(g->d_bp_hdr);
    cudaFree(g->d_bp_ent);
    g->d_fp_hdr = nullptr;
    g->d_fp_ent = nullptr;
    g->d_bp_blk = nullptr;
    g->d_bp_hdr = nullptr;
    g->d_bp_ent = nullptr;
    g->matrix_bytes = 0;
}

}  // namespace oslalm

using namespace oslalm;

extern "C" int oslalm_geom_build_matrix(oslalm_geom *g, size_t *bytes, void *stream) {
    clear_error();
    if (!g) return fail(OSLALM_ERR_ARG, "geometry handle is NULL");
    if (is_3d(g)) return fail(OSLALM_ERR_ARG, "the device system matrix is built for 2D geometries only");
    if (g->d.nviews > 65535) return fail(OSLALM_ERR_RANGE, "system matrix: at most 65535 views");
    cudaStream_t st = (cudaStream_t)stream;
    free_matrix2d(g);  // geo2() below must describe the evaluating path
    const Geo2 geo = g->geo2();
    const size_t nrays = (size_t)geo.nviews * geo.ns;
    const int ntx = (geo.nx + kBpTile - 1) / kBpTile;
    const size_t ntiles = (size_t)ntx * ((geo.ny + kBpTile - 1) / kBpTile);
    const size_t nblk = (size_t)geo.nviews * 2 * ntiles;

    DevBuf err_b, cnt_b, fph_b, fpe_b, bpb_b, bph_b, bpe_b;
    OSL_CUDA_TRY(cudaMalloc(&err_b.p, sizeof(int)));
    OSL_CUDA_TRY(cudaMemsetAsync(err_b.p, 0, sizeof(int), st));
    int *d_err = (int *)err_b.p;

    // forward layout: rows per ray, their offsets, the entries
    OSL_CUDA_TRY(cudaMalloc(&cnt_b.p, sizeof(unsigned) * nrays));
    const unsigned nb = (unsigned)((nrays + 255) / 256);
    mat_fp_count_kernel<<<nb, 256, 0, st>>>(geo, (unsigned *)cnt_b.p);
    OSL_LAUNCH_CHECK("mat_fp_count_kernel");
    std::vector<unsigned> rows(nrays);
    OSL_CUDA_TRY(cudaMemcpyAsync(rows.data(), cnt_b.p, sizeof(unsigned) * nrays, cudaMemcpyDeviceToHost, st));
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned long long total = 0;
    for (size_t i = 0; i < nrays; ++i) {
        const unsigned n = rows[i];
        rows[i] = (unsigned)total;
        total += n;
        if (total > 0xffffffffull) return fail(OSLALM_ERR_RANGE, "system matrix: more than 2^32 forward entries");
    }
    OSL_CUDA_TRY(cudaMemcpyAsync(cnt_b.p, rows.data(), sizeof(unsigned) * nrays, cudaMemcpyHostToDevice, st));
    OSL_CUDA_TRY(cudaMalloc(&fph_b.p, sizeof(uint4) * nrays));
    OSL_CUDA_TRY(cudaMalloc(&fpe_b.p, sizeof(uint2) * (total ? total : 1)));
    mat_fp_fill_kernel<<<nb, 256, 0, st>>>(geo, (const unsigned *)cnt_b.p, (uint4 *)fph_b.p, (uint2 *)fpe_b.p,
                                           d_err);
    OSL_LAUNCH_CHECK("mat_fp_fill_kernel");
    const size_t fp_bytes = sizeof(uint4) * nrays + sizeof(uint2) * total;

    // back-projection layout: lane headers and block lengths, offsets, entries
    OSL_CUDA_TRY(cudaMalloc(&bpb_b.p, sizeof(uint2) * nblk));
    OSL_CUDA_TRY(cudaMalloc(&bph_b.p, sizeof(unsigned) * nblk * 32));
    dim3 grid((unsigned)ntiles, (unsigned)geo.nviews);
    mat_bp_kernel<0><<<grid, 64, 0, st>>>(geo, (unsigned *)bph_b.p, (uint2 *)bpb_b.p, nullptr, d_err);
    OSL_LAUNCH_CHECK("mat_bp_kernel<count>");
    std::vector<uint2> blk(nblk);
    OSL_CUDA_TRY(cudaMemcpyAsync(blk.data(), bpb_b.p, sizeof(uint2) * nblk, cudaMemcpyDeviceToHost, st));
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    unsigned long long brows = 0;
    for (size_t i = 0; i < nblk; ++i) {
        blk[i].x = (unsigned)brows;
        brows += blk[i].y;
        if (brows > 0xffffffffull) return fail(OSLALM_ERR_RANGE, "system matrix: more than 2^32 entry rows");
    }
    OSL_CUDA_TRY(cudaMemcpyAsync(bpb_b.p, blk.data(), sizeof(uint2) * nblk, cudaMemcpyHostToDevice, st));
    const size_t ent_bytes = sizeof(uint2) * 32 * (brows ? brows : 1);
    OSL_CUDA_TRY(cudaMalloc(&bpe_b.p, ent_bytes));
    OSL_CUDA_TRY(cudaMemsetAsync(bpe_b.p, 0, ent_bytes, st));
    mat_bp_kernel<1><<<grid, 64, 0, st>>>(geo, (unsigned *)bph_b.p, (uint2 *)bpb_b.p, (uint2 *)bpe_b.p, d_err);
    OSL_LAUNCH_CHECK("mat_bp_kernel<fill>");
    const size_t bp_bytes = sizeof(uint2) * nblk + sizeof(unsigned) * nblk * 32 + ent_bytes;

    int herr = 0;
    OSL_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    OSL_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr)
        return fail(OSLALM_ERR_RANGE,
                    "system matrix: the geometry breaks an assumption of the stored layout (code %d: %s)", herr,
                    herr & 1 ? "a ray's first pixel moves by more than three per row"
                             : "a strip's rays are not consecutive channels, or step by more than 3 pixels");
    g->d_fp_hdr = (uint4 *)fph_b.release();
    g->d_fp_ent = (uint2 *)fpe_b.release();
    g->d_bp_blk = (uint2 *)bpb_b.release();
    g->d_bp_hdr = (unsigned *)bph_b.release();
    g->d_bp_ent = (uint2 *)bpe_b.release();
    g->matrix_bytes = fp_bytes + bp_bytes;
    if (bytes) {
        bytes[0] = fp_bytes;
        bytes[1] = bp_bytes;
    }
    return OSLALM_OK;
}

extern "C" int oslalm_geom_drop_matrix(oslalm_geom *g) {
    clear_error();
    if (!g) return fail(OSLALM_ERR_ARG, "geometry handle is NULL");
    OSL_CUDA_TRY(cudaDeviceSynchronize());  // no launch may still read the tables
    free_matrix2d(g);
    return OSLALM_OK;
}
