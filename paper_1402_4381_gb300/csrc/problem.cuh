// The PWLS problem state (shared by the single-problem driver and the batch).
#pragma once

#include <vector>

#include "common.cuh"

struct oslalm_problem {
    const oslalm_geom *g;
    oslalm_params p;
    long npix;
    int per_view;  // nt * ns
    std::vector<int> order, off, cnt;  // subset order; view offset / count of subset m (subset-major layout)
    int max_cnt;
    int *d_views = nullptr;  // subset-major global view ids [nviews]
    float *d_y = nullptr;    // subset-major [nviews][nt][ns]
    void *d_w = nullptr;     // same, storage dtype p.w_dtype
    float *d_wscale = nullptr;
    void *d_D = nullptr;     // image, storage dtype p.d_dtype
    float *d_dscale = nullptr;
    unsigned int *d_maxbits = nullptr;
    float *d_g = nullptr, *d_zeta = nullptr, *d_xalt = nullptr;
    float *d_fu[2] = {nullptr, nullptr}, *d_fv[2] = {nullptr, nullptr};  // inner FISTA iterates (n_inner > 1)
    std::vector<float> fista_gamma;                                     // momentum weights of the inner steps
    float *d_bbx = nullptr, *d_bbz = nullptr;  // Barzilai-Borwein: per subset, last gradient's iterate and value [M][npix]
    int *d_bbhave = nullptr;                   // [M]: 1 once subset m has a stored pair
    float *d_r = nullptr;    // residual of one subset
    float *d_tmp = nullptr;  // full-sinogram scratch (set_data staging)
    oslalm::DevState *d_state = nullptr;
    oslalm::RhoEnt *d_rho_tab = nullptr;  // continuation: rho_l and g-update weights for l < rho_tab_n
    int rho_tab_n = 0;
    double *d_partials = nullptr;
    int n_partials = 0;
    oslalm_stats *d_stats = nullptr;
    int stats_cap = 0;
    signed char *d_replay = nullptr;
    int replay_n = 0;
    bool d_valid = false, initialized = false;
    long j_host = 0;  // subset-iterations done
    // CUDA graph of whole iterations
    cudaGraphExec_t gexec = nullptr;
    const float *g_x = nullptr;
    int g_iters = 0;
    cudaStream_t g_stream = nullptr;
    oslalm_stats *g_stats_ptr = nullptr;
};

namespace oslalm {
// helpers of problem.cu used by other translation units
int problem_update_step(oslalm_problem *p, const float *x_in, float *x_out, cudaStream_t st);
}  // namespace oslalm
