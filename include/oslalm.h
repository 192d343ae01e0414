/*
 * liboslalm -- C ABI of the GB300 (sm_103a) OS-LALM reconstruction library.
 *
 * Nien & Fessler, "Fast X-ray CT image reconstruction using the linearized
 * augmented Lagrangian method with ordered subsets" (OS-LALM).  The library
 * solves the penalized weighted least-squares problem of Sec. IV
 * (Eq. ct_recon)
 *
 *     x_hat = argmin_{x >= 0} 1/2 ||y - A x||_W^2 + R(x),
 *     R(x)  = beta sum_{j<k neighbours} w_jk psi(x_j - x_k),
 *     psi(t) = delta^2 (sqrt(1 + (t/delta)^2) - 1),
 *
 * with the OS-LALM iterates of Eq. os_lalm_iterates, the diagonal majorizer
 * L_diag = diag{A' W A 1} and bit-reversal subset order of Sec. IV-A, and the
 * deterministic downward continuation of Sec. III-B (Eq. rho_l_formula_qp,
 * restart when the indicator of Eq. period_indicator_qp is positive).
 *
 * Conventions for every entry point:
 *  - Return value: OSLALM_OK (0) or a negative OSLALM_ERR_* code; nothing
 *    aborts or throws across the ABI.  oslalm_last_error() gives a message
 *    for the calling thread's most recent failure.
 *  - Device pointers ("dev") are allocated and owned by the caller, must stay
 *    valid until the work queued on `stream` has finished, and are only read
 *    or written on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *    default stream).  Calls are asynchronous on that stream unless stated.
 *  - Host pointers ("host") are read or written before the call returns.
 *  - Layouts: image [nz][ny][nx] (x fastest), FP32; sinogram
 *    [view][row][channel] (channel fastest), FP32.  Units: mm, radians, 1/mm.
 *  - Opaque handles own their device buffers; *_destroy frees them.  A handle
 *    may be used from one host thread at a time.
 *
 * Scan geometry (the paper leaves the system matrix unspecified; Sec. IV):
 *  - view v has angle phi_v = pi tau_v, tau_v = angle_start/pi +
 *    v (angle_span/pi)/nviews, with cos/sin evaluated by exact quarter-turn
 *    reduction; u = (cos phi, sin phi) is the beam direction,
 *    e = (-sin phi, cos phi) the detector's lateral axis;
 *  - PAR2D: ray c is the line through s_c e along u,
 *    s_c = (c - (ns-1)/2 + offset_s) ds;
 *  - FAN2D_ARC: source at -dso u, channel angle gamma_c = s_c / dsd, ray
 *    direction cos(gamma_c) u + sin(gamma_c) e;
 *  - CONE3D_FLAT: source at (-dso u, 0), cell centre (dsd-dso) u + s_c e +
 *    t_t z, t_t = (t - (nt-1)/2 + offset_t) dt;
 *  - pixel (ix,iy,iz) centred at ((ix-(nx-1)/2) dx + offset_x, ...);
 *  - a_ij = length of ray i inside pixel j (exact ray/pixel intersection);
 *    pixels are half-open boxes [lo, hi).
 */
#ifndef OSLALM_H
#define OSLALM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OSLALM_OK 0
#define OSLALM_ERR_ARG (-1)     /* invalid argument, shape or handle */
#define OSLALM_ERR_CUDA (-2)    /* a CUDA runtime call or kernel launch failed */
#define OSLALM_ERR_RANGE (-3)   /* value outside the supported range */
#define OSLALM_ERR_TIMEOUT (-4) /* a bounded device-side wait gave up */
#define OSLALM_ERR_STATE (-5)   /* call out of order (e.g. iterate before init) */
#define OSLALM_ERR_ALLOC (-6)   /* device or host allocation failed */

#define OSLALM_PAR2D 0
#define OSLALM_FAN2D_ARC 1
#define OSLALM_CONE3D_FLAT 2

#define OSLALM_F32 0
#define OSLALM_F16 1
#define OSLALM_BF16 2

#define OSLALM_RHO_CONTINUATION 0 /* Sec. III-B downward continuation */
#define OSLALM_RHO_FIXED 1        /* fixed rho (rho = 1: ordered-subsets SQS) */
#define OSLALM_RHO_REPLAY 2       /* continuation with restarts read from a list */

#define OSLALM_CURV_HUBER 0 /* D_R from psi'(t)/t at the current x */
#define OSLALM_CURV_MAX 1   /* D_R from the maximum curvature psi''(0) = 1 */

typedef struct oslalm_geom_desc {
    int kind;                         /* OSLALM_PAR2D | OSLALM_FAN2D_ARC | OSLALM_CONE3D_FLAT */
    int nx, ny, nz;                   /* image size; nz = 1 for 2D */
    double dx, dy, dz;                /* pixel size (mm) */
    double offset_x, offset_y, offset_z; /* image centre (mm) */
    int nviews;
    double angle_start, angle_span;   /* radians */
    int ns, nt;                       /* channels, detector rows (nt = 1 for 2D) */
    double ds, dt;                    /* channel / row pitch (mm at the detector) */
    double offset_s, offset_t;        /* detector offsets in channels / rows */
    double dso, dsd;                  /* source-isocentre, source-detector (mm) */
    double pitch;                     /* cone beam: 0 = circular orbit; > 0 = helix whose
                                         source and detector rise by pitch * nt * dt (mm)
                                         per turn, centred on the scanned angle range:
                                         z_v = pitch nt dt (phi_v - phi_mid) / (2 pi) */
} oslalm_geom_desc;

typedef struct oslalm_params {
    double beta;      /* regularization weight */
    double delta;     /* hyperbola edge parameter (1/mm) */
    int nbr;          /* 4 or 8 (2D); 6 or 26 (3D); w_jk = 1/index distance */
    int M;            /* number of ordered subsets (views v with v mod M = m) */
    double rho_min;   /* continuation floor (Sec. III-B uses 1e-3) */
    int n_inner;      /* FISTA steps (1..64) on the constrained denoising problem of the
                         x-update (Sec. IV-A) from the previous image, each a projected
                         SQS step from the extrapolated point with denominators
                         rho D + D_R(v); 1 = the single projected SQS step.  Batches
                         (oslalm_batch_*) take n_inner = 1 only. */
    int rho_mode;     /* OSLALM_RHO_* */
    double rho_fixed; /* rho for OSLALM_RHO_FIXED */
    int curvature;    /* OSLALM_CURV_* */
    int w_dtype;      /* storage of W: OSLALM_F32 | OSLALM_F16 | OSLALM_BF16 */
    int d_dtype;      /* storage of the SQS denominator D: same choices */
    int use_graph;    /* 1: replay whole iterations from a captured CUDA graph */
    int bb;           /* 1: Barzilai-Borwein scaling of the majorizer (supplement Sec. II-A,
                         Eqs. secant_eq and scale_factor_alpha_k): the x-updates of
                         iteration k+1 use H = alpha D in place of D, with alpha =
                         min(sum_m s_m'y_m / sum_m s_m'D s_m, 1) fitted at the end of
                         iteration k from each subset's secant pair over that iteration
                         (s_m = change of the iterate at which subset m's gradient was
                         taken, y_m = change of that gradient); 1 until pairs exist and
                         when sum s'y <= 0.  Holds 2 M images of history.  0: plain SQS
                         majorizer.  Batches take bb = 0 only. */
} oslalm_params;

/* One record per subset-iteration (filled by oslalm_iterate when asked). */
typedef struct oslalm_stats {
    double xi;        /* restart indicator of Eq. period_indicator_qp (subset gradients) */
    double rho_used;  /* rho of this subset-iteration */
    int l;            /* continuation counter after the update */
    int restart;      /* 1 if l was reset */
    int subset;       /* subset whose gradient was computed (sigma(j+1)) */
    int pad;
    double alpha;     /* Barzilai-Borwein scale after this subset-iteration (1 without bb) */
} oslalm_stats;

typedef struct oslalm_geom oslalm_geom;
typedef struct oslalm_problem oslalm_problem;

/* Message of the calling thread's last failure ("" if none).  Never NULL. */
const char *oslalm_last_error(void);

/* Library ABI version (major*100 + minor). */
int oslalm_version(void);

/* ---- geometry / system model -------------------------------------------
 * Builds the per-ray parameter tables on the current CUDA device (host FP64
 * set-up, one synchronous upload).  Requires the image box to lie strictly
 * between source and detector (fan/cone) and nx, ny, nz, nviews, ns, nt > 0.
 * Errors: ARG (bad descriptor), ALLOC, CUDA.  *out is NULL on failure. */
int oslalm_geom_create(const oslalm_geom_desc *desc, oslalm_geom **out);
int oslalm_geom_destroy(oslalm_geom *g);

/* Host-only view of the 2D system model: the per-ray parameters that the
 * projector pair reads for view `view` (arrays [host, ns] each).  Ray c is
 * written along its major index axis a as b(a) = n0 + f0 + a (k/2048 +
 * kappa_lo), with packed = (k << 16) | ((n0 & 0x7fff) << 1) | axis (axis 0:
 * a = x index, 1: a = y index) and lrow = ray length (mm) per unit of a
 * (0 for a ray that misses the image).  The length of the ray inside pixel
 * (ia, jb) is lrow times the fraction of row [ia, ia+1] whose b lies in
 * [jb, jb+1).  No GPU needed.  Errors: ARG, RANGE. */
int oslalm_ray_table(const oslalm_geom_desc *desc, int view, float *f0, float *kappa_lo, float *lrow, int *packed);

/* ---- subsets (Sec. IV-A bit-reversal order; Sec. IV-B interleaved views) --
 * order[host, M]: subset visiting order by bit reversal; for M not a power of
 * two the bit-reversed values of 0..2^ceil(log2 M)-1 that are < M.
 * views[host, capacity ceil(nviews/M)]: views of subset m (v = m, m+M, ...);
 * *n receives their count.  Errors: ARG. */
int oslalm_subset_order(int M, int *order);

/* Largest number of subsets that still gives every voxel of the central
 * transaxial region s views per subset (Sec. IV-B): *m_max = nviews / s on a
 * circular orbit (Eq. max_M_axial; the paper uses s = 40), and
 * (views per turn) dso / (pitch s dsd) on a helix (Eq. max_M_helical;
 * s = 24), views per turn = nviews 2 pi / angle_span.  A guideline (not
 * enforced by oslalm_problem_create).  Host only.  Errors: ARG. */
int oslalm_max_subsets(const oslalm_geom_desc *desc, double s, double *m_max);
int oslalm_subset_views(const oslalm_geom *g, int M, int m, int *views, int *n);

/* ---- projector pair (A_m and its exact transpose) -------------------------
 * oslalm_project: sino[dev, nv][nt][ns] = A_views x[dev, image].
 * oslalm_backproject: x[dev, image] (=|+=) A_views' sino[dev, nv][nt][ns]
 *   (accumulate = 0 overwrites, 1 adds).
 * views[dev, nv]: global view indices (each in [0, nviews)); nv >= 0 (0 is a
 * no-op / zero image).  The back-projector evaluates the same per-ray/pixel
 * weights as the projector, so it is the transpose up to summation order.
 * Errors: ARG, CUDA. */
int oslalm_project(const oslalm_geom *g, const float *x, float *sino,
                   const int *views, int nv, void *stream);
int oslalm_backproject(const oslalm_geom *g, const float *sino, float *x,
                       const int *views, int nv, int accumulate, void *stream);

/* ---- initial image ---------------------------------------------------------
 * x[dev, image] = filtered back-projection of sino[dev, nviews][nt][ns] (all
 * views).  The paper initialises from an FBP image (Sec. V) without giving
 * the filter; this is the textbook analytic reconstruction: Ram-Lak parallel
 * FBP, equiangular fan FBP over 360 degrees, Feldkamp for the flat cone
 * detector (fan/cone need angle_span = 2 pi).  clip_nonneg = 1 clips to
 * x >= 0.  Allocates a filtered-sinogram buffer with cudaMallocAsync on
 * `stream` and frees it before returning.  Errors: ARG, RANGE, CUDA. */
int oslalm_fbp(const oslalm_geom *g, const float *sino, float *x, int clip_nonneg, void *stream);

/* Same as oslalm_fbp, for callers that cannot allocate device memory while
 * they run (a service whose memory pool took the whole GPU at start-up, or a
 * real-time pipeline that forbids cudaMalloc after initialisation because it
 * may synchronize the device).  The paper has no counterpart: this is a
 * deployment variant.  The filtered sinogram lives in a fixed 16 MiB buffer
 * (2^22 FP32 samples) inside the library; nviews*nt*ns above 2^22 returns
 * OSLALM_ERR_RANGE.  The call itself allocates nothing.
 * The buffer is reserved on a device when the library's FBP code is first
 * loaded there (the CUDA runtime loads device code lazily), i.e. by the first
 * oslalm_fbp_noalloc_prepare or oslalm_fbp_noalloc on that device, and stays
 * until the process exits.  Call oslalm_fbp_noalloc_prepare() once per
 * device, with that device current, during initialisation: before reserving
 * your own memory pool and before any stream capture.  It loads the FBP
 * kernels and looks up the buffer's device address (cudaGetSymbolAddress);
 * synchronous; errors: CUDA, RANGE (device ordinal >= 64).
 * All calls share the one buffer and the next call overwrites it: calls whose
 * work overlaps on the GPU (other streams, other host threads) race, so
 * serialize them.  The result is bit-identical to oslalm_fbp's.  Errors:
 * ARG, RANGE, CUDA. */
int oslalm_fbp_noalloc_prepare(void);
int oslalm_fbp_noalloc(const oslalm_geom *g, const float *sino, float *x, int clip_nonneg, void *stream);

/* ---- PWLS problem and OS-LALM (Eq. os_lalm_iterates, Sec. III-IV) --------
 * oslalm_problem_create: copies y[dev, sino] and w[dev, sino] (FP32,
 *   w >= 0) into library-owned subset-major buffers, storing W as
 *   params->w_dtype (FP16/BF16 with a power-of-two per-array scale).  The
 *   problem keeps a reference to g (g must outlive it).  Synchronizes the
 *   current device once.  Errors: ARG, RANGE, ALLOC, CUDA.
 * oslalm_problem_set_data: replaces y and W (same shapes) on `stream`; the
 *   SQS denominator is recomputed by the next oslalm_init only.
 * oslalm_init: on `stream`, computes D = A'WA1 (first call or after
 *   set_data), zeta = M grad l_{sigma(0)}(x) (Eq. os_lalm_iterates), g = zeta,
 *   l = 0, rho = 1 (or rho_fixed).  x[dev, image] is read only.
 * oslalm_iterate: runs n_iter full iterations (n_iter*M subset-iterations)
 *   updating x[dev, image] in place; each subset-iteration is the inner SQS
 *   step with the hyperbola regularizer and the non-negativity projection,
 *   the forward projection with the weighted residual, the exact-transpose
 *   back-projection with the split-gradient update and the restart
 *   indicator, and the continuation update (rho lives on the device, no host
 *   round trip).  stats[host, n_iter*M] or NULL: when given, the call
 *   synchronizes `stream` and fills one record per subset-iteration.
 *   Errors: STATE (no init), ARG, CUDA.
 * oslalm_set_replay: restart decisions for OSLALM_RHO_REPLAY, restarts[host,
 *   n] (0/1) indexed by the global subset-iteration counter; copied.
 * oslalm_cost: *out[host] = Psi(x) = 1/2 sum_i w_i (y_i - [Ax]_i)^2 + R(x),
 *   projections accumulated and reduced in FP64; synchronizes `stream`.
 * oslalm_get_state / oslalm_set_state: the iteration state for an exact
 *   resume: g and zeta [dev, image each, FP32], rho_l_j[host, 4 doubles] =
 *   {rho, l, j, alpha} (j = subset-iterations done, alpha the
 *   Barzilai-Borwein scale).  With bb the per-subset secant history is not
 *   part of the state: after oslalm_set_state it starts again (alpha is kept
 *   for the next iteration).  Both synchronize `stream`. */
int oslalm_problem_create(const oslalm_geom *g, const float *y, const float *w,
                          const oslalm_params *params, oslalm_problem **out);
int oslalm_problem_destroy(oslalm_problem *p);
int oslalm_problem_set_data(oslalm_problem *p, const float *y, const float *w, void *stream);
int oslalm_init(oslalm_problem *p, const float *x, void *stream);
int oslalm_iterate(oslalm_problem *p, float *x, int n_iter, oslalm_stats *stats, void *stream);
int oslalm_set_replay(oslalm_problem *p, const int *restarts, int n);
int oslalm_cost(oslalm_problem *p, const float *x, double *out, void *stream);
int oslalm_get_state(oslalm_problem *p, float *g, float *zeta, double *rho_l_j, void *stream);
int oslalm_set_state(oslalm_problem *p, const float *g, const float *zeta, const double *rho_l_j, void *stream);

/* Gradient of the PWLS cost of Sec. IV (Eq. ct_recon) at x:
 * grad[dev, image] = A'W(Ax - y) + grad R(x), with W as stored (w_dtype),
 * FP32 projections summed subset by subset.  For optimality (KKT) checks of
 * a converged image: at a minimiser over x >= 0, grad = 0 where x > 0 and
 * grad >= 0 where x = 0.  Does not change the iteration state.  Errors: ARG,
 * CUDA. */
int oslalm_gradient(oslalm_problem *p, const float *x, float *grad, void *stream);

/* The SQS denominator D = A'WA1 as stored (dequantized to FP32) into
 * d[dev, image]; valid after oslalm_init.  Errors: STATE, CUDA. */
int oslalm_get_denominator(oslalm_problem *p, float *d, void *stream);

/* Timing pass for roofline reports: runs n_iter full iterations exactly as
 * oslalm_iterate does without a graph, with CUDA events recorded on `stream`
 * around every kernel launch, and returns the summed device time (ms) per
 * kernel kind in ms_out[host, 3] = {update, forward+residual,
 * back-projection+split-gradient}; launches_out[host, 3] receives the launch
 * counts.  Synchronizes `stream`.  Errors: STATE, ARG, CUDA. */
int oslalm_profile_iterate(oslalm_problem *p, float *x, int n_iter, double *ms_out, int *launches_out,
                           void *stream);

/* ---- batched reconstruction (many independent 2D scans) ------------------
 * A batch advances several initialised 2D problems (oslalm_init done, each at
 * a whole iteration) together: every subset-iteration step runs four
 * persistent launches (update, forward projection + residual, back-projection
 * + split gradient, restart test + continuation) whose grids of resident
 * blocks walk a work list covering all scans still running, so scans of
 * different image sizes, view counts and numbers of subsets share the GPU.
 * Each scan follows exactly the single-problem algorithm (Eq. os_lalm_iterates,
 * Sec. III-B continuation); with launch shape 0 a batched scan is
 * bit-identical to the same problem iterated alone.  The batch references the
 * problems' buffers: the problems must outlive it and must not be iterated
 * by other calls while a batch call on them is queued.
 * oslalm_batch_create: probs[host, n] problem handles.  Errors: ARG, STATE, ALLOC.
 * oslalm_batch_iterate: x[host, n] device image pointers (one per problem,
 *   updated in place); every problem runs n_iter full iterations (n_iter*M_i
 *   subset-iterations; scans with fewer subsets finish earlier).  use_graph =
 *   1 replays the whole call from a CUDA graph (captured on first use of the
 *   same x pointers, n_iter and shape).  Errors: ARG, CUDA.
 * oslalm_batch_autotune: times every launch shape (image tile, forward lanes
 *   per ray) at two occupancies over probe_iters iterations, keeps the fastest
 *   and restores every problem's image and state; ms_out[host, 2 x number of
 *   shapes] or NULL receives the timings.  Allocates and frees backups;
 *   synchronizes.  Errors: ARG, ALLOC, CUDA.
 * oslalm_batch_set_shape / oslalm_batch_get_shape: shape index and blocks per
 *   SM (0 = occupancy maximum).  oslalm_batch_shape_info: tile and lanes of a
 *   shape; oslalm_batch_shape_count: number of shapes. */
typedef struct oslalm_batch oslalm_batch;
int oslalm_batch_create(oslalm_problem *const *probs, int n, oslalm_batch **out);
int oslalm_batch_destroy(oslalm_batch *b);
int oslalm_batch_iterate(oslalm_batch *b, float *const *x, int n_iter, int use_graph, void *stream);
int oslalm_batch_autotune(oslalm_batch *b, float *const *x, int probe_iters, double *ms_out, void *stream);
int oslalm_batch_set_shape(oslalm_batch *b, int shape, int blocks_per_sm);
int oslalm_batch_get_shape(const oslalm_batch *b, int *shape, int *blocks_per_sm);
int oslalm_batch_shape_count(void);
int oslalm_batch_shape_info(int shape, int *tile_x, int *tile_y, int *lanes);

/* ---- learned warm start (no counterpart in the paper) ----------------------
 * A 4-level U-Net (3x3 convs with 32/64/128/256 channels, ReLU, 2x2 average
 * pooling, nearest 2x upsampling, skip concatenation, 1x1 output conv plus
 * the input as a residual; 1,946,305 parameters) mapping an FBP image to an
 * estimate of the converged PWLS image, used as the initial image x0 of
 * OS-LALM (the minimiser is unchanged).  BF16 activations and weights, FP32
 * accumulation on the tensor cores, FP32 master weights, Adam
 * (beta 0.9 / 0.999, eps 1e-8), mean-squared-error loss.
 * Images are FP32 [n][height][width] on the device; the network sees
 * x * scale (scale ~ 1/mu_water puts water at 1) and returns y / scale.
 * oslalm_cnn_create: buffers for exactly `batch` images of height x width
 *   (multiples of 8); seeded He-normal initialisation.  Errors: ARG, ALLOC.
 * oslalm_cnn_param_count: parameters in the exchange layout of get/set:
 *   per layer (e0a, e0b, e1a, e1b, e2a, e2b, b3a, b3b, d2a, d2b, d1a, d1b, d0a,
 *   d0b) weights [cout][3][3][cin] then biases [cout]; then out.w[32], out.b.
 * oslalm_cnn_get_params / oslalm_cnn_set_params: host copies (set also resets
 *   the Adam state).  oslalm_cnn_forward: y[dev] = net(x[dev]).
 * oslalm_cnn_gradients: loss and parameter gradients (host, exchange layout)
 *   without an update.  oslalm_cnn_train_step: one Adam step on (x, target);
 *   *loss (host, may be NULL; when given the call synchronizes).
 * oslalm_cnn_flops_per_image: multiply-add count x 2 of one forward pass.
 * Errors: the convolutions' tensor-core waits are bounded; one that runs out
 *   marks the network (the block stops issuing work, waits a bounded time for
 *   its own MMAs, frees its tensor memory and exits without writing its
 *   outputs), and the next call that synchronizes (get_params, gradients,
 *   train_step with a loss) returns OSLALM_ERR_TIMEOUT and clears the mark
 *   (the outputs since the previous check are invalid).
 * oslalm_cnn_mark_timeout: sets that mark from the host, exactly as a
 *   convolution whose wait ran out would (synchronous), so that callers can
 *   test their handling of OSLALM_ERR_TIMEOUT without a device fault.
 *   Errors: ARG, CUDA.
 * oslalm_cnn_set_tma: enable (default) or disable the TMA forms of the
 *   convolutions and weight gradients.  Convolutions take their tiles by TMA
 *   where a level's 128-pixel blocks are whole rows or row segments (width a
 *   multiple of 128, or 128 / width rows with the height a multiple of that),
 *   and on widths that are a multiple of 128 load each input row once for its
 *   three horizontal taps; weight gradients likewise for 64-pixel stages
 *   (three taps per block on widths that are a multiple of 64).  Disabled,
 *   every kernel stages its tiles with cp.async.  The convolutions run the
 *   same MMAs in the same order on every path, so their outputs are
 *   identical; the weight gradients agree to the rounding of their FP32
 *   atomic sums.  Errors: ARG. */
typedef struct oslalm_cnn oslalm_cnn;
long oslalm_cnn_param_count(void);
int oslalm_cnn_create(int batch, int height, int width, unsigned long long seed, oslalm_cnn **out);
int oslalm_cnn_destroy(oslalm_cnn *c);
int oslalm_cnn_get_params(oslalm_cnn *c, float *host);
int oslalm_cnn_set_params(oslalm_cnn *c, const float *host);
int oslalm_cnn_forward(oslalm_cnn *c, const float *x, float *y, int n, float scale, void *stream);
int oslalm_cnn_gradients(oslalm_cnn *c, const float *x, const float *target, int n, float scale, float *grad_host,
                         double *loss, void *stream);
int oslalm_cnn_train_step(oslalm_cnn *c, const float *x, const float *target, int n, float scale, float lr,
                          double *loss, void *stream);
double oslalm_cnn_flops_per_image(int height, int width);
int oslalm_cnn_mark_timeout(oslalm_cnn *c);
int oslalm_cnn_set_tma(oslalm_cnn *c, int enable);
/* oslalm_cnn_launch_count: kernel launches issued so far by the network
 * functions of this process (all networks, all devices); differences of two
 * readings count the launches of the calls between them.  Never fails. */
long oslalm_cnn_launch_count(void);

/* ---- monitoring ----------------------------------------------------------
 * *out[host] = sqrt(sum_{mask} (x - xref)^2 / count(mask)) over the pixels
 * where mask[dev, image, uint8] != 0 (FP64 reduction); synchronizes.  Sec. V
 * measures convergence by this RMS difference (reported in HU by callers). */
int oslalm_rmsd(const float *x, const float *xref, const uint8_t *mask, long n,
                double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OSLALM_H */
