/*
 * lt.h -- C ABI of the GB300 (sm_103a) image-plane chi^2 library for
 * LENSTOOL-style parametric strong-lens modelling.
 *
 * Method: Rexroth, Schaefer, Fourestey & Kneib (2019), "High Performance
 * Computing for gravitational lens modeling: single vs double precision on
 * GPUs and CPUs".  For each lens-parameter sample the library
 *   - sums the scaled deflection of all potentials at every node of an
 *     image-plane grid (Sect. 2.2.2, Algorithm 1 and its superposition),
 *   - maps nodes to the source plane, beta = theta - (D_ls/D_s) alpha
 *     (Eq. 13),
 *   - splits every cell into two triangles and tests each mapped triangle
 *     for containing each source / system barycentre (Sect. 2.2.2, Fig. 1),
 *   - interpolates predicted image positions by barycentric weights,
 *   - reduces chi^2 = sum_ij |x_obs,ij - x_ij|^2 / sigma_ij^2 (Eq. 11),
 *   - and differentiates chi^2 w.r.t. the lens parameters with the triangle
 *     assignment held fixed.
 *
 * Conventions shared by every call
 *   Angles in arcsec, velocity dispersions in km/s, position angles in rad.
 *   Node (i, j) of an lt_grid sits at (x0 + i*dx, y0 + j*dy).
 *   Cell (i, j) with corners v00, v10, v01, v11 has triangles
 *   T0 = (v00, v10, v11) and T1 = (v00, v11, v01); tri = 2*(j*(nx-1)+i) + t.
 *   A point on a shared edge belongs to the triangle whose edge, traversed
 *   counter-clockwise in the source plane, has dy > 0 (or dy == 0, dx < 0);
 *   a mapped triangle with zero FP64 determinant is skipped.
 *   Buffers marked "device" are CUDA device pointers (e.g. from torch);
 *   "host" buffers are ordinary host memory.  The caller owns every buffer
 *   it passes.  Streams are cudaStream_t values cast to uintptr_t (0 = the
 *   legacy default stream).  All compute calls are stream-ordered and
 *   asynchronous: the returned status covers argument and launch errors;
 *   errors detected on the device (hit overflow, non-finite or invalid
 *   parameters) are latched in the model and returned by lt_model_sync.
 *   A model is not thread-safe; use one model per host thread.
 */
#ifndef LT_H
#define LT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LT_OK = 0,
  LT_ERR_INVALID_ARG = 1, /* bad pointer, size, grid or enum */
  LT_ERR_CUDA = 2,        /* a CUDA runtime call failed (see lt_last_error) */
  LT_ERR_NOMEM = 3,       /* device allocation failed */
  LT_ERR_OVERFLOW = 4,    /* more hits / FP64 work items than capacity */
  LT_ERR_TIMEOUT = 5,     /* reserved: no kernel of this library spin-waits */
  LT_ERR_NONFINITE = 6    /* non-finite or out-of-domain lens parameter or source */
} lt_status;

typedef enum { LT_SIS = 0, LT_PIEMD = 1, LT_SIE = 2 } lt_kind;

/* LT_PREC_FP64: deflection, mapping and predicate in FP64 throughout.
 * LT_PREC_MIXED: deflection, mapping and triangle test in FP32 with a
 * per-node running error bound; a (triangle, source) pair whose FP32
 * orientation signs are not certain under that bound, and a hit whose FP32
 * position bound exceeds LT_POS_TOL, are re-evaluated in FP64 with the three
 * vertex deflections recomputed in FP64.  Image sets equal the FP64 ones. */
typedef enum { LT_PREC_FP64 = 0, LT_PREC_MIXED = 1, LT_PREC_PAPER = 2 } lt_precision;

/* LT_PREC_PAPER (lt_deflect_grid only): the paper's own mixed-precision rule
 * for the deflection grid (Sect. 3.3 and App. A.3).  Every node is computed
 * in FP32; then every node is recomputed in FP64 that lies
 *   - in a square patch centred on a halo: 400 x 400 nodes around
 *     cluster-scale halos (b0 >= LT_PAPER_CLUSTER_B0 arcsec), 20 x 20 around
 *     the others (galaxy scale), or
 *   - where the distortion criteria fire on the FP32 grid (Eqs. 23-28):
 *     |h - d1| or |h - d2| < 0.0092 h/0.03, or |d3| or |d4| > 0.0104 h/0.03,
 *     with d1 = a1(i,j) - a1(i-1,j), d2 = a2(i,j) - a2(i,j-1),
 *     d3 = a1(i,j) - a1(i,j-1), d4 = a2(i,j) - a2(i-1,j), h the node spacing
 *     (the paper's thresholds for 0.03" pixels, scaled with the spacing;
 *     nodes in the first row or column have no criteria).
 * alpha_out is then double [ny][nx][2]; err_out (optional) receives 1.0 at
 * the nodes recomputed in FP64 and 0.0 elsewhere. */
#define LT_PAPER_CLUSTER_B0 1.0

/* Position tolerance (arcsec) that an FP32 interpolated image must provably
 * meet; otherwise the hit is re-interpolated in FP64. */
#define LT_POS_TOL 2.5e-5

/* Parameter rows of the params array (see lt_model_set_params). */
enum { LT_ROW_KIND = 0, LT_ROW_X, LT_ROW_Y, LT_ROW_E, LT_ROW_PHI, LT_ROW_RCORE,
       LT_ROW_RCUT, LT_ROW_SIGMA, LT_N_ROWS };
/* Gradient columns of lt_chi2_grad's output. */
enum { LT_GRAD_X = 0, LT_GRAD_Y, LT_GRAD_E, LT_GRAD_PHI, LT_GRAD_RCORE, LT_GRAD_SIGMA,
       LT_N_GRAD };

typedef struct {
  double x0, y0, dx, dy; /* node (i,j) = (x0 + i*dx, y0 + j*dy) */
  int32_t nx, ny;        /* nodes per row / column, each >= 1 */
} lt_grid;

typedef struct {
  int32_t n_pot;        /* potentials per sample, >= 1 */
  int32_t batch;        /* samples, >= 1 */
  int64_t hit_capacity; /* per-sample capacity of the internal hit and FP64
                           work lists used by lt_chi2 / lt_chi2_grad;
                           0 selects 4096 */
} lt_model_desc;

typedef struct lt_model lt_model;

/* One predicted image (lt_find_images output), 64 bytes. */
typedef struct {
  int32_t sample, src; /* sample index, source index */
  int64_t tri;         /* triangle id within the sample's grid */
  double x, y;         /* interpolated image position (arcsec) */
  double w[3];         /* barycentric weights of the triangle's vertices */
  int32_t fp64;        /* 1 if the containment or the position was decided
                          in FP64 (mixed precision only) */
  int32_t reserved;
} lt_image;

/* Observed multiple images, shared by every sample of a batch (the data an
 * MCMC fits).  All pointers are device pointers. */
typedef struct {
  int32_t n_obs;        /* observed images, >= 1 */
  int32_t n_sys;        /* multiple-image systems, >= 1 */
  const double* x;      /* [n_obs] observed positions (arcsec) */
  const double* y;      /* [n_obs] */
  const double* sigma;  /* [n_obs] positional error budget sigma_ij (arcsec) */
  const int32_t* sys;   /* [n_obs] system index in [0, n_sys) */
  const double* dls_ds; /* [n_sys] D_ls/D_s of each system's source */
} lt_obs;

/* Counters of the last compute call, for reporting. */
typedef struct {
  int64_t hits;          /* predicted images found (all samples) */
  int64_t ambiguous;     /* (triangle, source) pairs the search's coarse FP32
                            bound left undecided */
  int64_t refined;       /* certain FP32 hits whose position bound was too large */
  int64_t fp64_nodes;    /* node deflections evaluated in FP64 */
  int64_t work_overflow; /* items dropped for lack of capacity (0 when OK) */
  int64_t tight_nodes;   /* distinct nodes of those items re-evaluated in FP32
                            with the tight bound */
  int64_t fp64_items;    /* items the tight bound left undecided, decided in FP64 */
} lt_stats;

/* Create a model for `batch` samples of `n_pot` potentials.  Allocates the
 * parameter buffers on the current CUDA device; workspaces grow on demand.
 * Errors: LT_ERR_INVALID_ARG (null pointers, n_pot < 1, batch < 1),
 * LT_ERR_NOMEM, LT_ERR_CUDA.  On error *out is NULL. */
lt_status lt_model_create(const lt_model_desc* desc, lt_model** out);

/* Destroy a model and free its device memory (synchronises its work). */
void lt_model_destroy(lt_model* model);

/* Text of the last error seen by this model (never NULL). */
const char* lt_last_error(const lt_model* model);
const char* lt_status_string(lt_status status);

/* Load the lens parameters of every sample and run parameter preparation.
 * params: float64 [batch][LT_N_ROWS][n_pot] (SoA per sample, Sect. 2.3):
 *   kind (LT_SIS / LT_PIEMD / LT_SIE, stored as a double), x, y (arcsec),
 *   e (PIEMD: ellipticity 1 - b/a, axis ratio q = 1 - e, 0 <= e < 1;
 *      SIE: pseudo-ellipticity eps, 0 <= eps < 1), phi (rad, major axis
 *   counter-clockwise from the x axis), r_core, r_cut (PIEMD only,
 *   0 < r_core < r_cut, arcsec), sigma_v (km/s, >= 0).
 * on_device != 0: params is a device pointer, read in place by the
 * preparation kernel (it must stay valid and unchanged until the stream
 * reaches that kernel); else a host pointer (copied asynchronously; the host
 * buffer must stay valid until the stream reaches the copy).  Invalid or non-finite values are latched as LT_ERR_NONFINITE
 * (reported by lt_model_sync). */
lt_status lt_model_set_params(lt_model* model, const double* params, int on_device,
                              uintptr_t stream);

/* Deflection field of one sample over one grid (Sect. 2.2.2: the gradient of
 * the lensing potential summed over all potentials at every node).
 * alpha_out: device, [ny][nx][2] of float (LT_PREC_MIXED) or double
 * (LT_PREC_FP64, LT_PREC_PAPER).  err_out: optional device [ny][nx] float
 * receiving the FP32 running error bound of each node (LT_PREC_MIXED; 1e30
 * at a node whose FP32 coordinates coincide with an SIS or SIE centre, where
 * the deflection's direction is undefined) or the FP64-recomputation map
 * (LT_PREC_PAPER); NULL with LT_PREC_FP64.
 * Errors: LT_ERR_INVALID_ARG. */
lt_status lt_deflect_grid(lt_model* model, int32_t sample, const lt_grid* grid,
                          lt_precision precision, void* alpha_out, float* err_out,
                          uintptr_t stream);

/* Predicted images of explicit source positions (Fig. 1 relensing).
 * grids: host [batch]; src_xy: device [batch][n_src][2]; dls_ds: device
 * [batch][n_src]; out: device [batch][capacity] lt_image records, each
 * sample's images sorted by (src, tri); n_out: device [batch] int64, the
 * number of images of each sample (may exceed capacity: then only capacity
 * records are written and LT_ERR_OVERFLOW is latched).  A source needs a
 * finite position and a ratio 0 <= D_ls/D_s < 1e30 (0: a source in the lens
 * plane, whose image is the source position itself); any other source has
 * no images and LT_ERR_NONFINITE is latched.
 * Errors: LT_ERR_INVALID_ARG. */
lt_status lt_find_images(lt_model* model, const lt_grid* grids, int32_t n_src,
                         const double* src_xy, const double* dls_ds, lt_precision precision,
                         int64_t capacity, lt_image* out, int64_t* n_out, uintptr_t stream);

/* chi^2 of Eq. 11 for every sample: observed images mapped to the source
 * plane, per-system barycentres (FP64), triangle search for each barycentre,
 * barycentric image positions, and for each observed image the nearest
 * predicted image of its system (ties to the lower triangle id); a system
 * with no predicted image contributes (L_diag/sigma)^2 per observed image,
 * L_diag the diagonal of its sample's grid.  A system whose barycentre is not
 * finite or whose D_ls/D_s lies outside [0, 1e30) has no predicted images
 * (LT_ERR_NONFINITE latched), as in lt_find_images.
 * grids: host [batch]; obs: host struct of device pointers; chi2_out: device
 * [batch] double.  Errors: LT_ERR_INVALID_ARG; overflow latched. */
lt_status lt_chi2(lt_model* model, const lt_grid* grids, const lt_obs* obs,
                  lt_precision precision, double* chi2_out, uintptr_t stream);

/* chi^2 and its gradient w.r.t. (x, y, e, phi, r_core, sigma_v) of every
 * potential with the triangle assignment and matching of this evaluation
 * held fixed (hand-written adjoint; FP32 derivatives, FP64 accumulation).
 * grad_out: device [batch][n_pot][LT_N_GRAD] double.  Derivatives that a
 * potential kind does not depend on are 0. */
lt_status lt_chi2_grad(lt_model* model, const lt_grid* grids, const lt_obs* obs,
                       lt_precision precision, double* chi2_out, double* grad_out,
                       uintptr_t stream);

/* Copy the intermediates of the last lt_chi2 / lt_chi2_grad call (device
 * pointers, any may be NULL): match_tri [batch][n_obs] int64 (-1 = none),
 * match_xy [batch][n_obs][2], bary [batch][n_sys][2].  Errors:
 * LT_ERR_INVALID_ARG if no chi^2 call has run. */
lt_status lt_last_matches(lt_model* model, int64_t* match_tri, double* match_xy,
                          double* bary, uintptr_t stream);

/* Wait for the model's work on `stream`, fill *stats (may be NULL) with the
 * counters of the last compute call, and return (then clear) the latched
 * device status: LT_OK, LT_ERR_OVERFLOW or LT_ERR_NONFINITE. */
lt_status lt_model_sync(lt_model* model, uintptr_t stream, lt_stats* stats);

/* Capture the whole lt_chi2 sequence for these grids, observations, precision
 * and output pointer into a CUDA graph owned by the model, and launch it on
 * `stream`; later calls with the same arguments replay the graph.  Same
 * results and errors as lt_chi2. */
lt_status lt_chi2_graph(lt_model* model, const lt_grid* grids, const lt_obs* obs,
                        lt_precision precision, double* chi2_out, uintptr_t stream);

/* Choose the launch shape of the FP32 deflection kernel by index, in
 * [0, lt_num_shapes()): (threads per block, nodes per thread, resident blocks
 * per SM its register budget allows) of (256, 4, 3) (the default),
 * (256, 2, 5), (256, 3, 4), (128, 8, 3), (128, 8, 4), (128, 4, 7), (128, 4, 8),
 * (256, 2, 6).  A thread's nodes are consecutive rows of one grid column.
 * Every shape computes the same values; only speed differs.  lt_autotune
 * picks one by timing.  Errors: LT_ERR_INVALID_ARG. */
lt_status lt_model_set_shape(lt_model* model, int32_t shape);
int32_t lt_num_shapes(void);

/* Autotune the FP32 deflection kernel's launch shape for this model's
 * potential mix (sample 0) on a representative grid: each candidate shape's
 * kernel alone is timed with CUDA events on `stream`, the minimum of five
 * launches after a warm-up; a later candidate replaces an earlier one only
 * when it is faster by more than 0.5 %.  The fastest is kept for later calls;
 * *choice (optional) receives its index.  Synchronises the stream. */
lt_status lt_autotune(lt_model* model, const lt_grid* grid, uintptr_t stream, int32_t* choice);

/* Per-kernel timing of later compute calls (off by default).  When enabled,
 * every launch of the deflection, search, FP64-resolution, chi^2 and
 * barycentre kernels issued by lt_chi2 / lt_find_images is bracketed by CUDA
 * events recorded on the stream it runs on (not inside lt_chi2_graph).
 * Stages 0-3 run one after another on the caller's stream, so their times
 * add up; stage 4 runs on the model's side stream, overlapping stage 0.
 * lt_profile_read waits for the recorded events and returns the totals since
 * the last reset. */
typedef struct {
  int64_t launches[5]; /* kernel launches of [0] the deflection, [1] the
                          search, [2] the FP64 resolution (3 kernels per
                          chunk), [3] matching + chi^2 (2 per chunk), [4] the
                          barycentres (2, on the side stream) */
  double ms[5];        /* summed event durations of those stages (one event
                          pair per stage and chunk) */
  double node_pot[2];  /* node x potential evaluations by the deflection
                          launches: [0] FP32, [1] FP64 */
} lt_profile;
lt_status lt_profile_enable(lt_model* model, int on);
lt_status lt_profile_read(lt_model* model, lt_profile* out, int reset);

/* Like lt_profile_enable, for a subset of the stages: bit k of mask brackets
 * stage k (0 deflection, 1 search, 2 FP64 resolution, 3 matching + chi^2,
 * 4 barycentres); 0 turns timing off.  Each bracketed stage records two events per chunk on
 * the stream, so timing only the stage of interest keeps the overhead of a
 * measured evaluation small.  Errors: LT_ERR_INVALID_ARG. */
lt_status lt_profile_stages(lt_model* model, uint32_t mask);

/* Allocation-free deflection grid, for callers that cannot allocate device
 * memory (code inside an allocator hook or memory-pool callback, plugins of
 * an application that owns every device allocation, processes that reserve
 * all device memory at start-up).  The paper has no counterpart: it is an
 * integration variant of lt_deflect_grid in mixed precision for one lens
 * model, and needs no lt_model.
 * params: device, float64 [LT_N_ROWS][n_pot] (the layout of one sample of
 * lt_model_set_params), 1 <= n_pot <= 4096.  grid: host.  alpha_out: device
 * [ny][nx][2] float; err_out: optional device [ny][nx] float (the FP32
 * running error bound); status_out: optional device int32 receiving LT_OK or
 * LT_ERR_NONFINITE (invalid parameters, which are neutralised to zero mass).
 * Returns LT_ERR_INVALID_ARG for null pointers, a bad grid or n_pot outside
 * [1, 4096]; LT_ERR_CUDA if a runtime call fails.
 * Its scratch is a fixed file-scope device array of about 0.9 MiB that every
 * GPU loading the library holds until exit; the call itself allocates
 * nothing.  The first call on a device resolves that array's address
 * (cudaGetSymbolAddress, with the device current).  Under CUDA's lazy module
 * loading (the default) that first call is also when the library's device
 * code and this array are loaded onto the device, which does take device
 * memory: make one warm-up call before the process reserves its device
 * memory, outside any allocator hook, and before any stream capture; later
 * calls allocate nothing.  The address is kept per device index for the life
 * of the process: do not call this entry point after cudaDeviceReset, or with
 * a context other than the device's primary context current.  All calls on a
 * device share the array, so calls that overlap on the GPU (different
 * streams, or threads) race; order them on one stream. */
lt_status lt_deflect_grid_noalloc(const double* params, int32_t n_pot, const lt_grid* grid,
                                  float* alpha_out, float* err_out, int32_t* status_out,
                                  uintptr_t stream);

/* Source-plane chi^2 of every sample: each observed image is mapped to the
 * source plane (beta = theta - (D_ls/D_s) alpha, Eq. 13) and each system's
 * barycentre formed as in lt_chi2 (Fig. 1); the scatter about it is weighted
 * by the squared point magnification at the observed image,
 *   chi2_S = sum_m |beta_m - beta_bar|^2 mu_m^2 / sigma_m^2,
 *   mu_m = 1 / det(I - (D_ls/D_s) d alpha/d theta),
 * the LENSTOOL source-plane fit (Jullo et al. 2007, which the paper cites for
 * the chi^2).  d alpha/d theta is the sum of closed-form second derivatives
 * of every potential.  FP64 throughout; needs no grid.
 * obs: host struct of device pointers; chi2_out: device [batch] double;
 * mu_out: device [batch][n_obs] double (the point magnifications) or NULL.
 * Errors: LT_ERR_INVALID_ARG. */
lt_status lt_chi2_source(lt_model* model, const lt_obs* obs, double* chi2_out, double* mu_out,
                         uintptr_t stream);

/* Signed triangle magnification of the predicted image each observed image
 * was matched to in the last lt_chi2 / lt_chi2_grad / lt_chi2_graph call: the
 * image-plane area of the grid triangle over the signed area of the triangle
 * lensed into the source plane (Fig. 1), from FP64 deflections of its three
 * nodes; negative for images of odd parity; NaN for an observed image without
 * a match.  Uses the model's current parameters: call it before
 * lt_model_set_params changes them.  obs: the same observations as that call
 * (host struct of device pointers); mu_out: device [batch][n_obs] double.
 * Errors: LT_ERR_INVALID_ARG (no evaluation yet, or other observations). */
lt_status lt_last_magnifications(lt_model* model, const lt_obs* obs, double* mu_out,
                                 uintptr_t stream);

/* D_ls/D_s of a source at redshift z_s behind a lens at z_l (Sect. 4: the
 * paper's benchmark puts the lens at 0.3 and the sources at 2.0 in flat
 * LambdaCDM, Omega_m = 0.3, Omega_Lambda = 0.7), the ratio that scales the
 * deflection in the lens equation (Eq. 13).  Host computation: angular
 * diameter distances from the comoving distance integral (Gauss-Legendre
 * quadrature); H0 cancels.  Requires 0 <= z_l < z_s, Omega_m >= 0 and
 * Omega_k = 1 - Omega_m - Omega_Lambda >= 0 (flat or open); otherwise
 * LT_ERR_INVALID_ARG.  No model or GPU is needed. */
lt_status lt_dls_ds(double z_l, double z_s, double omega_m, double omega_lambda,
                    double* dls_ds);

/* Library version string. */
const char* lt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LT_H */
