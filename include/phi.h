/*
 * phi.h - C ABI of the GB300 w-stacking w-projection measurement operator.
 *
 * Operator (Pratley, Johnston-Hollitt & McEwen, arXiv 1903.06555, Sec. 2-3):
 *
 *     y = Phi x,      Phi = W G C F Z S                         (Eq. matrix_equation)
 *     y_k = Phi_k x,  Phi_k = W_k [GC]_k F Z S~_k               (Sec. 3.1)
 *     x_dirty = [Phi_1^H ... Phi_K^H] [y_1; ...; y_K]          (Eq. stacked adjoint)
 *
 * for a real N x N image x and M visibilities y.  Visibilities are split into
 * K w-stacks by k-means on w (Algorithm 1) after an optional conjugate fold of
 * negative w onto positive w (Sec. 3.3).  Every w-projection kernel tap
 *
 *     [GC](rho, dw) = 2 pi int_0^R g(r) e^{-2 pi i dw (sqrt(1 - r^2/du^2) - 1)}
 *                              J0(2 pi rho r) r dr          (Eq. analytic_convolution_hankel)
 *
 * is computed on the fly by adaptive Gauss-Kronrod quadrature inside the
 * degridding and gridding kernels (PHI_KERNEL_QUADRATURE, the default); no
 * sparse G is ever stored.  Alternatives: pre-sampled 1-D w-planes with
 * bilinear interpolation (PHI_KERNEL_TABLE, Sec. 5.1.1), and a per-visibility
 * Chebyshev series in rho built from the same quadrature (PHI_KERNEL_RADIAL).
 * phi_degrid_dde / phi_grid_dde add a direction-dependent-effect kernel per
 * visibility by a further convolution (Sec. 5.2).
 *
 * Conventions shared by every call:
 *   - Pixels: l_j = (j - N/2) * dl, dl = fov_rad / N, for row (m) and column
 *     (l) index j; images are row-major N x N (row = m, column = l).
 *   - Grid: Npad = oversample * N (even), du = 1 / (Npad * dl) wavelengths.
 *     Grid frequency q (in [-Npad/2, Npad/2)) is stored at q mod Npad.
 *   - r = du * l (cycles per grid pixel); the kernel window is r <= R,
 *     R = alpha / 2.  The kernel is scaled by 2 pi (not the paper's
 *     2 pi / du^2) so that it matches the unnormalised DFT of the padded image.
 *   - g is the 2-D Fourier transform of the radial Kaiser-Bessel kernel
 *     k(rho) = I0(beta sqrt(1 - (2 rho / J)^2)) / I0(beta), |rho| <= J/2.
 *   - Visibility i of stack k takes the J_w x J_w grid taps q = q0 + (a, b),
 *     q0 = floor(u_i/du - J_w/2) + 1, wrapping circularly; its model value is
 *     y_i = W_i sum_taps [GC](|u_i/du - q|, w_i - wbar_k) Xhat_k[q], conjugated
 *     when the visibility was folded.  Visibilities whose own u/du or v/du lie
 *     outside [-Npad/2, Npad/2) are dropped: y_i = 0, and they add nothing to
 *     the adjoint.
 *   - Quadrature: Gauss-Kronrod 15/31 on equal panels of [0, R].  Acceptance
 *     per tap: sum over panels |K31 - G15| <= max(quad_abs_tol,
 *     quad_rel_tol * |K|) (paper: 1e-6 relative and absolute, Sec. 4).  Taps that do not converge within the refinement cap are
 *     counted (phi_plan_stats), never an error.
 *
 * Memory and streams: every pointer argument named *_dev is a device pointer
 * owned by the caller; the plan owns everything it allocates (sorted
 * visibility records, permutation, stack tables, per-pixel factors, the
 * padded grids of one group of stacks, cuFFT plans and their workspace);
 * the DDE calls may also take a transient buffer (see phi_degrid_dde).
 * Calls are asynchronous on the
 * given stream (a cudaStream_t passed as void*; NULL = legacy default stream)
 * and do not synchronise, except phi_plan_create (it reads the k-means
 * convergence test back every sweep) and the calls that return host values
 * (phi_plan_info, phi_plan_stats, phi_wkernel with a non-NULL counter).
 * A plan may be used by one stream at a time.
 *
 * Errors: every call returns PHI_OK (0) or a PHI_ERR_* code; no call traps or
 * aborts on the device.  phi_error_string() names a code.
 */
#ifndef PHI_H_
#define PHI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct phi_plan* phi_plan_t;

enum phi_status {
  PHI_OK = 0,
  PHI_ERR_ARG = 1,      /* invalid argument or descriptor field              */
  PHI_ERR_OOM = 2,      /* device allocation failed                          */
  PHI_ERR_CUDA = 3,     /* a CUDA runtime or cuFFT call failed               */
  PHI_ERR_HORIZON = 4,  /* image or kernel window reaches l^2 + m^2 >= 1      */
  PHI_ERR_SUPPORT = 5,  /* a stack needs J_w > max_support (raise K or cap),
                           or the radial / DDE per-warp storage for the largest
                           support exceeds a thread block's shared memory    */
  PHI_ERR_TIMEOUT = 6,  /* a bounded wait ran out                            */
  PHI_ERR_STATE = 7     /* the call does not apply to this plan              */
};

enum phi_precision {
  PHI_F32 = 0,  /* FP32 grid, FFT, kernel, accumulation and quadrature error
                   estimate; FP64 chirp phase argument                       */
  PHI_F64 = 1   /* everything in FP64                                        */
};

enum phi_kernel_mode {
  PHI_KERNEL_QUADRATURE = 0,  /* every tap by adaptive quadrature (Sec. 3.1)         */
  PHI_KERNEL_TABLE = 1,       /* pre-sampled 1-D w-planes, bilinear (Sec. 5.1.1)       */
  PHI_KERNEL_RADIAL = 2       /* per visibility: the same quadrature at Chebyshev radii,
                                 every tap from the resulting series in rho (no
                                 counterpart in the paper; same operator within the
                                 quadrature tolerance)                                 */
};

enum phi_support_rule {
  PHI_SUPPORT_STACK = 0,  /* J_w per stack from its largest |w - wbar_k|     */
  PHI_SUPPORT_VIS = 1     /* J_w per visibility from its own |w - wbar_k|    */
};

/* Plan descriptor.  phi_plan_desc_default() fills the paper's settings. */
typedef struct {
  int32_t image_n;          /* N, even                                       */
  int32_t support;          /* J, Kaiser-Bessel support in grid pixels, even */
  int32_t n_stacks;         /* K >= 1 (at most 126)                          */
  int32_t kmeans_max_iter;  /* Algorithm 1 sweep cap (default 100)           */
  int32_t conj_fold;        /* 1: fold w < 0 onto w > 0 (Sec. 3.3)           */
  int32_t max_support;      /* cap on J_w (default 64, at most 256)          */
  int32_t precision;        /* enum phi_precision                            */
  int32_t support_rule;     /* enum phi_support_rule                         */
  int32_t max_refine;       /* panel-count doublings allowed per tap chunk   */
  int32_t tile;             /* uv tile side used to sort visibilities (32)   */
  int32_t max_grid_mib;     /* device memory for the padded grids of stacks
                               processed together (0: 4096 MiB); at least
                               one grid is always held                      */
  int32_t kernel_mode;      /* enum phi_kernel_mode                          */
  int32_t grid_staging;     /* PHI_KERNEL_TABLE only: 0 = one warp per
                               visibility, table and grid read directly
                               (default); 1 = one thread block per uv tile
                               with its grid patch (tile + J_w cells a side)
                               staged in shared memory, gridding privatised
                               there and added to the grid once per tile;
                               2 = one thread block per w-row of the table:
                               the pair of w-planes around that row staged
                               in shared memory once for every visibility
                               whose |dw| falls on it (the plan keeps an
                               index of the records sorted by stack and
                               w-row; falls back to 0 when a row exceeds a
                               block's shared memory) */
  int32_t grid_deterministic; /* 0 = gridding adds FP values with FP atomics
                               (default; the order of the additions, and so
                               the last bits of the grid, vary from run to
                               run); 1 = every gridding contribution is
                               rounded to a 64-bit fixed-point integer of
                               the call's exponent e and added with integer
                               atomics, so phi_grid and phi_grid_dde return
                               the same bits on every run, alone or beside
                               other work.  e makes every cell's sum below
                               2^61 from the call's largest |W_i y_i| (times
                               the DDE kernels' sums), the number of
                               visibilities in the stack group and a bound
                               on |[GC]|, within the exponents of the grid's
                               precision; each term is off by at most 2^-e/2
                               (far below FP32 rounding, and below 1e-10 of
                               the largest term times the visibility count
                               in FP64).  Costs 16 bytes per resident grid
                               cell (counted against max_grid_mib) and a
                               conversion pass per group.  Not with
                               grid_staging 1 (PHI_ERR_ARG).  No
                               counterpart in the paper. */
  double oversample;        /* os; Npad = os * N must be an even integer     */
  double fov_rad;           /* full field of view in direction cosine        */
  double kmeans_tol;        /* Algorithm 1 convergence (default 1e-3)        */
  double alpha;             /* window radius R = alpha / 2 (default 1)       */
  double quad_rel_tol;      /* default 1e-6 (Sec. 4)                         */
  double quad_abs_tol;      /* default 1e-6 (Sec. 4)                         */
  double kb_beta;           /* 0: pi sqrt((J/os)^2 (os - 1/2)^2 - 0.8)        */
  double cycles_per_panel;  /* a-priori panel width in integrand cycles (0: auto) */
  double table_tol;         /* PHI_KERNEL_TABLE: bilinear interpolation error bound
                               (default 1e-4); sample spacing
                               h_rho = sqrt(4 tol) / (2 pi R),
                               h_w = sqrt(4 tol) / (2 pi (1 - n(R / du)))  */
} phi_plan_desc;

/* Plan summary filled by phi_plan_info. */
typedef struct {
  int64_t n_vis;            /* M as given                                    */
  int64_t n_kept;           /* M minus dropped visibilities                  */
  int64_t n_dropped;
  int64_t device_bytes;     /* device memory held by the plan                */
  int32_t image_n, npad, n_stacks, kmeans_sweeps, max_jw, precision;
  double du, dl, beta, window_radius, support_coeff;
  int32_t kernel_mode;      /* enum phi_kernel_mode                          */
  int32_t group;            /* stacks whose grids are processed together     */
  int64_t table_n_rho;      /* PHI_KERNEL_TABLE: samples in rho (0 otherwise) */
  int64_t table_n_w;        /* samples in |w|                                */
  double table_h_rho;       /* spacing in grid pixels                        */
  double table_h_w;         /* spacing in wavelengths                        */
} phi_plan_summary;

/* Fill *desc with the defaults (image size, FOV and stack count are 0 and
 * must be set by the caller).  Always PHI_OK unless desc is NULL. */
int phi_plan_desc_default(phi_plan_desc* desc);

/*
 * Build a plan (Sec. 3.2-3.3 and the per-visibility part of Eq. GC_k):
 * fold (conj_fold), Algorithm 1 on w, per-stack centres wbar_k, drop test,
 * support J_w, split u/du into integer base and fraction, sort by
 * (stack, uv tile), per-pixel image factors, cuFFT plan.  With
 * PHI_KERNEL_TABLE also the pre-sampled w-planes of Sec. 5.1.1:
 * [GC](i h_rho, j h_w) for 0 <= rho <= sqrt(2) max J_w / 2 + 2 and
 * 0 <= w <= max |w - wbar_k| (positive only: -w is the conjugate), computed
 * by the same adaptive quadrature, stored in pairs of adjacent w-planes;
 * degrid and grid then interpolate every tap bilinearly instead of
 * integrating it.  With PHI_KERNEL_RADIAL nothing extra is stored: for each
 * visibility the fused kernels integrate [GC](rho, dw_i) by the same
 * quadrature at the Chebyshev points of equal pieces of [0, rho_max]
 * (pieces of 2 / R grid pixels, 16 points each in FP32, 24 in FP64; the
 * kernel is band-limited to R cycles per pixel in rho, R the window radius)
 * and evaluate every tap from its piece's Chebyshev series; a piece whose
 * two trailing coefficients exceed the quadrature tolerance counts as
 * unconverged (phi_plan_stats).  PHI_ERR_SUPPORT if the per-warp series
 * storage for the largest support would exceed the shared memory of a
 * thread block.
 *   uvw_dev:     n_vis x 3 float64 (u, v, w in wavelengths), row-major, device.
 *   weights_dev: n_vis float64 weights W_i (Eq. matrix_equation), or NULL for 1.
 *   n_vis:       >= 0.
 * The input buffers are only read during the call; a non-finite u, v or w
 * is PHI_ERR_ARG.  Returns PHI_ERR_ARG,
 * PHI_ERR_HORIZON, PHI_ERR_SUPPORT, PHI_ERR_OOM or PHI_ERR_CUDA on failure
 * (then *out is NULL).  Synchronises `stream`.
 */
int phi_plan_create(phi_plan_t* out, const phi_plan_desc* desc, const double* uvw_dev,
                    const double* weights_dev, int64_t n_vis, void* stream);

/*
 * As phi_plan_create, but with the w-stack centres given instead of found by
 * Algorithm 1: each visibility joins its nearest centre by (wbar_k - w)^2
 * (lowest index on ties) and wbar_k = centres[k].  stack_jw, when non-NULL,
 * replaces the support rule with these per-stack supports (even, 2 ..
 * max_support; PHI_SUPPORT_STACK only), so that a plan over part of an
 * observation reproduces the operator of the plan over all of it (take the
 * centres and supports from phi_plan_info) for every visibility whose
 * nearest final centre is the stack Algorithm 1's last sweep gave it (all
 * but those within the last centre shift of a stack boundary; the plan built
 * here assigns by nearest centre).  centres and stack_jw are host
 * arrays of n_stacks entries.  PHI_ERR_ARG for non-finite centres or invalid
 * supports.
 */
int phi_plan_create_fixed(phi_plan_t* out, const phi_plan_desc* desc, const double* uvw_dev,
                          const double* weights_dev, int64_t n_vis, const double* centres,
                          const int32_t* stack_jw, void* stream);

/* Release the plan (after its last call has completed on its stream). */
void phi_plan_destroy(phi_plan_t plan);

/* Plan summary; per-stack arrays of n_stacks entries are filled when the
 * pointers are non-NULL: centre wbar_k (Algorithm 1), kept visibility count,
 * support J_w (per-stack maximum under PHI_SUPPORT_VIS).  Host pointers. */
int phi_plan_info(phi_plan_t plan, phi_plan_summary* info, double* wbar, int64_t* counts,
                  int32_t* jw);

/* Quadrature statistics accumulated since plan creation or the last reset:
 * taps that missed the tolerance at the refinement cap, taps evaluated, and
 * tap-node integrand evaluations (all refinements included).  Synchronises
 * `stream`.  reset != 0 zeroes the counters after reading.  NULL outputs are
 * skipped. */
int phi_plan_stats(phi_plan_t plan, int64_t* n_unconverged, int64_t* n_taps,
                   int64_t* n_tap_nodes, int reset, void* stream);

/* Stages of phi_degrid / phi_grid, for per-stage device timing. */
enum phi_stage {
  PHI_STAGE_PREP = 0,    /* S~_k and Z                                       */
  PHI_STAGE_FFT = 1,     /* cuFFT forward or inverse                         */
  PHI_STAGE_DEGRID = 2,  /* fused w-kernel quadrature + degridding           */
  PHI_STAGE_GRID = 3,    /* fused w-kernel quadrature + gridding             */
  PHI_STAGE_FINISH = 4,  /* crop, conj(S~_k), sum over stacks                */
  PHI_STAGE_CLEAR = 5,   /* zeroing of grid and outputs                      */
  PHI_NUM_STAGES = 6
};

/* Enable (1) or disable (0) per-stage timing: CUDA events are recorded on
 * the call's stream around every stage launch of later phi_degrid/phi_grid
 * calls.  Timing adds no synchronisation. */
int phi_plan_set_timing(phi_plan_t plan, int enable);

/* Elapsed device milliseconds and launch counts per stage (arrays of
 * PHI_NUM_STAGES, host) since the last reset.  Synchronises `stream`. */
int phi_plan_timings(phi_plan_t plan, double* ms, int64_t* launches, int reset, void* stream);

/*
 * y = Phi x (Sec. 3.1, Eq. matrix_equation): per stack k, S~_k and Z
 * (Eq. S~_k, a_k = 1), F (cuFFT, unnormalised forward), then fused
 * on-the-fly w-kernel quadrature + degridding + W + fold conjugation.
 *   image_dev: N x N real, float32 (PHI_F32) or float64 (PHI_F64), row-major.
 *   vis_dev:   n_vis complex (interleaved re, im) float32 / float64, written in
 *              the caller's visibility order; dropped visibilities get 0.
 */
int phi_degrid(phi_plan_t plan, const void* image_dev, void* vis_dev, void* stream);

/*
 * x = Re(Phi^H y) (Eq. stacked adjoint): per stack k, fused w-kernel
 * quadrature + gridding of conj([GC]) W y (y conjugated for folded
 * visibilities), unnormalised inverse FFT (= F^H), crop (Z^T), conj(S~_k),
 * summed over stacks.  The image is real, so the real part is returned.
 *   vis_dev:   n_vis complex, caller order (float32 / float64 per precision).
 *   image_dev: N x N real, overwritten.
 */
int phi_grid(phi_plan_t plan, const void* vis_dev, void* image_dev, void* stream);

/*
 * phi_degrid / phi_grid with a direction-dependent effect per visibility
 * (Sec. 5.2): a band-limited DDE kernel D_i given on the grid, separable as
 * D_i(s_u, s_v) = a_i(s_u) b_i(s_v) for offsets -h..h (dde_taps = 2 h + 1,
 * odd, 1..15), convolved with the w-kernel.  Visibility i then degrids with
 *     C_i(q) = sum_s D_i(s) [GC](|u_i/du - q - s|, w_i - wbar_k)
 * over the (J_w + dde_taps - 1)^2 box around it and grids with conj(C_i).
 * The w-kernel taps come from the per-tap quadrature, or from the
 * per-visibility Chebyshev series in a PHI_KERNEL_RADIAL plan (a
 * PHI_KERNEL_TABLE plan also integrates them per tap).  dde_taps = 1 with
 * a = b = 1 is phi_degrid / phi_grid.
 *   dde_a_dev, dde_b_dev: n_vis x dde_taps complex of the plan's precision
 *              (interleaved re, im), row-major, caller's visibility order;
 *              entry j of a row is offset j - h.  Read only; the caller owns
 *              them.
 * The fold's conjugate symmetry (Sec. 3.3) holds only for DDEs that are real
 * in the image domain, so a plan built with conj_fold = 1 gives PHI_ERR_ARG,
 * as do dde_taps outside 1..15 or even, and NULL kernels with n_vis > 0.
 * PHI_ERR_SUPPORT if one warp's w-kernel box for the plan's largest support
 * does not fit in a thread block's shared memory.  No counterpart for the
 * kernels' values: the paper gives no DDE model; they are the caller's.
 * Memory: in a quadrature plan whose largest box would leave few warps per
 * SM (J_w above about 24 in FP32, 10 in FP64) the boxes go through a
 * transient device buffer of at most 2 GiB, taken with cudaMallocAsync and
 * given back with cudaFreeAsync on `stream` (stream-ordered: no device-wide
 * synchronisation); when it cannot be had the call runs single-pass, with
 * the box in shared memory.  Nothing else is allocated.
 */
int phi_degrid_dde(phi_plan_t plan, const void* image_dev, const void* dde_a_dev,
                   const void* dde_b_dev, int32_t dde_taps, void* vis_dev, void* stream);
int phi_grid_dde(phi_plan_t plan, const void* vis_dev, const void* dde_a_dev,
                 const void* dde_b_dev, int32_t dde_taps, void* image_dev, void* stream);

/*
 * Evaluate [GC](rho_i, dw_i) (Eq. analytic_convolution_hankel) for n points
 * with the plan's geometry, taper and quadrature, by the same device routine
 * the degridder and gridder use.
 *   rho_dev: n float64 radii in grid pixels (>= 0); dw_dev: n float64 w offsets.
 *   k_dev:   n complex outputs (float32 or float64 pairs per precision).
 *   n_unconverged: host pointer or NULL; when non-NULL the call synchronises
 *   `stream` and stores the number of points that missed the tolerance (a
 *   synchronisation is not allowed while `stream` is being captured into a
 *   graph: such a call returns PHI_ERR_ARG and launches nothing).
 */
int phi_wkernel(phi_plan_t plan, const double* rho_dev, const double* dw_dev, int64_t n,
                void* k_dev, int64_t* n_unconverged, void* stream);

/*
 * Allocation-free kernel evaluation (no counterpart in the paper).
 *
 * For callers that must not allocate device memory once they are running:
 * a host application whose device memory is owned by another allocator
 * (for example a framework's caching pool that has reserved the GPU), or a
 * real-time imaging pipeline in which cudaMalloc's implicit device-wide
 * synchronisation would stall the streams that are already working.
 * phi_wkernel_noalloc evaluates [GC](rho_i, dw_i) like phi_wkernel, with the
 * same device routine, but without a plan and without allocating: its
 * scratch (the quadrature node tables and one counter) lives in a fixed
 * file-scope device array of PHI_WKERNEL_NOALLOC_SCRATCH_BYTES (about 384
 * KiB), which every GPU that loads the library holds until the process
 * exits.  The caller passes the inputs and outputs.
 *
 *   params:  geometry and quadrature settings (below); max_panels must be in
 *            1..PHI_WKERNEL_NOALLOC_MAX_PANELS, otherwise PHI_ERR_ARG and
 *            nothing runs.  Refinement doubles the panels up to max_panels;
 *            points still above the tolerance there (or after max_refine
 *            doublings) are counted as unconverged.
 *   rho_dev, dw_dev, n, k_dev, n_unconverged, stream: as for phi_wkernel.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call rebuilds the node tables for its own parameters and
 * zeroes the counter, so a call does not depend on the one before it, but
 * all calls on a device share the one array: calls whose work overlaps on
 * the GPU (different streams, or host threads racing) race on it and must be
 * serialised by the caller.
 */
#define PHI_WKERNEL_NOALLOC_MAX_PANELS 32
#define PHI_WKERNEL_NOALLOC_SCRATCH_BYTES (256 + 3 * 8 * (31 * 32 * 33 / 2))

typedef struct {
  double du;                /* grid spacing in wavelengths (phi_plan_info du)   */
  double window_radius;     /* R = alpha / 2 in r = du * l units                */
  double kb_beta;           /* Kaiser-Bessel shape, > 0                          */
  double quad_rel_tol;      /* > 0                                               */
  double quad_abs_tol;      /* > 0                                               */
  double cycles_per_panel;  /* a-priori panel width in integrand cycles, > 0    */
  int32_t support;          /* J, even, 2..64                                    */
  int32_t max_refine;       /* panel-count doublings allowed, 0..8               */
  int32_t max_panels;       /* 1..PHI_WKERNEL_NOALLOC_MAX_PANELS                 */
  int32_t precision;        /* PHI_F32 or PHI_F64 (output element type)          */
} phi_wkernel_params;

int phi_wkernel_noalloc(const phi_wkernel_params* params, const double* rho_dev,
                        const double* dw_dev, int64_t n, void* k_dev, int64_t* n_unconverged,
                        void* stream);

/* Static string naming a status code. */
const char* phi_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PHI_H_ */
