/*
 * bfsdf.h -- C ABI of the GB300 narrow-band posterior solver for
 * probabilistic signed-distance fusion (BayesFusion-SDF, arXiv 2602.19697).
 *
 * The library runs the method of Sec. 3 / Algorithm 1 of the paper on one
 * GPU: coarse TSDF and narrow band (Sec. 3.3, steps 1-2), sparse 8^3 bricks
 * (Sec. 3.4), depth-to-SDF observations (Sec. 3.5, step 3), the GMRF
 * posterior Q = Q0 + A^T W A, h = A^T W y + b0 (Sec. 3.6, step 4), the MAP
 * mean by PCG (Sec. 3.6, step 5), the probe estimate of diag(Q^-1) (Sec. 3.7,
 * step 6), marching cubes (Sec. 3.8, step 7) and next-best-view utilities
 * (Sec. 3.8, step 8).
 *
 * Conventions (all calls):
 *  - Grid: cubic n^3 lattice (n a multiple of 8) of voxel size `voxel`
 *    metres; voxel (i,j,k) has centre origin + (i + 1/2, j + 1/2, k + 1/2) h
 *    and linear index i + n (j + n k).  Bricks are 8^3 voxels; brick (bi,bj,bk)
 *    has linear index bi + nb (bj + nb bk), nb = n / 8.
 *  - Band layout: the N band voxels are stored compactly, ordered by (brick
 *    rank, local index lx + 8 ly + 64 lz), brick ranks ascending in linear
 *    brick index.  Every per-voxel array of the API ([N]) uses this order.
 *  - Units: the solver works in voxel units (paper's x divided by h): mu is
 *    in voxels, s in voxels^2.  Multiply by h (h^2) for metres (m^2).
 *    Camera poses are world<-camera [R | C] (row-major 3x4 floats), depth is
 *    z-depth in metres, 0 or non-finite = invalid pixel, SDF > 0 on the
 *    camera side.
 *  - Memory: every array argument may be HOST or DEVICE memory (the library
 *    asks the CUDA driver which).  Host inputs are staged through the
 *    library's device workspace; host outputs are written back before the
 *    call returns.  With device pointers only, calls are asynchronous on the
 *    context's stream except where a size must come back to the host
 *    (bf_build_band, bf_extract_surface, bf_score_views and the iteration
 *    counts of the solvers).  The caller owns every array it passes; the
 *    library owns the context, the band and their workspaces.
 *  - Devices: every call that takes a context first makes the context's
 *    device the calling thread's current device (and leaves it current), so
 *    one thread may drive contexts on several GPUs; bf_band_free and
 *    bf_net_destroy switch to the device that holds the object.
 *  - Errors: every call returns a bf_status; BF_OK is 0.  The text of the
 *    last error of a context is available from bf_last_error.  A call that
 *    fails leaves its outputs unspecified but the context usable, except
 *    after BF_ECUDA, which reports a CUDA error (the CUDA context may be lost).
 */
#ifndef BFSDF_H
#define BFSDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_ctx bf_ctx;   /* one GPU + one CUDA stream + workspace */
typedef struct bf_band bf_band; /* band, brick directory, system, solver state */

typedef enum {
  BF_OK = 0,
  BF_EINVAL = 1,          /* bad argument (null pointer, size, range)        */
  BF_ENOMEM = 2,          /* device allocation failed                        */
  BF_ECUDA = 3,           /* CUDA runtime error                              */
  BF_NOT_CONVERGED = 4,   /* iteration limit hit; best iterate written       */
  BF_BREAKDOWN = 5,       /* PCG breakdown (p.Qp <= 0 or non-finite)         */
  BF_ESTATE = 6           /* call order violated (e.g. solve before integrate) */
} bf_status;

typedef struct {
  int n;            /* voxels per axis, multiple of 8, 8..2048             */
  float voxel;      /* voxel size h in metres                              */
  float origin[3];  /* world position of the grid corner (metres)          */
} bf_grid;

typedef struct {
  float fx, fy, cx, cy; /* pinhole intrinsics (pixels)                       */
  int W, H;             /* image size (pixels)                               */
} bf_intrinsics;

typedef struct {
  double band_vox;   /* band half-width b (voxels): B = {|tsdf| <= b h}     */
  double trunc_vox;  /* coarse TSDF truncation tau_c (voxels), > band_vox  */
  double lambda;     /* smoothness weight (Sec. 3.6, Q0 equation)          */
  double lambda_b;   /* boundary anchor weight (Sec. 3.6, Q0 equation)     */
  double sig_a, sig_b;        /* sigma_depth(D) = sig_a + sig_b D^2 (m)    */
  double sig_pose, sig_model; /* sigma_pose, sigma_model (m), Sec. 3.5     */
} bf_params;

/* bf_solve_mean / bf_estimate_variance flags */
#define BF_SOLVE_FP64 1u  /* FP64 vectors and SpMV (default: FP32 vectors, FP64 inner products) */
#define BF_SOLVE_WARM 2u  /* mu holds the initial guess on entry (default: x0 = 0)              */

/* Create a context on CUDA device `device`, issuing work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  Returns BF_EINVAL for a
 * null `out`, BF_ECUDA if the device cannot be used. */
bf_status bf_create(int device, void* stream, bf_ctx** out);
void bf_destroy(bf_ctx* ctx);
const char* bf_last_error(const bf_ctx* ctx);
bf_status bf_set_stream(bf_ctx* ctx, void* stream);

/* Coarse TSDF bootstrap and narrow-band activation (Sec. 3.3, band equation
 * with alpha = 1, tau = band_vox h) on a sparse lattice of 8^3 bricks
 * (Sec. 3.4); Algorithm 1 steps 1-2.
 *   depth [T][H][W] float z-depth (m); poses [T][3][4] world<-camera.
 * TSDF: unit weight per frame, sample min(D - z_c, tau_c), samples below
 * -tau_c skipped.  Only bricks within r_B = floor((1.25 trunc_vox + 2)/8) + 1
 * bricks of a back-projected valid pixel are evaluated.  All decisions use
 * IEEE FP32 with separately rounded operations, so the band is reproducible
 * bit for bit.  *out receives a new band (free with bf_band_free).  Errors:
 * BF_EINVAL (T < 1, n not a multiple of 8, band_vox <= 0, trunc_vox <=
 * band_vox, null pointer), BF_ENOMEM. */
bf_status bf_build_band(bf_ctx* ctx, const float* depth, int T, const float* poses,
                        const bf_intrinsics* K, const bf_grid* grid, const bf_params* prm,
                        bf_band** out);
void bf_band_free(bf_band* band);

/* Sizes: band voxels N, active bricks, candidate bricks evaluated. */
bf_status bf_band_info(const bf_band* band, int64_t* n_vox, int32_t* n_bricks, int64_t* n_cand);

/* Copy band arrays out (any argument may be NULL to skip it):
 *   lin [N] int64 linear voxel index; tsdf [N] float metres; wcount [N]
 *   int32 TSDF samples; bdry [N] uint8 (1 = in dB: fewer than 6 band
 *   6-neighbours); brick_dir [nb^3] int32 rank or -1; mask [n_bricks][8]
 *   uint64 band bit of local voxel l at bit (l & 63) of word l >> 6. */
bf_status bf_export_band(bf_ctx* ctx, const bf_band* band, int64_t* lin, float* tsdf, int32_t* wcount,
                         uint8_t* bdry, int32_t* brick_dir, uint64_t* mask);

/* Depth-to-SDF observations and posterior assembly (Sec. 3.5 back-
 * projection, projective SDF, linear row and noise equations; Sec. 3.6 Q0,
 * precision and mean equations); Algorithm 1 steps 3-4.  For every valid
 * pixel the ray segment [s_p - tau, s_p + tau] around the back-projected
 * point is traversed voxel by voxel (3-D DDA, FP32 spec); each band voxel j
 * it enters receives one row a = e_j with y = clamp(r.(p - x_j), -tau, tau)/h
 * and precision w = h^2/sigma^2, sigma^2 = (sig_a + sig_b D^2)^2 + sig_pose^2
 * + sig_model^2.  Then Q_jj = lambda deg_j + lambda_b [j in dB] + sum w and
 * h_j = sum w y + lambda_b [j in dB] tsdf_j / h.  May be called several times
 * (observations accumulate; the system is reassembled after each call). */
bf_status bf_integrate_depth(bf_ctx* ctx, bf_band* band, const float* depth, int T, const float* poses,
                             const bf_intrinsics* K);

/* bf_integrate_depth with flags.  BF_INTEGRATE_DETERMINISTIC: the sums of w
 * and w y are accumulated as int64 in units of 2^-32 (each FP32 sample
 * rounded to the nearest unit, then added exactly), so they do not depend on
 * the order in which concurrent updates land and repeated runs give the same
 * bits; the FP32 sums of the default mode may differ in the last bits from
 * run to run.  The totals are converted to FP32 after each call.  A band
 * accumulates in one mode from its creation or its last
 * bf_reset_observations: a call in the other mode returns BF_ESTATE.
 * Totals must stay below 2^31 in magnitude.  Unknown flags: BF_EINVAL. */
#define BF_INTEGRATE_DETERMINISTIC 1u

/* Trilinear observation rows (Sec. 3.5: each observation is a linear row over
 * the voxel values holding the eight trilinear interpolation weights of the
 * sample point, one per corner of its cell; Sec. 3.6 precision equation: A^T W A then
 * couples each voxel with its 26 neighbours, so Q is a 27-point stencil with
 * per-voxel coefficients).  Flag of bf_integrate_depth_ex: the band
 * accumulates these rows instead of the voxel-binned ones.
 *   Samples: on every valid pixel's ray at s_p + k h for the integers k with
 *   |k| <= floor(band_vox) (2b + 1 per ray), observed value y = -k voxels
 *   (the projective SDF with n = -ray direction), precision w as in
 *   bf_integrate_depth.  Row: the weights of the sample in the cell of the 8
 *   voxel centres around it; used when every corner with a non-zero weight is
 *   a band voxel.  The cell and the weights follow an FP32 specification
 *   (each operation rounded separately, in this order): dx = ((u + 0.5) -
 *   cx)/fx, dy likewise, nrm = sqrt((dx dx + dy dy) + 1), r_i = ((R_i0 dx +
 *   R_i1 dy) + R_i2)/nrm, s = D nrm + k h, q_i = C_i + s r_i, g_i = (q_i -
 *   o_i)/h - 0.5, i0 = floor(g), f = g - i0, corner weight (w_x w_y) w_z with
 *   w = f (upper corner) or 1 - f (lower corner).
 *   Then bf_spmv, bf_solve_mean (FP32 PCG corrections inside FP64 refinement;
 *   no BF_SOLVE_WARM), bf_estimate_variance[_range] (blocks of 8 probes:
 *   rhs_block 0 or 8) and bf_export_system use the 27-point Q; bf_spmm,
 *   bf_solve_mean_static, bf_score_views_exact, bf_surrogate_variance,
 *   bf_autotune_rhs_block and bf_bench_kernel's block iteration return
 *   BF_ESTATE.  Not combinable with BF_INTEGRATE_DETERMINISTIC (BF_EINVAL); a
 *   band keeps one kind of rows until bf_reset_observations (the other kind:
 *   BF_ESTATE). */
#define BF_INTEGRATE_TRILINEAR 2u

/* The observation sums d = sum w and hdata = sum w y in FP64 ([N] double
 * each, device or host; NULL skips): after deterministic integration the
 * int64 fixed-point totals converted exactly (to 53 bits), else the FP32
 * sums widened.  BF_ESTATE before bf_integrate_depth. */
bf_status bf_export_observations_f64(bf_ctx* ctx, const bf_band* band, double* d, double* hdata);
bf_status bf_integrate_depth_ex(bf_ctx* ctx, bf_band* band, const float* depth, int T, const float* poses,
                                const bf_intrinsics* K, unsigned flags);

/* The trilinear rows of frames (depth [T][H][W], poses [T][3][4] as in
 * bf_integrate_depth; the band's own frames or any others), for checking the
 * FP32 specification above: M = T H W (2b + 1) rows in the order (frame,
 * pixel row by row, k = -b .. b); idx [M][8] int32 compact indices of the
 * cell corners (corner c at offset (c & 1, (c >> 1) & 1, (c >> 2) & 1) from
 * the cell's lowest centre; 0 for a zero-weight corner off the band), wts
 * [M][8] float weights, used [M] uint8; unused rows (invalid pixels
 * included) have idx and wts 0.  *M (host) receives M; with idx, wts and used
 * all NULL only M is returned (else all three are needed: BF_EINVAL). */
bf_status bf_export_trilinear_rows(bf_ctx* ctx, const bf_band* band, const float* depth, int T, const float* poses,
                                   const bf_intrinsics* K, int32_t* idx, float* wts, uint8_t* used, int64_t* M);

/* The 27-point precision of a band with trilinear rows (Sec. 3.6 precision
 * equation): coef [27][N] float, coef[o][j] = Q_{j, j + off(o)} with off(o) =
 * (o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1) in (i, j, k) voxel steps, 0 where
 * that neighbour is not a band voxel.  BF_ESTATE for other bands. */
bf_status bf_export_precision27(bf_ctx* ctx, const bf_band* band, float* coef);

/* Reset the accumulated observations of a band to zero. */
bf_status bf_reset_observations(bf_ctx* ctx, bf_band* band);

/* Copy the assembled system out ([N] float each; NULL skips):
 * d = sum w, hdata = sum w y, qdiag = Q_jj, rhs = h_j. */
bf_status bf_export_system(bf_ctx* ctx, const bf_band* band, float* d, float* hdata, float* qdiag, float* rhs);

/* y = Q x for x, y [N] float (Sec. 3.6 precision equation; matrix-free
 * 7-point stencil: (Qx)_j = Q_jj x_j - lambda sum_{6-nbrs k in B} x_k).
 * x, y device or host (host memory is staged; with a host y the call is
 * synchronous).  For x on a 16-byte boundary the kernel stages each brick's
 * runs by bulk copies whose waits are bounded: a wait that ran out (not
 * expected) is reported as BF_ECUDA by the next synchronous bf_spmv (host y)
 * or bf_bench_kernel call on the context. */
bf_status bf_spmv(bf_ctx* ctx, const bf_band* band, const float* x, float* y);

/* Y = Q X for R right-hand sides at once (Sec. 3.6 precision equation, the
 * same stencil and summation order as bf_spmv).  X, Y [N][R] float, the R
 * values of a voxel contiguous (device or host; host memory is staged).
 * R = 8, 16 or 32, else BF_EINVAL; BF_ESTATE before bf_integrate_depth.
 * The first call on a band builds its SpMM gather plan (kept with the band). */
bf_status bf_spmm(bf_ctx* ctx, bf_band* band, const float* X, int R, float* Y);

/* MAP mean: solve Q mu = h by Jacobi-preconditioned CG (Sec. 3.6, MAP
 * equation; Algorithm 1 step 5).  Stops when ||r||_2 <= rel_tol ||h||_2 on
 * the recursive residual, then recomputes the true residual in FP64 and
 * restarts from the current iterate (at most 64 refinement passes) if it
 * misses.
 *   mu [N] float (voxels); iters / rel_res (host, may be NULL) receive the
 *   iteration count and the final true relative residual.
 * Returns BF_NOT_CONVERGED after max_iter iterations (mu = last iterate),
 * BF_BREAKDOWN on p.Qp <= 0 or a non-finite scalar, BF_ESTATE before
 * bf_integrate_depth. */
bf_status bf_solve_mean(bf_ctx* ctx, bf_band* band, double rel_tol, int max_iter, unsigned flags, float* mu,
                        int* iters, double* rel_res);

/* Probe estimate of diag(Q^-1) (Sec. 3.7, diag equation; Algorithm 1 step 6):
 * s = (1/K) sum_k z_k (.) Q^-1 z_k with Rademacher probes z_k(j) = +1 if the
 * top bit of SplitMix64(SplitMix64(seed) ^ k * 0xD1B54A32D192ED03 ^ lin_j)
 * is 0, else -1 (lin_j the linear voxel index).  The K solves run as block
 * PCG over rhs_block columns at a time (8, 16 or 32; 0 = library choice by
 * bf_autotune_rhs_block),
 * every column to rel_tol as in bf_solve_mean; rhs_block = 1 solves the
 * probes one at a time with bf_solve_mean's single right-hand-side solver
 * (the unbatched form, for comparison).
 *   s [N] float (voxels^2); total_iters (host, may be NULL) = sum over
 *   probes of their iteration counts.
 * Errors as bf_solve_mean; BF_EINVAL for K < 1 or an unsupported block. */
bf_status bf_estimate_variance(bf_ctx* ctx, bf_band* band, int K, uint64_t seed, double rel_tol, int max_iter,
                               int rhs_block, unsigned flags, float* s, int* total_iters);

/* Scaled partial probe sum for sharding the estimator across devices or
 * calls (Sec. 3.7, diag equation): s_part = scale * sum_{k_begin <= k < k_end}
 * z_k (.) Q^-1 z_k with the probes of bf_estimate_variance (probe k is a
 * function of (seed, k, voxel) only).  With scale = 1/K, the parts of
 * disjoint ranges covering 0 .. K-1 add up to bf_estimate_variance's s (one
 * sum across ranks, no division after it); scale = 1 gives the plain sum.
 * scale must be finite and > 0 (else BF_EINVAL); other arguments and errors
 * as bf_estimate_variance. */
bf_status bf_estimate_variance_range(bf_ctx* ctx, bf_band* band, int k_begin, int k_end, double scale,
                                     uint64_t seed, double rel_tol, int max_iter, int rhs_block, unsigned flags,
                                     float* s_part, int* total_iters);

/* Marching cubes on mu (Sec. 3.8; Algorithm 1 step 7): every cube of 8 band
 * voxels, inside = mu < 0; per cube, polygons traced face by face
 * (ambiguous faces separate the inside corners) and fan-triangulated from
 * the lowest-numbered edge of each loop.  A vertex sits on each crossed
 * grid edge at t = mu_a / (mu_a - mu_b) from its lower voxel a.  Vertices
 * are ordered by (compact index of the lower voxel, axis), triangles by
 * (compact index of the cube's lower corner voxel, loop order); triangle
 * normals point to mu >= 0.  mu [N] float.  *nv, *nt (host) receive the
 * counts; the mesh is kept in the context until bf_get_surface. */
bf_status bf_extract_surface(bf_ctx* ctx, const bf_band* band, const float* mu, int64_t* nv, int64_t* nt);

/* Dual contouring on mu (Sec. 3.8: the surface is extracted by "MC or DC").
 * Cells are the cubes of 8 band voxels (inside = mu < 0).  A crossed grid
 * edge (a, b = a + e_axis, both band voxels) carries the point p = x_a + t
 * e_axis, t = mu_a / (mu_a - mu_b), and the normal n = g / |g| with g =
 * (1 - t) g_a + t g_b, g_v the central difference of mu over the voxel's
 * band neighbours along each axis (one-sided with one neighbour, 0 with
 * none; g = 0 adds the point but no plane).  Each cube with a crossed edge
 * gets one vertex, the minimiser of sum_e (n_e . (x - p_e))^2 + 0.01 |x -
 * c|^2 (c = the mean crossing point) clamped to the cube; each crossed edge
 * whose four cubes exist gives a quad of their vertices (cube offsets
 * (-1,-1), (0,-1), (0,0), (-1,0) along the two other axes taken cyclically,
 * reversed when the edge's lower end is outside), split into (q0, q1, q2),
 * (q0, q2, q3), so triangles face mu >= 0.  Hermite data and the QEF in FP64.
 * Vertices are ordered by the compact index of the cube's lower corner,
 * triangles by (compact index of the edge's lower voxel, axis).  mu [N] float
 * (voxels); *nv, *nt (host) receive the counts; the mesh is kept in the
 * context until bf_get_surface (replacing a marching-cubes mesh). */
bf_status bf_extract_surface_dc(bf_ctx* ctx, const bf_band* band, const float* mu, int64_t* nv, int64_t* nt);

/* Copy the last extracted mesh: verts [nv][3] float metres, tris [nt][3] int32. */
bf_status bf_get_surface(bf_ctx* ctx, float* verts, int32_t* tris);

/* Next-best-view utilities (Sec. 3.8, NBV equation; Algorithm 1 step 8).
 * For each candidate pose v (cand_poses [V][3][4], intrinsics K): the
 * predicted depth of each pixel is the first outside->inside zero crossing
 * of the trilinear interpolant of mu (march at h/2 from the grid entry, 10
 * bisection steps, FP32 spec); the pixel then adds predicted precision
 * dd_j = w(D) to the band voxels its DDA enters, as in bf_integrate_depth;
 * U(v) = sum_{|mu_j| <= eps} s_j^2 dd_j / (1 + s_j dd_j), with s_j floored at
 * 1/Q_jj.  mu [N] float (voxels), s [N] float (voxels^2); U [V] double
 * (host or device); *best (host, may be NULL) = argmax, lowest index on ties. */
bf_status bf_score_views(bf_ctx* ctx, const bf_band* band, const float* mu, const float* s,
                         const float* cand_poses, int V, const bf_intrinsics* K, double eps, double* U, int* best);

/* Exact view utilities: the marginal variances after a candidate's
 * observations re-estimated instead of approximated by the diagonal update
 * (s' of the Sec. 3.8 NBV equation).  For each candidate v the predicted
 * precision dd_v (as in bf_score_views) is added to the diagonal of Q and the
 * K_probes-probe estimate (seed, rel_tol, max_iter, rhs_block as in
 * bf_estimate_variance) is recomputed with the same probes;
 * U(v) = sum_{|mu_j| <= eps} (s_j - s'_j), s the estimate under Q with those
 * probes.  Costs V + 1 variance estimates.  mu [N] float (voxels);
 * U [V] double (host or device); *best (host, may be NULL) = argmax, lowest
 * index on ties; *total_iters (host, may be NULL) = probe iterations summed.
 * Errors as bf_estimate_variance and bf_score_views. */
bf_status bf_score_views_exact(bf_ctx* ctx, bf_band* band, const float* mu, const float* cand_poses, int V,
                               const bf_intrinsics* K, double eps, int K_probes, uint64_t seed, double rel_tol,
                               int max_iter, int rhs_block, double* U, int* best, int* total_iters);

/* Autotuner of the probe block width (the library choice rhs_block = 0 of
 * bf_estimate_variance uses it): times one block-PCG iteration on this band
 * at R = 8, 16, 32 (R not wider than K needs) and returns the R that
 * minimises ceil(K / R) x (time of one iteration at R).  The paper has no
 * counterpart (it solves probes one by one).  Choices are cached in the
 * context per (floor(log2 N), K class) unless force != 0, and, when the
 * environment variable BFSDF_TUNE_CACHE names a file, persisted there as
 * JSON lines and read back by later contexts on the same GPU model.
 *   *rhs_block (host) receives the choice; ms_per_iter (host [3], may be
 *   NULL) the measured ms per iteration at R = 8, 16, 32 (0 = not tried).
 * Overwrites the probe solver's workspace (no solve is in progress). */
bf_status bf_autotune_rhs_block(bf_ctx* ctx, bf_band* band, int K, int force, int* rhs_block, double* ms_per_iter);

/* Allocation-free mean solve, for callers that must not allocate device
 * memory while they run (a real-time loop with a fixed memory budget, or a
 * host application that owns the device allocator).  The paper has no
 * counterpart: it is bf_solve_mean's result (Jacobi PCG, FP32 vectors, FP64
 * inner products and FP64 true-residual refinement, same stopping rule)
 * computed with every scratch vector in one fixed array of device memory
 * that the library declares statically (about 7.4 MB per GPU, present from
 * library load until process exit).  No graph is used; the host launches
 * the iterations.
 *   Limits: band of at most 262,144 voxels (else BF_EINVAL); mu [N] must be
 *   DEVICE memory (else BF_EINVAL); x0 = 0.  Errors are reported through the
 *   status only (bf_last_error is updated only when the switch to the
 *   context's device fails).  At most 64 refinement passes, as in
 *   bf_solve_mean.
 *   The first call on a device looks up the array's device address (with
 *   the context's device current); make it before any stream capture.  All calls share the array: calls whose GPU
 *   work overlaps (other streams or threads) race and must be serialised by
 *   the caller. */
bf_status bf_solve_mean_static(bf_ctx* ctx, bf_band* band, double rel_tol, int max_iter, float* mu, int* iters,
                               double* rel_res);

/* ---- Learned warm start and variance surrogate ----------------------------
 * The paper has no counterpart: its Sec. 6 lists learned priors as future
 * work.  The network maps per-brick input tiles to a warm start for the mean
 * solve and an estimate of diag(Q^-1) that replaces the probe estimate on the
 * bricks where an independent probe judge agrees with it.
 *   Network: per band brick a 10^3 tile (the brick and a 1-voxel halo) with
 *   2 input channels, tsdf/h and log(1 + d) at band voxels and 0 elsewhere;
 *   four 3x3x3 convolutions 2 -> 32 -> 32 -> 32 -> 2 with bias, zero padding
 *   at the tile boundary, ReLU after the first three; at the brick's voxels
 *   mu_hat = tsdf/h + o0 (voxels) and log s_hat = o1 - log Q_jj (log
 *   voxels^2): residuals on the TSDF and on the Jacobi lower bound 1/Q_jj.
 *   Parameters: one float vector of bf_net_nparams() = 58,850 values,
 *   W1 b1 W2 b2 W3 b3 W4 b4 with W_l[tap][ci][co], tap = 9 (dz+1) + 3 (dy+1)
 *   + (dx+1), b_l[co].  The library keeps an FP32 master copy and Adam
 *   moments; the convolutions run on bf16 tensor-core operands (tcgen05) with FP32
 *   accumulation.
 *   Loss over the band voxels j (M of them):
 *   L = (1/M) sum_j (mu_hat_j - mu_j)^2 + (log s_hat_j - log max(s_j, 1/Q_jj))^2. */
typedef struct bf_net bf_net;

/* Number of network parameters (58,850). */
int64_t bf_net_nparams(void);

/* Create a network on the context's device with He-normal weights drawn from
 * a counter-based hash of `seed` (last layer scaled by 0.1), zero biases. */
bf_status bf_net_create(bf_ctx* ctx, uint64_t seed, bf_net** net);
void bf_net_destroy(bf_net* net);

/* Copy the FP32 parameters out / in ([nparams] floats, host or device).
 * Setting parameters resets the Adam moments and step count. */
bf_status bf_net_get_params(bf_ctx* ctx, const bf_net* net, float* params);
bf_status bf_net_set_params(bf_ctx* ctx, bf_net* net, const float* params);

/* Inference over the band (after bf_integrate_depth): mu_hat [N] float
 * (voxels; pass it to bf_solve_mean with BF_SOLVE_WARM as the initial guess)
 * and log_s_hat [N] float (pass it to bf_surrogate_variance). */
bf_status bf_net_forward(bf_ctx* ctx, bf_net* net, const bf_band* band, float* mu_hat, float* log_s_hat);

/* One training step on one band: forward, loss L (above) against targets
 * mu [N] float (voxels) and s [N] float (voxels^2; the fitted value is
 * log max(s, 1/Q_jj)), backward, then one Adam step (beta 0.9, 0.999,
 * eps 1e-8) with learning rate lr (0 = gradient only).  *loss (host, may be
 * NULL) receives L before the update; grad [nparams] float (may be NULL)
 * receives dL/dparams. */
bf_status bf_net_train_step(bf_ctx* ctx, bf_net* net, const bf_band* band, const float* mu, const float* s,
                            float lr, double* loss, float* grad);

/* diag(Q^-1) with the network's estimate where a probe judge accepts it.
 * The judge is the estimator of bf_estimate_variance restricted to probes
 * 0 .. K_judge-1 of `seed`: per voxel s_J (mean of the K_judge probe values
 * t_k = z_k (.) Q^-1 z_k), its standard error se (sample std / sqrt(K_judge)),
 * f = max(s_J, 1/Q_jj) and e = |exp(log_s_hat) - s_J|.  A brick is accepted
 * when the median over its voxels of e/f is <= 0.10 (brick_stat[b][0]) and
 * no voxel has e > 3 se + 0.1 f (brick_stat[b][1] = max e / (3 se + 0.1 f)
 * <= 1).  Output s [N] float: exp(log_s_hat) on accepted bricks; elsewhere
 * the K-probe estimate of bf_estimate_variance(K, seed), for which the
 * remaining probes K_judge .. K-1 are solved only if some brick is rejected.
 * accepted [NB] uint8 and brick_stat [NB][2] double may be NULL;
 * *n_accepted and *total_iters (host, may be NULL) receive the number of
 * accepted bricks and the summed probe iterations.  Needs 2 <= K_judge < K. */
bf_status bf_surrogate_variance(bf_ctx* ctx, bf_band* band, const float* log_s_hat, int K, int K_judge,
                                uint64_t seed, double rel_tol, int max_iter, int rhs_block, unsigned flags, float* s,
                                uint8_t* accepted, double* brick_stat, int* n_accepted, int* total_iters);

/* Timing of the network's kernels on the band's bricks (CUDA events on the
 * context stream, mean ms per repetition over `reps`):
 *   BF_NET_BENCH_FORWARD: bf_net_forward's kernels (features + 4 convolutions);
 *   BF_NET_BENCH_TRAIN: forward with loss + backward (no Adam step);
 *   BF_NET_BENCH_CONV: one 32 -> 32 forward convolution (layer 2; tcgen05 kernel);
 *   BF_NET_BENCH_WGRAD: one 32 x 32 weight-gradient pass (layer 2);
 *   BF_NET_BENCH_CONV_MMA: the same convolution on the mma.sync kernel.
 * Activations and gradients of the network are overwritten. */
#define BF_NET_BENCH_FORWARD 0
#define BF_NET_BENCH_TRAIN 1
#define BF_NET_BENCH_CONV 2
#define BF_NET_BENCH_WGRAD 3
#define BF_NET_BENCH_CONV_MMA 4
bf_status bf_net_bench(bf_ctx* ctx, bf_net* net, const bf_band* band, int which, int reps, double* ms_per_rep);

/* Kernel timing for roofline measurements: launches kernels of the solver
 * `reps` times back to back on the context stream between two CUDA events
 * and returns the mean time per repetition (ms).
 *   BF_KERNEL_SPMV: the 7-point SpMV y = Q x over the band (bf_spmv's kernel);
 *   BF_KERNEL_BLOCK_ITER: one probe-solver iteration over R = 8, 16 or 32
 *     columns (the single-pass kernel: vector updates and w = Q u);
 *   BF_KERNEL_SPMM: Y = Q X over R = 8, 16 or 32 columns (bf_spmm's kernel).
 * Inputs are the library's own workspaces (their values are not preserved). */
#define BF_KERNEL_SPMV 0
#define BF_KERNEL_BLOCK_ITER 1
#define BF_KERNEL_SPMM 2
bf_status bf_bench_kernel(bf_ctx* ctx, bf_band* band, int which, int R, int reps, double* ms_per_launch);

/* Number of GPU kernels this library has run in this process (host launches
 * plus the kernels executed inside its solver graphs); for accounting. */
bf_status bf_launch_count(int64_t* n);

#ifdef __cplusplus
}
#endif

#endif /* BFSDF_H */
