/*
 * rte.h - C ABI of the GB300 FC-DOM solver for the 2D time-domain radiative
 * transfer equation (Gaggioli & Bruno, "Parallel inverse-problem solver for
 * time-domain optical tomography with perfect parallel scaling").
 *
 * Method (paper sections): transport operator and Fresnel boundary problem,
 * Sec. 2 eqs. (Toper)/(RTE); Henyey-Greenstein phase, eq. (Henyey-
 * Greeinstein); discrete ordinates with trapezoid weights, Sec. 4.1 eq.
 * (RTETrapz); Adams-Bashforth 4, Sec. 4.2 eqs. (RTEAB4)/(RTEAB4L); FC-Gram
 * continuation and filtered spectral derivative, Sec. 4.3 eqs. (RTEFCSum),
 * (FFilter), (RTEFCSumder); loop order of Algorithm 1; laser beams, eqs.
 * (RTEsources)/(RTEsources2); detectors, eq. (OpMed); objective, eq. (FObj);
 * adjoint problem, eq. (AdjointProblem); gradient, eqs. (gradient_fin) and
 * (FDwin22).
 *
 * Conventions shared by every entry point
 *  - Units: cm and ps.  Grid point (i, j) sits at (xmin + i dx, ymin + j dy),
 *    i < nx, j < ny; nx and ny count points (N_x + 1 in the paper).
 *  - Ordinates theta_m = 2 pi m / M, m = 0..M-1 (M even, 8 <= M <= 64,
 *    M a multiple of 8).
 *  - Device arrays are FP32, row-major [j][i] (y outer, x inner), owned by
 *    the caller; the library copies what it keeps.  Host arrays are plain
 *    structs owned by the caller and read during the call only.
 *  - Every call is asynchronous on the context's CUDA stream except where
 *    noted (J_out synchronises).  The library allocates its own device
 *    scratch (state, history, checkpoints) with cudaMalloc and frees it in
 *    rte_destroy.
 *  - Errors are returned as rte_status; nothing is thrown across the ABI.
 *    After RTE_ERR_CUDA the context should be destroyed.
 */
#ifndef RTE_FCDOM_H
#define RTE_FCDOM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rte_status {
  RTE_OK = 0,
  RTE_ERR_INVALID_ARG = 1,  /* bad pointer, size or parameter */
  RTE_ERR_UNSTABLE_DT = 2,  /* dt outside the estimated AB4 stability region */
  RTE_ERR_OOM = 3,          /* cudaMalloc failed */
  RTE_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
  RTE_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
  RTE_ERR_STATE = 6,        /* call order violated (e.g. readout before forward) */
  RTE_ERR_UNSUPPORTED = 7   /* size outside what the kernels support */
} rte_status;

/* Uniform grid on [xmin, xmax] x [ymin, ymax] (Sec. 4.3, eq. square) and the
 * number of discrete ordinates M (Sec. 4.1).  Requires 16 <= nx, ny <= 512. */
typedef struct rte_grid {
  int nx, ny;
  double xmin, xmax, ymin, ymax;
  int M;
} rte_grid;

/* Optical constants: HG anisotropy g, refractive indices inside (n_in, the
 * paper's n_Omega) and outside (n_out, n_0), the HG denominator exponent
 * (1.5 as printed in the paper, 1.0 for the two-dimensional kernel), and the
 * speed of light in the medium c (cm/ps). */
typedef struct rte_optics {
  double g, n_in, n_out, hg_exponent, c;
} rte_optics;

/* Time step dt (ps); FC filter (alpha, beta) of eq. (FFilter), normally
 * (2, 55); checkpoint interval in steps for rte_adjoint_gradient (0: no
 * checkpoints are kept and the adjoint is unavailable); precision selects the
 * kernel family of the FC operator products:
 *   RTE_PREC_FP32   plain FP32 SIMT kernels (any supported size);
 *   RTE_PREC_TF32X3 tcgen05 tensor cores, split 3xTF32 operands (FP32-level
 *                   accuracy); requires M in {16, 32, 64} (nx, ny <= 512);
 *   RTE_PREC_TF32   tcgen05, single TF32 product (reduced precision, same
 *                   size limits);
 *   RTE_PREC_BF16X3 tcgen05 kind::f16 with BF16 operands split hi + lo, three
 *                   products (about 2^-16 relative per product);
 *   RTE_PREC_BF16   tcgen05, single BF16 product.
 * All tensor-core forms accumulate in FP32.  Every wait inside their kernels
 * is bounded; one that runs out sets the context's device timeout word, and
 * the passes launched while it is set return at once.  They synchronise the
 * stream at the end of every march (rte_forward, rte_forward_batch, both
 * adjoint gradients, rte_forward_static) to read and clear that word
 * (RTE_ERR_TIMEOUT).  Each context has its own word, so a timeout in one
 * context leaves the others' launches untouched. */
#define RTE_PREC_FP32 0
#define RTE_PREC_TF32X3 1
#define RTE_PREC_TF32 2
#define RTE_PREC_BF16X3 3
#define RTE_PREC_BF16 4
/* flags: RTE_FLAG_TC_SCATTER computes the x-pass scattering sum as a tcgen05
 * contraction into the operator accumulator (same operand split as the
 * precision; TF32 precisions and M <= 32 only, else UNSUPPORTED); without it the tensor-core forms evaluate the circulant
 * scattering sum in FP32 on the CUDA cores of the x-pass epilogue, which
 * measured faster on GB300 (0.158 vs 0.190 ms per x-pass at 256^2, M = 32,
 * 16 groups). */
#define RTE_FLAG_TC_SCATTER 1
/* RTE_FLAG_CUDA_GRAPH runs the forward march (rte_forward,
 * rte_forward_batch) as a CUDA graph: captured on the first call, replayed
 * while the step count, groups and buffers stay the same, re-captured when
 * they change.  The graph runs on a private stream ordered after the
 * context's stream by events, so the call stays asynchronous on that stream.
 * Off while per-kernel timing is on. */
#define RTE_FLAG_CUDA_GRAPH 2
/* RTE_FLAG_PHOTON_BALANCE makes rte_forward record, after every step, the
 * terms of the photon balance of every group in FP64 on the device (read
 * with rte_photon_balance).  One extra reduction launch per step, reading
 * the state once. */
#define RTE_FLAG_PHOTON_BALANCE 4
/* RTE_FLAG_TC_FUSED_STEP runs schedule 3 (the tile-local fused step of the
 * decomposed operator, Sec. 4.4) with its three contractions on the tensor
 * cores: the segment derivatives along x and y and the scattering sum as
 * tcgen05 MMAs with split 3xTF32 operands, the AB4 update, boundary
 * condition and exitance as in the FP32 form.  Requires RTE_PREC_TF32X3,
 * M = 32 and fc_parts_x, fc_parts_y >= 2 with every part owning exactly 16
 * points (else UNSUPPORTED at creation).  Without it schedule 3 runs the
 * FP32 form, which measured faster on GB300 (0.275 against 0.39-0.44 ms per
 * step at 256^2, M = 32, 16 x 16 parts, 16 groups): the form's 108 MMAs per
 * subdomain have N = 16 or 32 and cost more than the FMAs they replace. */
#define RTE_FLAG_TC_FUSED_STEP 8
/* fc_parts_x, fc_parts_y: the subdomain decomposition of Sec. 4.4 /
 * Algorithm 1 along each axis (0 or 1: one domain).  With P parts the n
 * points of a line are split into P owned ranges [k n / P, (k + 1) n / P);
 * each part continues and differentiates (eq. RTEFCSumder) its own segment,
 * the owned range plus two fringe points on every interior side, and a
 * point's derivative is its owner's (the fringe exchange of Algorithm 1).
 * The decomposed derivative is a different linear map from the global one;
 * it is built in FP64 on the host like the global operator and applied by
 * the same kernels.  Every segment must have at least 16 points. */
typedef struct rte_params {
  double dt;
  double filter_alpha, filter_beta;
  int ckpt_interval;
  int precision;
  int flags;
  int fc_parts_x, fc_parts_y;
} rte_params;

/* One laser beam s_k of eq. (RTEsources2): position (x, y) on the boundary,
 * direction theta (rad), spreads sigma_x (cm) and sigma_theta (rad), temporal
 * centre t_s and spread sigma_t (ps), delay tau (ps), amplitude; profile 0 is
 * a Gaussian in time, profile 1 the window w(|t - tau - t_s| / sigma_t) of
 * eq. (sourcelab). */
typedef struct rte_beam {
  double x, y, theta, sigma_x, sigma_theta, t_s, sigma_t, tau, amplitude;
  int profile;
} rte_beam;

/* A generalized source q_i of eq. (RTEsources): its beams fire together
 * (Transport Sweep: one beam; Multiple Staggered Sources: several, with
 * delays).  Each group is an independent forward solve. */
typedef struct rte_source_group {
  const rte_beam* beams;
  int n_beams;
} rte_source_group;

/* Detector of eq. (OpMed) at (x, y) on the boundary with window width
 * sigma_d (cm). */
typedef struct rte_detector {
  double x, y, sigma_d;
} rte_detector;

typedef struct rte_ctx rte_ctx;

/* Creates a context for one medium: builds in FP64 on the host the FC
 * derivative operators D_x, D_y (Sec. 4.3), the normalised phase matrix
 * (Sec. 4.1), the Fresnel/reflection tables of eq. (RTE) and the stability
 * estimate, and copies mua/mus ([ny][nx] device FP32, the paper's a and b).
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * The context belongs to the CUDA device current at this call.  A process
 * drives one GPU (one process per GPU, as torch.distributed launches them):
 * the kernels' shared-memory limits are set once per process, so creating a
 * context on a second device in the same process is refused.
 * dx and dy may differ; each axis gets its own operator.
 * Errors: INVALID_ARG (null pointers, M odd or not a multiple of 8, sizes
 * below 16, unknown precision or flags), UNSUPPORTED (nx or ny above 512, M
 * above 64; a tensor-core precision with M not in {16, 32, 64} or a flag it
 * does not support; a device other than the one of this process's first
 * context), UNSTABLE_DT, OOM, CUDA. */
rte_status rte_init_medium(rte_ctx** ctx, const rte_grid* grid,
                           const float* mua, const float* mus,
                           const rte_optics* optics, const rte_params* params,
                           void* cuda_stream);

/* Replaces the medium of an existing context (same grid); device FP32
 * [ny][nx].  Re-checks the stability estimate (UNSTABLE_DT). */
rte_status rte_set_medium(rte_ctx* ctx, const float* mua, const float* mus);

/* Runs n_steps AB4 steps (Algorithm 1) for every group at once, from the
 * paper's start-up (levels t^1..t^4 zero; step s produces t = (s + 4) dt and
 * imposes the boundary condition there).  Records the boundary exitance of
 * every step (input of rte_detector_readout) and, when the context has a
 * checkpoint interval, the AB4 checkpoints used by rte_adjoint_gradient.
 * snap_steps (host, n_snaps entries, each < n_steps) selects steps whose
 * fluence Phi = sum_m w_m u_m (eq. photondensity) is written to fluence_out
 * (device FP32 [group][snap][ny][nx]); fluence_out may be NULL when
 * n_snaps == 0.  Errors: INVALID_ARG, OOM, CUDA. */
rte_status rte_forward(rte_ctx* ctx, const rte_source_group* groups, int n_groups,
                       int n_steps, const int* snap_steps, int n_snaps,
                       float* fluence_out);

/* Batched forward: n_ctx contexts (media of their own grid sizes, at most
 * 64) advance through n_steps in lockstep, each with its own groups
 * (groups[i], n_groups[i] entries), exactly as rte_forward without snapshots
 * would advance each alone; afterwards rte_detector_readout, rte_objective
 * and rte_adjoint_gradient apply per context.  No counterpart in the paper
 * beyond its independent forward problems per source (Sec. 2.2); batching
 * fills the GPU with small media.  The contexts must share M, precision,
 * flags and stream.  In the tensor-core precisions every step is one x-pass
 * and one y-pass launch over the tiles of all media (longest lines first);
 * in RTE_PREC_FP32 each medium launches its own kernels.  Launches are
 * counted on ctxs[0] (in RTE_PREC_FP32 on each context).  Errors:
 * INVALID_ARG (also for mixed M, precision,
 * flags or stream, or a repeated context), OOM, CUDA, TIMEOUT. */
rte_status rte_forward_batch(rte_ctx* const* ctxs, int n_ctx,
                             const rte_source_group* const* groups,
                             const int* n_groups, int n_steps);

/* Detector curves of eq. (OpMed) for the last rte_forward: curves_out
 * (device FP32 [group][det][step]) receives G_j(t = (s + 4) dt) for every
 * step s, from the recorded exitance (trapezoid rule along each face,
 * accumulated in FP64).  Detectors may differ between calls.
 * Errors: INVALID_ARG, STATE (no forward yet), CUDA. */
rte_status rte_detector_readout(rte_ctx* ctx, const rte_detector* dets, int n_det,
                                float* curves_out);

/* Objective only: J = sum_i 1/2 sum_j sum_s (G_j - measured)^2 dt (eqs.
 * FObj/FObjpr, rectangle rule, FP64 on the device) for the last rte_forward,
 * written to *J_out (host double; synchronises the stream).  measured: device
 * FP32 [group][det][step].  Errors: INVALID_ARG, STATE, CUDA. */
rte_status rte_objective(rte_ctx* ctx, const rte_detector* dets, int n_det,
                         const float* measured, double* J_out);

/* Objective and gradient: J = sum_i 1/2 sum_j sum_s (G_j - measured)^2 dt
 * (eqs. FObj/FObjpr, rectangle rule) written to *J_out (host double; this
 * call synchronises the stream), and the continuous-adjoint gradient of
 * eqs. (AdjointProblem)/(FDwin22) summed over groups, per grid node:
 * dJ/dmua = -sum lambda u dtheta A_node dt, dJ/dmus = -sum lambda (u - Pu)
 * dtheta A_node dt (A_node the trapezoid area of the node), device FP32
 * [ny][nx] each (either may be NULL).  measured: device FP32
 * [group][det][step] for the last rte_forward's groups and steps.
 * Forward states are recomputed segment by segment from the checkpoints.
 * Errors: INVALID_ARG, STATE (no forward, or ckpt_interval == 0), OOM, CUDA. */
rte_status rte_adjoint_gradient(rte_ctx* ctx, const rte_detector* dets, int n_det,
                                const float* measured, double* J_out,
                                float* dJ_dmua, float* dJ_dmus);

/* Batched continuous adjoint: for n_ctx contexts whose last forward had the
 * same step count (rte_forward_batch, or each its own rte_forward), with the
 * same M, precision, flags, stream and checkpoint interval, computes for
 * each context i what rte_adjoint_gradient computes: J_out[i] (host double,
 * this call synchronises the stream) and the gradients dJ_dmua[i],
 * dJ_dmus[i] (device FP32 [ny_i][nx_i]; the arrays, or their entries, may be
 * NULL), from dets[i] (n_det[i] detectors) and measured[i] (device FP32
 * [group][det][step]).  No counterpart in the paper beyond its independent
 * forward/adjoint pairs per source (Sec. 3.4); batching fills the GPU with
 * small media.  In the tensor-core precisions the media march in lockstep:
 * each recomputed forward step and each adjoint step of eq.
 * (AdjointProblem) is one x-pass and one y-pass launch over the tiles of all
 * media, and each level's gradient terms (eq. FDwin22) and state saves are
 * one launch each.  Segments are recomputed before their adjoint steps, not
 * overlapped with them.  Each medium's results equal its own
 * rte_adjoint_gradient.  In RTE_PREC_FP32 the media run one after another.
 * Errors: INVALID_ARG (also mixed M, precision, flags, stream, step count or
 * checkpoint interval, a repeated context, more than 64 contexts), STATE (no
 * forward, or ckpt_interval == 0), OOM, CUDA, TIMEOUT. */
rte_status rte_adjoint_gradient_batch(rte_ctx* const* ctxs, int n_ctx, const rte_detector* const* dets,
                                      const int* n_det, const float* const* measured, double* J_out,
                                      float* const* dJ_dmua, float* const* dJ_dmus);

/* Objective and the exact gradient of the discrete objective: the same J as
 * rte_adjoint_gradient, and dJ/dmua, dJ/dmus with respect to the nodal values
 * of a and b of the discrete march itself (AB4 of eq. RTEAB4, the boundary
 * map of eq. RTE, the exitance of eq. OpMed and the rectangle rule of eq.
 * FObj), summed over groups, device FP32 [ny][nx] each (either may be NULL):
 *   dJ/dmua = -sum_s sum_m v^s u^s,  dJ/dmus = sum_s sum_m v^s (P~u^s - u^s),
 * where v^s is the adjoint of the AB4 increment of level s, found by the
 * reverse sweep of the march (the transposed FC operators D_x^T, D_y^T of
 * Sec. 4.3, the transposed boundary map and readout, the AB4 weights applied
 * backwards).  Unlike the continuous adjoint of eq. (AdjointProblem) it
 * agrees with finite differences of J to rounding, not to discretisation
 * level.  Arguments, ownership and synchronisation as rte_adjoint_gradient;
 * the transposed operators are built on the first call.  The passes run in
 * the context's precision with the one-tile-per-CTA schedule.
 * Errors: INVALID_ARG, STATE (no forward, or ckpt_interval == 0), OOM, CUDA,
 * TIMEOUT (tensor-core forms). */
rte_status rte_discrete_adjoint_gradient(rte_ctx* ctx, const rte_detector* dets, int n_det,
                                         const float* measured, double* J_out,
                                         float* dJ_dmua, float* dJ_dmus);

/* Photon balance of the last rte_forward (the context needs
 * RTE_FLAG_PHOTON_BALANCE).  Integrating eq. (RTE) over theta and Omega (the
 * scattering term integrates to zero by the normalisation of Sec. 4.1)
 * gives d/dt int Phi / c = - int a Phi - (net outward boundary flux), with
 * Phi of eq. (photondensity) and the incoming source entering the flux with
 * a negative sign.  For every group g and step s the library records, for
 * the post-boundary-condition state at t = (s + 4) dt, in FP64:
 *   out[(g n_steps + s) 3 + 0] = sum_nodes A_node Phi / c   (photons)
 *   out[(g n_steps + s) 3 + 1] = sum_nodes A_node a Phi     (absorption rate)
 *   out[(g n_steps + s) 3 + 2] = sum_faces sum_face nodes w_face
 *                                sum_m w (theta_m . nu) u_m (net outflux)
 * with the trapezoid node areas A_node, the face trapezoid weights w_face
 * (half at the face ends) and w = 2 pi / M.  The M ordinates of a node are
 * added in FP32 and every sum above that in FP64, in a fixed order (the
 * result does not depend on the schedule).  out: device double
 * [group][step][3], caller-owned.  Errors: INVALID_ARG, STATE (no forward
 * with the flag since the last forward, batched forward), CUDA. */
rte_status rte_photon_balance(rte_ctx* ctx, double* out);

/* Copies the current AB4 state of group g (u after the last step, FP32
 * [ny][nx][M]) into out (device).  Diagnostic; INVALID_ARG, STATE. */
rte_status rte_get_state(rte_ctx* ctx, int group, float* out);

/* Host-only helpers (no device work; they run without a GPU).
 * rte_host_fc_operator writes the dense FP64 FC derivative operator of a line
 * of n points at spacing h (row-major n x n, D[i*n + j] = d(out_i)/d(g_j);
 * Sec. 4.3 continuation with d = 5, C = 25 and the filtered derivative of
 * eqs. (RTEFCSum)-(RTEFCSumder)); 16 <= n <= 4096.
 * rte_host_phase_matrix writes P~[m*M + q] = w p_{m,q} normalised as in
 * Sec. 4.1.  Errors: INVALID_ARG. */
rte_status rte_host_fc_operator(int n, double h, double alpha, double beta, double* D_out);
/* The decomposed operator of rte_params.fc_parts_x / fc_parts_y for one
 * line (parts >= 1, every segment at least 16 points).  Errors: INVALID_ARG. */
rte_status rte_host_fc_operator_parts(int n, double h, double alpha, double beta, int parts,
                                      double* D_out);
rte_status rte_host_phase_matrix(int M, double g, double exponent, double* P_out);
/* The segment operators of the decomposed operator as the tensor-core fused
 * step (RTE_FLAG_TC_FUSED_STEP) takes them: for each part k, a hi tile then
 * a lo tile of 16 rows (owned point i) x 32 tf32 values (box position p,
 * the grid point lo - 2 + p), value (i, p) at i*32 + ((p/4) ^ (i%8))*4 + p%4
 * (K-major, 128-byte swizzle); hi = tf32(D), lo = tf32(D - hi), zero outside
 * the part's segment.  out: parts * 1024 floats.  Every part must own at
 * most 16 points.  Errors: INVALID_ARG. */
rte_status rte_host_segment_images(int n, double h, double alpha, double beta, int parts, float* out);
/* The transpose of the linear part of the boundary map of eq. (RTE) that
 * rte_discrete_adjoint_gradient applies, for M ordinates and the refractive
 * indices n_in -> n_out.  Tables 0..3 are the faces (left, right, bottom,
 * top), 4..7 the corners ((left, bottom), (right, bottom), (left, top),
 * (right, top)).  On a node of table t, the transposed map takes ubar[M] to
 * w[k] = sum_{q < 4} f_out[(t M + k) 4 + q] ubar[src_out[(t M + k) 4 + q]]:
 * slot 0 is the node's own value (f = 1 where ordinate k is not imposed,
 * 0 where it is), slots 1..3 the imposed ordinates that reflect into k with
 * their Fresnel coefficient (f = 0 in unused slots).  src_out and f_out hold
 * 8 * M * 4 entries (host).  Errors: INVALID_ARG (M odd or below 2, null
 * pointers, indices not positive), UNSUPPORTED (an ordinate that is the
 * reflection of more than three imposed ordinates). */
rte_status rte_host_bc_transpose(int M, double n_in, double n_out, int* src_out, double* f_out);

/* Per-kernel timing with CUDA events on the context's stream.  While on,
 * every AB4 step records events around its two passes (x-pass: scattering
 * and x-derivative; y-pass: y-derivative, AB4, boundary condition,
 * exitance).  rte_kernel_times synchronises the stream, writes the summed
 * device time in ms of each pass (ms_out[2]) and the number of timed launches
 * of each (count_out[2]), and restarts the count.  Errors: INVALID_ARG, CUDA. */
rte_status rte_set_kernel_timing(rte_ctx* ctx, int on);
rte_status rte_kernel_times(rte_ctx* ctx, double* ms_out, long long* count_out);

/* Name of the last CUDA error that a call of this library on the calling
 * thread reported as RTE_ERR_CUDA or RTE_ERR_OOM ("cudaSuccess" if none). */
const char* rte_last_cuda_error(void);

/* Number of kernels this context has launched since creation (kernels of
 * a replayed CUDA graph included). */
long long rte_kernel_launches(const rte_ctx* ctx);

/* Number of CUDA graphs captured by this context (RTE_FLAG_CUDA_GRAPH). */
long long rte_graph_captures(const rte_ctx* ctx);

/* Kernel schedule (no counterpart in the paper; a scheduling choice with
 * the same discrete operator, up to FP32 rounding and contraction order):
 *   0  persistent warp-specialised x- and y-passes, one CTA per SM, where
 *      supported (tensor-core precisions; nx, ny <= 256, M in {16, 32}, no
 *      RTE_FLAG_TC_SCATTER);
 *   1  (default) one-tile-per-CTA passes;
 *   2  one-tile-per-CTA x-pass and the pipelined persistent y-pass (the main
 *      loop of one tile and the epilogue of the previous one on two warp
 *      groups of one CTA per SM) where supported (tensor-core precisions,
 *      ny <= 256);
 *   3  tile-local fused step of the decomposed operator (Sec. 4.4,
 *      Algorithm 1): one launch per step, one CTA per subdomain and group,
 *      the whole step (segment derivatives, scattering, AB4, boundary
 *      condition, exitance) in shared memory with FP32 arithmetic, in every
 *      precision (with RTE_FLAG_TC_FUSED_STEP: its contractions on the
 *      tensor cores); where supported (fc_parts_x, fc_parts_y >= 2 with owned
 *      ranges of at most 16 points, M in {16, 32}) by rte_forward and
 *      rte_adjoint_gradient (rte_discrete_adjoint_gradient and the batched
 *      and allocation-free forwards run the one-tile-per-CTA passes);
 *   4  persistent TMA-fed x-pass (one CTA per SM; the raw slab arrives by
 *      tensor copies and converter warps split it into the tensor-core
 *      operands) and the one-tile-per-CTA y-pass, where supported
 *      (RTE_PREC_TF32X3 and RTE_PREC_TF32, nx <= 256, M in {16, 32}, no
 *      RTE_FLAG_TC_SCATTER);
 *   5  persistent TMA-fed x- and y-passes, where supported (as 4, and
 *      ny <= 256 for the y-pass).
 * Schedules 4 and 5 give the one-tile-per-CTA passes' results bit for bit.
 * rte_discrete_adjoint_gradient, rte_forward_batch and
 * rte_adjoint_gradient_batch run the one-tile-per-CTA passes under every
 * schedule.
 * Unsupported sizes run the one-tile-per-CTA passes (the plain FP32 passes
 * in RTE_PREC_FP32).  Errors: INVALID_ARG. */
rte_status rte_set_pass_variant(rte_ctx* ctx, int variant);

/* Failure injection for tests of the failure path (no counterpart in the
 * paper; host side, nothing on the device faults or hangs):
 *   RTE_FAULT_TIMEOUT_WORD  sets the context's timeout word, as a bounded
 *                           device wait that ran out would: the next march
 *                           launches tensor-core passes that return at once
 *                           and reports RTE_ERR_TIMEOUT (clearing the word);
 *   RTE_FAULT_EXPIRE_WAIT   the next march's first one-tile-per-CTA
 *                           tensor-core pass (rte_set_pass_variant 1) has one
 *                           CTA wait on a barrier that nothing arrives on,
 *                           before it issues any copy or MMA; the bounded
 *                           wait runs out after about 2 s and the march
 *                           reports RTE_ERR_TIMEOUT;
 *   RTE_FAULT_CLEAR         withdraws both.
 * Errors: INVALID_ARG (unknown kind), UNSUPPORTED (RTE_PREC_FP32: its
 * kernels have no device waits), CUDA. */
#define RTE_FAULT_CLEAR 0
#define RTE_FAULT_TIMEOUT_WORD 1
#define RTE_FAULT_EXPIRE_WAIT 2
rte_status rte_inject_fault(rte_ctx* ctx, int kind);

/* Autotuner (no counterpart in the paper): times every kernel configuration
 * the context's precision admits, with CUDA events around one forward of
 * n_trial_steps (>= 4) of the given groups after an untimed one, and keeps
 * the fastest in the context.  A configuration is choice = schedule +
 * 6 * (1 if the x-pass scattering is the tensor-core contraction), with the
 * schedule of rte_set_pass_variant (0, 1, 2, 4, 5; never 3, which is chosen
 * with the decomposition) and RTE_FLAG_TC_SCATTER.
 * Configurations a size does not support are skipped; all of them meet the
 * precision's parity bound.  *choice_out receives the chosen configuration,
 * ms_out (host, 12 entries, may be NULL) the time of each configuration tried
 * (entries of the others are untouched).  The trial forwards replace the
 * context's last-forward results.  In RTE_PREC_FP32 there is one
 * configuration and nothing is run.  Errors: INVALID_ARG, the errors of
 * rte_forward. */
rte_status rte_autotune(rte_ctx* ctx, const rte_source_group* groups, int n_groups,
                        int n_trial_steps, int* choice_out, float* ms_out);

/* Forward solve plus detector curves that allocate no device memory.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc/cudaFree while they run (device memory already reserved by
 * another allocator, latency-critical loops where an allocation may
 * synchronise the device, or a no-allocation policy after start-up).
 * It computes what rte_forward followed by rte_detector_readout computes,
 * the same discrete operator marched by the two-pass kernels of the
 * context's precision and schedule (the tile-local fused step of
 * rte_set_pass_variant 3 is not used here; it agrees with it to FP32
 * rounding): curves_out (device FP32 [group][det][step], at least
 * n_groups * n_det * n_steps floats) for n_groups groups of beams over
 * n_steps steps.  All per-call scratch
 * (state, history, exitance ring, source and detector tables) lives in one
 * file-scope device array of 64 MiB, reserved on every GPU that loads the
 * library until the process exits; a solve that needs more returns
 * RTE_ERR_UNSUPPORTED.  The context (operators and medium) must come from
 * rte_init_medium, called while allocation is allowed; this call does not
 * touch the context's rte_forward results.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress).  Every call
 * shares the array and finds the previous call's data there (it zeroes what
 * must start at zero); calls that overlap on the GPU race on it.  Host tables are copied from pageable
 * memory, so the call returns after they have left the host.  The calling
 * thread's current device must be the context's device (the array's address
 * is looked up there).  In the tensor-core precisions the call synchronises
 * the stream at the end to read the context's timeout word.
 * Errors: INVALID_ARG (also: current device is not the context's),
 * UNSUPPORTED (scratch too small), CUDA, TIMEOUT. */
rte_status rte_forward_static(rte_ctx* ctx, const rte_source_group* groups, int n_groups,
                              int n_steps, const rte_detector* dets, int n_det,
                              float* curves_out);

/* Frees the context and its device memory (synchronises its stream). */
rte_status rte_destroy(rte_ctx* ctx);

/* Static description of a status code. */
const char* rte_status_string(rte_status s);

#ifdef __cplusplus
}
#endif
#endif /* RTE_FCDOM_H */
