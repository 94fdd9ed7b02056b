// Kernel launchers of the FC-DOM step (internal to the library).
#pragma once
#include <cuda_runtime.h>

namespace rte_kern {

// Columns of one pass tile: (rows or columns of the grid) x ordinates.
constexpr int kTileCols = 64;
constexpr int kTM = 8, kTN = 8, kKC = 16;

// Boundary/source description shared by the y-pass epilogue.
struct BoundaryArgs {
  const int* face_refl;             // [4][M]
  const float* face_f;              // [4][M]
  const unsigned char* face_act;    // [4][M]
  const int* corner_refl;           // [4][M]
  const float* corner_f;
  const unsigned char* corner_act;
  const float* wexit;               // [4][M]
  // beam sources: q = sum_k S[g][k][node] * A[g][k][m] * T[g][k][step]
  const float* S;                   // [G][kmax][ring]
  const float* A;                   // [G][kmax][M]
  const float* T;                   // [G][kmax][T_len]
  int kmax, T_len;
  // adjoint injection: q += (1 - f) * rho[g][step][node]
  const float* rho;                 // [G][rho_len][ring] or null
  int rho_len;
  float* ring_out;                  // [G][ring_steps][ring] exitance, or null
  int ring_steps;
  // Transposed step of the exact discrete adjoint (bct_src non-null).  The
  // state buffers then hold v (U: the field the transposed operator acts
  // on) and the history w of transposed boundary values (L1 = w^{k+1},
  // L2 = w^{k+2}, L3 = w^{k+3}); the x-pass is unchanged (P~ is symmetric)
  // and the y-pass epilogue forms, with the transposed D operators,
  //   ubar = L1 + L^T v + readout^T(r^k)          (readout term on ring nodes)
  //   w^k  = BC^T ubar,  w^k[m] = sum_q bct_f[m][q] ubar[bct_src[m][q]]
  //   v'   = c dt (chi0 w^k + chi1 L1 + chi2 L2 + chi3 L3)
  // and writes v' to U and w^k to L3 (src_step = k).
  const int* bct_src;               // [8][M][4]: tables of faces 0..3, corners 4..7
  const float* bct_f;               // [8][M][4]
  const float* ebar;                // [G][ebar_len][ring]: dt sum_d Wd[d][node] r[d][k]
  int ebar_len;
};

struct StepArgs {
  int nx, ny, M, G;
  size_t plane;                     // ny*nx*M floats per group
  const float* DxT;                 // [nx][nx], DxT[k*nx + i] = D_x[i][k]
  const float* DyT;
  const float* PT;                  // [M][M], PT[q*M + m] = P~[m][q]
  const float* xi;                  // [M]
  const float* eta;
  const float* mua;                 // [ny][nx]
  const float* mus;
  float cdt;                        // c * dt
  // Tensor-core form: 0 = plain FP32 SIMT kernels, 1 = tcgen05 3xTF32,
  // 2 = tcgen05 TF32, 3 = tcgen05 bf16x3, 4 = tcgen05 BF16; DxImg/DyImg hold
  // the split, pre-swizzled operators (tf32 words or bf16 halves).
  int tc_mode;
  int tc_scatter;                   // x-pass scattering as a tcgen05 contraction
  int x_variant;                    // 0 persistent warp-specialised passes, 1 one tile per CTA, 2 pipelined y-pass,
                                    // 3 tile-local fused step, 4 TMA-fed persistent x-pass + one-tile y-pass,
                                    // 5 TMA-fed persistent x- and y-passes
  const void* DxImg;
  const void* DyImg;
  const float* PImg;                // phase matrix as the scattering operand
  // Tile-local fused step (x_variant 3) of the decomposed operator: per part
  // {lo, hi, slo, shi} (owned range, segment) and the part's segment operator
  // transposed and packed [part][k < kFusedOwnMax + 4][i < kFusedOwnMax]
  // (entry (k, i): derivative at owned point lo + i from segment point slo + k).
  int px, py;
  const int* fxp;
  const int* fyp;
  const float* FxT;
  const float* FyT;
  // The same segment operators as tensor-core B operands (3xTF32 split,
  // swizzled, indexed by box position): [part][hi, lo][16 rows][32], M = 32
  // and 16-point parts only; null otherwise.
  const float* FxImg;
  const float* FyImg;
  int fused_own_max;                // largest owned range over both axes
  int fused_exact;                  // every part owns exactly kFusedOwnMax points
  // The context's timeout word (device int): a tensor-core pass whose
  // bounded wait runs out sets it to 1, and every tensor-core pass launched
  // while it is set returns at once; the host reads and clears it after a
  // march.
  int* err;
  // Failure injection for tests: block (0, 0, 0) of the first
  // one-tile-per-CTA pass of the march waits on a barrier that nothing
  // arrives on, before it issues any copy or MMA, so that the bounded wait
  // runs out; the CTA then skips its work.
  int test_expire;
};

// Largest owned range per axis of the tile-local fused step.
constexpr int kFusedOwnMax = 16;

// One AB4 step on all groups: x-pass (R = b P u - (a+b) u - xi d_x u), then
// y-pass (L = R - eta d_y u, AB4 update, boundary condition, exitance).
// U is updated in place; Lk is written over L3 (the caller rotates the ring).
// ev (optional, 3 events) is recorded before the x-pass, between the passes
// and after the y-pass.
cudaError_t launch_step(const StepArgs& a, const BoundaryArgs& b, float* U, float* R,
                        const float* L1, const float* L2, float* L3, int step,
                        cudaStream_t s, long long* launches, cudaEvent_t* ev = nullptr);

// One medium of a batched step: its step and boundary arguments, its state
// buffers, and the CTA ranges of its tiles in the batched x- and y-pass
// launches (tiles_x = row tiles per group, tiles_y = column tiles per group).
struct BatchProblem {
  StepArgs a;
  BoundaryArgs b;
  float* U;
  float* R;
  float* L[3];
  int tile0_x, tiles_x, tile0_y, tiles_y;
};

// tcgen05 form of launch_step (a.tc_mode != 0); see rte_tc.cu.
bool tc_supported(int nx, int ny, int M, int precision, int flags);
cudaError_t launch_step_tc(const StepArgs& a, const BoundaryArgs& b, float* U, float* R,
                           const float* L1, const float* L2, float* L3, int step,
                           cudaStream_t s, long long* launches, cudaEvent_t* ev);
// Fills the CTA ranges of the problems (in order) and returns the launch
// sizes; every problem must share M, tc_mode and tc_scatter.
void tc_batch_layout(BatchProblem* probs, int n, int* ctas_x, int* ctas_y);
// One AB4 step of every problem with one x-pass and one y-pass launch;
// probs_dev is a device copy of the host table `probs`.
cudaError_t launch_step_tc_batched(const BatchProblem* probs, const BatchProblem* probs_dev, int n,
                                   int step, int hl, cudaStream_t s, long long* launches);

// Persistent warp-specialised passes (rte_tc_ws.cu): nx, ny <= 256, M in
// {16, 32}, without the tensor-core scattering flag.
bool tc_ws_supported(const StepArgs& a);
cudaError_t launch_pass_ws(bool xpass, const StepArgs& a, const BoundaryArgs& b, float* U, float* R,
                           const float* L1, const float* L2, float* L3, int src_step, int ring_step,
                           cudaStream_t s);

// Pipelined persistent y-pass (rte_tc_pipe.cu): ny <= 256, M in {16, 32, 64};
// the main loop of one tile and the epilogue of the previous one run on two
// warp groups of one CTA per SM.
bool tc_pipe_supported(const StepArgs& a);
cudaError_t launch_ypass_pipe(const StepArgs& a, const BoundaryArgs& b, float* U, const float* R, const float* L1,
                              const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s);

// Persistent TMA-fed passes (rte_tc_stream.cu): TF32 operand kinds, lines
// of at most 256 points, M in {16, 32} (the x-pass without the tensor-core
// scattering flag); the raw slab arrives by tensor copies and is split into
// operands by converter warps.  Neither has the transposed step.
bool tc_stream_supported(const StepArgs& a);
bool tc_ystream_supported(const StepArgs& a);
cudaError_t launch_xpass_stream(const StepArgs& a, const BoundaryArgs& b, const float* U, float* R,
                                cudaStream_t s);
cudaError_t launch_ypass_stream(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                                const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s);

// Tile-local fused step (rte_fused.cu): one launch per step over the
// subdomains of the decomposed operator (parts >= 2 on both axes, owned
// ranges <= kFusedOwnMax, M in {16, 32}); reads u^k from Uin and writes
// u^{k+1} to Uout (different buffers).
bool fused_supported(const StepArgs& a);
// Tensor-core form of the same step (rte_fused_tc.cu): precision 3xTF32,
// M = 32, every part owning 16 x 16 points.
bool fused_tc_supported(const StepArgs& a);
cudaError_t launch_step_fused(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                              const float* L1, const float* L2, float* L3, int step, cudaStream_t s,
                              long long* launches, cudaEvent_t* ev = nullptr);
cudaError_t launch_step_fused_tc(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                                 const float* L1, const float* L2, float* L3, int step, cudaStream_t s,
                                 long long* launches, cudaEvent_t* ev = nullptr);

// Phi[g][j][i] = w sum_m u_m  (eq. photondensity).
cudaError_t launch_fluence(const float* U, float* out, size_t out_group_stride, int nx, int ny,
                           int M, int G, size_t plane, float w, cudaStream_t s,
                           long long* launches);

// curves[g][d][s] = sum_node Wd[d][node] ring[g][s][node] over the node
// range [lo[d], hi[d]) in FP64.
cudaError_t launch_readout(const float* ring, int ring_len, int n_steps, int G,
                           const float* Wd, const int* lo, const int* hi, int n_det,
                           float* curves, double* curves64, cudaStream_t s,
                           long long* launches);

// J = 1/2 sum (curves - measured)^2 dt in FP64 (deterministic two-level
// reduction into *J_dev); resid = curves - measured.
cudaError_t launch_objective(const double* curves64, const float* measured, size_t n,
                             double dt, float* resid, double* partial, double* J_dev,
                             cudaStream_t s, long long* launches);

// rho[g][s][node] = scale * sum_d Wn[d][node] resid[g][d][s].
cudaError_t launch_rho(const float* resid, const float* Wn, int n_det, int ring_len,
                       int n_steps, int G, float scale, float* rho, cudaStream_t s,
                       long long* launches);

// grad_a[c] -= k sum_g sum_m lambda_m u_m; grad_b[c] -= k sum_g sum_m
// lambda_m (u - P u)_m, with k = scale * area[c] (scale alone when area is
// null) and lambda_m = mu_{m + M/2} when flip is set, mu_m otherwise.
cudaError_t launch_grad(const float* MU, const float* Useg, const float* PT, const float* area,
                        int nx, int ny, int M, int G, size_t plane, size_t useg_group_stride,
                        double scale, int flip, double* grad_a, double* grad_b, cudaStream_t s,
                        long long* launches);

// Photon-balance sums of the post-BC state U (every group) for one step:
// out[(g n_steps + step) 3 + k] = (photons int Phi / c, absorption int a Phi,
// net outward boundary flux) in FP64; partial holds G * balance_blocks(...)
// * 3 doubles, ticket G zeroed counters (left zeroed).
int balance_blocks(int nx, int ny, int M);
cudaError_t launch_balance(const float* U, size_t plane, int nx, int ny, int M, int G, const float* mua,
                           const double* trig, double dx, double dy, double w, double c, double* partial,
                           unsigned* ticket, double* out, int step, int n_steps, cudaStream_t s,
                           long long* launches);

// Batched gradient and state save for media that march in lockstep (one
// launch per step over all media).  Per medium: its adjoint field, the
// segment buffer of its recomputed forward states (slot k at
// seg + k * slot_floats), and what launch_grad takes; the gradient weight of
// a cell is scale * area[cell] (dtheta dt times the trapezoid node area of
// the continuous adjoint, eq. FDwin22).
struct GradJob {
  const float* MU;
  const float* seg;
  size_t slot_floats;
  const float* PT;
  const float* area;
  long long ncell;
  int M, G;
  size_t plane;
  double scale;
  double* grad_a;
  double* grad_b;
};
struct SaveJob {
  const float* src;
  float* seg;
  size_t n_floats;                  // a multiple of 4
};
// m_common: the ordinate count every job shares.
cudaError_t launch_grad_batch(const GradJob* jobs_dev, int n_jobs, int max_ncell, int m_common, int slot,
                              int flip, cudaStream_t s, long long* launches);
cudaError_t launch_save_batch(const SaveJob* jobs_dev, int n_jobs, int slot, cudaStream_t s, long long* launches);

cudaError_t launch_to_float(const double* in, float* out, size_t n, cudaStream_t s,
                            long long* launches);

}  // namespace rte_kern
