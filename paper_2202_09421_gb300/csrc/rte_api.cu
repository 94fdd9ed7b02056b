// C ABI of the FC-DOM library (include/rte.h): context, set-up uploads, the
// time-march driver, detector readout and the checkpointed adjoint gradient.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "../../include/rte.h"
#include "rte_kernels.cuh"
#include "rte_setup.h"

using rte_setup::kPi;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct rte_ctx {
  int nx = 0, ny = 0, M = 0;
  double xmin = 0, xmax = 0, ymin = 0, ymax = 0, dx = 0, dy = 0;
  rte_optics opt{};
  rte_params par{};
  cudaStream_t stream = nullptr;
  long long launches = 0;
  double rho_dx = 0, rho_dy = 0;   // spectral-radius estimates of D_x, D_y
  size_t plane = 0;                // ny * nx * M
  int ring_len = 0;
  std::vector<double> ring_x, ring_y, ring_w;
  // device tables
  DevBuf DxT, DyT, PT, xi, eta, mua, mus, area;
  DevBuf face_refl, corner_refl, face_f, corner_f, face_act, corner_act, wexit;
  DevBuf DxImg, DyImg, PImg;       // split, swizzled operators (tensor-core forms)
  // transposed operators D_x^T, D_y^T and the transposed boundary map of the
  // exact discrete adjoint (built on its first use)
  DevBuf DxTt, DyTt, DxImgT, DyImgT, bct_src, bct_f;
  bool transposed_ready = false;
  // tile-local fused step (decomposed operators): per-part ranges and the
  // packed segment operators of each axis
  DevBuf fxp, fyp, FxT, FyT;
  DevBuf FxImg, FyImg;             // the same as tensor-core operand images (16-point parts)
  int fused_own_max = 0;
  bool fused_exact = true;          // every part owns kFusedOwnMax points
  int tc_mode = 0;                 // the precision: 0 SIMT FP32, 1-4 tcgen05 forms
  int device = 0;                  // the CUDA device current at creation
  // timeout word of the tensor-core passes (one device int, see tc_check)
  // and the test-only request that the next march's first pass time out
  DevBuf err;
  bool inject_expire = false;
  // photon balance of the last rte_forward (RTE_FLAG_PHOTON_BALANCE):
  // [G][n_steps][3] FP64 terms, block partials, per-group tickets, and the
  // FP64 cos / sin of the ordinates
  DevBuf bal, bal_partial, bal_ticket, trig;
  bool bal_valid = false;
  int x_variant = 1;               // pass kernels: 0 persistent warp-specialised, 1 one tile per CTA, 2 pipelined y-pass
  // state of the last forward
  int G = 0, n_steps = -1, kmax = 0;
  int hl = 0;                      // history rotation index
  DevBuf U, R, L[3];
  DevBuf ring, S, A, T;
  DevBuf ckpt;
  int n_ckpt = 0;
  // per-kernel timing (events around every step's two passes)
  bool timing = false;
  std::vector<cudaEvent_t> events;   // 3 per timed step
  size_t n_timed = 0;
  // adjoint scratch
  DevBuf MU, RA, LA[3], seg, curves64, resid, partial, Jdev, rho, grad_a, grad_b, Wd, Wn, lohi;
  // batched forward: device copy of the problem table; batched adjoint: its
  // adjoint-march table and its gradient / state-save job tables
  DevBuf batch_tab, batch_tab_adj, batch_jobs;
  // CUDA-graph form of the forward march (RTE_FLAG_CUDA_GRAPH): the graph is
  // captured and replayed on a private stream ordered after the context's
  // stream by events, and re-captured when its key (sizes and every buffer
  // it touches) changes.
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned long long> gkey;
  long long glaunches = 0;         // kernels per replay
  long long graph_captures = 0;
  // adjoint pipeline: segment recompute on a second stream
  cudaStream_t astream = nullptr;
  cudaEvent_t aev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

// Last CUDA error a call of this library turned into a status.
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
// The CUDA device of this process's contexts (-1 until the first).
std::atomic<int> g_process_device{-1};

rte_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RTE_OK;
  g_last_cuda_error = e;
  if (e == cudaErrorMemoryAllocation) return RTE_ERR_OOM;
  return RTE_ERR_CUDA;
}

rte_status ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return RTE_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) return RTE_OK;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RTE_ERR_OOM;
  }
  b.bytes = bytes;
  return RTE_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

template <class T>
rte_status upload(DevBuf& b, const std::vector<T>& host, cudaStream_t s) {
  rte_status st = ensure(b, host.size() * sizeof(T));
  if (st != RTE_OK) return st;
  if (host.empty()) return RTE_OK;
  return cuda_status(cudaMemcpyAsync(b.p, host.data(), host.size() * sizeof(T),
                                     cudaMemcpyHostToDevice, s));
}

template <class T>
std::vector<float> to_f32(const std::vector<T>& v) {
  return std::vector<float>(v.begin(), v.end());
}

float* F(DevBuf& b) { return static_cast<float*>(b.p); }
double* D(DevBuf& b) { return static_cast<double*>(b.p); }

#define RTE_TRY(x)                      \
  do {                                  \
    rte_status _s = (x);                \
    if (_s != RTE_OK) return _s;        \
  } while (0)

// AB4 stability estimate: the transport eigenvalues lie within an ellipse
// with real semi-axis c dt max(a + b) and imaginary semi-axis
// c dt sqrt(2) rho(D); it must fit inside the ellipse through AB4's
// real-axis (0.3) and imaginary-axis (0.43) stability limits.
rte_status check_dt(rte_ctx* c, const float* mua, const float* mus) {
  std::vector<float> a(static_cast<size_t>(c->nx) * c->ny), b(a.size());
  cudaError_t e = cudaMemcpyAsync(a.data(), mua, a.size() * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b.data(), mus, b.size() * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return RTE_ERR_INVALID_ARG;
  double mx = 0.0;
  for (size_t k = 0; k < a.size(); ++k) {
    if (!(a[k] >= 0.f) || !(b[k] >= 0.f) || !std::isfinite(a[k]) || !std::isfinite(b[k]))
      return RTE_ERR_INVALID_ARG;
    mx = std::max(mx, static_cast<double>(a[k]) + b[k]);
  }
  const double cdt = c->opt.c * c->par.dt;
  const double z_abs = cdt * mx;
  const double z_adv = cdt * std::sqrt(2.0) * std::max(c->rho_dx, c->rho_dy);
  const double e2 = (z_abs / 0.3) * (z_abs / 0.3) + (z_adv / 0.43) * (z_adv / 0.43);
  return e2 <= 1.0 ? RTE_OK : RTE_ERR_UNSTABLE_DT;
}

rte_kern::StepArgs step_args(rte_ctx* c, int G) {
  rte_kern::StepArgs a;
  a.nx = c->nx; a.ny = c->ny; a.M = c->M; a.G = G; a.plane = c->plane;
  a.DxT = F(c->DxT); a.DyT = F(c->DyT); a.PT = F(c->PT);
  a.xi = F(c->xi); a.eta = F(c->eta); a.mua = F(c->mua); a.mus = F(c->mus);
  a.cdt = static_cast<float>(c->opt.c * c->par.dt);
  a.tc_mode = c->tc_mode;
  a.tc_scatter = (c->par.flags & RTE_FLAG_TC_SCATTER) ? 1 : 0;
  a.x_variant = c->x_variant;
  a.DxImg = c->DxImg.p;
  a.DyImg = c->DyImg.p;
  a.PImg = F(c->PImg);
  a.px = c->par.fc_parts_x;
  a.py = c->par.fc_parts_y;
  a.fxp = static_cast<const int*>(c->fxp.p);
  a.fyp = static_cast<const int*>(c->fyp.p);
  a.FxT = F(c->FxT);
  a.FyT = F(c->FyT);
  a.FxImg = F(c->FxImg);
  a.FyImg = F(c->FyImg);
  a.fused_own_max = c->fused_own_max;
  a.fused_exact = c->fused_exact ? 1 : 0;
  a.err = static_cast<int*>(c->err.p);
  a.test_expire = c->inject_expire ? 1 : 0;
  return a;
}

rte_kern::BoundaryArgs boundary_args(rte_ctx* c) {
  rte_kern::BoundaryArgs b;
  b.face_refl = static_cast<const int*>(c->face_refl.p);
  b.face_f = F(c->face_f);
  b.face_act = static_cast<const unsigned char*>(c->face_act.p);
  b.corner_refl = static_cast<const int*>(c->corner_refl.p);
  b.corner_f = F(c->corner_f);
  b.corner_act = static_cast<const unsigned char*>(c->corner_act.p);
  b.wexit = F(c->wexit);
  b.S = b.A = b.T = nullptr;
  b.kmax = 0; b.T_len = 0;
  b.rho = nullptr; b.rho_len = 0;
  b.ring_out = nullptr; b.ring_steps = 0;
  b.bct_src = nullptr; b.bct_f = nullptr;
  b.ebar = nullptr; b.ebar_len = 0;
  return b;
}

// Per-detector weights on the ring: trapezoid weight x window (with_trap),
// or the window alone (the pointwise term of the adjoint boundary condition).
void detector_weights(const rte_ctx* c, const rte_detector* dets, int n_det, bool with_trap,
                      std::vector<float>& W, std::vector<int>& lohi) {
  W.assign(static_cast<size_t>(n_det) * c->ring_len, 0.f);
  lohi.assign(2 * n_det, 0);
  for (int d = 0; d < n_det; ++d) {
    int lo = c->ring_len, hi = 0;
    for (int k = 0; k < c->ring_len; ++k) {
      const double r = std::hypot(c->ring_x[k] - dets[d].x, c->ring_y[k] - dets[d].y);
      const double w = rte_setup::window(r / dets[d].sigma_d) * (with_trap ? c->ring_w[k] : 1.0);
      if (w != 0.0) {
        W[static_cast<size_t>(d) * c->ring_len + k] = static_cast<float>(w);
        lo = std::min(lo, k);
        hi = std::max(hi, k + 1);
      }
    }
    if (lo > hi) lo = hi = 0;
    lohi[d] = lo;
    lohi[n_det + d] = hi;
  }
}

double temporal(const rte_beam& b, double t) {
  const double tt = t - b.tau - b.t_s;
  if (b.profile == 0) return std::exp(-tt * tt / (2.0 * b.sigma_t * b.sigma_t));
  return rte_setup::window(std::fabs(tt) / b.sigma_t);
}

double angdist(double a, double b) {
  double d = std::fmod(std::fabs(a - b), 2.0 * kPi);
  return std::min(d, 2.0 * kPi - d);
}

// Runs steps [s_begin, s_end) of the forward march on (U, R, L), starting
// from whatever state they hold; records checkpoints/exitance/fluence when
// asked.
rte_status march(rte_ctx* c, DevBuf& U, DevBuf& R, DevBuf* L, int& hl, int G, int s_begin,
                 int s_end, const rte_kern::BoundaryArgs& b, bool save_ckpt,
                 const std::vector<int>& snap_index, float* fluence_out,
                 std::vector<float*>* seg_out, double* balance_out = nullptr) {
  const rte_kern::StepArgs a = step_args(c, G);
  const size_t gbytes = static_cast<size_t>(G) * c->plane * sizeof(float);
  const int I = c->par.ckpt_interval;
  // The tile-local fused step reads u^k from one buffer and writes u^{k+1}
  // to the other (R, which it does not otherwise use); the state ends in U.
  const bool fused = a.x_variant == 3 && rte_kern::fused_supported(a);
  float* cur = F(U);
  float* oth = F(R);
  for (int s = s_begin; s < s_end; ++s) {
    float* L1 = F(L[hl]);
    float* L2 = F(L[(hl + 1) % 3]);
    float* L3 = F(L[(hl + 2) % 3]);
    if (save_ckpt && I > 0 && s % I == 0) {
      char* base = static_cast<char*>(c->ckpt.p) + static_cast<size_t>(s / I) * 4 * gbytes;
      const void* src[4] = {cur, L1, L2, L3};
      for (int q = 0; q < 4; ++q)
        RTE_TRY(cuda_status(cudaMemcpyAsync(base + q * gbytes, src[q], gbytes,
                                            cudaMemcpyDeviceToDevice, c->stream)));
    }
    cudaEvent_t* ev = nullptr;
    if (c->timing) {
      while (c->events.size() < 3 * (c->n_timed + 1)) {
        cudaEvent_t e;
        RTE_TRY(cuda_status(cudaEventCreate(&e)));
        c->events.push_back(e);
      }
      ev = &c->events[3 * c->n_timed++];
    }
    if (fused) {
      const auto step_fn = rte_kern::fused_tc_supported(a) ? rte_kern::launch_step_fused_tc
                                                           : rte_kern::launch_step_fused;
      RTE_TRY(cuda_status(step_fn(a, b, cur, oth, L1, L2, L3, s, c->stream, &c->launches, ev)));
      std::swap(cur, oth);
    } else {
      RTE_TRY(cuda_status(rte_kern::launch_step(a, b, cur, F(R), L1, L2, L3, s, c->stream,
                                                &c->launches, ev)));
    }
    hl = (hl + 2) % 3;
    if (fluence_out && snap_index[s] >= 0) {
      const size_t per = static_cast<size_t>(c->nx) * c->ny;
      const int n_snaps = static_cast<int>(std::count_if(snap_index.begin(), snap_index.end(),
                                                         [](int v) { return v >= 0; }));
      RTE_TRY(cuda_status(rte_kern::launch_fluence(
          cur, fluence_out + static_cast<size_t>(snap_index[s]) * per, per * n_snaps, c->nx,
          c->ny, c->M, G, c->plane, static_cast<float>(2.0 * kPi / c->M), c->stream,
          &c->launches)));
    }
    if (seg_out)
      RTE_TRY(cuda_status(cudaMemcpyAsync((*seg_out)[s - s_begin], cur, gbytes,
                                          cudaMemcpyDeviceToDevice, c->stream)));
    if (balance_out)
      RTE_TRY(cuda_status(rte_kern::launch_balance(
          cur, c->plane, c->nx, c->ny, c->M, G, F(c->mua), D(c->trig), c->dx, c->dy, 2.0 * kPi / c->M,
          c->opt.c, D(c->bal_partial), static_cast<unsigned*>(c->bal_ticket.p), balance_out, s, c->n_steps,
          c->stream, &c->launches)));
  }
  if (cur != F(U))
    RTE_TRY(cuda_status(cudaMemcpyAsync(U.p, cur, gbytes, cudaMemcpyDeviceToDevice, c->stream)));
  return RTE_OK;
}

// Uploads the operator E (row-major n x n, FP64) in the kernels' forms: the
// SIMT array ET[k n + i] = E[i][k] and, in the tensor-core forms, the split,
// swizzled image (synchronises: the host vectors must outlive the copies).
rte_status upload_operator(rte_ctx* c, const std::vector<double>& E, int n, DevBuf& simt, DevBuf& img) {
  std::vector<float> T(static_cast<size_t>(n) * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) T[static_cast<size_t>(k) * n + i] = static_cast<float>(E[static_cast<size_t>(i) * n + k]);
  RTE_TRY(upload(simt, T, c->stream));
  std::vector<float> im;
  std::vector<unsigned short> im16;
  if (c->tc_mode == RTE_PREC_BF16X3 || c->tc_mode == RTE_PREC_BF16) {
    rte_setup::tc_operator_image_bf16(E, n, im16);
    RTE_TRY(upload(img, im16, c->stream));
  } else if (c->tc_mode != 0) {
    rte_setup::tc_operator_image(E, n, im);
    RTE_TRY(upload(img, im, c->stream));
  }
  return cuda_status(cudaStreamSynchronize(c->stream));
}

// D_x^T, D_y^T and the transposed boundary tables of the exact discrete
// adjoint, built once per context.
rte_status ensure_transposed(rte_ctx* c) {
  if (c->transposed_ready) return RTE_OK;
  const int dims[2] = {c->nx, c->ny};
  const double hs[2] = {c->dx, c->dy};
  const int parts[2] = {c->par.fc_parts_x, c->par.fc_parts_y};
  DevBuf* simt[2] = {&c->DxTt, &c->DyTt};
  DevBuf* img[2] = {&c->DxImgT, &c->DyImgT};
  std::vector<double> Dm, Dt;
  for (int ax = 0; ax < 2; ++ax) {
    const int n = dims[ax];
    if (!rte_setup::fc_derivative_matrix_parts(n, hs[ax], c->par.filter_alpha, c->par.filter_beta, parts[ax], Dm))
      return RTE_ERR_INVALID_ARG;
    Dt.assign(Dm.size(), 0.0);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) Dt[static_cast<size_t>(k) * n + i] = Dm[static_cast<size_t>(i) * n + k];
    RTE_TRY(upload_operator(c, Dt, n, *simt[ax], *img[ax]));
  }
  rte_setup::BoundaryTables bt;
  rte_setup::boundary_tables(c->M, c->opt.n_in, c->opt.n_out, bt);
  std::vector<int> src;
  std::vector<double> f;
  if (!rte_setup::bc_transpose_tables(bt, c->M, src, f)) return RTE_ERR_UNSUPPORTED;
  RTE_TRY(upload(c->bct_src, src, c->stream));
  std::vector<float> f32 = to_f32(f);
  RTE_TRY(upload(c->bct_f, f32, c->stream));
  RTE_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  c->transposed_ready = true;
  return RTE_OK;
}

// The tcgen05 kernels bound every wait and, when one runs out, set the
// context's timeout word instead of hanging; passes launched while it is set
// return at once.  The tensor-core forms synchronise at the end of a march to
// read it, and clear it.
rte_status tc_check(rte_ctx* c) {
  c->inject_expire = false;
  if (c->tc_mode == 0) return RTE_OK;
  int flag = 0;
  RTE_TRY(cuda_status(cudaMemcpyAsync(&flag, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream)));
  RTE_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  if (!flag) return RTE_OK;
  RTE_TRY(cuda_status(cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream)));
  RTE_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  return RTE_ERR_TIMEOUT;
}

// Split, swizzled phase matrix for the tensor-core scattering contraction
// (built once, when the form is first used).
rte_status ensure_phase_image(rte_ctx* c) {
  if (c->PImg.p) return RTE_OK;
  std::vector<double> P;
  rte_setup::phase_matrix(c->M, c->opt.g, c->opt.hg_exponent, P);
  std::vector<float> img;
  rte_setup::tc_phase_image(P, c->M, img);
  RTE_TRY(upload(c->PImg, img, c->stream));
  return cuda_status(cudaStreamSynchronize(c->stream));   // img must outlive the copy
}

// Validates the beams and sets up a forward march of n_steps on G = n_groups
// groups: state buffers, checkpoint store, source factors, zero state.
rte_status prepare_forward(rte_ctx* c, const rte_source_group* groups, int n_groups, int n_steps) {
  int kmax = 0;
  for (int g = 0; g < n_groups; ++g) {
    if (groups[g].n_beams < 0 || (groups[g].n_beams > 0 && !groups[g].beams)) return RTE_ERR_INVALID_ARG;
    for (int k = 0; k < groups[g].n_beams; ++k) {
      const rte_beam& bm = groups[g].beams[k];
      if (!(bm.sigma_x > 0) || !(bm.sigma_theta > 0) || !(bm.sigma_t > 0)) return RTE_ERR_INVALID_ARG;
    }
    kmax = std::max(kmax, groups[g].n_beams);
  }
  const int G = n_groups;
  const size_t gbytes = static_cast<size_t>(G) * c->plane * sizeof(float);
  RTE_TRY(ensure(c->U, gbytes));
  RTE_TRY(ensure(c->R, gbytes));
  for (int q = 0; q < 3; ++q) RTE_TRY(ensure(c->L[q], gbytes));
  RTE_TRY(ensure(c->ring, static_cast<size_t>(G) * n_steps * c->ring_len * sizeof(float)));
  const int I = c->par.ckpt_interval;
  c->n_ckpt = I > 0 ? (n_steps + I - 1) / I : 0;
  if (I > 0) RTE_TRY(ensure(c->ckpt, static_cast<size_t>(c->n_ckpt) * 4 * gbytes));

  // Source factors q = S(node) A(m) T(step) per beam (eq. RTEsources2).
  const int kk = std::max(kmax, 1);
  std::vector<float> S(static_cast<size_t>(G) * kk * c->ring_len, 0.f),
      A(static_cast<size_t>(G) * kk * c->M, 0.f), T(static_cast<size_t>(G) * kk * n_steps, 0.f);
  for (int g = 0; g < G; ++g)
    for (int k = 0; k < groups[g].n_beams; ++k) {
      const rte_beam& bm = groups[g].beams[k];
      const size_t gk = static_cast<size_t>(g) * kk + k;
      for (int nd = 0; nd < c->ring_len; ++nd) {
        const double dx = c->ring_x[nd] - bm.x, dy = c->ring_y[nd] - bm.y;
        S[gk * c->ring_len + nd] = static_cast<float>(std::exp(-(dx * dx + dy * dy) / (2.0 * bm.sigma_x * bm.sigma_x)));
      }
      for (int m = 0; m < c->M; ++m)
        A[gk * c->M + m] = static_cast<float>(
            bm.amplitude * rte_setup::window(angdist(2.0 * kPi * m / c->M, bm.theta) / bm.sigma_theta));
      for (int s = 0; s < n_steps; ++s)
        T[gk * n_steps + s] = static_cast<float>(temporal(bm, (s + 4) * c->par.dt));
    }
  RTE_TRY(upload(c->S, S, c->stream));
  RTE_TRY(upload(c->A, A, c->stream));
  RTE_TRY(upload(c->T, T, c->stream));
  c->kmax = kmax;
  c->G = G;
  c->n_steps = n_steps;
  c->bal_valid = false;

  RTE_TRY(cuda_status(cudaMemsetAsync(c->U.p, 0, gbytes, c->stream)));
  for (int q = 0; q < 3; ++q) RTE_TRY(cuda_status(cudaMemsetAsync(c->L[q].p, 0, gbytes, c->stream)));
  c->hl = 0;
  return RTE_OK;
}

// Boundary arguments of the forward march set up by prepare_forward.
rte_kern::BoundaryArgs forward_bargs(rte_ctx* c) {
  rte_kern::BoundaryArgs b = boundary_args(c);
  b.S = F(c->S); b.A = F(c->A); b.T = F(c->T); b.kmax = c->kmax; b.T_len = c->n_steps;
  b.ring_out = F(c->ring); b.ring_steps = c->n_steps;
  return b;
}

// Checkpoint of the march state before step s (every ckpt_interval steps).
rte_status save_checkpoint(rte_ctx* c, int s, int hl) {
  const int I = c->par.ckpt_interval;
  if (I <= 0 || s % I != 0) return RTE_OK;
  const size_t gbytes = static_cast<size_t>(c->G) * c->plane * sizeof(float);
  char* base = static_cast<char*>(c->ckpt.p) + static_cast<size_t>(s / I) * 4 * gbytes;
  const void* src[4] = {c->U.p, c->L[hl].p, c->L[(hl + 1) % 3].p, c->L[(hl + 2) % 3].p};
  for (int q = 0; q < 4; ++q)
    RTE_TRY(cuda_status(cudaMemcpyAsync(base + q * gbytes, src[q], gbytes, cudaMemcpyDeviceToDevice, c->stream)));
  return RTE_OK;
}

// Runs `enqueue` (which puts the whole march on c->stream) directly, or, in
// the CUDA-graph form, replays the graph captured from it (capturing it when
// `key` differs from the cached one).  The kernel launch counter counts the
// replayed kernels.
template <class Fn>
rte_status run_march(rte_ctx* c, const std::vector<unsigned long long>& key, Fn&& enqueue) {
  if (!(c->par.flags & RTE_FLAG_CUDA_GRAPH) || c->timing) return enqueue();
  if (!c->gstream) {
    RTE_TRY(cuda_status(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)));
    for (int k = 0; k < 2; ++k)
      RTE_TRY(cuda_status(cudaEventCreateWithFlags(&c->gev[k], cudaEventDisableTiming)));
  }
  if (!c->gexec || key != c->gkey) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    const cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    c->stream = c->gstream;
    cudaGraph_t graph = nullptr;
    rte_status st = cuda_status(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    if (st == RTE_OK) {
      st = enqueue();
      const cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
      if (st == RTE_OK) st = cuda_status(e);
    }
    c->stream = user;
    c->glaunches = c->launches - l0;
    c->launches = l0;
    if (st == RTE_OK) st = cuda_status(cudaGraphInstantiate(&c->gexec, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    if (st != RTE_OK) {
      c->gexec = nullptr;
      return st;
    }
    c->gkey = key;
    ++c->graph_captures;
  }
  RTE_TRY(cuda_status(cudaEventRecord(c->gev[0], c->stream)));
  RTE_TRY(cuda_status(cudaStreamWaitEvent(c->gstream, c->gev[0], 0)));
  RTE_TRY(cuda_status(cudaGraphLaunch(c->gexec, c->gstream)));
  RTE_TRY(cuda_status(cudaEventRecord(c->gev[1], c->gstream)));
  RTE_TRY(cuda_status(cudaStreamWaitEvent(c->stream, c->gev[1], 0)));
  c->launches += c->glaunches;
  return RTE_OK;
}

unsigned long long key_ptr(const void* p) { return static_cast<unsigned long long>(reinterpret_cast<uintptr_t>(p)); }

// Key of the buffers a forward march of context c touches.
void append_forward_key(const rte_ctx* c, std::vector<unsigned long long>& key) {
  const void* ptrs[] = {c->U.p, c->R.p, c->L[0].p, c->L[1].p, c->L[2].p, c->ring.p, c->S.p, c->A.p,
                        c->T.p, c->ckpt.p, c->mua.p, c->mus.p};
  key.push_back(static_cast<unsigned long long>(c->n_steps));
  key.push_back(static_cast<unsigned long long>(c->G));
  key.push_back(static_cast<unsigned long long>(c->kmax));
  key.push_back(static_cast<unsigned long long>(c->x_variant));
  key.push_back(static_cast<unsigned long long>(c->par.flags));
  key.push_back(static_cast<unsigned long long>(c->inject_expire));
  for (const void* p : ptrs) key.push_back(key_ptr(p));
}

constexpr int kMaxBatch = 64;

}  // namespace

extern "C" {

const char* rte_status_string(rte_status s) {
  switch (s) {
    case RTE_OK: return "ok";
    case RTE_ERR_INVALID_ARG: return "invalid argument";
    case RTE_ERR_UNSTABLE_DT: return "dt outside the estimated AB4 stability region";
    case RTE_ERR_OOM: return "device memory allocation failed";
    case RTE_ERR_CUDA: return "CUDA error";
    case RTE_ERR_TIMEOUT: return "bounded device wait timed out";
    case RTE_ERR_STATE: return "call order violated";
    case RTE_ERR_UNSUPPORTED: return "size not supported by the kernels";
  }
  return "unknown status";
}

long long rte_kernel_launches(const rte_ctx* ctx) { return ctx ? ctx->launches : -1; }

const char* rte_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

long long rte_graph_captures(const rte_ctx* ctx) { return ctx ? ctx->graph_captures : -1; }

rte_status rte_set_pass_variant(rte_ctx* c, int variant) {
  if (!c || variant < 0 || variant > 5) return RTE_ERR_INVALID_ARG;
  c->x_variant = variant;
  return RTE_OK;
}

rte_status rte_inject_fault(rte_ctx* c, int kind) {
  if (!c || kind < RTE_FAULT_CLEAR || kind > RTE_FAULT_EXPIRE_WAIT) return RTE_ERR_INVALID_ARG;
  if (c->tc_mode == 0) return RTE_ERR_UNSUPPORTED;   // the FP32 kernels have no device waits
  c->inject_expire = kind == RTE_FAULT_EXPIRE_WAIT;
  return cuda_status(cudaMemsetAsync(c->err.p, kind == RTE_FAULT_TIMEOUT_WORD ? 1 : 0, sizeof(int), c->stream));
}

rte_status rte_autotune(rte_ctx* c, const rte_source_group* groups, int n_groups, int n_trial_steps,
                        int* choice_out, float* ms_out) {
  if (!c || !groups || n_groups <= 0 || n_trial_steps < 4 || !choice_out) return RTE_ERR_INVALID_ARG;
  *choice_out = c->x_variant + ((c->par.flags & RTE_FLAG_TC_SCATTER) ? 6 : 0);
  if (c->tc_mode == 0) return RTE_OK;                     // one kernel family, nothing to choose
  rte_kern::StepArgs probe = step_args(c, n_groups);
  // configurations: schedule (0, 1, 2, 4, 5) + 6 x (tensor-core scattering)
  std::vector<int> cands;
  for (int choice = 0; choice < 12; ++choice) {
    const int variant = choice % 6;
    const bool scat = choice >= 6;
    if (variant == 3) continue;                           // the fused step: chosen with the decomposition
    if (scat && !rte_kern::tc_supported(c->nx, c->ny, c->M, c->tc_mode, RTE_FLAG_TC_SCATTER)) continue;
    probe.x_variant = variant;
    probe.tc_scatter = scat ? 1 : 0;
    // skip configurations that would fall back to another one
    if (variant == 0 && !rte_kern::tc_ws_supported(probe)) continue;
    if (variant == 2 && !rte_kern::tc_pipe_supported(probe)) continue;
    if (variant == 4 && !rte_kern::tc_stream_supported(probe)) continue;
    if (variant == 5 && !rte_kern::tc_ystream_supported(probe)) continue;
    cands.push_back(choice);
  }
  const int keep_variant = c->x_variant, keep_flags = c->par.flags;
  const bool keep_timing = c->timing;
  c->timing = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rte_status st = cuda_status(cudaEventCreate(&e0));
  if (st == RTE_OK) st = cuda_status(cudaEventCreate(&e1));
  float best = 0.f;
  int best_choice = -1;
  for (size_t k = 0; k < cands.size() && st == RTE_OK; ++k) {
    const int choice = cands[k];
    c->x_variant = choice % 6;
    c->par.flags = (keep_flags & ~RTE_FLAG_TC_SCATTER) | (choice >= 6 ? RTE_FLAG_TC_SCATTER : 0);
    if (choice >= 6) st = ensure_phase_image(c);
    // one untimed forward, then a timed one
    if (st == RTE_OK) st = rte_forward(c, groups, n_groups, n_trial_steps, nullptr, 0, nullptr);
    if (st == RTE_OK) st = cuda_status(cudaEventRecord(e0, c->stream));
    if (st == RTE_OK) st = rte_forward(c, groups, n_groups, n_trial_steps, nullptr, 0, nullptr);
    if (st == RTE_OK) st = cuda_status(cudaEventRecord(e1, c->stream));
    if (st == RTE_OK) st = cuda_status(cudaEventSynchronize(e1));
    float ms = 0.f;
    if (st == RTE_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
    if (st == RTE_OK && ms_out) ms_out[choice] = ms;
    if (st == RTE_OK && (best_choice < 0 || ms < best)) {
      best = ms;
      best_choice = choice;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->timing = keep_timing;
  if (st != RTE_OK || best_choice < 0) {
    c->x_variant = keep_variant;
    c->par.flags = keep_flags;
    return st != RTE_OK ? st : RTE_ERR_STATE;
  }
  c->x_variant = best_choice % 6;
  c->par.flags = (keep_flags & ~RTE_FLAG_TC_SCATTER) | (best_choice >= 6 ? RTE_FLAG_TC_SCATTER : 0);
  *choice_out = best_choice;
  return RTE_OK;
}

rte_status rte_set_kernel_timing(rte_ctx* c, int on) {
  if (!c) return RTE_ERR_INVALID_ARG;
  c->timing = on != 0;
  c->n_timed = 0;
  return RTE_OK;
}

rte_status rte_kernel_times(rte_ctx* c, double* ms_out, long long* count_out) {
  if (!c || !ms_out || !count_out) return RTE_ERR_INVALID_ARG;
  RTE_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  double tx = 0.0, ty = 0.0;
  for (size_t k = 0; k < c->n_timed; ++k) {
    float a = 0.f, b = 0.f;
    RTE_TRY(cuda_status(cudaEventElapsedTime(&a, c->events[3 * k], c->events[3 * k + 1])));
    RTE_TRY(cuda_status(cudaEventElapsedTime(&b, c->events[3 * k + 1], c->events[3 * k + 2])));
    tx += a;
    ty += b;
  }
  ms_out[0] = tx;
  ms_out[1] = ty;
  count_out[0] = count_out[1] = static_cast<long long>(c->n_timed);
  c->n_timed = 0;
  return RTE_OK;
}

rte_status rte_host_fc_operator(int n, double h, double alpha, double beta, double* D_out) {
  if (n < 16 || n > 4096 || !(h > 0) || !D_out) return RTE_ERR_INVALID_ARG;
  std::vector<double> Dm;
  rte_setup::fc_derivative_matrix(n, h, alpha, beta, Dm);
  std::memcpy(D_out, Dm.data(), Dm.size() * sizeof(double));
  return RTE_OK;
}

rte_status rte_host_fc_operator_parts(int n, double h, double alpha, double beta, int parts, double* D_out) {
  if (n < 16 || n > 4096 || !(h > 0) || !D_out || parts < 1) return RTE_ERR_INVALID_ARG;
  std::vector<double> Dm;
  if (!rte_setup::fc_derivative_matrix_parts(n, h, alpha, beta, parts, Dm)) return RTE_ERR_INVALID_ARG;
  std::memcpy(D_out, Dm.data(), Dm.size() * sizeof(double));
  return RTE_OK;
}

rte_status rte_host_segment_images(int n, double h, double alpha, double beta, int parts, float* out) {
  if (n < 16 || n > 4096 || !(h > 0) || !out || parts < 2) return RTE_ERR_INVALID_ARG;
  std::vector<double> Dm;
  if (!rte_setup::fc_derivative_matrix_parts(n, h, alpha, beta, parts, Dm)) return RTE_ERR_INVALID_ARG;
  for (int k = 0; k < parts; ++k) {
    int lo, hi, slo, shi;
    rte_setup::part_range(n, parts, k, lo, hi, slo, shi);
    if (hi - lo > rte_kern::kFusedOwnMax) return RTE_ERR_INVALID_ARG;
  }
  for (int k = 0; k < parts; ++k) {
    int lo, hi, slo, shi;
    rte_setup::part_range(n, parts, k, lo, hi, slo, shi);
    rte_setup::tc_segment_image(Dm, n, lo, hi, slo, shi, out + static_cast<size_t>(k) * 2 * 16 * 32);
  }
  return RTE_OK;
}

rte_status rte_host_phase_matrix(int M, double g, double exponent, double* P_out) {
  if (M < 2 || !P_out || !(std::fabs(g) < 1.0)) return RTE_ERR_INVALID_ARG;
  std::vector<double> P;
  rte_setup::phase_matrix(M, g, exponent, P);
  std::memcpy(P_out, P.data(), P.size() * sizeof(double));
  return RTE_OK;
}

rte_status rte_host_bc_transpose(int M, double n_in, double n_out, int* src_out, double* f_out) {
  if (M < 2 || M % 2 != 0 || !src_out || !f_out || !(n_in > 0) || !(n_out > 0)) return RTE_ERR_INVALID_ARG;
  rte_setup::BoundaryTables bt;
  rte_setup::boundary_tables(M, n_in, n_out, bt);
  std::vector<int> src;
  std::vector<double> f;
  if (!rte_setup::bc_transpose_tables(bt, M, src, f)) return RTE_ERR_UNSUPPORTED;
  std::memcpy(src_out, src.data(), src.size() * sizeof(int));
  std::memcpy(f_out, f.data(), f.size() * sizeof(double));
  return RTE_OK;
}

rte_status rte_destroy(rte_ctx* c) {
  if (!c) return RTE_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  DevBuf* all[] = {&c->DxT, &c->DyT, &c->PT, &c->xi, &c->eta, &c->mua, &c->mus, &c->area,
                   &c->face_refl, &c->corner_refl, &c->face_f, &c->corner_f, &c->face_act,
                   &c->corner_act, &c->wexit, &c->U, &c->R, &c->L[0], &c->L[1], &c->L[2],
                   &c->ring, &c->S, &c->A, &c->T, &c->ckpt, &c->MU, &c->RA, &c->LA[0],
                   &c->LA[1], &c->LA[2], &c->seg, &c->curves64, &c->resid, &c->partial,
                   &c->Jdev, &c->rho, &c->grad_a, &c->grad_b, &c->Wd, &c->Wn, &c->lohi,
                   &c->DxImg, &c->DyImg, &c->PImg, &c->DxTt, &c->DyTt, &c->DxImgT, &c->DyImgT,
                   &c->bct_src, &c->bct_f, &c->fxp, &c->fyp, &c->FxT, &c->FyT, &c->FxImg, &c->FyImg};
  for (DevBuf* b : all) release(*b);
  release(c->batch_tab);
  release(c->batch_tab_adj);
  release(c->batch_jobs);
  release(c->err);
  release(c->bal);
  release(c->bal_partial);
  release(c->bal_ticket);
  release(c->trig);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (cudaEvent_t e : c->gev)
    if (e) cudaEventDestroy(e);
  if (c->gstream) {
    cudaStreamSynchronize(c->gstream);
    cudaStreamDestroy(c->gstream);
  }
  for (cudaEvent_t e : c->aev)
    if (e) cudaEventDestroy(e);
  if (c->astream) {
    cudaStreamSynchronize(c->astream);
    cudaStreamDestroy(c->astream);
  }
  delete c;
  return RTE_OK;
}

rte_status rte_set_medium(rte_ctx* c, const float* mua, const float* mus) {
  if (!c || !mua || !mus) return RTE_ERR_INVALID_ARG;
  RTE_TRY(check_dt(c, mua, mus));
  const size_t bytes = static_cast<size_t>(c->nx) * c->ny * sizeof(float);
  RTE_TRY(ensure(c->mua, bytes));
  RTE_TRY(ensure(c->mus, bytes));
  RTE_TRY(cuda_status(cudaMemcpyAsync(c->mua.p, mua, bytes, cudaMemcpyDeviceToDevice, c->stream)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(c->mus.p, mus, bytes, cudaMemcpyDeviceToDevice, c->stream)));
  return RTE_OK;
}

rte_status rte_init_medium(rte_ctx** out, const rte_grid* g, const float* mua, const float* mus,
                           const rte_optics* o, const rte_params* p, void* stream) {
  if (!out || !g || !mua || !mus || !o || !p) return RTE_ERR_INVALID_ARG;
  *out = nullptr;
  if (g->nx < 16 || g->ny < 16 || g->M < 8 || g->M % 8 != 0) return RTE_ERR_INVALID_ARG;
  if (g->nx > 512 || g->ny > 512 || g->M > 64) return RTE_ERR_UNSUPPORTED;
  if (!(g->xmax > g->xmin) || !(g->ymax > g->ymin)) return RTE_ERR_INVALID_ARG;
  if (!(p->dt > 0) || !(o->c > 0) || !(o->n_in > 0) || !(o->n_out > 0) || std::fabs(o->g) >= 1.0 ||
      p->ckpt_interval < 0 || (p->flags & ~(RTE_FLAG_TC_SCATTER | RTE_FLAG_CUDA_GRAPH | RTE_FLAG_PHOTON_BALANCE | RTE_FLAG_TC_FUSED_STEP)) != 0 ||
      p->precision < RTE_PREC_FP32 || p->precision > RTE_PREC_BF16 || p->fc_parts_x < 0 || p->fc_parts_y < 0)
    return RTE_ERR_INVALID_ARG;
  if (p->precision != RTE_PREC_FP32 && !rte_kern::tc_supported(g->nx, g->ny, g->M, p->precision, p->flags))
    return RTE_ERR_UNSUPPORTED;
  rte_ctx* c = new (std::nothrow) rte_ctx();
  if (!c) return RTE_ERR_OOM;
  c->nx = g->nx; c->ny = g->ny; c->M = g->M;
  c->xmin = g->xmin; c->xmax = g->xmax; c->ymin = g->ymin; c->ymax = g->ymax;
  c->dx = (g->xmax - g->xmin) / (g->nx - 1);
  c->dy = (g->ymax - g->ymin) / (g->ny - 1);
  c->opt = *o;
  c->par = *p;
  c->stream = static_cast<cudaStream_t>(stream);
  c->tc_mode = p->precision;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return RTE_ERR_CUDA;
  }
  // One GPU per process: the first context fixes the device (the kernels'
  // shared-memory limits are set once per process, on that device).
  {
    int expected = -1;
    if (!g_process_device.compare_exchange_strong(expected, c->device) && expected != c->device) {
      delete c;
      return RTE_ERR_UNSUPPORTED;
    }
  }
  c->plane = static_cast<size_t>(g->nx) * g->ny * g->M;
  c->ring_len = 2 * g->nx + 2 * g->ny;
  auto fail = [&](rte_status s) { rte_destroy(c); return s; };

  // FC derivative operators (Sec. 4.3), transposed for the kernels.
  std::vector<double> Dm;
  const int dims[2] = {g->nx, g->ny};
  const double hs[2] = {c->dx, c->dy};
  const int parts[2] = {p->fc_parts_x, p->fc_parts_y};
  DevBuf* dst[2] = {&c->DxT, &c->DyT};
  std::vector<int> part_tab[2];
  std::vector<float> seg_ops[2], seg_img[2];
  for (int ax = 0; ax < 2; ++ax) {
    const int n = dims[ax];
    if (!rte_setup::fc_derivative_matrix_parts(n, hs[ax], p->filter_alpha, p->filter_beta, parts[ax], Dm))
      return fail(RTE_ERR_INVALID_ARG);
    const rte_status s = upload_operator(c, Dm, n, *dst[ax], ax == 0 ? c->DxImg : c->DyImg);
    if (s != RTE_OK) return fail(s);
    // Tile-local fused step: each part's owned rows of its segment
    // operator, transposed and zero-padded to [kFusedOwnMax + 4][kFusedOwnMax].
    if (parts[ax] >= 2) {
      constexpr int kO = rte_kern::kFusedOwnMax, kS = kO + 4;
      part_tab[ax].assign(4 * parts[ax], 0);
      seg_ops[ax].assign(static_cast<size_t>(parts[ax]) * kS * kO, 0.f);
      seg_img[ax].assign(static_cast<size_t>(parts[ax]) * 2 * kO * 32, 0.f);
      for (int k = 0; k < parts[ax]; ++k) {
        int lo, hi, slo, shi;
        rte_setup::part_range(n, parts[ax], k, lo, hi, slo, shi);
        const int* v[4] = {&lo, &hi, &slo, &shi};
        for (int q = 0; q < 4; ++q) part_tab[ax][4 * k + q] = *v[q];
        c->fused_own_max = std::max(c->fused_own_max, hi - lo);
        if (hi - lo != rte_kern::kFusedOwnMax) c->fused_exact = false;
        if (hi - lo > kO) continue;   // the fused step is then unsupported
        for (int kk = 0; kk < shi - slo; ++kk)
          for (int i = 0; i < hi - lo; ++i)
            seg_ops[ax][(static_cast<size_t>(k) * kS + kk) * kO + i] =
                static_cast<float>(Dm[static_cast<size_t>(lo + i) * n + slo + kk]);
        rte_setup::tc_segment_image(Dm, n, lo, hi, slo, shi, seg_img[ax].data() + static_cast<size_t>(k) * 2 * kO * 32);
      }
    }
  }
  if ((p->flags & RTE_FLAG_TC_FUSED_STEP) && (parts[0] < 2 || parts[1] < 2)) return fail(RTE_ERR_UNSUPPORTED);
  if (parts[0] >= 2 && parts[1] >= 2) {
    rte_status s = upload(c->fxp, part_tab[0], c->stream);
    if (s == RTE_OK) s = upload(c->fyp, part_tab[1], c->stream);
    if (s == RTE_OK) s = upload(c->FxT, seg_ops[0], c->stream);
    if (s == RTE_OK) s = upload(c->FyT, seg_ops[1], c->stream);
    // operand images of the tensor-core fused step (3xTF32, M = 32, 16-point parts)
    if (s == RTE_OK && (p->flags & RTE_FLAG_TC_FUSED_STEP)) {
      if (!c->fused_exact || p->precision != RTE_PREC_TF32X3 || g->M != 32) s = RTE_ERR_UNSUPPORTED;
      if (s == RTE_OK) s = upload(c->FxImg, seg_img[0], c->stream);
      if (s == RTE_OK) s = upload(c->FyImg, seg_img[1], c->stream);
    }
    if (s == RTE_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
    if (s != RTE_OK) return fail(s);
  }
  c->rho_dx = rte_setup::fc_spectral_radius_parts(g->nx, c->dx, p->filter_alpha, p->filter_beta, p->fc_parts_x);
  c->rho_dy = rte_setup::fc_spectral_radius_parts(g->ny, c->dy, p->filter_alpha, p->filter_beta, p->fc_parts_y);

  // Phase matrix (Sec. 4.1), transposed: PT[q*M + m] = P~[m][q].
  std::vector<double> P;
  rte_setup::phase_matrix(g->M, o->g, o->hg_exponent, P);
  std::vector<float> PTf(P.size());
  for (int m = 0; m < g->M; ++m)
    for (int q = 0; q < g->M; ++q) PTf[static_cast<size_t>(q) * g->M + m] = static_cast<float>(P[static_cast<size_t>(m) * g->M + q]);
  std::vector<float> xi(g->M), eta(g->M);
  for (int m = 0; m < g->M; ++m) {
    xi[m] = static_cast<float>(std::cos(2.0 * kPi * m / g->M));
    eta[m] = static_cast<float>(std::sin(2.0 * kPi * m / g->M));
  }
  rte_setup::BoundaryTables bt;
  rte_setup::boundary_tables(g->M, o->n_in, o->n_out, bt);
  rte_setup::ring_geometry(g->nx, g->ny, g->xmin, g->xmax, g->ymin, g->ymax, c->ring_x, c->ring_y,
                           c->ring_w);
  std::vector<float> area(static_cast<size_t>(g->nx) * g->ny);
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      double wx = (i == 0 || i == g->nx - 1) ? 0.5 * c->dx : c->dx;
      double wy = (j == 0 || j == g->ny - 1) ? 0.5 * c->dy : c->dy;
      area[static_cast<size_t>(j) * g->nx + i] = static_cast<float>(wx * wy);
    }
  std::vector<double> trig(2 * static_cast<size_t>(g->M));
  for (int m = 0; m < g->M; ++m) {
    trig[m] = std::cos(2.0 * kPi * m / g->M);
    trig[g->M + m] = std::sin(2.0 * kPi * m / g->M);
  }
  rte_status s = ensure(c->err, sizeof(int));
  if (s == RTE_OK) s = upload(c->trig, trig, c->stream);
  if (s == RTE_OK) s = cuda_status(cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream));
  if (s == RTE_OK && c->tc_mode != 0 && (p->flags & RTE_FLAG_TC_SCATTER)) s = ensure_phase_image(c);
  if (s == RTE_OK && c->FxImg.p) s = ensure_phase_image(c);   // the tensor-core fused step's scattering operand
  if (s == RTE_OK) s = upload(c->PT, PTf, c->stream);
  if (s == RTE_OK) s = upload(c->xi, xi, c->stream);
  if (s == RTE_OK) s = upload(c->eta, eta, c->stream);
  if (s == RTE_OK) s = upload(c->area, area, c->stream);
  if (s == RTE_OK) s = upload(c->face_refl, bt.face_refl, c->stream);
  if (s == RTE_OK) s = upload(c->corner_refl, bt.corner_refl, c->stream);
  if (s == RTE_OK) s = upload(c->face_f, to_f32(bt.face_f), c->stream);
  if (s == RTE_OK) s = upload(c->corner_f, to_f32(bt.corner_f), c->stream);
  if (s == RTE_OK) s = upload(c->face_act, bt.face_act, c->stream);
  if (s == RTE_OK) s = upload(c->corner_act, bt.corner_act, c->stream);
  if (s == RTE_OK) s = upload(c->wexit, to_f32(bt.wexit), c->stream);
  if (s == RTE_OK) s = rte_set_medium(c, mua, mus);
  if (s == RTE_OK) s = cuda_status(cudaStreamSynchronize(c->stream));
  if (s != RTE_OK) return fail(s);
  *out = c;
  return RTE_OK;
}

rte_status rte_forward(rte_ctx* c, const rte_source_group* groups, int n_groups, int n_steps,
                       const int* snap_steps, int n_snaps, float* fluence_out) {
  if (!c || !groups || n_groups <= 0 || n_steps <= 0 || n_snaps < 0) return RTE_ERR_INVALID_ARG;
  if (n_snaps > 0 && (!snap_steps || !fluence_out)) return RTE_ERR_INVALID_ARG;
  std::vector<int> snap_index(n_steps, -1);
  for (int k = 0; k < n_snaps; ++k) {
    if (snap_steps[k] < 0 || snap_steps[k] >= n_steps || snap_index[snap_steps[k]] >= 0)
      return RTE_ERR_INVALID_ARG;
    snap_index[snap_steps[k]] = k;
  }
  RTE_TRY(prepare_forward(c, groups, n_groups, n_steps));
  double* balance = nullptr;
  if (c->par.flags & RTE_FLAG_PHOTON_BALANCE) {
    const int G = c->G;
    RTE_TRY(ensure(c->bal, static_cast<size_t>(G) * n_steps * 3 * sizeof(double)));
    RTE_TRY(ensure(c->bal_partial,
                   static_cast<size_t>(G) * rte_kern::balance_blocks(c->nx, c->ny, c->M) * 3 * sizeof(double)));
    RTE_TRY(ensure(c->bal_ticket, static_cast<size_t>(G) * sizeof(unsigned)));
    RTE_TRY(cuda_status(cudaMemsetAsync(c->bal_ticket.p, 0, static_cast<size_t>(G) * sizeof(unsigned), c->stream)));
    balance = D(c->bal);
  }
  const rte_kern::BoundaryArgs b = forward_bargs(c);
  std::vector<unsigned long long> key;
  append_forward_key(c, key);
  key.push_back(key_ptr(fluence_out));
  key.push_back(key_ptr(balance));
  key.push_back(key_ptr(c->bal_partial.p));
  for (int k = 0; k < n_snaps; ++k) key.push_back(static_cast<unsigned long long>(snap_steps[k]));
  RTE_TRY(run_march(c, key, [&]() {
    int hl = 0;
    return march(c, c->U, c->R, c->L, hl, c->G, 0, n_steps, b, true, snap_index, fluence_out, nullptr,
                 balance);
  }));
  c->hl = (2 * n_steps) % 3;
  const rte_status st = tc_check(c);
  if (st == RTE_OK && balance) c->bal_valid = true;
  return st;
}

rte_status rte_forward_batch(rte_ctx* const* ctxs, int n_ctx, const rte_source_group* const* groups,
                             const int* n_groups, int n_steps) {
  if (!ctxs || n_ctx <= 0 || n_ctx > kMaxBatch || !groups || !n_groups || n_steps <= 0)
    return RTE_ERR_INVALID_ARG;
  rte_ctx* c0 = ctxs[0];
  for (int i = 0; i < n_ctx; ++i) {
    rte_ctx* c = ctxs[i];
    if (!c || !groups[i] || n_groups[i] <= 0) return RTE_ERR_INVALID_ARG;
    if (c->M != c0->M || c->tc_mode != c0->tc_mode || c->par.flags != c0->par.flags || c->stream != c0->stream)
      return RTE_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == c) return RTE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_ctx; ++i) RTE_TRY(prepare_forward(ctxs[i], groups[i], n_groups[i], n_steps));
  std::vector<unsigned long long> key{static_cast<unsigned long long>(n_ctx)};
  for (int i = 0; i < n_ctx; ++i) {
    key.push_back(key_ptr(ctxs[i]));
    append_forward_key(ctxs[i], key);
  }
  const std::vector<int> no_snaps(n_steps, -1);
  std::vector<rte_kern::BoundaryArgs> bargs(n_ctx);
  for (int i = 0; i < n_ctx; ++i) bargs[i] = forward_bargs(ctxs[i]);
  if (c0->tc_mode == 0) {
    // Plain FP32 form: every medium's kernels, in lockstep.
    RTE_TRY(run_march(c0, key, [&]() {
      std::vector<int> hl(n_ctx, 0);
      for (int s = 0; s < n_steps; ++s)
        for (int i = 0; i < n_ctx; ++i) {
          rte_ctx* c = ctxs[i];
          const cudaStream_t keep = c->stream;
          c->stream = c0->stream;              // the capture stream while a graph is recorded
          const rte_status st = march(c, c->U, c->R, c->L, hl[i], c->G, s, s + 1, bargs[i], true, no_snaps,
                                      nullptr, nullptr);
          c->stream = keep;
          if (st != RTE_OK) return st;
        }
      return RTE_OK;
    }));
  } else {
    // Tensor-core form: one x-pass and one y-pass launch per step over the
    // tiles of every medium, the media with the longest lines first.
    std::vector<int> order(n_ctx);
    for (int i = 0; i < n_ctx; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return std::max(ctxs[x]->nx, ctxs[x]->ny) > std::max(ctxs[y]->nx, ctxs[y]->ny);
    });
    std::vector<rte_kern::BatchProblem> tab(n_ctx);
    for (int r = 0; r < n_ctx; ++r) {
      rte_ctx* c = ctxs[order[r]];
      rte_kern::BatchProblem& P = tab[r];
      P.a = step_args(c, c->G);
      P.b = bargs[order[r]];
      P.U = F(c->U);
      P.R = F(c->R);
      for (int q = 0; q < 3; ++q) P.L[q] = F(c->L[q]);
    }
    int ctas_x = 0, ctas_y = 0;
    rte_kern::tc_batch_layout(tab.data(), n_ctx, &ctas_x, &ctas_y);
    RTE_TRY(upload(c0->batch_tab, tab, c0->stream));
    // the table must reach the device before the host vector goes away
    RTE_TRY(cuda_status(cudaStreamSynchronize(c0->stream)));
    key.push_back(key_ptr(c0->batch_tab.p));
    const auto* dev = static_cast<const rte_kern::BatchProblem*>(c0->batch_tab.p);
    RTE_TRY(run_march(c0, key, [&]() {
      int hl = 0;
      for (int s = 0; s < n_steps; ++s) {
        for (int i = 0; i < n_ctx; ++i) {
          rte_ctx* c = ctxs[i];
          const cudaStream_t keep = c->stream;
          c->stream = c0->stream;
          const rte_status st = save_checkpoint(c, s, hl);
          c->stream = keep;
          if (st != RTE_OK) return st;
        }
        RTE_TRY(cuda_status(rte_kern::launch_step_tc_batched(tab.data(), dev, n_ctx, s, hl, c0->stream,
                                                              &c0->launches)));
        hl = (hl + 2) % 3;
      }
      return RTE_OK;
    }));
  }
  for (int i = 0; i < n_ctx; ++i) ctxs[i]->hl = (2 * n_steps) % 3;
  rte_status st = RTE_OK;
  for (int i = 0; i < n_ctx; ++i) {
    const rte_status si = tc_check(ctxs[i]);
    if (st == RTE_OK) st = si;
  }
  return st;
}

rte_status rte_detector_readout(rte_ctx* c, const rte_detector* dets, int n_det, float* curves_out) {
  if (!c || !dets || n_det <= 0 || !curves_out) return RTE_ERR_INVALID_ARG;
  if (c->n_steps <= 0) return RTE_ERR_STATE;
  for (int d = 0; d < n_det; ++d)
    if (!(dets[d].sigma_d > 0)) return RTE_ERR_INVALID_ARG;
  std::vector<float> W;
  std::vector<int> lohi;
  detector_weights(c, dets, n_det, true, W, lohi);
  RTE_TRY(upload(c->Wd, W, c->stream));
  RTE_TRY(upload(c->lohi, lohi, c->stream));
  const int* lo = static_cast<const int*>(c->lohi.p);
  return cuda_status(rte_kern::launch_readout(F(c->ring), c->ring_len, c->n_steps, c->G, F(c->Wd), lo,
                                              lo + n_det, n_det, curves_out, nullptr, c->stream,
                                              &c->launches));
}

rte_status rte_get_state(rte_ctx* c, int group, float* out) {
  if (!c || !out || group < 0) return RTE_ERR_INVALID_ARG;
  if (c->n_steps <= 0 || group >= c->G) return RTE_ERR_STATE;
  return cuda_status(cudaMemcpyAsync(out, F(c->U) + static_cast<size_t>(group) * c->plane,
                                     c->plane * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
}

rte_status rte_photon_balance(rte_ctx* c, double* out) {
  if (!c || !out) return RTE_ERR_INVALID_ARG;
  if (!c->bal_valid) return RTE_ERR_STATE;
  return cuda_status(cudaMemcpyAsync(out, c->bal.p, static_cast<size_t>(c->G) * c->n_steps * 3 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c->stream));
}

rte_status rte_objective(rte_ctx* c, const rte_detector* dets, int n_det, const float* measured,
                         double* J_out) {
  if (!c || !dets || n_det <= 0 || !measured || !J_out) return RTE_ERR_INVALID_ARG;
  if (c->n_steps <= 0) return RTE_ERR_STATE;
  for (int d = 0; d < n_det; ++d)
    if (!(dets[d].sigma_d > 0)) return RTE_ERR_INVALID_ARG;
  const size_t ncurve = static_cast<size_t>(c->G) * n_det * c->n_steps;
  std::vector<float> Wd;
  std::vector<int> lohi;
  detector_weights(c, dets, n_det, true, Wd, lohi);
  RTE_TRY(upload(c->Wd, Wd, c->stream));
  RTE_TRY(upload(c->lohi, lohi, c->stream));
  RTE_TRY(ensure(c->curves64, ncurve * sizeof(double)));
  RTE_TRY(ensure(c->resid, ncurve * sizeof(float)));
  RTE_TRY(ensure(c->partial, 256 * sizeof(double)));
  RTE_TRY(ensure(c->Jdev, sizeof(double)));
  const int* lo = static_cast<const int*>(c->lohi.p);
  RTE_TRY(cuda_status(rte_kern::launch_readout(F(c->ring), c->ring_len, c->n_steps, c->G, F(c->Wd), lo,
                                               lo + n_det, n_det, nullptr, D(c->curves64), c->stream,
                                               &c->launches)));
  RTE_TRY(cuda_status(rte_kern::launch_objective(D(c->curves64), measured, ncurve, c->par.dt, F(c->resid),
                                                 D(c->partial), D(c->Jdev), c->stream, &c->launches)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(J_out, c->Jdev.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream)));
  return cuda_status(cudaStreamSynchronize(c->stream));
}

// Objective and gradient after a forward march: the continuous adjoint of
// eq. (AdjointProblem) (discrete = false) or the exact discrete adjoint, the
// transpose of the discrete march (discrete = true).  Both recompute the
// forward levels segment by segment from the checkpoints, on a second stream,
// while the adjoint march consumes the previous segment.
static rte_status adjoint_impl(rte_ctx* c, const rte_detector* dets, int n_det, const float* measured,
                               double* J_out, float* dJ_dmua, float* dJ_dmus, bool discrete) {
  if (!c || !dets || n_det <= 0 || !measured || !J_out) return RTE_ERR_INVALID_ARG;
  if (c->n_steps <= 0 || c->par.ckpt_interval <= 0) return RTE_ERR_STATE;
  for (int d = 0; d < n_det; ++d)
    if (!(dets[d].sigma_d > 0)) return RTE_ERR_INVALID_ARG;
  if (discrete) RTE_TRY(ensure_transposed(c));
  const int G = c->G, N = c->n_steps, I = c->par.ckpt_interval;
  const size_t gfloats = static_cast<size_t>(G) * c->plane, gbytes = gfloats * sizeof(float);
  const size_t ncurve = static_cast<size_t>(G) * n_det * N;
  const size_t ncell = static_cast<size_t>(c->nx) * c->ny;
  std::vector<float> Wd, Wn;
  std::vector<int> lohi, lohi_n;
  detector_weights(c, dets, n_det, true, Wd, lohi);
  detector_weights(c, dets, n_det, false, Wn, lohi_n);
  RTE_TRY(upload(c->Wd, Wd, c->stream));
  RTE_TRY(upload(c->Wn, Wn, c->stream));
  RTE_TRY(upload(c->lohi, lohi, c->stream));
  RTE_TRY(ensure(c->curves64, ncurve * sizeof(double)));
  RTE_TRY(ensure(c->resid, ncurve * sizeof(float)));
  RTE_TRY(ensure(c->partial, 256 * sizeof(double)));
  RTE_TRY(ensure(c->Jdev, sizeof(double)));
  RTE_TRY(ensure(c->rho, static_cast<size_t>(G) * N * c->ring_len * sizeof(float)));
  RTE_TRY(ensure(c->grad_a, ncell * sizeof(double)));
  RTE_TRY(ensure(c->grad_b, ncell * sizeof(double)));
  RTE_TRY(ensure(c->MU, gbytes));
  RTE_TRY(ensure(c->RA, gbytes));
  for (int q = 0; q < 3; ++q) RTE_TRY(ensure(c->LA[q], gbytes));
  RTE_TRY(ensure(c->seg, 2 * static_cast<size_t>(I) * gbytes));   // two segment buffers
  if (!c->astream) {
    RTE_TRY(cuda_status(cudaStreamCreateWithFlags(&c->astream, cudaStreamNonBlocking)));
    for (int k = 0; k < 4; ++k) RTE_TRY(cuda_status(cudaEventCreateWithFlags(&c->aev[k], cudaEventDisableTiming)));
  }
  const int* lo = static_cast<const int*>(c->lohi.p);

  // Detector curves (FP64), residual and objective (eq. FObj), then the
  // adjoint boundary data rho = sum_j r_j w(|x - x_j| / sigma_d).
  RTE_TRY(cuda_status(rte_kern::launch_readout(F(c->ring), c->ring_len, N, G, F(c->Wd), lo, lo + n_det,
                                               n_det, nullptr, D(c->curves64), c->stream, &c->launches)));
  RTE_TRY(cuda_status(rte_kern::launch_objective(D(c->curves64), measured, ncurve, c->par.dt, F(c->resid),
                                                 D(c->partial), D(c->Jdev), c->stream, &c->launches)));
  // Discrete form: ebar = dt sum_j Wd_j r_j, the transpose of the readout
  // (trapezoid weights included) applied to dJ/dG = dt r.
  RTE_TRY(cuda_status(rte_kern::launch_rho(F(c->resid), discrete ? F(c->Wd) : F(c->Wn), n_det, c->ring_len,
                                           N, G, discrete ? static_cast<float>(c->par.dt) : 1.0f, F(c->rho),
                                           c->stream, &c->launches)));
  RTE_TRY(cuda_status(cudaMemsetAsync(c->grad_a.p, 0, ncell * sizeof(double), c->stream)));
  RTE_TRY(cuda_status(cudaMemsetAsync(c->grad_b.p, 0, ncell * sizeof(double), c->stream)));
  RTE_TRY(cuda_status(cudaMemsetAsync(c->MU.p, 0, gbytes, c->stream)));
  for (int q = 0; q < 3; ++q) RTE_TRY(cuda_status(cudaMemsetAsync(c->LA[q].p, 0, gbytes, c->stream)));

  rte_kern::BoundaryArgs bf = boundary_args(c);
  bf.S = F(c->S); bf.A = F(c->A); bf.T = F(c->T); bf.kmax = c->kmax; bf.T_len = N;
  rte_kern::BoundaryArgs ba = boundary_args(c);
  rte_kern::StepArgs sa = step_args(c, G);
  if (discrete) {
    ba.bct_src = static_cast<const int*>(c->bct_src.p);
    ba.bct_f = F(c->bct_f);
    ba.ebar = F(c->rho);
    ba.ebar_len = N;
    sa.DxT = F(c->DxTt); sa.DyT = F(c->DyTt);
    sa.DxImg = c->DxImgT.p; sa.DyImg = c->DyImgT.p;
    sa.x_variant = 1;
  } else {
    ba.rho = F(c->rho); ba.rho_len = N;
  }
  const double scale = (2.0 * kPi / c->M) * c->par.dt;
  // continuous form with the tile-local fused step: MU and RA alternate as
  // input and output state
  const bool fused_adj = !discrete && sa.x_variant == 3 && rte_kern::fused_supported(sa);
  float* mcur = F(c->MU);
  float* moth = F(c->RA);
  int hl_adj = 0;
  std::vector<int> no_snaps(N, -1);
  // Levels needed: forward steps 0 .. N-2 (the adjoint vanishes at the last).
  const int last = N - 2;
  // Segments in reverse order.  The forward recompute of a segment (second
  // stream, into segment buffer b = k % 2) overlaps the adjoint march of the
  // segment before it in this order (context stream, reading the other
  // buffer).  Events: done_fwd[b] (recompute into b finished) orders the
  // adjoint after it; done_adj[b] (adjoint that read b finished) orders the
  // next recompute into b after it.
  std::vector<int> segs;
  for (int seg = c->n_ckpt - 1; seg >= 0; --seg)
    if (seg * I <= last) segs.push_back(seg);
  cudaEvent_t* done_fwd = c->aev;
  cudaEvent_t* done_adj = c->aev + 2;
  // the recompute stream starts after everything queued so far
  RTE_TRY(cuda_status(cudaEventRecord(done_adj[0], c->stream)));
  RTE_TRY(cuda_status(cudaStreamWaitEvent(c->astream, done_adj[0], 0)));
  auto seg_ptrs = [&](int k, int s0, int s_end) {
    std::vector<float*> segp(s_end - s0);
    const size_t base = static_cast<size_t>(k % 2) * I * gfloats;
    for (int q = 0; q < s_end - s0; ++q) segp[q] = F(c->seg) + base + static_cast<size_t>(q) * gfloats;
    return segp;
  };
  auto recompute = [&](int k) -> rte_status {
    const int seg = segs[k];
    const int s0 = seg * I, s_end = std::min(s0 + I, last + 1);
    const cudaStream_t keep = c->stream;
    c->stream = c->astream;
    const bool keep_timing = c->timing;
    c->timing = false;
    // Restore the AB4 state of the checkpoint and recompute the segment.
    const char* base = static_cast<const char*>(c->ckpt.p) + static_cast<size_t>(seg) * 4 * gbytes;
    rte_status st = cuda_status(cudaMemcpyAsync(c->U.p, base, gbytes, cudaMemcpyDeviceToDevice, c->stream));
    for (int q = 0; q < 3 && st == RTE_OK; ++q)
      st = cuda_status(cudaMemcpyAsync(c->L[q].p, base + (q + 1) * gbytes, gbytes, cudaMemcpyDeviceToDevice,
                                       c->stream));
    int hl = 0;
    std::vector<float*> segp = seg_ptrs(k, s0, s_end);
    if (st == RTE_OK) st = march(c, c->U, c->R, c->L, hl, G, s0, s_end, bf, false, no_snaps, nullptr, &segp);
    if (st == RTE_OK) st = cuda_status(cudaEventRecord(done_fwd[k % 2], c->stream));
    c->stream = keep;
    c->timing = keep_timing;
    return st;
  };
  if (!segs.empty()) RTE_TRY(recompute(0));
  // Discrete form: the transposed step with src_step N-1 on the zero state
  // gives v^{N-1} = c dt chi0 BC^T(readout^T r^{N-1}), the field that the
  // gradient of level N-1 takes.
  if (discrete && !segs.empty())
    RTE_TRY(cuda_status(rte_kern::launch_step(sa, ba, F(c->MU), F(c->RA), F(c->LA[0]), F(c->LA[1]),
                                              F(c->LA[2]), N - 1, c->stream, &c->launches)));
  if (discrete) hl_adj = 2;
  for (size_t k = 0; k < segs.size(); ++k) {
    const int seg = segs[k];
    const int s0 = seg * I, s_end = std::min(s0 + I, last + 1);
    // next segment's recompute may start once the adjoint that read its
    // buffer (segment k - 1) is done
    if (k + 1 < segs.size()) {
      if (k >= 1) RTE_TRY(cuda_status(cudaStreamWaitEvent(c->astream, done_adj[(k + 1) % 2], 0)));
      RTE_TRY(recompute(static_cast<int>(k + 1)));
    }
    RTE_TRY(cuda_status(cudaStreamWaitEvent(c->stream, done_fwd[k % 2], 0)));
    std::vector<float*> segp = seg_ptrs(static_cast<int>(k), s0, s_end);
    // Adjoint steps for levels s_end-1 .. s0.  Continuous form: the step of
    // eq. (AdjointProblem) on the flipped field, then its gradient term
    // (eq. FDwin22, area-weighted).  Discrete form: the gradient term of
    // level lvl+1 (v^{lvl+1} against u^{lvl+1}, unweighted), then the
    // transposed step that gives v^{lvl} (not needed at lvl = 0: u^0 = 0).
    for (int lvl = s_end - 1; lvl >= s0; --lvl) {
      float* L1 = F(c->LA[hl_adj]);
      float* L2 = F(c->LA[(hl_adj + 1) % 3]);
      float* L3 = F(c->LA[(hl_adj + 2) % 3]);
      if (fused_adj) {
        const auto step_fn = rte_kern::fused_tc_supported(sa) ? rte_kern::launch_step_fused_tc
                                                              : rte_kern::launch_step_fused;
        RTE_TRY(cuda_status(step_fn(sa, ba, mcur, moth, L1, L2, L3, lvl, c->stream, &c->launches, nullptr)));
        std::swap(mcur, moth);
        hl_adj = (hl_adj + 2) % 3;
      } else if (!discrete) {
        RTE_TRY(cuda_status(rte_kern::launch_step(sa, ba, F(c->MU), F(c->RA), L1, L2, L3, lvl, c->stream,
                                                  &c->launches)));
        hl_adj = (hl_adj + 2) % 3;
      }
      RTE_TRY(cuda_status(rte_kern::launch_grad(mcur, segp[lvl - s0], F(c->PT),
                                                discrete ? nullptr : F(c->area), c->nx, c->ny, c->M, G,
                                                c->plane, c->plane, discrete ? 1.0 : scale, discrete ? 0 : 1,
                                                dJ_dmua ? D(c->grad_a) : nullptr,
                                                dJ_dmus ? D(c->grad_b) : nullptr, c->stream,
                                                &c->launches)));
      if (discrete && lvl >= 1) {
        RTE_TRY(cuda_status(rte_kern::launch_step(sa, ba, F(c->MU), F(c->RA), L1, L2, L3, lvl, c->stream,
                                                  &c->launches)));
        hl_adj = (hl_adj + 2) % 3;
      }
    }
    RTE_TRY(cuda_status(cudaEventRecord(done_adj[k % 2], c->stream)));
  }
  // The forward state buffers now hold a recomputed state; mark them stale.
  if (dJ_dmua)
    RTE_TRY(cuda_status(rte_kern::launch_to_float(D(c->grad_a), dJ_dmua, ncell, c->stream, &c->launches)));
  if (dJ_dmus)
    RTE_TRY(cuda_status(rte_kern::launch_to_float(D(c->grad_b), dJ_dmus, ncell, c->stream, &c->launches)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(J_out, c->Jdev.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream)));
  RTE_TRY(cuda_status(cudaStreamSynchronize(c->stream)));
  return tc_check(c);
}

rte_status rte_adjoint_gradient(rte_ctx* c, const rte_detector* dets, int n_det, const float* measured,
                                double* J_out, float* dJ_dmua, float* dJ_dmus) {
  return adjoint_impl(c, dets, n_det, measured, J_out, dJ_dmua, dJ_dmus, false);
}

rte_status rte_discrete_adjoint_gradient(rte_ctx* c, const rte_detector* dets, int n_det,
                                         const float* measured, double* J_out, float* dJ_dmua,
                                         float* dJ_dmus) {
  return adjoint_impl(c, dets, n_det, measured, J_out, dJ_dmua, dJ_dmus, true);
}

rte_status rte_adjoint_gradient_batch(rte_ctx* const* ctxs, int n_ctx, const rte_detector* const* dets,
                                      const int* n_det, const float* const* measured, double* J_out,
                                      float* const* dJ_dmua, float* const* dJ_dmus) {
  if (!ctxs || n_ctx <= 0 || n_ctx > kMaxBatch || !dets || !n_det || !measured || !J_out) return RTE_ERR_INVALID_ARG;
  rte_ctx* c0 = ctxs[0];
  if (!c0) return RTE_ERR_INVALID_ARG;
  for (int i = 0; i < n_ctx; ++i) {
    rte_ctx* c = ctxs[i];
    if (!c || !dets[i] || n_det[i] <= 0 || !measured[i]) return RTE_ERR_INVALID_ARG;
    if (c->M != c0->M || c->tc_mode != c0->tc_mode || c->par.flags != c0->par.flags || c->stream != c0->stream)
      return RTE_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == c) return RTE_ERR_INVALID_ARG;
    if (c->n_steps <= 0 || c->par.ckpt_interval <= 0) return RTE_ERR_STATE;
    if (c->n_steps != c0->n_steps || c->par.ckpt_interval != c0->par.ckpt_interval) return RTE_ERR_INVALID_ARG;
    for (int d = 0; d < n_det[i]; ++d)
      if (!(dets[i][d].sigma_d > 0)) return RTE_ERR_INVALID_ARG;
  }
  if (c0->tc_mode == 0) {
    // plain FP32 form: one medium after another
    for (int i = 0; i < n_ctx; ++i)
      RTE_TRY(adjoint_impl(ctxs[i], dets[i], n_det[i], measured[i], &J_out[i], dJ_dmua ? dJ_dmua[i] : nullptr,
                           dJ_dmus ? dJ_dmus[i] : nullptr, false));
    return RTE_OK;
  }
  const int N = c0->n_steps, I = c0->par.ckpt_interval;
  const cudaStream_t st = c0->stream;
  // Per medium: detector curves, objective, adjoint boundary data rho of eq.
  // (AdjointProblem), zeroed gradients and adjoint state (as adjoint_impl).
  int max_ncell = 0;
  // gradient-term and state-save jobs, one set per segment buffer
  std::vector<rte_kern::GradJob> gjobs(2 * n_ctx);
  std::vector<rte_kern::SaveJob> sjobs(2 * n_ctx);
  std::vector<std::vector<float>> keep_f;               // host tables alive until the copies are done
  std::vector<std::vector<int>> keep_i;
  for (int i = 0; i < n_ctx; ++i) {
    rte_ctx* c = ctxs[i];
    const int G = c->G;
    const size_t gfloats = static_cast<size_t>(G) * c->plane, gbytes = gfloats * sizeof(float);
    const size_t ncurve = static_cast<size_t>(G) * n_det[i] * N;
    const size_t ncell = static_cast<size_t>(c->nx) * c->ny;
    std::vector<float> Wd, Wn;
    std::vector<int> lohi, lohi_n;
    detector_weights(c, dets[i], n_det[i], true, Wd, lohi);
    detector_weights(c, dets[i], n_det[i], false, Wn, lohi_n);
    RTE_TRY(upload(c->Wd, Wd, st));
    RTE_TRY(upload(c->Wn, Wn, st));
    RTE_TRY(upload(c->lohi, lohi, st));
    keep_f.push_back(std::move(Wd));
    keep_f.push_back(std::move(Wn));
    keep_i.push_back(std::move(lohi));
    RTE_TRY(ensure(c->curves64, ncurve * sizeof(double)));
    RTE_TRY(ensure(c->resid, ncurve * sizeof(float)));
    RTE_TRY(ensure(c->partial, 256 * sizeof(double)));
    RTE_TRY(ensure(c->Jdev, sizeof(double)));
    RTE_TRY(ensure(c->rho, static_cast<size_t>(G) * N * c->ring_len * sizeof(float)));
    RTE_TRY(ensure(c->grad_a, ncell * sizeof(double)));
    RTE_TRY(ensure(c->grad_b, ncell * sizeof(double)));
    RTE_TRY(ensure(c->MU, gbytes));
    RTE_TRY(ensure(c->RA, gbytes));
    for (int q = 0; q < 3; ++q) RTE_TRY(ensure(c->LA[q], gbytes));
    RTE_TRY(ensure(c->seg, 2 * static_cast<size_t>(I) * gbytes));   // two segments of recomputed states
    const int* lo = static_cast<const int*>(c->lohi.p);
    RTE_TRY(cuda_status(rte_kern::launch_readout(F(c->ring), c->ring_len, N, G, F(c->Wd), lo, lo + n_det[i],
                                                 n_det[i], nullptr, D(c->curves64), st, &c0->launches)));
    RTE_TRY(cuda_status(rte_kern::launch_objective(D(c->curves64), measured[i], ncurve, c->par.dt, F(c->resid),
                                                   D(c->partial), D(c->Jdev), st, &c0->launches)));
    RTE_TRY(cuda_status(rte_kern::launch_rho(F(c->resid), F(c->Wn), n_det[i], c->ring_len, N, G, 1.0f, F(c->rho),
                                             st, &c0->launches)));
    RTE_TRY(cuda_status(cudaMemsetAsync(c->grad_a.p, 0, ncell * sizeof(double), st)));
    RTE_TRY(cuda_status(cudaMemsetAsync(c->grad_b.p, 0, ncell * sizeof(double), st)));
    RTE_TRY(cuda_status(cudaMemsetAsync(c->MU.p, 0, gbytes, st)));
    for (int q = 0; q < 3; ++q) RTE_TRY(cuda_status(cudaMemsetAsync(c->LA[q].p, 0, gbytes, st)));
    for (int bsel = 0; bsel < 2; ++bsel) {
      float* segb = F(c->seg) + static_cast<size_t>(bsel) * I * gfloats;
      rte_kern::GradJob& gj = gjobs[bsel * n_ctx + i];
      gj.MU = F(c->MU);
      gj.seg = segb;
      gj.slot_floats = gfloats;
      gj.PT = F(c->PT);
      gj.area = F(c->area);
      gj.ncell = static_cast<long long>(ncell);
      gj.M = c->M;
      gj.G = G;
      gj.plane = c->plane;
      gj.scale = (2.0 * kPi / c->M) * c->par.dt;
      gj.grad_a = (dJ_dmua && dJ_dmua[i]) ? D(c->grad_a) : nullptr;
      gj.grad_b = (dJ_dmus && dJ_dmus[i]) ? D(c->grad_b) : nullptr;
      sjobs[bsel * n_ctx + i] = rte_kern::SaveJob{F(c->U), segb, gfloats};
    }
    max_ncell = std::max(max_ncell, static_cast<int>(ncell));
  }
  // Tables of the recompute (forward boundary data, no exitance ring) and of
  // the adjoint march (residual injection), media with the longest lines
  // first, as in rte_forward_batch.
  std::vector<int> order(n_ctx);
  for (int i = 0; i < n_ctx; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return std::max(ctxs[x]->nx, ctxs[x]->ny) > std::max(ctxs[y]->nx, ctxs[y]->ny);
  });
  std::vector<rte_kern::BatchProblem> tf(n_ctx), ta(n_ctx);
  for (int r = 0; r < n_ctx; ++r) {
    rte_ctx* c = ctxs[order[r]];
    rte_kern::BatchProblem& P = tf[r];
    P.a = step_args(c, c->G);
    P.b = boundary_args(c);
    P.b.S = F(c->S); P.b.A = F(c->A); P.b.T = F(c->T); P.b.kmax = c->kmax; P.b.T_len = N;
    P.U = F(c->U);
    P.R = F(c->R);
    for (int q = 0; q < 3; ++q) P.L[q] = F(c->L[q]);
    rte_kern::BatchProblem& Q = ta[r];
    Q.a = step_args(c, c->G);
    Q.b = boundary_args(c);
    Q.b.rho = F(c->rho); Q.b.rho_len = N;
    Q.U = F(c->MU);
    Q.R = F(c->RA);
    for (int q = 0; q < 3; ++q) Q.L[q] = F(c->LA[q]);
  }
  int cx = 0, cy = 0;
  rte_kern::tc_batch_layout(tf.data(), n_ctx, &cx, &cy);
  rte_kern::tc_batch_layout(ta.data(), n_ctx, &cx, &cy);
  RTE_TRY(upload(c0->batch_tab, tf, st));
  RTE_TRY(upload(c0->batch_tab_adj, ta, st));
  const size_t jg = gjobs.size() * sizeof(rte_kern::GradJob), js = sjobs.size() * sizeof(rte_kern::SaveJob);
  RTE_TRY(ensure(c0->batch_jobs, jg + js));
  RTE_TRY(cuda_status(cudaMemcpyAsync(c0->batch_jobs.p, gjobs.data(), jg, cudaMemcpyHostToDevice, st)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(static_cast<char*>(c0->batch_jobs.p) + jg, sjobs.data(), js,
                                      cudaMemcpyHostToDevice, st)));
  RTE_TRY(cuda_status(cudaStreamSynchronize(st)));      // the host tables can go
  const auto* tf_dev = static_cast<const rte_kern::BatchProblem*>(c0->batch_tab.p);
  const auto* ta_dev = static_cast<const rte_kern::BatchProblem*>(c0->batch_tab_adj.p);
  const auto* gj_dev = static_cast<const rte_kern::GradJob*>(c0->batch_jobs.p);
  const auto* sj_dev = reinterpret_cast<const rte_kern::SaveJob*>(static_cast<const char*>(c0->batch_jobs.p) + jg);
  if (!c0->astream) {
    RTE_TRY(cuda_status(cudaStreamCreateWithFlags(&c0->astream, cudaStreamNonBlocking)));
    for (int k = 0; k < 4; ++k) RTE_TRY(cuda_status(cudaEventCreateWithFlags(&c0->aev[k], cudaEventDisableTiming)));
  }
  const cudaStream_t rs = c0->astream;

  // Segments in reverse order, as adjoint_impl: the forward levels of a
  // segment are recomputed from every medium's checkpoint on a second stream
  // (one x- and one y-pass launch per step over all media, then one launch
  // saving every medium's state into segment buffer k % 2), overlapping the
  // adjoint march of the segment before it in this order on the context
  // stream (the adjoint steps of eq. (AdjointProblem) for levels s_end - 1 ..
  // s0, one launch of each kind per level for all media, and their gradient
  // terms, eq. FDwin22, read from the other buffer).  done_fwd[b] orders an
  // adjoint after the recompute into b; done_adj[b] orders the next
  // recompute into b after the adjoint that read it.
  const int last = N - 2;
  std::vector<int> segs;
  for (int seg = c0->n_ckpt - 1; seg >= 0; --seg)
    if (seg * I <= last) segs.push_back(seg);
  cudaEvent_t* done_fwd = c0->aev;
  cudaEvent_t* done_adj = c0->aev + 2;
  RTE_TRY(cuda_status(cudaEventRecord(done_adj[0], st)));
  RTE_TRY(cuda_status(cudaStreamWaitEvent(rs, done_adj[0], 0)));
  auto recompute = [&](int k) -> rte_status {
    const int s0 = segs[k] * I, s_end = std::min(s0 + I, last + 1);
    for (int i = 0; i < n_ctx; ++i) {
      rte_ctx* c = ctxs[i];
      const size_t gbytes = static_cast<size_t>(c->G) * c->plane * sizeof(float);
      const char* base = static_cast<const char*>(c->ckpt.p) + static_cast<size_t>(segs[k]) * 4 * gbytes;
      RTE_TRY(cuda_status(cudaMemcpyAsync(c->U.p, base, gbytes, cudaMemcpyDeviceToDevice, rs)));
      for (int q = 0; q < 3; ++q)
        RTE_TRY(cuda_status(cudaMemcpyAsync(c->L[q].p, base + (q + 1) * gbytes, gbytes, cudaMemcpyDeviceToDevice, rs)));
    }
    int hl = 0;
    for (int s = s0; s < s_end; ++s) {
      RTE_TRY(cuda_status(rte_kern::launch_step_tc_batched(tf.data(), tf_dev, n_ctx, s, hl, rs, &c0->launches)));
      RTE_TRY(cuda_status(rte_kern::launch_save_batch(sj_dev + (k % 2) * n_ctx, n_ctx, s - s0, rs, &c0->launches)));
      hl = (hl + 2) % 3;
    }
    return cuda_status(cudaEventRecord(done_fwd[k % 2], rs));
  };
  int hl_adj = 0;
  if (!segs.empty()) RTE_TRY(recompute(0));
  for (size_t k = 0; k < segs.size(); ++k) {
    const int s0 = segs[k] * I, s_end = std::min(s0 + I, last + 1);
    if (k + 1 < segs.size()) {
      if (k >= 1) RTE_TRY(cuda_status(cudaStreamWaitEvent(rs, done_adj[(k + 1) % 2], 0)));
      RTE_TRY(recompute(static_cast<int>(k + 1)));
    }
    RTE_TRY(cuda_status(cudaStreamWaitEvent(st, done_fwd[k % 2], 0)));
    for (int lvl = s_end - 1; lvl >= s0; --lvl) {
      RTE_TRY(cuda_status(rte_kern::launch_step_tc_batched(ta.data(), ta_dev, n_ctx, lvl, hl_adj, st, &c0->launches)));
      hl_adj = (hl_adj + 2) % 3;
      RTE_TRY(cuda_status(rte_kern::launch_grad_batch(gj_dev + (k % 2) * n_ctx, n_ctx, max_ncell, c0->M, lvl - s0, 1,
                                                      st, &c0->launches)));
    }
    RTE_TRY(cuda_status(cudaEventRecord(done_adj[k % 2], st)));
  }
  for (int i = 0; i < n_ctx; ++i) {
    rte_ctx* c = ctxs[i];
    const size_t ncell = static_cast<size_t>(c->nx) * c->ny;
    if (dJ_dmua && dJ_dmua[i])
      RTE_TRY(cuda_status(rte_kern::launch_to_float(D(c->grad_a), dJ_dmua[i], ncell, st, &c0->launches)));
    if (dJ_dmus && dJ_dmus[i])
      RTE_TRY(cuda_status(rte_kern::launch_to_float(D(c->grad_b), dJ_dmus[i], ncell, st, &c0->launches)));
    RTE_TRY(cuda_status(cudaMemcpyAsync(&J_out[i], c->Jdev.p, sizeof(double), cudaMemcpyDeviceToHost, st)));
  }
  RTE_TRY(cuda_status(cudaStreamSynchronize(st)));
  rte_status res = RTE_OK;
  for (int i = 0; i < n_ctx; ++i) {
    const rte_status si = tc_check(ctxs[i]);
    if (res == RTE_OK) res = si;
  }
  return res;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward solve without any device allocation.
//
// Some callers cannot call cudaMalloc (or cudaFree) once they are running:
// code whose device memory is already fully reserved by another allocator
// (a framework's caching pool), latency-critical loops where an allocation
// call may synchronise the device, and hosts whose policy forbids allocator
// calls after start-up.  For them rte_forward_static runs a whole forward
// solve (state, history, exitance ring, source and detector tables) inside
// one file-scope device array instead of memory from cudaMalloc.  The
// context still comes from rte_init_medium, created while allocation is
// allowed; this call only reads its operators and medium.
//
// The array is kStaticScratchBytes (64 MiB) on every GPU that loads the
// library and stays reserved until the process exits.  Every call shares it
// and it keeps the previous call's contents, so each call zeroes the state it
// needs first; calls that overlap on the GPU (other streams, other threads,
// other contexts on the same device) race on it.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (host code only
// sees a host-side stand-in under that name).  Looked up once per device.
rte_status static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return RTE_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return RTE_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" rte_status rte_forward_static(rte_ctx* c, const rte_source_group* groups, int n_groups,
                                         int n_steps, const rte_detector* dets, int n_det,
                                         float* curves_out) {
  if (!c || !groups || n_groups <= 0 || n_steps <= 0 || !dets || n_det <= 0 || !curves_out)
    return RTE_ERR_INVALID_ARG;
  // The array's address is looked up on the current device; the kernels run
  // on the context's stream, which belongs to the context's device.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RTE_ERR_CUDA;
  }
  if (dev != c->device) return RTE_ERR_INVALID_ARG;
  int kmax = 0;
  for (int g = 0; g < n_groups; ++g) {
    if (groups[g].n_beams < 0 || (groups[g].n_beams > 0 && !groups[g].beams)) return RTE_ERR_INVALID_ARG;
    for (int k = 0; k < groups[g].n_beams; ++k) {
      const rte_beam& bm = groups[g].beams[k];
      if (!(bm.sigma_x > 0) || !(bm.sigma_theta > 0) || !(bm.sigma_t > 0)) return RTE_ERR_INVALID_ARG;
    }
    kmax = std::max(kmax, groups[g].n_beams);
  }
  for (int d = 0; d < n_det; ++d)
    if (!(dets[d].sigma_d > 0)) return RTE_ERR_INVALID_ARG;
  const int G = n_groups, kk = std::max(kmax, 1);
  // Carve the scratch: U, R, L1..L3, exitance ring, S, A, T, detector
  // weights and ranges, each 256-byte aligned.
  const size_t gbytes = align256(static_cast<size_t>(G) * c->plane * sizeof(float));
  const size_t ring_b = align256(static_cast<size_t>(G) * n_steps * c->ring_len * sizeof(float));
  const size_t S_b = align256(static_cast<size_t>(G) * kk * c->ring_len * sizeof(float));
  const size_t A_b = align256(static_cast<size_t>(G) * kk * c->M * sizeof(float));
  const size_t T_b = align256(static_cast<size_t>(G) * kk * n_steps * sizeof(float));
  const size_t W_b = align256(static_cast<size_t>(n_det) * c->ring_len * sizeof(float));
  const size_t lh_b = align256(2 * static_cast<size_t>(n_det) * sizeof(int));
  const size_t need = 5 * gbytes + ring_b + S_b + A_b + T_b + W_b + lh_b;
  if (need > kStaticScratchBytes) return RTE_ERR_UNSUPPORTED;

  void* base = nullptr;
  RTE_TRY(static_scratch_address(&base));
  char* p = static_cast<char*>(base);
  float* U = reinterpret_cast<float*>(p); p += gbytes;
  float* R = reinterpret_cast<float*>(p); p += gbytes;
  float* L[3];
  for (int q = 0; q < 3; ++q) { L[q] = reinterpret_cast<float*>(p); p += gbytes; }
  float* ring = reinterpret_cast<float*>(p); p += ring_b;
  float* Sd = reinterpret_cast<float*>(p); p += S_b;
  float* Ad = reinterpret_cast<float*>(p); p += A_b;
  float* Td = reinterpret_cast<float*>(p); p += T_b;
  float* Wdd = reinterpret_cast<float*>(p); p += W_b;
  int* lohi_d = reinterpret_cast<int*>(p);

  // Source factors q = S(node) A(m) T(step) per beam (eq. RTEsources2) and
  // detector weights (eq. OpMed), built on the host as in rte_forward.
  std::vector<float> S(static_cast<size_t>(G) * kk * c->ring_len, 0.f),
      A(static_cast<size_t>(G) * kk * c->M, 0.f), T(static_cast<size_t>(G) * kk * n_steps, 0.f);
  for (int g = 0; g < G; ++g)
    for (int k = 0; k < groups[g].n_beams; ++k) {
      const rte_beam& bm = groups[g].beams[k];
      const size_t gk = static_cast<size_t>(g) * kk + k;
      for (int nd = 0; nd < c->ring_len; ++nd) {
        const double dx = c->ring_x[nd] - bm.x, dy = c->ring_y[nd] - bm.y;
        S[gk * c->ring_len + nd] = static_cast<float>(std::exp(-(dx * dx + dy * dy) / (2.0 * bm.sigma_x * bm.sigma_x)));
      }
      for (int m = 0; m < c->M; ++m)
        A[gk * c->M + m] = static_cast<float>(
            bm.amplitude * rte_setup::window(angdist(2.0 * kPi * m / c->M, bm.theta) / bm.sigma_theta));
      for (int s = 0; s < n_steps; ++s)
        T[gk * n_steps + s] = static_cast<float>(temporal(bm, (s + 4) * c->par.dt));
    }
  std::vector<float> W;
  std::vector<int> lohi;
  detector_weights(c, dets, n_det, true, W, lohi);
  // Pageable host sources: each copy has left the host vector when it returns.
  RTE_TRY(cuda_status(cudaMemcpyAsync(Sd, S.data(), S.size() * 4, cudaMemcpyHostToDevice, c->stream)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(Ad, A.data(), A.size() * 4, cudaMemcpyHostToDevice, c->stream)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(Td, T.data(), T.size() * 4, cudaMemcpyHostToDevice, c->stream)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(Wdd, W.data(), W.size() * 4, cudaMemcpyHostToDevice, c->stream)));
  RTE_TRY(cuda_status(cudaMemcpyAsync(lohi_d, lohi.data(), lohi.size() * sizeof(int),
                                      cudaMemcpyHostToDevice, c->stream)));
  // The array keeps the previous call's contents: the march starts from zero.
  RTE_TRY(cuda_status(cudaMemsetAsync(U, 0, gbytes, c->stream)));
  for (int q = 0; q < 3; ++q) RTE_TRY(cuda_status(cudaMemsetAsync(L[q], 0, gbytes, c->stream)));

  rte_kern::BoundaryArgs b = boundary_args(c);
  b.S = Sd; b.A = Ad; b.T = Td; b.kmax = kmax; b.T_len = n_steps;
  b.ring_out = ring; b.ring_steps = n_steps;
  const rte_kern::StepArgs a = step_args(c, G);
  int hl = 0;
  for (int s = 0; s < n_steps; ++s) {
    RTE_TRY(cuda_status(rte_kern::launch_step(a, b, U, R, L[hl], L[(hl + 1) % 3], L[(hl + 2) % 3], s,
                                              c->stream, &c->launches)));
    hl = (hl + 2) % 3;
  }
  RTE_TRY(cuda_status(rte_kern::launch_readout(ring, c->ring_len, n_steps, G, Wdd, lohi_d, lohi_d + n_det,
                                               n_det, curves_out, nullptr, c->stream, &c->launches)));
  // tensor-core forms: read (and clear) the context's timeout word
  return tc_check(c);
}
