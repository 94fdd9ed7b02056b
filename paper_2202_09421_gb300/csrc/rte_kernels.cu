// Plain FP32 SIMT kernels of the FC-DOM step (Algorithm 1 loop body).
//
// Layout: U[g][j][i][m] (group, y, x, ordinate), FP32, ordinate innermost so
// that one grid node's M intensities are contiguous (the scattering sum and
// the boundary reflections are node-local) and both line directions are
// dense: an x-line tile is rows (j) x all i x all m; a y-line tile is all j x
// a few columns (i) x all m, contiguous per row.
//
// x-pass: for a block of rows, R = b P~u - (a + b) u - xi_m (D_x u)  [one GEMM
//         D_x (nx x nx) times the rows' (nx x rows*M) slab, plus the node-local
//         M x M scattering]
// y-pass: for a block of columns, L^k = R - eta_m (D_y u); AB4 update of
//         eq. (RTEAB4); boundary condition of eq. (RTE) on Gamma_-; exitance
//         of eq. (OpMed) on the boundary ring.  U is updated in place; the
//         new L^k overwrites the oldest history slot.
// The same passes take the transposed step of the exact discrete adjoint
// (BoundaryArgs::bct_src set): transposed D operators in the GEMMs and the
// transposed AB4 / boundary / readout bookkeeping in the y-pass epilogue.
#include <cstdint>

#include "rte_kernels.cuh"

namespace rte_kern {

namespace {

constexpr float kAB0 = 55.0f / 24.0f, kAB1 = -59.0f / 24.0f, kAB2 = 37.0f / 24.0f,
                kAB3 = -9.0f / 24.0f;

__host__ __device__ inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Output rows of a tile are padded to 32 so that a block (8 x rows/8
// threads) is a whole number of warps: the epilogue works warp by warp.
constexpr int kRowPad = 32;

// acc[r][c] += sum_k A[row0 + r][k] * B[k][col0 + c] over the whole K range,
// with A given transposed in global memory (AT[k * n + row]) and staged in
// shared memory chunk by chunk; B is the full slab already in shared memory.
__device__ inline void gemm_rows(const float* __restrict__ AT, int n, int npad, int kpad,
                                 const float* Bs, float* As, int row0, int col0,
                                 float acc[kTM][kTN]) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  for (int k0 = 0; k0 < kpad; k0 += kKC) {
    __syncthreads();
    for (int idx = tid; idx < kKC * npad; idx += nthr) {
      const int k = idx / npad, r = idx - k * npad;
      const int kk = k0 + k;
      As[idx] = (kk < n && r < n) ? __ldg(AT + static_cast<size_t>(kk) * n + r) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kKC; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(As + k * npad + row0);
      const float4 a1 = *reinterpret_cast<const float4*>(As + k * npad + row0 + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(Bs + (k0 + k) * kTileCols + col0);
      const float4 b1 = *reinterpret_cast<const float4*>(Bs + (k0 + k) * kTileCols + col0 + 4);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < kTM; ++r)
#pragma unroll
        for (int c = 0; c < kTN; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
  }
}

__global__ void __launch_bounds__(512) xpass_kernel(StepArgs a, const float* __restrict__ U,
                                                     float* __restrict__ R) {
  extern __shared__ __align__(16) float smem[];
  const int n = a.nx, M = a.M;
  const int npad = round_up(n, kRowPad), kpad = round_up(n, kKC);
  const int rows_per_tile = kTileCols / M;
  float* Bs = smem;                                   // [kpad][64]
  float* As = Bs + kpad * kTileCols;                  // [kKC][npad]
  float* Ps = As + kKC * npad;                        // [M][M] (P~ transposed)
  const int g = blockIdx.z;
  const int j0 = blockIdx.x * rows_per_tile;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  const float* Ug = U + static_cast<size_t>(g) * a.plane;

  // Stage the rows' slab: Bs[i'][r*M + m] = u[j0 + r][i'][m].
  for (int idx = tid; idx < kpad * (kTileCols / 4); idx += nthr) {
    const int k = idx / (kTileCols / 4), c = (idx - k * (kTileCols / 4)) * 4;
    const int r = c / M, m = c - r * M, j = j0 + r;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < n && r < rows_per_tile && j < a.ny)
      v = __ldg(reinterpret_cast<const float4*>(Ug + (static_cast<size_t>(j) * n + k) * M + m));
    *reinterpret_cast<float4*>(Bs + k * kTileCols + c) = v;
  }
  for (int idx = tid; idx < M * M; idx += nthr) Ps[idx] = __ldg(a.PT + idx);

  const int row0 = threadIdx.y * kTM, col0 = threadIdx.x * kTN;
  float acc[kTM][kTN];
#pragma unroll
  for (int r = 0; r < kTM; ++r)
#pragma unroll
    for (int c = 0; c < kTN; ++c) acc[r][c] = 0.f;
  gemm_rows(a.DxT, n, npad, kpad, Bs, As, row0, col0, acc);

  // Epilogue: node-local scattering and absorption, minus xi * d_x u.
  // Columns past rows_per_tile * M (M not dividing 64) belong to no row of
  // this tile.
  const int r = col0 / M, mb = col0 - r * M, j = j0 + r;
  if (r >= rows_per_tile || j >= a.ny) return;
  float xi[kTN];
#pragma unroll
  for (int t = 0; t < kTN; ++t) xi[t] = __ldg(a.xi + mb + t);
#pragma unroll
  for (int ii = 0; ii < kTM; ++ii) {
    const int i = row0 + ii;
    if (i >= n) break;
    const float* ucell = Bs + i * kTileCols + r * M;
    float s[kTN];
#pragma unroll
    for (int t = 0; t < kTN; ++t) s[t] = 0.f;
    for (int q = 0; q < M; ++q) {
      const float uq = ucell[q];
      const float4 p0 = *reinterpret_cast<const float4*>(Ps + q * M + mb);
      const float4 p1 = *reinterpret_cast<const float4*>(Ps + q * M + mb + 4);
      s[0] = fmaf(p0.x, uq, s[0]); s[1] = fmaf(p0.y, uq, s[1]);
      s[2] = fmaf(p0.z, uq, s[2]); s[3] = fmaf(p0.w, uq, s[3]);
      s[4] = fmaf(p1.x, uq, s[4]); s[5] = fmaf(p1.y, uq, s[5]);
      s[6] = fmaf(p1.z, uq, s[6]); s[7] = fmaf(p1.w, uq, s[7]);
    }
    const float av = __ldg(a.mua + static_cast<size_t>(j) * n + i);
    const float bv = __ldg(a.mus + static_cast<size_t>(j) * n + i);
    float out[kTN];
#pragma unroll
    for (int t = 0; t < kTN; ++t)
      out[t] = bv * s[t] - (av + bv) * ucell[mb + t] - xi[t] * acc[ii][t];
    float* dst = R + static_cast<size_t>(g) * a.plane + (static_cast<size_t>(j) * n + i) * M + mb;
    reinterpret_cast<float4*>(dst)[0] = make_float4(out[0], out[1], out[2], out[3]);
    reinterpret_cast<float4*>(dst)[1] = make_float4(out[4], out[5], out[6], out[7]);
  }
}

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// TR: the transposed step of the discrete adjoint (BoundaryArgs::bct_src);
// a separate instance, so that the forward step compiles without it.
template <bool TR>
__global__ void __launch_bounds__(512) ypass_kernel(StepArgs a, BoundaryArgs b, float* __restrict__ U,
                                                     const float* __restrict__ R,
                                                     const float* __restrict__ L1,
                                                     const float* __restrict__ L2,
                                                     float* __restrict__ L3, int src_step,
                                                     int ring_step) {
  extern __shared__ __align__(16) float smem[];
  const int nx = a.nx, n = a.ny, M = a.M;
  const int npad = round_up(n, kRowPad), kpad = round_up(n, kKC);
  const int cols_per_tile = kTileCols / M;
  float* Bs = smem;                                   // [kpad][64]
  float* As = Bs + kpad * kTileCols;                  // [kKC][npad]
  const int g = blockIdx.z;
  const int i0 = blockIdx.x * cols_per_tile;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  const size_t goff = static_cast<size_t>(g) * a.plane;
  float* Ug = U + goff;

  // Stage the columns' slab: Bs[j'][w*M + m] = u[j'][i0 + w][m] (contiguous).
  const int valid_cols = min(cols_per_tile, nx - i0) * M;
  for (int idx = tid; idx < kpad * (kTileCols / 4); idx += nthr) {
    const int k = idx / (kTileCols / 4), c = (idx - k * (kTileCols / 4)) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < n && c < valid_cols)
      v = *reinterpret_cast<const float4*>(Ug + (static_cast<size_t>(k) * nx + i0) * M + c);
    *reinterpret_cast<float4*>(Bs + k * kTileCols + c) = v;
  }

  const int row0 = threadIdx.y * kTM, col0 = threadIdx.x * kTN;
  float acc[kTM][kTN];
#pragma unroll
  for (int r = 0; r < kTM; ++r)
#pragma unroll
    for (int c = 0; c < kTN; ++c) acc[r][c] = 0.f;
  gemm_rows(a.DyT, n, npad, kpad, Bs, As, row0, col0, acc);

  // AB4 update (eq. RTEAB4) for this thread's outputs.
  const int w = col0 / M, mb = col0 - w * M, i = i0 + w;
  const bool col_ok = w < cols_per_tile && i < nx;
  float eta[kTN];
#pragma unroll
  for (int t = 0; t < kTN; ++t) eta[t] = __ldg(a.eta + mb + t);
#pragma unroll
  for (int jj = 0; jj < kTM; ++jj) {
    const int j = row0 + jj;
    if (!col_ok || j >= n) {
#pragma unroll
      for (int t = 0; t < kTN; ++t) acc[jj][t] = 0.f;
      continue;
    }
    const size_t base = goff + (static_cast<size_t>(j) * nx + i) * M + mb;
    const float4 r0 = *reinterpret_cast<const float4*>(R + base);
    const float4 r1 = *reinterpret_cast<const float4*>(R + base + 4);
    const float4 p0 = *reinterpret_cast<const float4*>(L1 + base);
    const float4 p1 = *reinterpret_cast<const float4*>(L1 + base + 4);
    const float4 q0 = *reinterpret_cast<const float4*>(L2 + base);
    const float4 q1 = *reinterpret_cast<const float4*>(L2 + base + 4);
    const float4 s0 = *reinterpret_cast<const float4*>(L3 + base);
    const float4 s1 = *reinterpret_cast<const float4*>(L3 + base + 4);
    const float rv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    const float l1[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
    const float l2[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
    const float l3[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    if constexpr (TR) {
      // transposed step: ubar = w^{k+1} + L^T v (readout term and BC^T below)
#pragma unroll
      for (int t = 0; t < kTN; ++t) acc[jj][t] = rv[t] - eta[t] * acc[jj][t] + l1[t];
      continue;
    }
    float lk[8];
#pragma unroll
    for (int t = 0; t < kTN; ++t) {
      lk[t] = rv[t] - eta[t] * acc[jj][t];
      const float incr = kAB0 * lk[t] + kAB1 * l1[t] + kAB2 * l2[t] + kAB3 * l3[t];
      acc[jj][t] = fmaf(a.cdt, incr, Bs[j * kTileCols + col0 + t]);   // u^{k+1}, pre-BC
    }
    reinterpret_cast<float4*>(L3 + base)[0] = make_float4(lk[0], lk[1], lk[2], lk[3]);
    reinterpret_cast<float4*>(L3 + base)[1] = make_float4(lk[4], lk[5], lk[6], lk[7]);
  }
  __syncthreads();   // every thread has read u^k from Bs
#pragma unroll
  for (int jj = 0; jj < kTM; ++jj) {
    const int j = row0 + jj;
    if (j < kpad) {
      *reinterpret_cast<float4*>(Bs + j * kTileCols + col0) =
          make_float4(acc[jj][0], acc[jj][1], acc[jj][2], acc[jj][3]);
      *reinterpret_cast<float4*>(Bs + j * kTileCols + col0 + 4) =
          make_float4(acc[jj][4], acc[jj][5], acc[jj][6], acc[jj][7]);
    }
  }
  __syncthreads();

  // Boundary condition (eq. RTE third line) from the pre-BC values in Bs,
  // store, and the exitance of eq. (OpMed) on boundary nodes.  One warp per
  // grid node, lanes over ordinates.
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int ncols = min(cols_per_tile, nx - i0);
  const int ring_len = 2 * n + 2 * nx;
  for (int cell = warp; cell < n * ncols; cell += nwarps) {
    const int j = cell / ncols, wc = cell - j * ncols, ic = i0 + wc;
    float* pre = Bs + j * kTileCols + wc * M;
    const bool lf = ic == 0, rt = ic == nx - 1, bt = j == 0, tp = j == n - 1;
    const bool bnd = lf || rt || bt || tp;
    float* dst = Ug + (static_cast<size_t>(j) * nx + ic) * M;
    if constexpr (TR) {
      // Transposed step on this node: the readout transpose on the ring
      // (every face the node lies on), w = BC^T ubar, then the transposed
      // AB4 combination v' = c dt (chi0 w + chi1 w^{k+1} + chi2 w^{k+2} + chi3 w^{k+3}).
      int tb = -1;
      if (bnd) {
        const float* eb = b.ebar + (static_cast<size_t>(g) * b.ebar_len + src_step) * ring_len;
        for (int m = lane; m < M; m += 32) {
          float v = pre[m];
          if (lf || rt) v = fmaf(b.wexit[(lf ? 0 : 1) * M + m], eb[lf ? j : n + j], v);
          if (bt || tp) v = fmaf(b.wexit[(bt ? 2 : 3) * M + m], eb[bt ? 2 * n + ic : 2 * n + nx + ic], v);
          pre[m] = v;
        }
        __syncwarp();
        tb = ((lf || rt) && (bt || tp)) ? 4 + (rt ? 1 : 0) + (tp ? 2 : 0) : (lf ? 0 : rt ? 1 : bt ? 2 : 3);
      }
      const size_t e0 = goff + (static_cast<size_t>(j) * nx + ic) * M;
      for (int m = lane; m < M; m += 32) {
        float wv = pre[m];
        if (tb >= 0) {
          const int* src = b.bct_src + (tb * M + m) * 4;
          const float* cf = b.bct_f + (tb * M + m) * 4;
          wv = 0.f;
#pragma unroll
          for (int q = 0; q < 4; ++q) wv = fmaf(cf[q], pre[src[q]], wv);
        }
        const float incr = kAB0 * wv + kAB1 * L1[e0 + m] + kAB2 * L2[e0 + m] + kAB3 * L3[e0 + m];
        L3[e0 + m] = wv;
        dst[m] = a.cdt * incr;
      }
      continue;
    }
    if (!bnd) {
      for (int m = lane; m < M; m += 32) dst[m] = pre[m];
      continue;
    }
    const int* refl;
    const float* fco;
    const unsigned char* act;
    if ((lf || rt) && (bt || tp)) {
      const int c = (rt ? 1 : 0) + (tp ? 2 : 0);
      refl = b.corner_refl + c * M; fco = b.corner_f + c * M; act = b.corner_act + c * M;
    } else {
      const int F = lf ? 0 : rt ? 1 : bt ? 2 : 3;
      refl = b.face_refl + F * M; fco = b.face_f + F * M; act = b.face_act + F * M;
    }
    // ring node used for the source data (x-face index at corners)
    const int node = lf ? j : rt ? n + j : bt ? 2 * n + ic : 2 * n + nx + ic;
    float ex_x = 0.f, ex_y = 0.f;
    for (int m = lane; m < M; m += 32) {
      float v = pre[m];
      if (act[m]) {
        float q = 0.f;
        for (int k = 0; k < b.kmax; ++k) {
          const size_t gk = static_cast<size_t>(g) * b.kmax + k;
          q = fmaf(b.S[gk * ring_len + node] * b.A[gk * M + m], b.T[gk * b.T_len + src_step], q);
        }
        if (b.rho)
          q = fmaf(1.0f - fco[m], b.rho[(static_cast<size_t>(g) * b.rho_len + src_step) * ring_len + node], q);
        v = fmaf(fco[m], pre[refl[m]], q);
      }
      dst[m] = v;
      if (lf || rt) ex_x = fmaf(b.wexit[(lf ? 0 : 1) * M + m], v, ex_x);
      if (bt || tp) ex_y = fmaf(b.wexit[(bt ? 2 : 3) * M + m], v, ex_y);
    }
    if (b.ring_out && ring_step >= 0) {
      float* ro = b.ring_out + (static_cast<size_t>(g) * b.ring_steps + ring_step) * ring_len;
      if (lf || rt) {
        ex_x = warp_sum(ex_x);
        if (lane == 0) ro[lf ? j : n + j] = ex_x;
      }
      if (bt || tp) {
        ex_y = warp_sum(ex_y);
        if (lane == 0) ro[bt ? 2 * n + ic : 2 * n + nx + ic] = ex_y;
      }
    }
  }
}

size_t pass_smem(int n, int M, bool xpass) {
  const int npad = round_up(n, kRowPad), kpad = round_up(n, kKC);
  size_t f = static_cast<size_t>(kpad) * kTileCols + static_cast<size_t>(kKC) * npad;
  if (xpass) f += static_cast<size_t>(M) * M;
  return f * sizeof(float);
}

__global__ void fluence_kernel(const float* __restrict__ U, float* __restrict__ out,
                               size_t out_gs, int ncell, int M, size_t plane, float w) {
  const int lane = threadIdx.x & 31;
  const long long warp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int g = blockIdx.y;
  if (warp >= ncell) return;
  const float* u = U + static_cast<size_t>(g) * plane + static_cast<size_t>(warp) * M;
  float s = 0.f;
  for (int m = lane; m < M; m += 32) s += u[m];
  s = warp_sum(s);
  if (lane == 0) out[static_cast<size_t>(g) * out_gs + warp] = w * s;
}

__global__ void readout_kernel(const float* __restrict__ ring, int ring_len, int n_steps, int G,
                               const float* __restrict__ Wd, const int* __restrict__ lo,
                               const int* __restrict__ hi, int n_det, float* curves,
                               double* curves64) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long total = static_cast<long long>(G) * n_det * n_steps;
  if (idx >= total) return;
  const int s = static_cast<int>(idx % n_steps);
  const int d = static_cast<int>((idx / n_steps) % n_det);
  const int g = static_cast<int>(idx / (static_cast<long long>(n_steps) * n_det));
  const float* r = ring + (static_cast<size_t>(g) * n_steps + s) * ring_len;
  double acc = 0.0;
  for (int k = lo[d]; k < hi[d]; ++k) {
    const float wv = Wd[static_cast<size_t>(d) * ring_len + k];
    if (wv != 0.f) acc += static_cast<double>(wv) * static_cast<double>(r[k]);
  }
  if (curves) curves[idx] = static_cast<float>(acc);
  if (curves64) curves64[idx] = acc;
}

__global__ void objective_partial(const double* __restrict__ c64, const float* __restrict__ meas,
                                  size_t n, float* __restrict__ resid, double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const double r = c64[k] - static_cast<double>(meas[k]);
    resid[k] = static_cast<float>(r);
    s += r * r;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void objective_final(const double* __restrict__ partial, int nb, double scale,
                                double* J) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s += partial[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = scale * sh[0];
}

__global__ void rho_kernel(const float* __restrict__ resid, const float* __restrict__ Wn, int n_det,
                           int ring_len, int n_steps, int G, float scale, float* __restrict__ rho) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long total = static_cast<long long>(G) * n_steps * ring_len;
  if (idx >= total) return;
  const int node = static_cast<int>(idx % ring_len);
  const int s = static_cast<int>((idx / ring_len) % n_steps);
  const int g = static_cast<int>(idx / (static_cast<long long>(ring_len) * n_steps));
  float acc = 0.f;
  for (int d = 0; d < n_det; ++d)
    acc = fmaf(Wn[static_cast<size_t>(d) * ring_len + node],
               resid[(static_cast<size_t>(g) * n_det + d) * n_steps + s], acc);
  rho[idx] = scale * acc;
}

// The gradient terms of eq. (FDwin22) at one grid cell, summed over the
// groups and the ordinates (see launch_grad):
//   sa = sum_g sum_m lam_m u_m,  sb = sum_g sum_m lam_m (u_m - (P~u)_m),
// lam the adjoint field (its ordinates flipped by M/2 in the continuous form).
// One thread per cell for M in {16, 32}: the node's M values of u and lam
// arrive as 32-byte loads, and P~u uses the circulant's first column p_d =
// P~[d][0] (P~[m][q] = p_{(m - q) mod M}) from registers, summed over q in
// order for every m.
// 32 bytes of read-only data into 8 registers (32-byte aligned address).
__device__ __forceinline__ void ld32b(const float* ptr, float* v) {
  asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(ptr));
}

template <int MM>
__device__ __forceinline__ void grad_node(const float* __restrict__ MU, const float* __restrict__ Useg,
                                          const float* __restrict__ PT, const float* __restrict__ area,
                                          long long cell, int G, size_t plane, size_t useg_gs, double scale,
                                          int flip, double* __restrict__ grad_a, double* __restrict__ grad_b) {
  float p[MM];
#pragma unroll
  for (int d = 0; d < MM; ++d) p[d] = __ldg(PT + d);            // P~[0][d] = p_d (symmetric circulant)
  float sa = 0.f, sb = 0.f;
  for (int g = 0; g < G; ++g) {
    const float* u = Useg + static_cast<size_t>(g) * useg_gs + static_cast<size_t>(cell) * MM;
    const float* mu = MU + static_cast<size_t>(g) * plane + static_cast<size_t>(cell) * MM;
    float uu[MM], lam[MM];
#pragma unroll
    for (int k = 0; k < MM / 8; ++k) {
      ld32b(u + 8 * k, uu + 8 * k);
      ld32b(mu + 8 * k, lam + 8 * k);
    }
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      float pu = 0.f;
#pragma unroll
      for (int q = 0; q < MM; ++q) pu = fmaf(p[(m - q + MM) % MM], uu[q], pu);
      const float l = flip ? lam[(m + MM / 2) % MM] : lam[m];
      sa = fmaf(l, uu[m], sa);
      sb = fmaf(l, uu[m] - pu, sb);
    }
  }
  const double k = area ? scale * static_cast<double>(area[cell]) : scale;
  if (grad_a) grad_a[cell] -= k * static_cast<double>(sa);
  if (grad_b) grad_b[cell] -= k * static_cast<double>(sb);
}

// Any M: one warp per cell, the lanes over the ordinates, the row of P~ from
// memory.
__device__ __forceinline__ void grad_cell(const float* __restrict__ MU, const float* __restrict__ Useg,
                                          const float* __restrict__ PT, const float* __restrict__ area,
                                          long long cell, int M, int G, size_t plane, size_t useg_gs,
                                          double scale, int flip, double* __restrict__ grad_a,
                                          double* __restrict__ grad_b) {
  __shared__ float ubuf[8][64];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  float sa = 0.f, sb = 0.f;
  for (int g = 0; g < G; ++g) {
    const float* u = Useg + static_cast<size_t>(g) * useg_gs + static_cast<size_t>(cell) * M;
    const float* mu = MU + static_cast<size_t>(g) * plane + static_cast<size_t>(cell) * M;
    for (int m = lane; m < M; m += 32) ubuf[wl][m] = u[m];
    __syncwarp();
    for (int m = lane; m < M; m += 32) {
      float pu = 0.f;
      for (int q = 0; q < M; ++q) pu = fmaf(PT[q * M + m], ubuf[wl][q], pu);
      const float lam = flip ? mu[(m + M / 2) % M] : mu[m];
      sa = fmaf(lam, ubuf[wl][m], sa);
      sb = fmaf(lam, ubuf[wl][m] - pu, sb);
    }
    __syncwarp();
  }
  sa = warp_sum(sa);
  sb = warp_sum(sb);
  if (lane == 0) {
    const double k = area ? scale * static_cast<double>(area[cell]) : scale;
    if (grad_a) grad_a[cell] -= k * static_cast<double>(sa);
    if (grad_b) grad_b[cell] -= k * static_cast<double>(sb);
  }
}

// M in {16, 32}: one thread per cell; other M: one warp per cell.
__device__ __forceinline__ bool grad_by_thread(int M) { return M == 16 || M == 32; }

__global__ void grad_kernel(const float* __restrict__ MU, const float* __restrict__ Useg,
                            const float* __restrict__ PT, const float* __restrict__ area, int ncell,
                            int M, int G, size_t plane, size_t useg_gs, double scale, int flip,
                            double* __restrict__ grad_a, double* __restrict__ grad_b) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (grad_by_thread(M)) {
    if (t >= ncell) return;
    if (M == 32) grad_node<32>(MU, Useg, PT, area, t, G, plane, useg_gs, scale, flip, grad_a, grad_b);
    else grad_node<16>(MU, Useg, PT, area, t, G, plane, useg_gs, scale, flip, grad_a, grad_b);
    return;
  }
  const long long cell = t >> 5;
  if (cell >= ncell) return;   // whole warp exits together
  grad_cell(MU, Useg, PT, area, cell, M, G, plane, useg_gs, scale, flip, grad_a, grad_b);
}

// Batched forms for media that march in lockstep: blockIdx.y picks the
// medium; its forward state of the level sits in slot `slot` of its segment
// buffer.
__global__ void grad_batch_kernel(const GradJob* __restrict__ jobs, int slot, int flip) {
  const GradJob& j = jobs[blockIdx.y];
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const float* useg = j.seg + static_cast<size_t>(slot) * j.slot_floats;
  if (grad_by_thread(j.M)) {
    if (t >= j.ncell) return;
    if (j.M == 32) grad_node<32>(j.MU, useg, j.PT, j.area, t, j.G, j.plane, j.plane, j.scale, flip, j.grad_a, j.grad_b);
    else grad_node<16>(j.MU, useg, j.PT, j.area, t, j.G, j.plane, j.plane, j.scale, flip, j.grad_a, j.grad_b);
    return;
  }
  const long long cell = t >> 5;
  if (cell >= j.ncell) return;
  grad_cell(j.MU, useg, j.PT, j.area, cell, j.M, j.G, j.plane, j.plane, j.scale, flip, j.grad_a, j.grad_b);
}

__global__ void save_batch_kernel(const SaveJob* __restrict__ jobs, int slot) {
  const SaveJob& j = jobs[blockIdx.y];
  const size_t n4 = j.n_floats / 4;
  const float4* src = reinterpret_cast<const float4*>(j.src);
  float4* dst = reinterpret_cast<float4*>(j.seg + static_cast<size_t>(slot) * j.n_floats);
  // four independent 16-byte loads in flight per thread and pass
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; k + 3 * stride < n4; k += 4 * stride) {
    const float4 v0 = __ldg(src + k), v1 = __ldg(src + k + stride), v2 = __ldg(src + k + 2 * stride),
                 v3 = __ldg(src + k + 3 * stride);
    dst[k] = v0;
    dst[k + stride] = v1;
    dst[k + 2 * stride] = v2;
    dst[k + 3 * stride] = v3;
  }
  for (; k < n4; k += stride) dst[k] = __ldg(src + k);
}

__global__ void to_float_kernel(const double* in, float* out, size_t n) {
  const size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) out[k] = static_cast<float>(in[k]);
}

// Photon balance of one post-BC state (eq. RTE integrated over theta and
// Omega; the scattering term integrates to zero): per group,
//   S0 = sum_nodes A_node sum_m u_m,   S1 = sum_nodes A_node a sum_m u_m,
//   S2 = sum_faces sum_face nodes w_face sum_m (theta_m . nu) u_m,
// with the trapezoid node areas A_node and face weights w_face (half at the
// face ends).  One thread per float4 of the state: the M/4 lanes of a node
// add its ordinates in FP32 (a pairwise tree of M terms) and the node's first
// lane adds A_node sum_m u_m and a A_node sum_m u_m to its own compensated
// (Kahan) FP32 sums, at most kBalItems nodes a thread (32); the boundary fluxes
// are formed in FP64 from a double table of cos and sin of the ordinates.
// GB300's FP64 pipe issues a warp instruction in tens of clocks, so FP64
// work runs once per thread and per boundary node, not per node.  From the
// threads up everything is FP64: warp and block sums in a fixed order, then
// the last block of a group to finish (ticket counter) adds the block
// partials in block order, so the sums do not depend on the schedule.
// out[(g n_steps + step) 3 + k] = (w S0 / c, w S1, w S2).
constexpr int kBalThreads = 256, kBalItems = 32;

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
  const float y = x - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

__global__ void __launch_bounds__(kBalThreads)
    balance_kernel(const float* __restrict__ U, size_t plane, int nx, int ny, int M,
                   const float* __restrict__ mua, const double* __restrict__ trig, double dx, double dy,
                   double w, double inv_c, double* __restrict__ partial, unsigned* __restrict__ ticket,
                   double* __restrict__ out, int step, int n_steps) {
  __shared__ double red[3][kBalThreads / 32];
  __shared__ int last;
  const int g = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
  const int V = M / 4;                                  // lanes per node: 2, 4, 8 or 16
  const int lv = __ffs(V) - 1;                          // log2 V
  // at most 512 x 512 nodes x 16 float4: 32-bit indices
  const int n4 = nx * ny * V;
  const float4* u4 = reinterpret_cast<const float4*>(U + static_cast<size_t>(g) * plane);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float fdx = static_cast<float>(dx), fdy = static_cast<float>(dy);
  float a0 = 0.f, c0 = 0.f, a1 = 0.f, c1 = 0.f;        // Kahan sums of A sum_m u and a A sum_m u
  double s2 = 0.0;
  const int base = b * kBalItems * kBalThreads;
  for (int k = 0; k < kBalItems; ++k) {
    const int q = base + k * kBalThreads + static_cast<int>(threadIdx.x);
    const bool valid = q < n4;                          // node groups never straddle the end
    const float4 v = valid ? __ldcs(u4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    float su = (v.x + v.y) + (v.z + v.w);
    for (int o = 1; o < V; o <<= 1) su += __shfl_xor_sync(0xffffffffu, su, o);
    if (!valid) continue;
    const int node = q >> lv;
    const int r = q & (V - 1);
    const int j = node / nx, i = node - j * nx;
    const bool xe = i == 0 || i == nx - 1, ye = j == 0 || j == ny - 1;
    if (r == 0) {
      // trapezoid node area: dx dy, halved on each face the node lies on
      const float area = (xe ? 0.5f * fdx : fdx) * (ye ? 0.5f * fdy : fdy);
      const float t = area * su;
      kahan_add(a0, c0, t);
      kahan_add(a1, c1, t * __ldg(mua + node));
    }
    if (xe || ye) {
      const double wx = (i == 0 || i == nx - 1) ? 0.5 * dx : dx;
      const double wy = (j == 0 || j == ny - 1) ? 0.5 * dy : dy;
      const int m0 = 4 * r;
      const double e[4] = {v.x, v.y, v.z, v.w};
      double fx = 0.0, fy = 0.0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        fx += __ldg(trig + m0 + t) * e[t];
        fy += __ldg(trig + M + m0 + t) * e[t];
      }
      if (i == 0) s2 -= wy * fx;
      if (i == nx - 1) s2 += wy * fx;
      if (j == 0) s2 -= wx * fy;
      if (j == ny - 1) s2 += wx * fy;
    }
  }
  double s0 = static_cast<double>(a0) - static_cast<double>(c0);
  double s1 = static_cast<double>(a1) - static_cast<double>(c1);
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    red[0][warp] = s0;
    red[1][warp] = s1;
    red[2][warp] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k)
      for (int wv = 0; wv < kBalThreads / 32; ++wv) t[k] += red[k][wv];
    double* pp = partial + (static_cast<size_t>(g) * nb + b) * 3;
    pp[0] = t[0];
    pp[1] = t[1];
    pp[2] = t[2];
    __threadfence();
    last = atomicAdd(ticket + g, 1u) == static_cast<unsigned>(nb - 1);
  }
  __syncthreads();
  if (!last || warp != 0) return;
  // the group's last block: lane l adds blocks l, l + 32, ... in order, then
  // a fixed butterfly combines the lanes
  __threadfence();
  const volatile double* pg = partial + static_cast<size_t>(g) * nb * 3;
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
  for (int bb = lane; bb < nb; bb += 32) {
    t0 += pg[3 * bb];
    t1 += pg[3 * bb + 1];
    t2 += pg[3 * bb + 2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    t0 += __shfl_xor_sync(0xffffffffu, t0, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    t2 += __shfl_xor_sync(0xffffffffu, t2, o);
  }
  if (lane == 0) {
    double* o = out + (static_cast<size_t>(g) * n_steps + step) * 3;
    o[0] = w * inv_c * t0;
    o[1] = w * t1;
    o[2] = w * t2;
    ticket[g] = 0u;
  }
}

}  // namespace

cudaError_t launch_step(const StepArgs& a, const BoundaryArgs& b, float* U, float* R,
                        const float* L1, const float* L2, float* L3, int step,
                        cudaStream_t s, long long* launches, cudaEvent_t* ev) {
  if (a.tc_mode != 0) return launch_step_tc(a, b, U, R, L1, L2, L3, step, s, launches, ev);
  static bool attr_done = false;
  const size_t smx = pass_smem(a.nx, a.M, true), smy = pass_smem(a.ny, a.M, false);
  if (!attr_done) {
    cudaFuncSetAttribute(xpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    cudaFuncSetAttribute(ypass_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    cudaFuncSetAttribute(ypass_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    attr_done = true;
  }
  const int per_tile = kTileCols / a.M;
  // npad / kTM rows of threads: 8 x (multiple of 4) = whole warps.
  dim3 bx(kTileCols / kTN, round_up(a.nx, kRowPad) / kTM);
  dim3 gx((a.ny + per_tile - 1) / per_tile, 1, a.G);
  if (ev) cudaEventRecord(ev[0], s);
  xpass_kernel<<<gx, bx, smx, s>>>(a, U, R);
  if (ev) cudaEventRecord(ev[1], s);
  dim3 by(kTileCols / kTN, round_up(a.ny, kRowPad) / kTM);
  dim3 gy((a.nx + per_tile - 1) / per_tile, 1, a.G);
  const int ring_step = b.ring_out ? step : -1;
  if (b.bct_src)
    ypass_kernel<true><<<gy, by, smy, s>>>(a, b, U, R, L1, L2, L3, step, ring_step);
  else
    ypass_kernel<false><<<gy, by, smy, s>>>(a, b, U, R, L1, L2, L3, step, ring_step);
  if (ev) cudaEventRecord(ev[2], s);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_fluence(const float* U, float* out, size_t out_group_stride, int nx, int ny,
                           int M, int G, size_t plane, float w, cudaStream_t s,
                           long long* launches) {
  const int ncell = nx * ny;
  dim3 grid((ncell * 32 + 255) / 256, G);
  fluence_kernel<<<grid, 256, 0, s>>>(U, out, out_group_stride, ncell, M, plane, w);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_readout(const float* ring, int ring_len, int n_steps, int G,
                           const float* Wd, const int* lo, const int* hi, int n_det,
                           float* curves, double* curves64, cudaStream_t s,
                           long long* launches) {
  const long long total = static_cast<long long>(G) * n_det * n_steps;
  if (total == 0) return cudaSuccess;
  readout_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
      ring, ring_len, n_steps, G, Wd, lo, hi, n_det, curves, curves64);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_objective(const double* curves64, const float* measured, size_t n,
                             double dt, float* resid, double* partial, double* J_dev,
                             cudaStream_t s, long long* launches) {
  const int nb = 256;
  objective_partial<<<nb, 256, 0, s>>>(curves64, measured, n, resid, partial);
  objective_final<<<1, 256, 0, s>>>(partial, nb, 0.5 * dt, J_dev);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_rho(const float* resid, const float* Wn, int n_det, int ring_len,
                       int n_steps, int G, float scale, float* rho, cudaStream_t s,
                       long long* launches) {
  const long long total = static_cast<long long>(G) * n_steps * ring_len;
  if (total == 0) return cudaSuccess;
  rho_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(resid, Wn, n_det, ring_len,
                                                                         n_steps, G, scale, rho);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_grad_batch(const GradJob* jobs_dev, int n_jobs, int max_ncell, int m_common, int slot,
                              int flip, cudaStream_t s, long long* launches) {
  // one thread per cell for M in {16, 32} (every medium of a batch shares M)
  dim3 grid((max_ncell * 32 + 255) / 256, n_jobs);
  if (m_common == 16 || m_common == 32) grid.x = (max_ncell + 255) / 256;
  grad_batch_kernel<<<grid, 256, 0, s>>>(jobs_dev, slot, flip);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_save_batch(const SaveJob* jobs_dev, int n_jobs, int slot, cudaStream_t s, long long* launches) {
  dim3 grid(4 * 152, n_jobs);
  save_batch_kernel<<<grid, 256, 0, s>>>(jobs_dev, slot);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

int balance_blocks(int nx, int ny, int M) {
  const long long n4 = static_cast<long long>(nx) * ny * (M / 4);
  return static_cast<int>((n4 + kBalItems * kBalThreads - 1) / (kBalItems * kBalThreads));
}

cudaError_t launch_balance(const float* U, size_t plane, int nx, int ny, int M, int G, const float* mua,
                           const double* trig, double dx, double dy, double w, double c, double* partial,
                           unsigned* ticket, double* out, int step, int n_steps, cudaStream_t s,
                           long long* launches) {
  dim3 grid(balance_blocks(nx, ny, M), G);
  balance_kernel<<<grid, kBalThreads, 0, s>>>(U, plane, nx, ny, M, mua, trig, dx, dy, w, 1.0 / c, partial,
                                              ticket, out, step, n_steps);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_grad(const float* MU, const float* Useg, const float* PT, const float* area,
                        int nx, int ny, int M, int G, size_t plane, size_t useg_group_stride,
                        double scale, int flip, double* grad_a, double* grad_b, cudaStream_t s,
                        long long* launches) {
  const int ncell = nx * ny;
  const long long threads = (M == 16 || M == 32) ? ncell : 32LL * ncell;
  grad_kernel<<<static_cast<int>((threads + 255) / 256), 256, 0, s>>>(MU, Useg, PT, area, ncell, M, G, plane,
                                                                      useg_group_stride, scale, flip, grad_a,
                                                                      grad_b);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_to_float(const double* in, float* out, size_t n, cudaStream_t s,
                            long long* launches) {
  to_float_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(in, out, n);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

}  // namespace rte_kern
