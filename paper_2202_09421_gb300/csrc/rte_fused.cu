// Tile-local fused FC-DOM step for the decomposed FC operator of Sec. 4.4
// (Algorithm 1's subdomains): one CTA owns one subdomain of one group, all M
// ordinates, and does the whole step of eq. (RTEAB4) in shared memory.
//
// Subdomain (kx, ky) owns x in [x_lo, x_hi), y in [y_lo, y_hi); its FC
// segments add two fringe points on interior sides.  The derivative at an
// owned point is the row of the owner's segment operator (ox x sx, dense, a
// few KB), so the x- and y-derivatives of the whole subdomain need only the
// owned block plus a two-point halo: the "box".  Per step the CTA
//   1. copies the box of u^k (owned + halo, from the input state buffer)
//      into shared memory (cp.async);
//   2. x-lines (row, m): lbuf = -xi_m D_x,seg u    (two lines per thread,
//      sharing float4 operator loads, paired FP32 FMAs);
//   3. y-lines (column, m): lbuf += -eta_m D_y,seg u;
//   4. per node (one warp, or half a warp at M = 16, over the ordinates):
//      L^k = lbuf + b P~u - (a + b) u, the AB4 update, the Fresnel boundary
//      condition with beam or adjoint injection on physical boundary nodes
//      (eq. RTE), the exitance ring (eq. OpMed); writes u^{k+1} to the output
//      state buffer and L^k over the oldest history slot.
// Neighbouring CTAs read this CTA's owned values as their halo during the
// same step, so input and output states are different buffers.
//
// Per update: 4 B of u (plus the halo share) + 12 B of history read, 8 B
// written: about 25 B against the two-pass form's 36 B, and 2 (s_x + s_y) +
// 2 M flops of operator and scattering work instead of 2 (n_x + n_y) + 2 M.
// The history is not staged in shared memory (that would leave one CTA per
// SM): each warp streams it through registers one batch of nodes ahead, the
// first batch while the derivatives are formed.
#include <cstdint>

#include "rte_kernels.cuh"

namespace rte_kern {

namespace {

constexpr float kAB0 = 55.0f / 24.0f, kAB1 = -59.0f / 24.0f, kAB2 = 37.0f / 24.0f,
                kAB3 = -9.0f / 24.0f;
constexpr int kFThreads = 256;
constexpr int kHalo = 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Shared-memory layout (floats) of one CTA for MM ordinates and at most OM
// owned points per axis; every region starts on a 16-byte boundary.  About
// 88 KB at M = 32: two CTAs per SM.
template <int MM, int OM>
struct FusedSmem {
  static constexpr int kBox = OM + 2 * kHalo;                      // box side (nodes)
  static constexpr int kRow = kBox * MM + (MM == 16 ? 16 : 0);     // box row stride
  static constexpr int kOwn = OM * OM * MM;                        // owned values
  static constexpr int kBoxF = kBox * kRow;
  static constexpr int kOpF = (OM + 2 * kHalo) * OM;               // [k < seg][i < OM]
  static constexpr int kTotal = kBoxF + kOwn + 2 * kOpF + 2 * OM * OM;
  static constexpr size_t kBytes = static_cast<size_t>(kTotal) * sizeof(float);
};

// Two FP32 fused multiply-adds in one instruction (each rounded as fmaf).
__device__ __forceinline__ float2 fma2(float2 x, float2 y, float2 z) { return __ffma2_rn(x, y, z); }

__device__ __forceinline__ float group_sum(float v, int width) {
  for (int o = width / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Node passes of the per-node phase whose history loads are in flight
// together (a register pipeline one batch ahead; larger batches spill at
// 128 registers).

template <int MM, int OM, bool EXACT>
__global__ void __launch_bounds__(kFThreads, 2)
    fused_step_kernel(StepArgs a, BoundaryArgs b, const float* __restrict__ Uin, float* __restrict__ Uout,
                      const float* __restrict__ L1, const float* __restrict__ L2, float* __restrict__ L3,
                      int src_step, int ring_step) {
  using S = FusedSmem<MM, OM>;
  constexpr int kPerWarp = 32 / MM;                  // nodes per warp pass
  constexpr int kWarps = kFThreads / 32;
  constexpr int kBatch = 4;
  extern __shared__ __align__(16) float sm[];
  float* box = sm;                                  // [kBox][kRow]: node (x_lo-2+ib, y_lo-2+jb)
  float* lbuf = box + S::kBoxF;                     // [ny_own][nx_own][MM]
  float* dxs = lbuf + S::kOwn;                      // [k < sx][i < OM]
  float* dys = dxs + S::kOpF;                       // [k < sy][j < OM]
  float* abs_ = dys + S::kOpF;                      // [2][ny_own][nx_own]: a, b

  const int nx = a.nx, ny = a.ny, M = MM;
  const int part = blockIdx.x, g = blockIdx.y;
  const int kx = part % a.px, ky = part / a.px;
  const int x_lo = a.fxp[4 * kx], x_hi = a.fxp[4 * kx + 1], x_slo = a.fxp[4 * kx + 2], x_shi = a.fxp[4 * kx + 3];
  const int y_lo = a.fyp[4 * ky], y_hi = a.fyp[4 * ky + 1], y_slo = a.fyp[4 * ky + 2], y_shi = a.fyp[4 * ky + 3];
  // EXACT: every part owns OM x OM points (compile-time loop bounds)
  const int ox = EXACT ? OM : x_hi - x_lo, oy = EXACT ? OM : y_hi - y_lo;
  const int sx = x_shi - x_slo, sy = y_shi - y_slo;
  const int own = ox * oy;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = lane % MM, sub = lane / MM;
  const size_t goff = static_cast<size_t>(g) * a.plane;
  const float* Ug = Uin + goff;

  // 1. The box of u^k by cp.async: rows of the y-segment; owned rows span the
  //    x-segment, fringe rows the owned columns.
  {
    constexpr int V = MM / 4;                       // float4 per node
    for (int r = 0; r < sy; ++r) {
      const int gj = y_slo + r;
      const bool owned_row = gj >= y_lo && gj < y_hi;
      const int c0 = owned_row ? x_slo : x_lo, c1 = owned_row ? x_shi : x_hi;
      const int items = (c1 - c0) * V;
      const float* src = Ug + (static_cast<size_t>(gj) * nx + c0) * M;
      float* dst = box + (gj - y_lo + kHalo) * S::kRow + (c0 - x_lo + kHalo) * MM;
      for (int e = tid; e < items; e += kFThreads) cp16(dst + 4 * e, src + 4 * e);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // Node passes of the per-node phase: warp w takes the owned rows
  // w, w + kWarps, ..., each in ppr passes of kPerWarp nodes (lane group sub
  // takes column pass * kPerWarp + sub).  A cursor (row, column) walks them
  // without divisions; columns past the row end mirror node (0, 0).
  const int ppr = (ox + kPerWarp - 1) / kPerWarp;
  const int n_pass = (warp < oy ? (oy - warp + kWarps - 1) / kWarps : 0) * ppr;
  auto advance = [&](int& jl, int& il) {
    il += kPerWarp;
    if (il >= ppr * kPerWarp) {
      il = sub;
      jl += kWarps;
    }
  };
  auto hist_index = [&](int jl, int il) {
    const bool ok = jl < oy && il < ox;
    return goff + (static_cast<size_t>(y_lo + (ok ? jl : 0)) * nx + x_lo + (ok ? il : 0)) * M + m;
  };
  // History of this warp's first batch of passes, in flight while the
  // derivatives are formed.
  int pj = warp, pi = sub;                          // prefetch cursor
  float h1[kBatch], h2[kBatch], h3[kBatch];
#pragma unroll
  for (int t = 0; t < kBatch; ++t) {
    const size_t e = hist_index(pj, pi);
    h1[t] = __ldg(L1 + e);
    h2[t] = __ldg(L2 + e);
    h3[t] = L3[e];
    advance(pj, pi);
  }
  // Segment operators of this part (transposed: [k][i]), the phase matrix,
  // and the owned block of a and b.
  {
    const float* fx = a.FxT + static_cast<size_t>(kx) * S::kOpF;
    const float* fy = a.FyT + static_cast<size_t>(ky) * S::kOpF;
    for (int e = tid; e < S::kOpF; e += kFThreads) {
      dxs[e] = __ldg(fx + e);
      dys[e] = __ldg(fy + e);
    }
    for (int e = tid; e < own; e += kFThreads) {
      const int jl = e / ox, il = e - jl * ox;
      const size_t cell = static_cast<size_t>(y_lo + jl) * nx + x_lo + il;
      abs_[e] = __ldg(a.mua + cell);
      abs_[OM * OM + e] = __ldg(a.mus + cell);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();

  // 2. x-lines: line l = (row jl, ordinate m); outputs i < ox.
  {
    const int nl = oy * MM;
    const int xoff = (x_slo - x_lo + kHalo) * MM;
    for (int l0 = tid; l0 < nl; l0 += 2 * kFThreads) {
      const int l1 = l0 + kFThreads < nl ? l0 + kFThreads : l0;
      const int j0 = l0 / MM, m0 = l0 - j0 * MM, j1 = l1 / MM, m1 = l1 - j1 * MM;
      const float* r0 = box + (j0 + kHalo) * S::kRow + xoff + m0;
      const float* r1 = box + (j1 + kHalo) * S::kRow + xoff + m1;
      float2 acc0[OM / 2], acc1[OM / 2];
#pragma unroll
      for (int i = 0; i < OM / 2; ++i) acc0[i] = acc1[i] = make_float2(0.f, 0.f);
      // interior parts have the full segment (owned range + two fringe
      // points on each side): a fixed trip count
      const int kx_n = (EXACT && sx == OM + 2 * kHalo) ? OM + 2 * kHalo : sx;
#pragma unroll 4
      for (int k = 0; k < kx_n; ++k) {
        const float u0 = r0[k * MM], u1 = r1[k * MM];
        const float2 uu0 = make_float2(u0, u0), uu1 = make_float2(u1, u1);
        const float4* dk = reinterpret_cast<const float4*>(dxs + k * OM);
#pragma unroll
        for (int q = 0; q < OM / 4; ++q) {
          if (4 * q < ox) {
            const float4 c = dk[q];
            const float2 clo = make_float2(c.x, c.y), chi = make_float2(c.z, c.w);
            acc0[2 * q] = fma2(clo, uu0, acc0[2 * q]);
            acc0[2 * q + 1] = fma2(chi, uu0, acc0[2 * q + 1]);
            acc1[2 * q] = fma2(clo, uu1, acc1[2 * q]);
            acc1[2 * q + 1] = fma2(chi, uu1, acc1[2 * q + 1]);
          }
        }
      }
      const float xi0 = -__ldg(a.xi + m0), xi1 = -__ldg(a.xi + m1);
#pragma unroll
      for (int i = 0; i < OM; ++i) {
        if (i < ox) {
          const float v0 = (i & 1) ? acc0[i / 2].y : acc0[i / 2].x;
          const float v1 = (i & 1) ? acc1[i / 2].y : acc1[i / 2].x;
          lbuf[(j0 * ox + i) * MM + m0] = xi0 * v0;
          if (l1 != l0) lbuf[(j1 * ox + i) * MM + m1] = xi1 * v1;
        }
      }
    }
  }
  __syncthreads();

  // 3. y-lines: line l = (column il, ordinate m); outputs j < oy.
  {
    const int nl = ox * MM;
    const int yoff = (y_slo - y_lo + kHalo) * S::kRow;
    for (int l0 = tid; l0 < nl; l0 += 2 * kFThreads) {
      const int l1 = l0 + kFThreads < nl ? l0 + kFThreads : l0;
      const int i0 = l0 / MM, m0 = l0 - i0 * MM, i1 = l1 / MM, m1 = l1 - i1 * MM;
      const float* c0 = box + yoff + (i0 + kHalo) * MM + m0;
      const float* c1 = box + yoff + (i1 + kHalo) * MM + m1;
      float2 acc0[OM / 2], acc1[OM / 2];
#pragma unroll
      for (int j = 0; j < OM / 2; ++j) acc0[j] = acc1[j] = make_float2(0.f, 0.f);
      const int ky_n = (EXACT && sy == OM + 2 * kHalo) ? OM + 2 * kHalo : sy;
#pragma unroll 4
      for (int k = 0; k < ky_n; ++k) {
        const float u0 = c0[k * S::kRow], u1 = c1[k * S::kRow];
        const float2 uu0 = make_float2(u0, u0), uu1 = make_float2(u1, u1);
        const float4* dk = reinterpret_cast<const float4*>(dys + k * OM);
#pragma unroll
        for (int q = 0; q < OM / 4; ++q) {
          if (4 * q < oy) {
            const float4 c = dk[q];
            const float2 clo = make_float2(c.x, c.y), chi = make_float2(c.z, c.w);
            acc0[2 * q] = fma2(clo, uu0, acc0[2 * q]);
            acc0[2 * q + 1] = fma2(chi, uu0, acc0[2 * q + 1]);
            acc1[2 * q] = fma2(clo, uu1, acc1[2 * q]);
            acc1[2 * q + 1] = fma2(chi, uu1, acc1[2 * q + 1]);
          }
        }
      }
      const float et0 = -__ldg(a.eta + m0), et1 = -__ldg(a.eta + m1);
#pragma unroll
      for (int j = 0; j < OM; ++j) {
        if (j < oy) {
          const float v0 = (j & 1) ? acc0[j / 2].y : acc0[j / 2].x;
          const float v1 = (j & 1) ? acc1[j / 2].y : acc1[j / 2].x;
          lbuf[(j * ox + i0) * MM + m0] = fmaf(et0, v0, lbuf[(j * ox + i0) * MM + m0]);
          if (l1 != l0) lbuf[(j * ox + i1) * MM + m1] = fmaf(et1, v1, lbuf[(j * ox + i1) * MM + m1]);
        }
      }
    }
  }
  __syncthreads();

  // 4. Per node: scattering, L^k, AB4, boundary condition, exitance; the
  //    history of the next batch of passes is loaded while this one runs.
  {
    float prow[MM];
#pragma unroll
    for (int q = 0; q < MM; ++q) prow[q] = __ldg(a.PT + q * MM + m);   // P~[m][q]: lanes read consecutive words
    const int ring_len = 2 * ny + 2 * nx;
    // An interior subdomain of the exact size has no node on the physical
    // boundary, and its passes form a fixed grid (each warp's owned rows x the
    // column passes), so every index below is a constant offset from the
    // thread's bases.  Same arithmetic, in the same order, as the general
    // loop that follows; the first batch's history (loaded before the
    // derivatives) is for the same nodes.
    const bool interior = EXACT && x_lo > 0 && x_hi < nx && y_lo > 0 && y_hi < ny;   // CTA-uniform
    if (interior) {
      constexpr int kRowsW = OM / kWarps;                        // owned rows per warp
      constexpr int kColP = OM / kPerWarp;                       // column passes per row
      constexpr int kPass = kRowsW * kColP;
      const size_t hbase = goff + (static_cast<size_t>(y_lo + warp) * nx + x_lo + sub) * M + m;
      const size_t hrow = static_cast<size_t>(kWarps) * nx * M;
      auto hidx = [&](int pp) {
        return hbase + static_cast<size_t>(pp / kColP) * hrow + static_cast<size_t>((pp % kColP) * kPerWarp) * M;
      };
      const float* unb = box + (warp + kHalo) * S::kRow + (sub + kHalo) * MM;
#pragma unroll
      for (int p0 = 0; p0 < kPass; p0 += kBatch) {
        float g1[kBatch], g2[kBatch], g3[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
          const int pp = p0 + kBatch + t;
          g1[t] = g2[t] = g3[t] = 0.f;
          if (pp < kPass) {
            const size_t e = hidx(pp);
            g1[t] = __ldg(L1 + e);
            g2[t] = __ldg(L2 + e);
            g3[t] = L3[e];
          }
        }
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
          const int pp = p0 + t, rr = pp / kColP, cc = pp % kColP;
          const float* un = unb + rr * kWarps * S::kRow + cc * kPerWarp * MM;
          float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < MM; q += 4) {
            const float4 v = *reinterpret_cast<const float4*>(un + q);
            s01 = fma2(make_float2(prow[q], prow[q + 1]), make_float2(v.x, v.y), s01);
            s23 = fma2(make_float2(prow[q + 2], prow[q + 3]), make_float2(v.z, v.w), s23);
          }
          const float sc = (s01.x + s01.y) + (s23.x + s23.y);
          const float u = un[m];
          const int n = (warp + kWarps * rr) * OM + sub + kPerWarp * cc;
          const float av = abs_[n], bv = abs_[OM * OM + n];
          const float lk = fmaf(bv, sc, lbuf[n * MM + m] - (av + bv) * u);
          const float pre = fmaf(a.cdt, kAB0 * lk + kAB1 * h1[t] + kAB2 * h2[t] + kAB3 * h3[t], u);
          const size_t e = hidx(pp);
          L3[e] = lk;
          Uout[e] = pre;
        }
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
          h1[t] = g1[t];
          h2[t] = g2[t];
          h3[t] = g3[t];
        }
      }
      return;
    }
    int cj = warp, ci = sub;                         // compute cursor
    for (int t0 = 0; t0 < n_pass; t0 += kBatch) {
      float g1[kBatch], g2[kBatch], g3[kBatch];
      const bool more = t0 + kBatch < n_pass;
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        const size_t e = hist_index(pj, pi);
        g1[t] = more ? __ldg(L1 + e) : 0.f;
        g2[t] = more ? __ldg(L2 + e) : 0.f;
        g3[t] = more ? L3[e] : 0.f;
        advance(pj, pi);
      }
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        if (t0 + t >= n_pass) break;                   // warp-uniform
        const bool valid = ci < ox;
        const int jl = valid ? cj : 0, il = valid ? ci : 0;
        advance(cj, ci);
        const int n = jl * ox + il;
        const int gj = y_lo + jl, gi = x_lo + il;
        const float* un = box + (jl + kHalo) * S::kRow + (il + kHalo) * MM;
        float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < MM; q += 4) {
          const float4 v = *reinterpret_cast<const float4*>(un + q);
          s01 = fma2(make_float2(prow[q], prow[q + 1]), make_float2(v.x, v.y), s01);
          s23 = fma2(make_float2(prow[q + 2], prow[q + 3]), make_float2(v.z, v.w), s23);
        }
        const float sc = (s01.x + s01.y) + (s23.x + s23.y);
        const float u = un[m];
        const float av = abs_[n], bv = abs_[OM * OM + n];
        const int o = n * MM + m;
        const float lk = fmaf(bv, sc, lbuf[o] - (av + bv) * u);
        const float pre = fmaf(a.cdt, kAB0 * lk + kAB1 * h1[t] + kAB2 * h2[t] + kAB3 * h3[t], u);
        const size_t e = goff + (static_cast<size_t>(gj) * nx + gi) * M + m;
        const bool lf = gi == 0, rt = gi == nx - 1, bt = gj == 0, tp = gj == ny - 1;
        const bool bnd = valid && (lf || rt || bt || tp);
        if (valid) L3[e] = lk;
        if (!__any_sync(0xffffffffu, bnd)) {
          if (valid) Uout[e] = pre;
          continue;
        }
        // Boundary nodes in this pass: pre-BC values through shared memory
        // (this node's lbuf entries are no longer needed).
        if (valid) lbuf[o] = pre;
        __syncwarp();
        float v = pre;
        if (bnd) {
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
          const int node = lf ? gj : rt ? ny + gj : bt ? 2 * ny + gi : 2 * ny + nx + gi;
          if (act[m]) {
            float q = 0.f;
            for (int k = 0; k < b.kmax; ++k) {
              const size_t gk = static_cast<size_t>(g) * b.kmax + k;
              q = fmaf(__ldg(b.S + gk * ring_len + node) * __ldg(b.A + gk * M + m),
                       __ldg(b.T + gk * b.T_len + src_step), q);
            }
            if (b.rho)
              q = fmaf(1.0f - fco[m], __ldg(b.rho + (static_cast<size_t>(g) * b.rho_len + src_step) * ring_len + node), q);
            v = fmaf(fco[m], lbuf[n * MM + refl[m]], q);
          }
        }
        if (valid) Uout[e] = v;
        // exitance of the node's faces (eq. OpMed), summed over its ordinates
        float ex = 0.f, ey = 0.f;
        if (bnd && (lf || rt)) ex = b.wexit[(lf ? 0 : 1) * M + m] * v;
        if (bnd && (bt || tp)) ey = b.wexit[(bt ? 2 : 3) * M + m] * v;
        ex = group_sum(ex, MM);
        ey = group_sum(ey, MM);
        if (bnd && m == 0 && b.ring_out && ring_step >= 0) {
          float* ro = b.ring_out + (static_cast<size_t>(g) * b.ring_steps + ring_step) * ring_len;
          if (lf || rt) ro[lf ? gj : ny + gj] = ex;
          if (bt || tp) ro[bt ? 2 * ny + gi : 2 * ny + nx + gi] = ey;
        }
        __syncwarp();
      }
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        h1[t] = g1[t];
        h2[t] = g2[t];
        h3[t] = g3[t];
      }
    }
  }
}

template <int MM, int OM, bool EXACT>
cudaError_t launch_fused_t(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                           const float* L1, const float* L2, float* L3, int src_step, int ring_step,
                           cudaStream_t s) {
  using S = FusedSmem<MM, OM>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<MM, OM, EXACT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(S::kBytes));
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  dim3 grid(a.px * a.py, a.G);
  fused_step_kernel<MM, OM, EXACT><<<grid, kFThreads, S::kBytes, s>>>(a, b, Uin, Uout, L1, L2, L3, src_step,
                                                                      ring_step);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_fused_m(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                           const float* L1, const float* L2, float* L3, int src_step, int ring_step,
                           cudaStream_t s) {
  return a.fused_exact ? launch_fused_t<MM, kFusedOwnMax, true>(a, b, Uin, Uout, L1, L2, L3, src_step, ring_step, s)
                       : launch_fused_t<MM, kFusedOwnMax, false>(a, b, Uin, Uout, L1, L2, L3, src_step, ring_step, s);
}

}  // namespace

bool fused_supported(const StepArgs& a) {
  if (a.px < 2 || a.py < 2 || !a.FxT || !a.FyT || !a.fxp || !a.fyp) return false;
  return (a.M == 16 || a.M == 32) && a.fused_own_max <= kFusedOwnMax;
}

cudaError_t launch_step_fused(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                              const float* L1, const float* L2, float* L3, int step, cudaStream_t s,
                              long long* launches, cudaEvent_t* ev) {
  const int ring_step = b.ring_out ? step : -1;
  if (ev) {
    cudaEventRecord(ev[0], s);
    cudaEventRecord(ev[1], s);
  }
  const cudaError_t e = a.M == 16 ? launch_fused_m<16>(a, b, Uin, Uout, L1, L2, L3, step, ring_step, s)
                                  : launch_fused_m<32>(a, b, Uin, Uout, L1, L2, L3, step, ring_step, s);
  if (ev) cudaEventRecord(ev[2], s);
  if (launches) *launches += 1;
  return e;
}

}  // namespace rte_kern
