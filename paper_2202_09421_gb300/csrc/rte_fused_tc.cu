// Tensor-core (tcgen05, split 3xTF32) form of the tile-local fused step of
// the decomposed FC operator (Sec. 4.4, Algorithm 1's subdomains), for
// M = 32 ordinates and parts that all own 16 x 16 points.
//
// One CTA takes one subdomain of one group and does the whole step of
// eq. (RTEAB4) on it, like the FP32 form in rte_fused.cu; the three
// contractions of the step run on the tensor cores, accumulated in FP32 in
// tensor memory:
//   x-derivative  dX[(j, m)][i] = sum_p u(j, p, m) Dx[i][p]
//                 A rows (owned row j, ordinate m), 128 per tile (4 rows),
//                 K = box position p along x (20 positions, padded to 24);
//                 B = the part's segment operator, rows i (N = 16);
//   y-derivative  dY[(i, m)][j] = sum_p u(p, i, m) Dy[j][p]
//                 A rows (owned column i, m), K = box position along y;
//   scattering    S[n][m] = sum_q u(n, q) P~[m][q]
//                 A rows = owned node n (128 per tile), K = q; B = P~.
// The "box" is the owned block plus a two-point halo on each side; box
// position p is grid point lo - 2 + p.  The segment operators are images
// indexed by box position: entry (i, p) is the derivative at owned point i
// from the segment point at box position p, zero outside the segment.
// Positions outside the part's segment are never read and enter the
// operands as zeros.
//
// Operands are split as hi = r(x), lo = r(x - hi) (r: round to tf32) and
// the products hi*hi + hi*lo + lo*hi accumulated (about 2^-22 relative per
// product).  The CTA copies the box of u^k into shared memory (cp.async)
// and converts ten A tiles from it (4 x-tiles, 4 y-tiles, 2 scattering
// tiles), each in two halves: the hi tile goes to staging slot 0 and one
// thread issues the MMAs that take A_hi, then the lo tile goes to slot 1
// and the MMAs that take A_lo follow; a slot is rewritten only after the
// MMAs of the previous tile on it have completed, so the conversion of one
// half overlaps the MMAs of the other.  Slots are 16 KB (K-major, 128-byte
// swizzle).  Two CTAs share an SM (about 101 KB of shared memory and 256
// tensor-memory columns each).
//
// Epilogue: the two staging slots become a [node][m] buffer (bank-conflict-free
// XOR layout, address n * 32 + (m ^ (n & 31))): -eta_m dY is written there
// by the threads holding dY (lane = (i, m)), then b S is added by the
// threads holding S (lane = node); the threads of the final combine own (row
// j, ordinate m) for 16 nodes of the row, hold dX from tensor memory and
// form L^k = -xi dX - eta dY + b P~u - (a + b) u, the AB4 update, the Fresnel
// boundary condition with beam or adjoint injection on physical boundary
// nodes (eq. RTE; the reflected ordinate is a lane of the same warp), and
// the exitance ring (eq. OpMed).  u^{k+1} goes to the output state buffer
// and L^k over the oldest history slot.  The history goes to L2 on entry
// and into registers one batch of 8 nodes ahead of the combine.
#include <cstdint>

#include "rte_tc_common.cuh"

namespace rte_kern {

namespace {

using namespace tc;

constexpr int kFM = 32;                 // ordinates
constexpr int kFO = 16;                 // owned points per axis
constexpr int kFB = kFO + 4;            // box positions per axis (two halo points each side)
constexpr int kFT = 256;                // threads

// Shared-memory layout in bytes from a 1024-byte-aligned base.
constexpr int kSlot0 = 0;                           // A staging: hi tile (16 KB)
constexpr int kSlot1 = 16384;                       //            lo tile (16 KB); both: [node][m] buffer
constexpr int kOpX = 32768;                         // x segment operator: hi 16 rows x 128 B, lo
constexpr int kOpY = kOpX + 4096;                   // y segment operator
constexpr int kOpP = kOpY + 4096;                   // P~: hi 32 rows x 128 B, lo
constexpr int kBoxOff = kOpP + 8192;                // u^k box [kFB][kFB][kFM] floats
constexpr int kAOff = kBoxOff + kFB * kFB * kFM * 4;   // a of the owned nodes
constexpr int kBOff = kAOff + kFO * kFO * 4;        // b of the owned nodes
constexpr int kEnd = kBOff + kFO * kFO * 4;
constexpr size_t kSmemTc = static_cast<size_t>(kEnd) + 1024;   // alignment slack
constexpr int kTmemCols = 256;          // dX 64 + dY 64 + S 64 columns
constexpr int kColX = 0, kColY = 64, kColS = 128;
constexpr int kOpImgFloats = 2 * kFO * 32;          // one part's segment image (hi + lo)
constexpr int kRounds = 10;             // 4 x-tiles, 4 y-tiles, 2 scattering tiles

__device__ __forceinline__ bool mbar_wait_t(uint32_t bar, uint32_t parity, int* err) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  return true;
}

__device__ __forceinline__ void cp16(void* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(void* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Bulk copy that adds no arrival (the caller arrives once with the total).
__device__ __forceinline__ void bulk_copy_noarrive(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Prefetch of a contiguous range into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ int nb_idx(int n, int m) { return n * kFM + (m ^ (n & 31)); }

__global__ void __launch_bounds__(kFT, 2)
    fused_step_tc_kernel(StepArgs a, BoundaryArgs b, const float* __restrict__ Uin, float* __restrict__ Uout,
                         const float* __restrict__ L1, const float* __restrict__ L2, float* __restrict__ L3,
                         int src_step, int ring_step) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bars[3];          // operator images, hi slot, lo slot
  __shared__ uint32_t tmem_slot;
  __shared__ int skip;
  // A launch after a timed-out one does nothing (one read, so that the whole
  // CTA takes the same branch).
  if (threadIdx.x == 0) skip = *static_cast<volatile int*>(a.err);
  __syncthreads();
  if (skip) return;

  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  float* box = reinterpret_cast<float*>(sm + kBoxOff);
  float* asm_ = reinterpret_cast<float*>(sm + kAOff);
  float* bsm = reinterpret_cast<float*>(sm + kBOff);
  float* nbuf = reinterpret_cast<float*>(sm + kSlot0);

  const int nx = a.nx, ny = a.ny;
  const int part = blockIdx.x, g = blockIdx.y;
  const int kx = part % a.px, ky = part / a.px;
  const int x_lo = a.fxp[4 * kx], x_hi = a.fxp[4 * kx + 1], x_slo = a.fxp[4 * kx + 2], x_shi = a.fxp[4 * kx + 3];
  const int y_lo = a.fyp[4 * ky], y_hi = a.fyp[4 * ky + 1], y_slo = a.fyp[4 * ky + 2], y_shi = a.fyp[4 * ky + 3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t goff = static_cast<size_t>(g) * a.plane;
  const float* Ug = Uin + goff;
  const uint32_t bar_ops = smem_u32(&bars[0]);
  const uint32_t bar_slot[2] = {smem_u32(&bars[1]), smem_u32(&bars[2])};
  bool ok = true;

  if (tid == 0) {
    for (int k = 0; k < 3; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // The box of u^k by cp.async: rows of the y-segment; owned rows span the
  // x-segment, fringe rows the owned columns.  Then a and b of the owned
  // nodes.
  {
    const int sy = y_shi - y_slo;
    for (int r = 0; r < sy; ++r) {
      const int gj = y_slo + r;
      const bool owned_row = gj >= y_lo && gj < y_hi;
      const int c0 = owned_row ? x_slo : x_lo, c1 = owned_row ? x_shi : x_hi;
      const int items = (c1 - c0) * (kFM / 4);
      const float* src = Ug + (static_cast<size_t>(gj) * nx + c0) * kFM;
      float* dst = box + ((gj - y_lo + 2) * kFB + (c0 - x_lo + 2)) * kFM;
      for (int e = tid; e < items; e += kFT) cp16(dst + 4 * e, src + 4 * e);
    }
    const size_t cell = static_cast<size_t>(y_lo + (tid >> 4)) * nx + x_lo + (tid & 15);   // kFT == 256 nodes
    cp4(asm_ + tid, a.mua + cell);
    cp4(bsm + tid, a.mus + cell);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // The history of the owned block goes to L2 now (threads 0..47: one row
  // of L^{k-1}, L^{k-2} or L^{k-3} each); the final combine reads it.
  if (tid < 3 * kFO) {
    const float* hsrc = tid < kFO ? L1 : tid < 2 * kFO ? L2 : L3;
    prefetch_l2(hsrc + goff + (static_cast<size_t>(y_lo + tid % kFO) * nx + x_lo) * kFM, kFO * kFM * 4);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();                                   // barriers initialised, TMEM allocated
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_ops), "r"(4096 + 4096 + 8192)
                 : "memory");
    bulk_copy_noarrive(smem_u32(sm + kOpX), a.FxImg + static_cast<size_t>(kx) * kOpImgFloats, 4096, bar_ops);
    bulk_copy_noarrive(smem_u32(sm + kOpY), a.FyImg + static_cast<size_t>(ky) * kOpImgFloats, 4096, bar_ops);
    bulk_copy_noarrive(smem_u32(sm + kOpP), a.PImg, 8192, bar_ops);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();                                   // box and coefficients in place

  // ---------------- rounds: split one A tile, hi then lo ----------------
  // Each round converts one tile: its hi values go to slot 0 and the MMAs
  // that take A_hi (A_hi B_hi, A_hi B_lo) are issued; then its lo values go
  // to slot 1 and the MMAs that take A_lo (A_lo B_hi).  A slot is rewritten
  // only after the previous round's MMAs on it have completed (round r
  // waits for phase r - 1 of the slot's barrier).
  const uint32_t idesc16 = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  const uint32_t idesc32 = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
#pragma unroll 1
  for (int r = 0; r < kRounds; ++r) {
    float4 vh[4], vl[4];
    const bool der = r < 8;
    if (der) {
      // rows (owned line l = 4t + row / 32, m = lane); K = box position
      // along the axis, three groups of 4 (20 positions + 4 zeros)
      const bool xt = r < 4;
      const int t = xt ? r : r - 4;
      const int line = 4 * t + ((tid & 127) >> 5) + 2;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int grp = (tid >> 7) + 2 * k;
        float4 v;
        float* vp = reinterpret_cast<float*>(&v);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p = 4 * grp + e;
          const int gp = (xt ? x_lo : y_lo) - 2 + p;
          const bool valid = p < kFB && gp >= (xt ? x_slo : y_slo) && gp < (xt ? x_shi : y_shi);
          const int pc = valid ? p : 2;              // box index inside the loaded block
          const float x = box[(xt ? line * kFB + pc : pc * kFB + line) * kFM + lane];
          vp[e] = valid ? x : 0.f;
        }
        split4(v, 1.0f, vh[k], vl[k]);
      }
    } else {
      // rows = owned nodes n = 128 t + row; K = q
      const int t = r - 8;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int it = tid + k * kFT;
        const int n = 128 * t + (it >> 3);
        const float4 v =
            *reinterpret_cast<const float4*>(box + (((n >> 4) + 2) * kFB + (n & 15) + 2) * kFM + 4 * (it & 7));
        split4(v, 1.0f, vh[k], vl[k]);
      }
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      unsigned char* slot = sm + (half ? kSlot1 : kSlot0);
      if (r > 0) ok = mbar_wait_t(bar_slot[half], (r - 1) & 1, a.err) && ok;
      if (der) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          *reinterpret_cast<float4*>(slot + sw128_off(tid & 127, (tid >> 7) + 2 * k)) = half ? vl[k] : vh[k];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int it = tid + k * kFT;
          *reinterpret_cast<float4*>(slot + sw128_off(it >> 3, it & 7)) = half ? vl[k] : vh[k];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        if (r == 0 && half == 0) ok = mbar_wait_t(bar_ops, 0, a.err) && ok;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t dA = sw128_desc(smem_u32(slot));
        if (der) {
          const unsigned char* Bop = sm + (r < 4 ? kOpX : kOpY);
          const uint64_t dBh = sw128_desc(smem_u32(Bop)), dBl = sw128_desc(smem_u32(Bop + 2048));
          const uint32_t acc = tmem + (r < 4 ? kColX + 16 * r : kColY + 16 * (r - 4));
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);   // 32 bytes per K step
            if (half == 0) {
              mma<false>(acc, dA + o, dBh + o, idesc16, kk > 0 ? 1u : 0u);
              mma<false>(acc, dA + o, dBl + o, idesc16, 1u);
            } else {
              mma<false>(acc, dA + o, dBh + o, idesc16, 1u);
            }
          }
        } else {
          const uint64_t dPh = sw128_desc(smem_u32(sm + kOpP)), dPl = sw128_desc(smem_u32(sm + kOpP + 4096));
          const uint32_t acc = tmem + kColS + 32 * (r - 8);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);
            if (half == 0) {
              mma<false>(acc, dA + o, dPh + o, idesc32, kk > 0 ? 1u : 0u);
              mma<false>(acc, dA + o, dPl + o, idesc32, 1u);
            } else {
              mma<false>(acc, dA + o, dPh + o, idesc32, 1u);
            }
          }
        }
        mma_commit(bar_slot[half]);
      }
    }
  }
  // Epilogue rows of this thread: warp w (quarter q = w % 4, half h = w / 4)
  // combines owned rows j0 = 8h + q and j1 = j0 + 4 for ordinate m = lane, in
  // four batches of 8 nodes; each batch's history is loaded one batch ahead
  // (the first while the last MMAs run).
  const int qw = warp & 3, hw = warp >> 2;
  const int j0 = 8 * hw + qw, j1 = j0 + 4;
  float hb[8][3], hn[8][3];                          // L^{k-1}, L^{k-2}, L^{k-3} of 8 nodes
  auto load_batch = [&](int beta, float (&h)[8][3]) {
    const int j = beta < 2 ? j0 : j1, i0 = 8 * (beta & 1);
    const size_t e0 = goff + (static_cast<size_t>(y_lo + j) * nx + x_lo + i0) * kFM + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q][0] = __ldg(L1 + e0 + q * kFM);
      h[q][1] = __ldg(L2 + e0 + q * kFM);
      h[q][2] = L3[e0 + q * kFM];
    }
  };
  load_batch(0, hb);
  ok = mbar_wait_t(bar_slot[0], (kRounds - 1) & 1, a.err) && ok;
  ok = mbar_wait_t(bar_slot[1], (kRounds - 1) & 1, a.err) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---------------- epilogue ----------------
  const uint32_t tq = tmem + (static_cast<uint32_t>(32 * qw) << 16);   // this warp's lane quarter
  // -eta_m dY: y-tiles 2h, 2h + 1; lane = (column i = 4t + q, m), columns j
  {
    const float neta = -__ldg(a.eta + lane);
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
      const int t = 2 * hw + tt, i = 4 * t + qw;
      float v[16];
      tmem_ld16(tq + kColY + 16 * t, v);
#pragma unroll
      for (int j = 0; j < kFO; ++j) nbuf[nb_idx(j * kFO + i, lane)] = neta * v[j];
    }
  }
  __syncthreads();
  // + b S: scattering tile h; lane = node n = 128h + 32q + lane, columns m
  {
    const int n = 128 * hw + 32 * qw + lane;
    float s[32];
    tmem_ld16(tq + kColS + 32 * hw, s);
    tmem_ld16(tq + kColS + 32 * hw + 16, s + 16);
    const float bn = bsm[n];
#pragma unroll
    for (int m = 0; m < kFM; ++m) {
      const int idx = nb_idx(n, m);
      nbuf[idx] = fmaf(bn, s[m], nbuf[idx]);
    }
  }
  __syncthreads();
  // Final combine.
  const float nxi = -__ldg(a.xi + lane);
  const int ring_len = 2 * ny + 2 * nx;
#pragma unroll
  for (int beta = 0; beta < 4; ++beta) {
    if (beta + 1 < 4) load_batch(beta + 1, hn);
    const int j = beta < 2 ? j0 : j1, i0 = 8 * (beta & 1);
    float dxv[8];
    tmem_ld8(tq + kColX + 16 * (j >> 2) + i0, dxv);   // x-tile j / 4, lane quarter j % 4
    const int gj = y_lo + j;
    const size_t erow = goff + (static_cast<size_t>(gj) * nx + x_lo + i0) * kFM + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = i0 + q, n = j * kFO + i;
      const float u = box[((j + 2) * kFB + i + 2) * kFM + lane];
      const float lk = fmaf(-(asm_[n] + bsm[n]), u, fmaf(nxi, dxv[q], nbuf[nb_idx(n, lane)]));
      const float pre = ab4_node(a.cdt, lk, hb[q][0], hb[q][1], hb[q][2], u);
      const size_t e = erow + static_cast<size_t>(q) * kFM;
      const int gi = x_lo + i;
      const bool lf = gi == 0, rt = gi == nx - 1, bt = gj == 0, tp = gj == ny - 1;
      if (ok) L3[e] = lk;
      if (!(lf || rt || bt || tp)) {                 // warp-uniform
        if (ok) Uout[e] = pre;
        continue;
      }
      // physical boundary node: Fresnel condition with injection (eq. RTE)
      const int* refl;
      const float* fco;
      const unsigned char* act;
      if ((lf || rt) && (bt || tp)) {
        const int c = (rt ? 1 : 0) + (tp ? 2 : 0);
        refl = b.corner_refl + c * kFM; fco = b.corner_f + c * kFM; act = b.corner_act + c * kFM;
      } else {
        const int F = lf ? 0 : rt ? 1 : bt ? 2 : 3;
        refl = b.face_refl + F * kFM; fco = b.face_f + F * kFM; act = b.face_act + F * kFM;
      }
      const int node = lf ? gj : rt ? ny + gj : bt ? 2 * ny + gi : 2 * ny + nx + gi;
      const float pr = __shfl_sync(0xffffffffu, pre, refl[lane]);
      float v = pre;
      if (act[lane]) {
        float qs = 0.f;
        for (int k = 0; k < b.kmax; ++k) {
          const size_t gk = static_cast<size_t>(g) * b.kmax + k;
          qs = fmaf(__ldg(b.S + gk * ring_len + node) * __ldg(b.A + gk * kFM + lane),
                    __ldg(b.T + gk * b.T_len + src_step), qs);
        }
        if (b.rho)
          qs = fmaf(1.0f - fco[lane],
                    __ldg(b.rho + (static_cast<size_t>(g) * b.rho_len + src_step) * ring_len + node), qs);
        v = fmaf(fco[lane], pr, qs);
      }
      if (ok) Uout[e] = v;
      // exitance of the node's faces (eq. OpMed), summed over the ordinates
      float ex = (lf || rt) ? b.wexit[(lf ? 0 : 1) * kFM + lane] * v : 0.f;
      float ey = (bt || tp) ? b.wexit[(bt ? 2 : 3) * kFM + lane] * v : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ex += __shfl_xor_sync(0xffffffffu, ex, o);
        ey += __shfl_xor_sync(0xffffffffu, ey, o);
      }
      if (ok && lane == 0 && b.ring_out && ring_step >= 0) {
        float* ro = b.ring_out + (static_cast<size_t>(g) * b.ring_steps + ring_step) * ring_len;
        if (lf || rt) ro[lf ? gj : ny + gj] = ex;
        if (bt || tp) ro[bt ? 2 * ny + gi : 2 * ny + nx + gi] = ey;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) hb[q][c] = hn[q][c];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

bool fused_tc_supported(const StepArgs& a) {
  return a.tc_mode == 1 && a.M == kFM && a.fused_exact && a.FxImg && a.FyImg && a.PImg && fused_supported(a);
}

static cudaError_t launch_fused_tc(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                                   const float* L1, const float* L2, float* L3, int src_step, int ring_step,
                                   cudaStream_t s) {
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(fused_step_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(kSmemTc));
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  dim3 grid(a.px * a.py, a.G);
  fused_step_tc_kernel<<<grid, kFT, kSmemTc, s>>>(a, b, Uin, Uout, L1, L2, L3, src_step, ring_step);
  return cudaGetLastError();
}

cudaError_t launch_step_fused_tc(const StepArgs& a, const BoundaryArgs& b, const float* Uin, float* Uout,
                                 const float* L1, const float* L2, float* L3, int step, cudaStream_t s,
                                 long long* launches, cudaEvent_t* ev) {
  const int ring_step = b.ring_out ? step : -1;
  if (ev) {
    cudaEventRecord(ev[0], s);
    cudaEventRecord(ev[1], s);
  }
  const cudaError_t e = launch_fused_tc(a, b, Uin, Uout, L1, L2, L3, step, ring_step, s);
  if (ev) cudaEventRecord(ev[2], s);
  if (launches) *launches += 1;
  return e;
}

}  // namespace rte_kern
