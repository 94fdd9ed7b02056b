// Tensor-core (tcgen05) form of the two FC-DOM passes for sm_103a.
//
// Each CTA owns one slab tile: 128 slab columns c (x-pass: grid rows j0 ..
// j0 + 128/M - 1 times the M ordinates, M in {16, 32, 64}; y-pass: grid
// columns i0 .. times M) over a whole line of n <= 512 positions, K = input
// positions.
//   x-pass: per 128-position tile t of the line, the dense FC operator D
//     (n x n, Sec. 4.3) is the A operand (M = 128 output positions) and the
//     transposed slab the B operand (N = 128 slab columns): tensor memory
//     holds acc_t[lane = output position i][column = (row, m)], so the
//     epilogue's lanes walk the contiguous x direction of the grid.
//   y-pass: the slab is the A operand (M = 128 slab columns) and D the B
//     operand (N = output positions, issued as N <= 256 halves):
//     acc[lane = (column, m)][column = j], so the epilogue's lanes walk the
//     contiguous (column, m) run of a grid row.
//
// x-pass: the node-local scattering sum b P~ u (Sec. 4.1) is accumulated into
// the same tensor-memory tile as a second contraction: for each grid row r of
// the tile, A = b(r, i) u(r, i, q) (rows i, K = ordinates q) and B = P~ (rows
// m, K = q); the -xi_m factor of the streaming term is folded into the slab
// operand.  The epilogue adds -(a + b) u:  R = b P~u - (a+b) u - xi_m D_x u.
// y-pass: acc = -eta_m D_y u; the epilogue forms L = R + acc, the AB4 update
// (eq. RTEAB4), the Fresnel boundary condition with beam or adjoint
// injection (eq. RTE), the exitance ring (eq. OpMed), and updates u in place.
// Transposed step of the exact discrete adjoint (BoundaryArgs::bct_src set,
// operator images of D_x^T and D_y^T): the y-pass epilogue forms
// ubar = w^{k+1} + R + acc (+ the readout transpose on ring nodes), the
// transposed boundary map w^k = BC^T ubar and v = c dt sum_i chi_i w^{k+i}.
//
// Precision: kind::tf32 or kind::f16 (BF16 operands) with split operands.
// Every operand x is split as hi = r(x), lo = r(x - hi), r the rounding to
// the operand type (D and P~ on the host, the slab and the scattering operand
// while staged), and the products hi*hi + hi*lo + lo*hi are accumulated in
// FP32: 3xTF32 (about 2^-22 relative per product) and bf16x3 (about 2^-16);
// the single-product forms (TF32, BF16) are the reduced-precision variants.
//
// Operands use the K-major 128-byte-swizzle layout (rows of 32 tf32 or 64
// bf16 values; 8-row atoms of 1024 B).  D and P~ chunks are pre-swizzled in global memory
// and copied with cp.async.bulk; the slab is converted and swizzled by all
// threads.  K runs in chunks of one 128-byte row (32 tf32 / 64 bf16
// positions); the next chunk's slab values are loaded into registers while
// the tensor core works on the current one.  One thread issues the MMAs
// and commits them to mbarriers; every wait is bounded and sets the context's
// timeout word (StepArgs::err) instead of spinning forever.
#include <cstdint>

#include "rte_tc_common.cuh"

namespace rte_kern {

namespace {

using namespace tc;

// Bounded wait (kWaitNs of wall clock); false, and the timeout word set,
// when the limit runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  return true;
}

constexpr int kPBytes = 2 * 32 * 128;   // P~ operand image: hi and lo, 32 rows x 128 B
constexpr int kMaxM = 64;
// y-pass epilogue: two 5-array buffers, three [16][128] tiles, boundary tables
constexpr size_t kEpiBytes = (2 * 5 * 16 + 3 * 16) * 128 * 4 + (8 + 4 + 8) * kMaxM * 4 + 8 * kMaxM;

// One CTA's work on slab tile `tile` of group g (x-pass: grid rows
// tile * 128/M ...; y-pass: grid columns).  Shared by the single-medium and
// the batched kernels below.
template <bool XPASS, int PREC, int MM, bool SCAT_TC>
__device__ __forceinline__ void tc_pass_body(const StepArgs& a, const BoundaryArgs& b, float* __restrict__ U,
                                             float* __restrict__ R, const float* __restrict__ L1,
                                             const float* __restrict__ L2, float* __restrict__ L3, int src_step,
                                             int ring_step, int tile, int g) {
  using K = Kind<PREC>;
  constexpr bool X3 = K::X3, BF = K::BF;
  constexpr int KC = K::KC, GV = K::GV;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bars[4];   // full, done, p_full, scat_done
  __shared__ uint32_t tmem_slot;
  __shared__ float pcs[kMaxM];                 // P~[k][0]: the x-pass scattering weights
  const int nx = a.nx, ny = a.ny;
  constexpr int M = MM;
  const int n = XPASS ? nx : ny;
  const TcLayout L(n, X3, KC);
  constexpr int per_tile = kNC / M;           // grid rows (x) or columns (y) per tile
  const int t0 = tile * per_tile;             // first grid row (x) / column (y) of the tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t goff = static_cast<size_t>(g) * a.plane;
  const unsigned char* Dimg = static_cast<const unsigned char*>(XPASS ? a.DxImg : a.DyImg);
  const float* scale = XPASS ? a.xi : a.eta;
  const int n_lines = XPASS ? ny : nx;        // rows (x) / columns (y) of the grid

  // A launch after a timed-out one does nothing (the march reports the error).
  if (*static_cast<volatile int*>(a.err)) return;
  // x-pass: the y-pass that follows may be scheduled as soon as CTAs leave.
  if (XPASS) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  unsigned char* Psm = sm + L.stage_bytes;    // P~ image (x-pass, TC scattering)
  const uint32_t bar_full = smem_u32(&bars[0]), bar_done = smem_u32(&bars[1]);
  const uint32_t bar_p = smem_u32(&bars[2]), bar_scat = smem_u32(&bars[3]);

  if (tid == 0) {
    for (int k = 0; k < 4; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (XPASS)
    for (int k = tid; k < M; k += kThreads) pcs[k] = __ldg(a.PT + k);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(L.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // Failure injection (tests): one CTA waits on a barrier that nothing
  // arrives on, before this CTA has issued any copy or MMA, so that the
  // bounded wait runs out and sets the timeout word; the CTA then frees its
  // tensor memory and leaves without touching any output.
  if (a.test_expire && tile == 0 && g == 0) {
    __shared__ int gave_up;
    if (tid == 0) gave_up = mbar_wait(bar_scat, 0, a.err) ? 0 : 1;
    __syncthreads();
    if (gave_up) {
      if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L.tmem_cols));
      return;
    }
  }
  if constexpr (XPASS && SCAT_TC) {
    if (tid == 0) bulk_copy(smem_u32(Psm), a.PImg, kPBytes, bar_p);
  }

  const int nrows_img = L.nrows_img;                    // rows of the operator image
  // idesc: D = F32, A = B = TF32 (2) or BF16 (1), K-major, M = 128; N = 128
  // slab columns (x-pass) or output positions (y-pass, set per half).
  constexpr uint32_t kFmt = BF ? 1u : 2u;
  const uint32_t idesc_base = (1u << 4) | (kFmt << 7) | (kFmt << 10) | (static_cast<uint32_t>(kMT >> 4) << 24);
  const uint32_t idesc_x = idesc_base | (static_cast<uint32_t>(kNC >> 3) << 17);
  const size_t chunk_bytes = static_cast<size_t>(2) * nrows_img * 128;   // hi + lo tiles of one K chunk
  bool ok = true;

  // ---------------- main loop over K chunks ----------------
  // Slab^T chunk: S[c][kk] = -scale_m u(c, k0 + kk).  Each thread owns 4
  // (column, 16-byte group) items; the next chunk's loads are issued before
  // this chunk's MMAs so that their latency overlaps the tensor core.
  constexpr int kItems = kNC * (KC / GV) / kThreads;   // 4
  float v[kItems][GV];
  const uint64_t pol_keep = policy_evict_last();
  auto load_chunk = [&](int q) {
    const int k0 = q * KC;
#pragma unroll
    for (int t = 0; t < kItems; ++t) {
      const int it = tid + t * kThreads;
      const int c = it % kNC, grp = it / kNC;
      const int rc = c / M, m = c - rc * M;
      const int line = t0 + rc;
      const bool valid = line < n_lines;
#pragma unroll
      for (int e = 0; e < GV; ++e) {
        const int k = k0 + grp * GV + e;
        v[t][e] = 0.f;
        if (valid && k < n) {
          const size_t idx = XPASS ? goff + (static_cast<size_t>(line) * nx + k) * M + m
                                   : goff + (static_cast<size_t>(k) * nx + line) * M + m;
          v[t][e] = ld_hint(U + idx, pol_keep);
        }
      }
    }
  };
  unsigned char* Dhi = sm;                                        // n_mt tiles
  unsigned char* Dlo = sm + L.n_mt * kTileBytes;                  // (split forms)
  unsigned char* Shi = sm + (X3 ? 2 : 1) * L.n_mt * kTileBytes;
  unsigned char* Slo = Shi + kTileBytes;
  load_chunk(0);
  for (int q = 0; q < L.n_kc; ++q) {
    if (q >= 1) ok = mbar_wait(bar_done, (q - 1) & 1, a.err) && ok;    // stage free again
    if (tid == 0) {
      // image chunk: [hi: nrows_img rows][lo: nrows_img rows] -> Dhi, Dlo contiguous
      bulk_copy(smem_u32(Dhi), Dimg + q * chunk_bytes, (X3 ? 2 : 1) * nrows_img * 128, bar_full);
    }
#pragma unroll
    for (int t = 0; t < kItems; ++t) {
      const int it = tid + t * kThreads;
      const int c = it % kNC, grp = it / kNC;
      const float sc = -__ldg(scale + (c % M));
      const int off = sw128_off(c, grp);
      if constexpr (BF) {
        uint4 hi, lo;
        split8_bf16(v[t], sc, hi, lo);
        *reinterpret_cast<uint4*>(Shi + off) = hi;
        if (X3) *reinterpret_cast<uint4*>(Slo + off) = lo;
      } else {
        float4 hi, lo;
        split4(make_float4(v[t][0], v[t][1], v[t][2], v[t][3]), sc, hi, lo);
        *reinterpret_cast<float4*>(Shi + off) = hi;
        if (X3) *reinterpret_cast<float4*>(Slo + off) = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (q + 1 < L.n_kc) load_chunk(q + 1);
    if (tid == 0) {
      ok = mbar_wait(bar_full, q & 1, a.err) && ok;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dSh = sw128_desc(smem_u32(Shi)), dSl = sw128_desc(smem_u32(Slo));
      if (XPASS) {
        for (int t = 0; t < L.n_mt; ++t) {
          const uint64_t dDh = sw128_desc(smem_u32(Dhi + t * kTileBytes));
          const uint64_t dDl = sw128_desc(smem_u32(Dlo + t * kTileBytes));
          const uint32_t acc_t = tmem + t * kNC;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);   // 32 bytes per K step
            mma<BF>(acc_t, dDh + o, dSh + o, idesc_x, (q > 0 || kk > 0) ? 1u : 0u);
            if (X3) {
              mma<BF>(acc_t, dDh + o, dSl + o, idesc_x, 1u);
              mma<BF>(acc_t, dDl + o, dSh + o, idesc_x, 1u);
            }
          }
        }
      } else {
        // N = output positions in halves of at most 256 (rows 256 h .. of D).
        for (int h = 0; 256 * h < nrows_img; ++h) {
          const int nh = min(256, nrows_img - 256 * h);
          const uint32_t idesc_y = idesc_base | (static_cast<uint32_t>(nh >> 3) << 17);
          const uint64_t dDh = sw128_desc(smem_u32(Dhi + h * 256 * 128));
          const uint64_t dDl = sw128_desc(smem_u32(Dlo + h * 256 * 128));
          const uint32_t acc_h = tmem + 256 * h;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);
            mma<BF>(acc_h, dSh + o, dDh + o, idesc_y, (q > 0 || kk > 0) ? 1u : 0u);
            if (X3) {
              mma<BF>(acc_h, dSh + o, dDl + o, idesc_y, 1u);
              mma<BF>(acc_h, dSl + o, dDh + o, idesc_y, 1u);
            }
          }
        }
      }
      mma_commit(bar_done);
    }
  }
  ok = mbar_wait(bar_done, (L.n_kc - 1) & 1, a.err) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // y-pass launched as a dependent of the x-pass: its main loop read only
  // u^k and D_y; the epilogue reads R and rewrites u, so it waits here for
  // the x-pass to have completed (no-op for an ordinary launch).
  if (!XPASS) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // an x-pass wait that ran out while this CTA's main loop ran: write nothing
    if (*static_cast<volatile int*>(a.err)) ok = false;
  }

  // ---------------- x-pass: scattering contraction into the same tiles ----------------
  if constexpr (XPASS && SCAT_TC) {
    // (t, r) pairs: 128 output positions of tile t on grid row j0 + r.  A =
    // b(r, i) u(r, i, q) (K = q padded to 32), B = P~ rows m; N = max(M, 16).
    // TF32 operands and M <= 32 only.
    const uint32_t idesc_s = (1u << 4) | (2u << 7) | (2u << 10) |
                             (static_cast<uint32_t>((M < 16 ? 16 : M) >> 3) << 17) |
                             (static_cast<uint32_t>(kMT >> 4) << 24);
    const int slot_bytes = (X3 ? 2 : 1) * kTileBytes;
    const int slots = min(4, L.stage_bytes / slot_bytes);
    const int pairs = L.n_mt * per_tile;
    if (tid == 0) ok = mbar_wait(bar_p, 0, a.err) && ok;
    const uint64_t dPh = sw128_desc(smem_u32(Psm)), dPl = sw128_desc(smem_u32(Psm + 32 * 128));
    int round = 0;
    for (int p0 = 0; p0 < pairs; p0 += slots, ++round) {
      const int np = min(slots, pairs - p0);
      // Stage np pairs; each is 128 rows x 8 groups of 4 ordinates.  All of
      // a thread's loads are issued before any is converted.
      constexpr int kMaxItems = 16;                        // slots <= 4 -> <= 16 items per thread
      float4 val[kMaxItems];
      float bv[kMaxItems];
#pragma unroll
      for (int h = 0; h < kMaxItems; ++h) {
        const int it = tid + h * kThreads;
        val[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        bv[h] = 0.f;
        if (it >= np * kMT * 8) continue;
        const int pp = it / (kMT * 8), rem = it - pp * (kMT * 8);
        const int row = rem >> 3, grp = rem & 7;
        const int p = p0 + pp, t = p / per_tile, r = p - t * per_tile;
        const int i = t * kMT + row, j = t0 + r, m0 = grp * 4;
        if (i < nx && j < ny && m0 < M) {
          const size_t cell = static_cast<size_t>(j) * nx + i;
          val[h] = *reinterpret_cast<const float4*>(U + goff + cell * M + m0);
          bv[h] = __ldg(a.mus + cell);
        }
      }
#pragma unroll
      for (int h = 0; h < kMaxItems; ++h) {
        const int it = tid + h * kThreads;
        if (it >= np * kMT * 8) continue;
        const int pp = it / (kMT * 8), rem = it - pp * (kMT * 8);
        const int row = rem >> 3, grp = rem & 7;
        float4 hi, lo;
        split4(val[h], bv[h], hi, lo);
        unsigned char* slot = sm + pp * slot_bytes;
        const int off = sw128_off(row, grp);
        *reinterpret_cast<float4*>(slot + off) = hi;
        if (X3) *reinterpret_cast<float4*>(slot + kTileBytes + off) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int pp = 0; pp < np; ++pp) {
          const int p = p0 + pp, t = p / per_tile, r = p - t * per_tile;
          if (t0 + r >= ny) continue;
          unsigned char* slot = sm + pp * slot_bytes;
          const uint64_t dAh = sw128_desc(smem_u32(slot)), dAl = sw128_desc(smem_u32(slot + kTileBytes));
          const uint32_t acc = tmem + t * kNC + r * M;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);
            mma<false>(acc, dAh + o, dPh + o, idesc_s, 1u);
            if (X3) {
              mma<false>(acc, dAh + o, dPl + o, idesc_s, 1u);
              mma<false>(acc, dAl + o, dPh + o, idesc_s, 1u);
            }
          }
        }
        mma_commit(bar_scat);
      }
      ok = mbar_wait(bar_scat, round & 1, a.err) && ok;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }

  // ---------------- epilogues ----------------
  const int quarter = warp & 3;
  if (XPASS) {
    // lane = output position i, columns = (row, m).  The (tile t, row rc)
    // pairs of the CTA, p = t * per_tile + rc, alternate between warps 0-3
    // and warps 4-7; warp w reads TMEM lanes 32 (w % 4) ...
    const int half = warp >> 2;
    const int n_pairs = L.n_mt * per_tile;
    const uint32_t tq = tmem + (static_cast<uint32_t>(32 * quarter) << 16);
    auto pair_cell = [&](int p, int& t, int& rc, int& i, int& j) {
      t = p / per_tile;
      rc = p - t * per_tile;
      i = t * kMT + 32 * quarter + lane;
      j = t0 + rc;
    };
    if constexpr (MM == 64) {
      // 64 ordinates: the node's u and the scattering sums in registers,
      // P~[k][0] from shared memory (one broadcast value per k).
      for (int p = half; p < n_pairs; p += 2) {
        int t, rc, i, j;
        pair_cell(p, t, rc, i, j);
        const bool valid = ok && i < nx && j < ny;
        const size_t cell = static_cast<size_t>(j) * nx + i;
        float uu[MM];
        float ab = 0.f, bb = 0.f;
#pragma unroll
        for (int k = 0; k < MM / 4; ++k) {
          float4 u4 = make_float4(0.f, 0.f, 0.f, 0.f);
          if (valid) u4 = reinterpret_cast<const float4*>(U + goff + cell * M)[k];
          uu[4 * k] = u4.x; uu[4 * k + 1] = u4.y; uu[4 * k + 2] = u4.z; uu[4 * k + 3] = u4.w;
        }
        if (valid) {
          bb = __ldg(a.mus + cell);
          ab = __ldg(a.mua + cell) + bb;
        }
        float sc[MM];
#pragma unroll
        for (int m = 0; m < MM; ++m) sc[m] = 0.f;
#pragma unroll
        for (int k = 0; k < MM; ++k) {
          const float pk = pcs[k];
#pragma unroll
          for (int m = 0; m < MM; ++m) sc[m] = fmaf(pk, uu[(m - k + MM) % MM], sc[m]);
        }
        float4* rp = reinterpret_cast<float4*>(R + goff + cell * M);
#pragma unroll
        for (int gq = 0; gq < MM / 16; ++gq) {
          float acc[16];
          tmem_ld16(tq + t * kNC + rc * M + 16 * gq, acc);
          if (valid) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int m = 16 * gq + 4 * e;
              rp[m / 4] = make_float4(fmaf(bb, sc[m], acc[4 * e] - ab * uu[m]),
                                      fmaf(bb, sc[m + 1], acc[4 * e + 1] - ab * uu[m + 1]),
                                      fmaf(bb, sc[m + 2], acc[4 * e + 2] - ab * uu[m + 2]),
                                      fmaf(bb, sc[m + 3], acc[4 * e + 3] - ab * uu[m + 3]));
            }
          }
        }
      }
    } else {
      // Per pair: the node's u (M floats) and a + b; with the tensor-core
      // scattering the next pair's values are loaded before this one is
      // finished, otherwise right after it.
      float4 ucur[MM / 4], unext[MM / 4];
#pragma unroll
      for (int k = 0; k < MM / 4; ++k) ucur[k] = unext[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      float abcur = 0.f, abnext = 0.f, bcur = 0.f;
      auto load_pair = [&](int p, float4* u4, float& ab, float& bv) {
        int t, rc, i, j;
        pair_cell(p, t, rc, i, j);
        if (!ok || p >= n_pairs || i >= nx || j >= ny) return;
        const size_t cell = static_cast<size_t>(j) * nx + i;
        bv = __ldg(a.mus + cell);
        ab = __ldg(a.mua + cell) + bv;
        const float4* up = reinterpret_cast<const float4*>(U + goff + cell * M);
#pragma unroll
        for (int k = 0; k < MM / 4; ++k) u4[k] = up[k];
      };
      load_pair(half, ucur, abcur, bcur);
      for (int p = half; p < n_pairs; p += 2) {
        int t, rc, i, j;
        pair_cell(p, t, rc, i, j);
        float bdummy = 0.f;
        if (SCAT_TC) load_pair(p + 2, unext, abnext, bdummy);
        float acc[MM];
        tmem_ld16(tq + t * kNC + rc * M, acc);
        if (MM > 16) tmem_ld16(tq + t * kNC + rc * M + 16, acc + 16);
        if (ok && i < nx && j < ny) {
          const size_t cell = static_cast<size_t>(j) * nx + i;
          float4* rp = reinterpret_cast<float4*>(R + goff + cell * M);
          if (SCAT_TC) {
#pragma unroll
            for (int k = 0; k < MM / 4; ++k)
              rp[k] = make_float4(acc[4 * k] - abcur * ucur[k].x, acc[4 * k + 1] - abcur * ucur[k].y,
                                  acc[4 * k + 2] - abcur * ucur[k].z, acc[4 * k + 3] - abcur * ucur[k].w);
          } else {
            float uu[MM];
#pragma unroll
            for (int k = 0; k < MM / 4; ++k) {
              uu[4 * k] = ucur[k].x; uu[4 * k + 1] = ucur[k].y; uu[4 * k + 2] = ucur[k].z; uu[4 * k + 3] = ucur[k].w;
            }
            xpass_node_rhs<MM>(acc, uu, pcs, abcur, bcur);
#pragma unroll
            for (int k = 0; k < MM / 4; ++k)
              st_hint(reinterpret_cast<float*>(rp + k), make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]),
                      pol_keep);   // R is read by the y-pass that follows
          }
        }
        if (SCAT_TC) {
#pragma unroll
          for (int k = 0; k < MM / 4; ++k) ucur[k] = unext[k];
          abcur = abnext;
        } else {
          load_pair(p + 2, ucur, abcur, bcur);
        }
      }
    }
  } else {
    // acc[lane = slab column c][column = output row j].  Per chunk of 16 grid
    // rows: every thread copies its own float4 items of u, R, L1, L2, L3 into
    // a shared double buffer with cp.async one chunk ahead (so a chunk's loads
    // overlap the previous chunk's work, and each thread reads back only what
    // it copied); warps 0-3 copy the accumulator to a shared [16][128] tile;
    // all threads form AB4 with float4 accesses; boundary nodes are finished
    // from the pre-BC values kept in shared memory.  Uses the stage and P~
    // regions, free after the main loop.
    constexpr int kEpiArr = 5;                                   // u, R, L1, L2, L3
    constexpr int kBufFloats = kEpiArr * 16 * kNC;               // 40 KB
    float* ebuf = reinterpret_cast<float*>(sm);                  // [2][5][16][128]
    float* acc_s = ebuf + 2 * kBufFloats;                        // [16][128]
    float* un_s = acc_s + 16 * kNC;                              // [16][128] pre-BC u^{k+1}
    float* bc_s = un_s + 16 * kNC;                               // [16][128] post-BC values
    const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * quarter) << 16);
    const bool tile_has_xface = (t0 == 0) || (t0 + per_tile > nx - 1);
    const int ring_len = 2 * ny + 2 * nx;
    const int wcols = min(per_tile, nx - t0);                    // valid grid columns of the tile
    const int nchunks = min(nrows_img / 16, (ny + 15) / 16);
    const float* srcs[kEpiArr] = {U, R, L1, L2, L3};
    // Boundary tables (faces 0..3, corners 4..7) staged once per CTA.
    float* bc_f = bc_s + 16 * kNC;                               // [8][M]
    float* bc_wexit = bc_f + 8 * kMaxM;                          // [4][M]
    int* bc_refl = reinterpret_cast<int*>(bc_wexit + 4 * kMaxM); // [8][M]
    unsigned char* bc_act = reinterpret_cast<unsigned char*>(bc_refl + 8 * kMaxM);   // [8][M]
    for (int e = tid; e < 8 * M; e += kThreads) {
      const int tb = e / M, m = e - tb * M;
      const bool face = tb < 4;
      const int k = (face ? tb : tb - 4) * M + m;
      bc_f[e] = face ? b.face_f[k] : b.corner_f[k];
      bc_refl[e] = face ? b.face_refl[k] : b.corner_refl[k];
      bc_act[e] = face ? b.face_act[k] : b.corner_act[k];
      if (face) bc_wexit[e] = b.wexit[k];
    }
    const uint64_t pol_once = policy_evict_first();
    auto issue_chunk = [&](int cc, int bsel) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int item = tid + h * kThreads;                   // 16 rows x 32 float4
        const int t = item >> 5, c = (item & 31) * 4;
        const int j = cc * 16 + t;
        if (c / M >= wcols || j >= ny) continue;
        const size_t gidx = goff + (static_cast<size_t>(j) * nx + t0) * M + c;
#pragma unroll
        for (int arr = 0; arr < kEpiArr; ++arr) {
          float* dst = ebuf + bsel * kBufFloats + (arr * 16 + t) * kNC + c;
          asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                       "l"(srcs[arr] + gidx), "l"(pol_once)
                       : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (ok) issue_chunk(0, 0);
    for (int ci = 0; ci < nchunks; ++ci) {
      const int j0c = ci * 16;
      const int bsel = ci & 1;
      if (ok && ci + 1 < nchunks) issue_chunk(ci + 1, bsel ^ 1);
      if (warp < 4) {
        float acc[16];
        tmem_ld16(tbase + j0c, acc);
        const int c = 32 * warp + lane;
#pragma unroll
        for (int t = 0; t < 16; ++t) acc_s[t * kNC + c] = acc[t];
      }
      if (ci + 1 < nchunks)
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      else
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
      // CTA-uniform (barriers below depend on it).
      const bool chunk_bnd = j0c == 0 || j0c + 16 > ny - 1 || tile_has_xface;
      const float* buf = ebuf + bsel * kBufFloats;
      const bool got = ok;
      if (got) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int item = tid + h * kThreads;               // this thread's own copies
          const int t = item >> 5, c = (item & 31) * 4;
          const int w = c / M, j = j0c + t, i = t0 + w;
          if (w >= wcols || j >= ny) continue;
          const float4 u4 = *reinterpret_cast<const float4*>(buf + (0 * 16 + t) * kNC + c);
          const float4 r4 = *reinterpret_cast<const float4*>(buf + (1 * 16 + t) * kNC + c);
          const float4 p4 = *reinterpret_cast<const float4*>(buf + (2 * 16 + t) * kNC + c);
          const float4 q4 = *reinterpret_cast<const float4*>(buf + (3 * 16 + t) * kNC + c);
          const float4 s4 = *reinterpret_cast<const float4*>(buf + (4 * 16 + t) * kNC + c);
          const float4 ac = *reinterpret_cast<const float4*>(acc_s + t * kNC + c);
          const size_t gidx = goff + (static_cast<size_t>(j) * nx + t0) * M + c;
          const bool bnd = i == 0 || i == nx - 1 || j == 0 || j == ny - 1;
          if (b.bct_src) {
            // ubar = w^{k+1} + L^T v; the boundary finish adds the readout
            // transpose and applies BC^T across the node's ordinates
            float ub[4] = {r4.x + ac.x + p4.x, r4.y + ac.y + p4.y, r4.z + ac.z + p4.z, r4.w + ac.w + p4.w};
            if (bnd) {
              const int m0 = c - w * M;
              const float* eb = b.ebar + (static_cast<size_t>(g) * b.ebar_len + src_step) * ring_len;
              if (i == 0 || i == nx - 1) {
                const float e = __ldg(eb + (i == 0 ? j : ny + j));
                const float* wx = bc_wexit + (i == 0 ? 0 : 1) * M + m0;
#pragma unroll
                for (int q = 0; q < 4; ++q) ub[q] = fmaf(wx[q], e, ub[q]);
              }
              if (j == 0 || j == ny - 1) {
                const float e = __ldg(eb + (j == 0 ? 2 * ny + i : 2 * ny + nx + i));
                const float* wy = bc_wexit + (j == 0 ? 2 : 3) * M + m0;
#pragma unroll
                for (int q = 0; q < 4; ++q) ub[q] = fmaf(wy[q], e, ub[q]);
              }
              *reinterpret_cast<float4*>(un_s + t * kNC + c) = make_float4(ub[0], ub[1], ub[2], ub[3]);
            } else {
              const float4 wn = make_float4(ub[0], ub[1], ub[2], ub[3]);
              float4 v;
              v.x = a.cdt * (kAB0 * wn.x + kAB1 * p4.x + kAB2 * q4.x + kAB3 * s4.x);
              v.y = a.cdt * (kAB0 * wn.y + kAB1 * p4.y + kAB2 * q4.y + kAB3 * s4.y);
              v.z = a.cdt * (kAB0 * wn.z + kAB1 * p4.z + kAB2 * q4.z + kAB3 * s4.z);
              v.w = a.cdt * (kAB0 * wn.w + kAB1 * p4.w + kAB2 * q4.w + kAB3 * s4.w);
              *reinterpret_cast<float4*>(L3 + gidx) = wn;
              st_hint(U + gidx, v, pol_keep);
            }
            continue;
          }
          float4 lk, un;
          lk.x = r4.x + ac.x; lk.y = r4.y + ac.y; lk.z = r4.z + ac.z; lk.w = r4.w + ac.w;
          un.x = ab4_node(a.cdt, lk.x, p4.x, q4.x, s4.x, u4.x);
          un.y = ab4_node(a.cdt, lk.y, p4.y, q4.y, s4.y, u4.y);
          un.z = ab4_node(a.cdt, lk.z, p4.z, q4.z, s4.z, u4.z);
          un.w = ab4_node(a.cdt, lk.w, p4.w, q4.w, s4.w, u4.w);
          *reinterpret_cast<float4*>(L3 + gidx) = lk;
          if (chunk_bnd) *reinterpret_cast<float4*>(un_s + t * kNC + c) = un;
          if (!bnd) st_hint(U + gidx, un, pol_keep);   // u^{k+1} is read by the next x-pass
        }
      }
      if (chunk_bnd) {
        // eq. (RTE) third line on the chunk's boundary nodes, from the pre-BC
        // values of the node (un_s); results in bc_s and in U.  Boundary
        // nodes of the chunk: the x-face column (tiles at i = 0 / nx-1) on
        // every row, and the y-face rows j = 0 / ny-1 on every column.
        __syncthreads();
        const int xcol = (t0 == 0) ? 0 : (t0 + wcols - 1 == nx - 1 ? wcols - 1 : -1);
        const int yrow0 = (j0c == 0) ? 0 : -1;
        const int yrow1 = (ny - 1 >= j0c && ny - 1 < j0c + 16) ? ny - 1 - j0c : -1;
        const int rows = min(16, ny - j0c);
        // cells: [x-face column on each row][y-face rows on each column]
        const int n_xcells = xcol >= 0 ? rows : 0;
        const int n_ycells = ((yrow0 >= 0) + (yrow1 >= 0 && yrow1 != yrow0)) * wcols;
        for (int e = tid; e < (n_xcells + n_ycells) * M; e += kThreads) {
          const int cidx = e / M, m = e - cidx * M;
          int t, w;
          if (cidx < n_xcells) {
            t = cidx;
            w = xcol;
          } else {
            const int yc = cidx - n_xcells;
            t = (yc / wcols == 0 && yrow0 >= 0) ? yrow0 : yrow1;
            w = yc % wcols;
            if (xcol >= 0 && w == xcol) continue;                // corner: done as x-face cell
          }
          const int j = j0c + t, i = t0 + w;
          if (!got) continue;
          const bool lf = i == 0, rt = i == nx - 1, bt = j == 0, tp = j == ny - 1;
          int tb;                                                // table: face 0..3 or corner 4..7
          if ((lf || rt) && (bt || tp)) tb = 4 + (rt ? 1 : 0) + (tp ? 2 : 0);
          else tb = lf ? 0 : rt ? 1 : bt ? 2 : 3;
          const float* pre = un_s + t * kNC + w * M;
          if (b.bct_src) {
            // transposed step: w^k = BC^T ubar, v = c dt sum_i chi_i w^{k+i}
            const int* src = b.bct_src + (tb * M + m) * 4;
            const float* cf = b.bct_f + (tb * M + m) * 4;
            float wv = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) wv = fmaf(__ldg(cf + q), pre[__ldg(src + q)], wv);
            const int col = w * M + m;
            const float w1 = buf[(2 * 16 + t) * kNC + col], w2 = buf[(3 * 16 + t) * kNC + col],
                        w3 = buf[(4 * 16 + t) * kNC + col];
            const size_t gi = goff + (static_cast<size_t>(j) * nx + i) * M + m;
            L3[gi] = wv;
            U[gi] = a.cdt * (kAB0 * wv + kAB1 * w1 + kAB2 * w2 + kAB3 * w3);
            continue;
          }
          float val = pre[m];
          if (bc_act[tb * M + m]) {
            const int node = lf ? j : rt ? ny + j : bt ? 2 * ny + i : 2 * ny + nx + i;
            float qv = 0.f;
            for (int k = 0; k < b.kmax; ++k) {
              const size_t gk = static_cast<size_t>(g) * b.kmax + k;
              qv = fmaf(__ldg(b.S + gk * ring_len + node) * __ldg(b.A + gk * M + m),
                        __ldg(b.T + gk * b.T_len + src_step), qv);
            }
            const float fco = bc_f[tb * M + m];
            if (b.rho)
              qv = fmaf(1.0f - fco, __ldg(b.rho + (static_cast<size_t>(g) * b.rho_len + src_step) * ring_len + node), qv);
            val = fmaf(fco, pre[bc_refl[tb * M + m]], qv);
          }
          bc_s[t * kNC + w * M + m] = val;
          U[goff + (static_cast<size_t>(j) * nx + i) * M + m] = val;
        }
        __syncthreads();
        // Exitance of eq. (OpMed): one thread per (boundary node, face), in a
        // fixed summation order.
        if (got && b.ring_out && ring_step >= 0) {
          float* ro = b.ring_out + (static_cast<size_t>(g) * b.ring_steps + ring_step) * ring_len;
          for (int e = tid; e < 16 * wcols * 2; e += kThreads) {
            const int t = e / (wcols * 2), rem = e - t * (wcols * 2), w = rem >> 1, fy = rem & 1;
            const int j = j0c + t, i = t0 + w;
            if (j >= ny) continue;
            const bool lf = i == 0, rt = i == nx - 1, bt = j == 0, tp = j == ny - 1;
            if (fy == 0 && !(lf || rt)) continue;
            if (fy == 1 && !(bt || tp)) continue;
            const int F = fy == 0 ? (lf ? 0 : 1) : (bt ? 2 : 3);
            const float* val = bc_s + t * kNC + w * M;
            float ex = 0.f;
            for (int m = 0; m < M; ++m) ex = fmaf(bc_wexit[F * M + m], val[m], ex);
            ro[fy == 0 ? (lf ? j : ny + j) : (bt ? 2 * ny + i : 2 * ny + nx + i)] = ex;
          }
        }
      }
      __syncthreads();   // acc_s / un_s / bc_s are reused by the next chunk
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L.tmem_cols));
}

template <bool XPASS, int PREC, int MM, bool SCAT_TC>
__global__ void __launch_bounds__(kThreads, MM == 64 ? 1 : 2)
    tc_pass_kernel(StepArgs a, BoundaryArgs b, float* __restrict__ U, float* __restrict__ R,
                   const float* __restrict__ L1, const float* __restrict__ L2, float* __restrict__ L3,
                   int src_step, int ring_step) {
  // The y-pass walks the groups last to first: it starts on the groups whose
  // R the x-pass wrote last (still in L2) and ends on the groups whose
  // u^{k+1} the next x-pass reads first.
  const int g = XPASS ? static_cast<int>(blockIdx.z) : static_cast<int>(gridDim.z - 1 - blockIdx.z);
  tc_pass_body<XPASS, PREC, MM, SCAT_TC>(a, b, U, R, L1, L2, L3, src_step, ring_step, blockIdx.x, g);
}

// Batched form: the CTAs of one launch cover the tiles of several media
// (problems sorted by first CTA index); each CTA copies its problem's
// descriptor to shared memory and runs the same body.  The history ring of
// every problem is at the same rotation hl (the problems step in lockstep).
template <bool XPASS, int PREC, int MM, bool SCAT_TC>
__global__ void __launch_bounds__(kThreads, MM == 64 ? 1 : 2)
    tc_pass_batched(const BatchProblem* __restrict__ probs, int n_probs, int step, int hl) {
  __shared__ BatchProblem sp;
  __shared__ int sp_tile, sp_g;
  if (threadIdx.x == 0) {
    const int bid = blockIdx.x;
    int p = 0;
    while (p + 1 < n_probs && bid >= (XPASS ? probs[p + 1].tile0_x : probs[p + 1].tile0_y)) ++p;
    sp = probs[p];
    const int local = bid - (XPASS ? sp.tile0_x : sp.tile0_y);
    const int tiles = XPASS ? sp.tiles_x : sp.tiles_y;
    sp_g = local / tiles;
    sp_tile = local - sp_g * tiles;
  }
  __syncthreads();
  const int h1 = hl, h2 = (hl + 1) % 3, h3 = (hl + 2) % 3;
  tc_pass_body<XPASS, PREC, MM, SCAT_TC>(sp.a, sp.b, sp.U, sp.R, sp.L[h1], sp.L[h2], sp.L[h3], step,
                                         sp.b.ring_out ? step : -1, sp_tile, sp_g);
}


template <bool XPASS, int PREC, int MM, bool SCAT_TC>
cudaError_t launch_one(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                       const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s, bool pdl) {
  using K = Kind<PREC>;
  const TcLayout L(XPASS ? a.nx : a.ny, K::X3, K::KC);
  // The y-pass epilogue reuses the stage and P~ regions for its buffers.
  const size_t body = static_cast<size_t>(L.stage_bytes) + kPBytes;
  size_t smem = 1024 + (XPASS ? body : (body > kEpiBytes ? body : kEpiBytes));
  // A CTA holding all 512 TMEM columns keeps the SM to itself, so that a
  // second resident CTA does not sit in tcgen05.alloc.
  if (L.tmem_cols == 512 && smem < 120 * 1024) smem = 120 * 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_pass_kernel<XPASS, PREC, MM, SCAT_TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         232448 - 2048);
    attr = true;
  }
  constexpr int per_tile = kNC / MM;
  const int lines = XPASS ? a.ny : a.nx;
  dim3 grid((lines + per_tile - 1) / per_tile, 1, a.G);
  if (!pdl) {
    tc_pass_kernel<XPASS, PREC, MM, SCAT_TC><<<grid, kThreads, smem, s>>>(a, b, U, R, L1, L2, L3, src_step,
                                                                          ring_step);
    return cudaGetLastError();
  }
  // programmatic dependent launch: may start while the preceding x-pass's
  // last CTAs run (see the wait before the y epilogue)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr_pdl[1];
  attr_pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr_pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr_pdl;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_pass_kernel<XPASS, PREC, MM, SCAT_TC>, a, b, U, R, L1, L2, L3, src_step,
                            ring_step);
}

template <bool XPASS, int PREC>
cudaError_t launch_pass(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                        const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s, bool pdl) {
  constexpr bool kScatOk = XPASS && !Kind<PREC>::BF;   // TC scattering: TF32 operands, M <= 32
  const bool st = kScatOk && a.tc_scatter != 0;
  if (a.M == 16)
    return st ? launch_one<XPASS, PREC, 16, kScatOk>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl)
              : launch_one<XPASS, PREC, 16, false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
  if (a.M == 32)
    return st ? launch_one<XPASS, PREC, 32, kScatOk>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl)
              : launch_one<XPASS, PREC, 32, false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
  return launch_one<XPASS, PREC, 64, false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
}

template <bool XPASS>
cudaError_t launch_mode(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                        const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s,
                        bool pdl = false) {
  switch (a.tc_mode) {
    case 1: return launch_pass<XPASS, 1>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
    case 2: return launch_pass<XPASS, 2>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
    case 3: return launch_pass<XPASS, 3>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
    default: return launch_pass<XPASS, 4>(a, b, U, R, L1, L2, L3, src_step, ring_step, s, pdl);
  }
}

template <bool XPASS, int PREC, int MM, bool SCAT_TC>
cudaError_t launch_batched_one(const BatchProblem* probs, const BatchProblem* dev, int n, int step, int hl,
                               cudaStream_t s) {
  using K = Kind<PREC>;
  size_t smem = 0;
  int ctas = 0;
  for (int p = 0; p < n; ++p) {
    const TcLayout L(XPASS ? probs[p].a.nx : probs[p].a.ny, K::X3, K::KC);
    const size_t body = static_cast<size_t>(L.stage_bytes) + kPBytes;
    const size_t need = 1024 + (XPASS ? body : (body > kEpiBytes ? body : kEpiBytes));
    if (need > smem) smem = need;
    ctas += (XPASS ? probs[p].tiles_x : probs[p].tiles_y) * probs[p].a.G;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_pass_batched<XPASS, PREC, MM, SCAT_TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         232448 - 2048);
    attr = true;
  }
  if (XPASS) {
    tc_pass_batched<XPASS, PREC, MM, SCAT_TC><<<ctas, kThreads, smem, s>>>(dev, n, step, hl);
    return cudaGetLastError();
  }
  // the y-pass as a programmatic dependent of the batched x-pass before it
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr_pdl[1];
  attr_pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr_pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr_pdl;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_pass_batched<XPASS, PREC, MM, SCAT_TC>, dev, n, step, hl);
}

template <bool XPASS, int PREC>
cudaError_t launch_batched_pass(const BatchProblem* probs, const BatchProblem* dev, int n, int step, int hl,
                                cudaStream_t s) {
  constexpr bool kScatOk = XPASS && !Kind<PREC>::BF;
  const bool st = kScatOk && probs[0].a.tc_scatter != 0;
  const int M = probs[0].a.M;
  if (M == 16)
    return st ? launch_batched_one<XPASS, PREC, 16, kScatOk>(probs, dev, n, step, hl, s)
              : launch_batched_one<XPASS, PREC, 16, false>(probs, dev, n, step, hl, s);
  if (M == 32)
    return st ? launch_batched_one<XPASS, PREC, 32, kScatOk>(probs, dev, n, step, hl, s)
              : launch_batched_one<XPASS, PREC, 32, false>(probs, dev, n, step, hl, s);
  return launch_batched_one<XPASS, PREC, 64, false>(probs, dev, n, step, hl, s);
}

template <bool XPASS>
cudaError_t launch_batched_mode(const BatchProblem* probs, const BatchProblem* dev, int n, int step, int hl,
                                cudaStream_t s) {
  switch (probs[0].a.tc_mode) {
    case 1: return launch_batched_pass<XPASS, 1>(probs, dev, n, step, hl, s);
    case 2: return launch_batched_pass<XPASS, 2>(probs, dev, n, step, hl, s);
    case 3: return launch_batched_pass<XPASS, 3>(probs, dev, n, step, hl, s);
    default: return launch_batched_pass<XPASS, 4>(probs, dev, n, step, hl, s);
  }
}

}  // namespace

void tc_batch_layout(BatchProblem* probs, int n, int* ctas_x, int* ctas_y) {
  int cx = 0, cy = 0;
  for (int p = 0; p < n; ++p) {
    const int per_tile = kNC / probs[p].a.M;
    probs[p].tiles_x = (probs[p].a.ny + per_tile - 1) / per_tile;
    probs[p].tiles_y = (probs[p].a.nx + per_tile - 1) / per_tile;
    probs[p].tile0_x = cx;
    probs[p].tile0_y = cy;
    cx += probs[p].tiles_x * probs[p].a.G;
    cy += probs[p].tiles_y * probs[p].a.G;
  }
  *ctas_x = cx;
  *ctas_y = cy;
}

cudaError_t launch_step_tc_batched(const BatchProblem* probs, const BatchProblem* probs_dev, int n, int step,
                                   int hl, cudaStream_t s, long long* launches) {
  cudaError_t e = launch_batched_mode<true>(probs, probs_dev, n, step, hl, s);
  if (e != cudaSuccess) return e;
  e = launch_batched_mode<false>(probs, probs_dev, n, step, hl, s);
  if (launches) *launches += 2;
  return e;
}

bool tc_supported(int nx, int ny, int M, int precision, int flags) {
  if (nx < 16 || ny < 16 || nx > 512 || ny > 512) return false;
  if (M != 16 && M != 32 && M != 64) return false;
  if (precision < 1 || precision > 4) return false;
  // The tensor-core scattering contraction exists for TF32 operands and M <= 32.
  if ((flags & 1) && (precision > 2 || M > 32)) return false;
  return true;
}

cudaError_t launch_step_tc(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                           const float* L2, float* L3, int step, cudaStream_t s, long long* launches,
                           cudaEvent_t* ev) {
  const int ring_step = b.ring_out ? step : -1;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  // the transposed step exists in the one-tile-per-CTA passes only
  const bool ws = a.x_variant == 0 && tc_ws_supported(a) && !b.bct_src;
  const bool pipe = a.x_variant == 2 && tc_pipe_supported(a) && !b.bct_src;
  // the TMA-fed passes (the same arithmetic as the one-tile passes; the
  // transposed step uses the one-tile passes throughout)
  const bool tma = (a.x_variant == 4 || a.x_variant == 5) && !b.bct_src && !a.test_expire;
  const bool stream = tma && tc_stream_supported(a);
  const bool ystream = tma && a.x_variant == 5 && tc_ystream_supported(a);
  e = ws       ? launch_pass_ws(true, a, b, U, R, L1, L2, L3, step, ring_step, s)
      : stream ? launch_xpass_stream(a, b, U, R, s)
               : launch_mode<true>(a, b, U, R, L1, L2, L3, step, ring_step, s);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  e = ws        ? launch_pass_ws(false, a, b, U, R, L1, L2, L3, step, ring_step, s)
      : pipe    ? launch_ypass_pipe(a, b, U, R, L1, L2, L3, step, ring_step, s)
      : ystream ? launch_ypass_stream(a, b, U, R, L1, L2, L3, step, ring_step, s)
                : launch_mode<false>(a, b, U, R, L1, L2, L3, step, ring_step, s, !ev);
  if (ev) cudaEventRecord(ev[2], s);
  if (launches) *launches += 2;
  return e;
}

}  // namespace rte_kern
