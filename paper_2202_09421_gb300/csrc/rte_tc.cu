// Tensor-core (tcgen05) form of the two FC-DOM passes for sm_103a.
//
// Each CTA owns one slab tile: 128 slab columns c (x-pass: grid rows j0 ..
// j0 + 128/M - 1 times the M ordinates; y-pass: grid columns i0 .. times M)
// over a whole line of n <= 256 positions, K = input positions.
//   x-pass: per 128-position tile t of the line, the dense FC operator D
//     (n x n, Sec. 4.3) is the A operand (M = 128 output positions) and the
//     transposed slab the B operand (N = 128 slab columns): tensor memory
//     holds acc_t[lane = output position i][column = (row, m)], so the
//     epilogue's lanes walk the contiguous x direction of the grid.
//   y-pass: the slab is the A operand (M = 128 slab columns) and D the B
//     operand (N = output positions): acc[lane = (column, m)][column = j], so
//     the epilogue's lanes walk the contiguous (column, m) run of a grid row.
//
// x-pass: the node-local scattering sum b P~ u (Sec. 4.1) is accumulated into
// the same tensor-memory tile as a second contraction: for each grid row r of
// the tile, A = b(r, i) u(r, i, q) (rows i, K = ordinates q) and B = P~ (rows
// m, K = q); the -xi_m factor of the streaming term is folded into the slab
// operand.  The epilogue adds -(a + b) u:  R = b P~u - (a+b) u - xi_m D_x u.
// y-pass: acc = -eta_m D_y u; the epilogue forms L = R + acc, the AB4 update
// (eq. RTEAB4), the Fresnel boundary condition with beam or adjoint
// injection (eq. RTE), the exitance ring (eq. OpMed), and updates u in place.
//
// Precision: kind::tf32 with split operands.  Every operand x is split as
// hi = tf32(x), lo = tf32(x - hi) (D and P~ on the host, the slab and the
// scattering operand while staged) and the products hi*hi + hi*lo + lo*hi
// are accumulated in FP32 (3xTF32, about 2^-22 relative per product); the
// single-product form (1xTF32) is the reduced-precision variant.
//
// Operands use the K-major 128-byte-swizzle layout (rows of 32 tf32 values;
// 8-row atoms of 1024 B).  D and P~ chunks are pre-swizzled in global memory
// and copied with cp.async.bulk; the slab is converted and swizzled by all
// threads.  K runs in chunks of 32 through a two-stage ring, so chunk q+1 is
// staged while the tensor core works on chunk q.  One thread issues the MMAs
// and commits them to mbarriers; every wait is bounded and sets g_tc_error
// instead of spinning forever.
#include <cstdint>

#include "rte_kernels.cuh"

namespace rte_kern {

__device__ int g_tc_error;

namespace {

constexpr int kNC = 128;          // slab columns per tile (MMA N)
constexpr int kMT = 128;          // output positions per accumulator tile (MMA M)
constexpr int kKC = 32;           // K per chunk: one 128-byte row of tf32
constexpr int kThreads = 256;
constexpr int kTileBytes = 128 * 128;   // one 128-row x 128-byte operand tile
constexpr long kWaitLimit = 1L << 26;
constexpr float kAB0 = 55.0f / 24.0f, kAB1 = -59.0f / 24.0f, kAB2 = 37.0f / 24.0f,
                kAB3 = -9.0f / 24.0f;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row group
// stride 1024 B (start address in 16-byte units).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFF) | (static_cast<uint64_t>(1024 >> 4) << 32) |
         (static_cast<uint64_t>(1) << 46) | (static_cast<uint64_t>(2) << 61);
}

// Byte offset of the 16-byte group grp (4 tf32 values) of row `row` in a
// K-major 128-byte-swizzle tile.
__device__ __forceinline__ int sw128_off(int row, int grp) { return row * 128 + ((grp ^ (row & 7)) << 4); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false (and the error flag set) when the limit runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try(bar, parity)) return true;
  atomicExch(&g_tc_error, 1);
  return false;
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[t]);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split4(float4 v, float s, float4& hi, float4& lo) {
  hi.x = tf32_rna(s * v.x); lo.x = tf32_rna(s * v.x - hi.x);
  hi.y = tf32_rna(s * v.y); lo.y = tf32_rna(s * v.y - hi.y);
  hi.z = tf32_rna(s * v.z); lo.z = tf32_rna(s * v.z - hi.z);
  hi.w = tf32_rna(s * v.w); lo.w = tf32_rna(s * v.w - hi.w);
}

struct TcLayout {
  int n, n_mt, n_kc, stage_bytes, tmem_cols;
  __host__ __device__ TcLayout(int n_, bool x3) : n(n_) {
    n_mt = (n + kMT - 1) / kMT;
    n_kc = (n + kKC - 1) / kKC;
    stage_bytes = (x3 ? 2 : 1) * (n_mt + 1) * kTileBytes;   // D tiles + slab tile, hi (+ lo)
    tmem_cols = n_mt == 1 ? 128 : 256;
  }
};

constexpr int kPBytes = 2 * 32 * 128;   // P~ operand image: hi and lo, 32 rows x 128 B
// y-pass epilogue: two 5-array buffers, three [16][128] tiles, boundary tables
constexpr size_t kEpiBytes = (2 * 5 * 16 + 3 * 16) * 128 * 4 + (8 + 4 + 8) * 32 * 4 + 8 * 32;

template <bool XPASS, bool X3, int NSTAGE, int MM, bool SCAT_TC>
__global__ void __launch_bounds__(kThreads, NSTAGE == 1 ? 2 : 1)
    tc_pass_kernel(StepArgs a, BoundaryArgs b, float* __restrict__ U, float* __restrict__ R,
                   const float* __restrict__ L1, const float* __restrict__ L2, float* __restrict__ L3,
                   int src_step, int ring_step) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bars[6];   // full[2], done[2], p_full, scat_done
  __shared__ uint32_t tmem_slot;
  const int nx = a.nx, ny = a.ny;
  constexpr int M = MM;
  const int n = XPASS ? nx : ny;
  const TcLayout L(n, X3);
  const int per_tile = kNC / M;               // grid rows (x) or columns (y) per tile
  const int g = blockIdx.z;
  const int t0 = blockIdx.x * per_tile;       // first grid row (x) / column (y) of the tile
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t goff = static_cast<size_t>(g) * a.plane;
  const float* Dimg = XPASS ? a.DxImg : a.DyImg;
  const float* scale = XPASS ? a.xi : a.eta;
  const int n_lines = XPASS ? ny : nx;        // rows (x) / columns (y) of the grid

  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  unsigned char* Psm = sm + NSTAGE * L.stage_bytes;     // P~ image (x-pass)
  const uint32_t bar_full0 = smem_u32(&bars[0]), bar_done0 = smem_u32(&bars[2]);
  const uint32_t bar_p = smem_u32(&bars[4]), bar_scat = smem_u32(&bars[5]);

  if (tid == 0) {
    for (int k = 0; k < 6; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(L.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (XPASS && tid == 0) bulk_copy(smem_u32(Psm), a.PImg, kPBytes, bar_p);

  const int nrows_img = L.n_mt * kMT;                   // rows of the operator image
  // idesc: D = F32, A = B = TF32, K-major, M = 128; N = 128 slab columns
  // (x-pass) or all output positions (y-pass).
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                         (static_cast<uint32_t>((XPASS ? kNC : nrows_img) >> 3) << 17) |
                         (static_cast<uint32_t>(kMT >> 4) << 24);
  const size_t chunk_floats = static_cast<size_t>(2) * nrows_img * kKC;
  bool ok = true;

  // ---------------- main loop over K chunks ----------------
  // Slab^T chunk: S[c][kk] = -scale_m u(c, k0 + kk).  Each thread owns 4
  // (column, 4-value group) items; the next chunk's 16 loads are issued
  // before this chunk's MMAs so that their latency overlaps the tensor core.
  constexpr int kItems = kNC * (kKC / 4) / kThreads;   // 4
  float v[kItems][4];
  auto load_chunk = [&](int q) {
    const int k0 = q * kKC;
#pragma unroll
    for (int t = 0; t < kItems; ++t) {
      const int it = tid + t * kThreads;
      const int c = it % kNC, grp = it / kNC;
      const int rc = c / M, m = c - rc * M;
      const int line = t0 + rc;
      const bool valid = rc < per_tile && line < n_lines;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = k0 + grp * 4 + e;
        v[t][e] = 0.f;
        if (valid && k < n) {
          const size_t idx = XPASS ? goff + (static_cast<size_t>(line) * nx + k) * M + m
                                   : goff + (static_cast<size_t>(k) * nx + line) * M + m;
          v[t][e] = U[idx];
        }
      }
    }
  };
  load_chunk(0);
  for (int q = 0; q < L.n_kc; ++q) {
    const int s = q % NSTAGE;
    unsigned char* stage = sm + s * L.stage_bytes;
    unsigned char* Dhi = stage;                                   // n_mt tiles
    unsigned char* Dlo = stage + L.n_mt * kTileBytes;             // (3xTF32)
    unsigned char* Shi = stage + (X3 ? 2 : 1) * L.n_mt * kTileBytes;
    unsigned char* Slo = Shi + kTileBytes;
    if (q >= NSTAGE) ok = mbar_wait(bar_done0 + 8 * s, ((q - NSTAGE) / NSTAGE) & 1) && ok;
    if (tid == 0) {
      // image chunk: [hi: nrows_img x 32][lo: nrows_img x 32] -> Dhi, Dlo contiguous
      bulk_copy(smem_u32(Dhi), Dimg + q * chunk_floats, (X3 ? 2 : 1) * nrows_img * 128, bar_full0 + 8 * s);
    }
#pragma unroll
    for (int t = 0; t < kItems; ++t) {
      const int it = tid + t * kThreads;
      const int c = it % kNC, grp = it / kNC;
      float4 hi, lo;
      split4(make_float4(v[t][0], v[t][1], v[t][2], v[t][3]), -__ldg(scale + (c % M)), hi, lo);
      const int off = sw128_off(c, grp);
      *reinterpret_cast<float4*>(Shi + off) = hi;
      if (X3) *reinterpret_cast<float4*>(Slo + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (q + 1 < L.n_kc) load_chunk(q + 1);
    if (tid == 0) {
      ok = mbar_wait(bar_full0 + 8 * s, (q / NSTAGE) & 1) && ok;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dSh = sw128_desc(smem_u32(Shi)), dSl = sw128_desc(smem_u32(Slo));
      if (XPASS) {
        for (int t = 0; t < L.n_mt; ++t) {
          const uint64_t dDh = sw128_desc(smem_u32(Dhi + t * kTileBytes));
          const uint64_t dDl = sw128_desc(smem_u32(Dlo + t * kTileBytes));
          const uint32_t acc_t = tmem + t * kNC;
#pragma unroll
          for (int kk = 0; kk < kKC / 8; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);   // 32 bytes per K step
            mma_tf32(acc_t, dDh + o, dSh + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
            if (X3) {
              mma_tf32(acc_t, dDh + o, dSl + o, idesc, 1u);
              mma_tf32(acc_t, dDl + o, dSh + o, idesc, 1u);
            }
          }
        }
      } else {
        const uint64_t dDh = sw128_desc(smem_u32(Dhi)), dDl = sw128_desc(smem_u32(Dlo));
#pragma unroll
        for (int kk = 0; kk < kKC / 8; ++kk) {
          const uint64_t o = static_cast<uint64_t>(kk * 2);
          mma_tf32(tmem, dSh + o, dDh + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
          if (X3) {
            mma_tf32(tmem, dSh + o, dDl + o, idesc, 1u);
            mma_tf32(tmem, dSl + o, dDh + o, idesc, 1u);
          }
        }
      }
      mma_commit(bar_done0 + 8 * s);
    }
  }
  ok = mbar_wait(bar_done0 + 8 * ((L.n_kc - 1) % NSTAGE), ((L.n_kc - 1) / NSTAGE) & 1) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // ---------------- x-pass: scattering contraction into the same tiles ----------------
  if (XPASS && SCAT_TC) {
    // (t, r) pairs: 128 output positions of tile t on grid row j0 + r.  A =
    // b(r, i) u(r, i, q) (K = q padded to 32), B = P~ rows m; N = max(M, 16).
    const uint32_t idesc_s = (1u << 4) | (2u << 7) | (2u << 10) |
                             (static_cast<uint32_t>((M < 16 ? 16 : M) >> 3) << 17) |
                             (static_cast<uint32_t>(kMT >> 4) << 24);
    const int slot_bytes = (X3 ? 2 : 1) * kTileBytes;
    const int slots = min(4, (NSTAGE * L.stage_bytes) / slot_bytes);
    const int pairs = L.n_mt * per_tile;
    if (tid == 0) ok = mbar_wait(bar_p, 0) && ok;
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
          for (int kk = 0; kk < kKC / 8; ++kk) {
            const uint64_t o = static_cast<uint64_t>(kk * 2);
            mma_tf32(acc, dAh + o, dPh + o, idesc_s, 1u);
            if (X3) {
              mma_tf32(acc, dAh + o, dPl + o, idesc_s, 1u);
              mma_tf32(acc, dAl + o, dPh + o, idesc_s, 1u);
            }
          }
        }
        mma_commit(bar_scat);
      }
      ok = mbar_wait(bar_scat, round & 1) && ok;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }

  // ---------------- epilogues ----------------
  const int quarter = warp & 3;
  if (XPASS) {
    // lane = output position i, columns = (row, m).  Warps 0-3 take tile 0
    // and warps 4-7 tile 1; with one tile they split the slab's rows.
    const int t = L.n_mt == 2 ? (warp >> 2) : 0;
    const int line_first = L.n_mt == 2 ? 0 : (warp >> 2);
    const int line_step = L.n_mt == 2 ? 1 : 2;
    const int i = t * kMT + 32 * quarter + lane;
    const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + t * kNC;
    // Per grid row of the slab: the next row's u (M floats of the node) and
    // a + b are loaded while this row is finished.
    float4 ucur[8], unext[8];
    float abcur = 0.f, abnext = 0.f;
    auto load_row = [&](int rc, float4* u4, float& ab) {
      const int j = t0 + rc;
      if (!ok || rc >= per_tile || i >= nx || j >= ny) return;
      const size_t cell = static_cast<size_t>(j) * nx + i;
      ab = __ldg(a.mua + cell) + __ldg(a.mus + cell);
      const float4* up = reinterpret_cast<const float4*>(U + goff + cell * M);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (4 * k < M) u4[k] = up[k];
    };
    // Scattering weights p_k = P~[k][0]; P~[m][q] = p_{(m - q) mod M}
    // (symmetric circulant), used by the FP32 form of the scattering sum.
    float pc[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) pc[k] = SCAT_TC ? 0.f : __ldg(a.PT + k);
    float bcur = 0.f;
    auto load_b = [&](int rc) {
      const int j = t0 + rc;
      return (ok && rc < per_tile && i < nx && j < ny) ? __ldg(a.mus + static_cast<size_t>(j) * nx + i) : 0.f;
    };
    load_row(line_first, ucur, abcur);
    if (!SCAT_TC) bcur = load_b(line_first);
    for (int rc = line_first; rc < per_tile; rc += line_step) {
      const int j = t0 + rc;
      float bnext = 0.f;
      if (SCAT_TC) {
        load_row(rc + line_step, unext, abnext);
      }
      float acc[MM];
      tmem_ld16(tbase + rc * M, acc);
      if (MM > 16) tmem_ld16(tbase + rc * M + 16, acc + 16);
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
#pragma unroll
          for (int m = 0; m < MM; ++m) {
            float sc = 0.f;
#pragma unroll
            for (int q = 0; q < MM; ++q) sc = fmaf(pc[(m - q + MM) % MM], uu[q], sc);
            acc[m] = fmaf(bcur, sc, acc[m] - abcur * uu[m]);
          }
#pragma unroll
          for (int k = 0; k < MM / 4; ++k) rp[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
        }
      }
      if (SCAT_TC) {
#pragma unroll
        for (int k = 0; k < 8; ++k) ucur[k] = unext[k];
        abcur = abnext;
      } else if (rc + line_step < per_tile) {
        load_row(rc + line_step, ucur, abcur);
        bnext = load_b(rc + line_step);
        bcur = bnext;
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
    // regions (104 KB), free after the main loop.
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
    float* bc_wexit = bc_f + 8 * 32;                             // [4][M]
    int* bc_refl = reinterpret_cast<int*>(bc_wexit + 4 * 32);    // [8][M]
    unsigned char* bc_act = reinterpret_cast<unsigned char*>(bc_refl + 8 * 32);   // [8][M]
    for (int e = tid; e < 8 * M; e += kThreads) {
      const int tb = e / M, m = e - tb * M;
      const bool face = tb < 4;
      const int k = (face ? tb : tb - 4) * M + m;
      bc_f[e] = face ? b.face_f[k] : b.corner_f[k];
      bc_refl[e] = face ? b.face_refl[k] : b.corner_refl[k];
      bc_act[e] = face ? b.face_act[k] : b.corner_act[k];
      if (face) bc_wexit[e] = b.wexit[k];
    }
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
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(srcs[arr] + gidx)
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
          float4 lk, un;
          lk.x = r4.x + ac.x; lk.y = r4.y + ac.y; lk.z = r4.z + ac.z; lk.w = r4.w + ac.w;
          un.x = fmaf(a.cdt, kAB0 * lk.x + kAB1 * p4.x + kAB2 * q4.x + kAB3 * s4.x, u4.x);
          un.y = fmaf(a.cdt, kAB0 * lk.y + kAB1 * p4.y + kAB2 * q4.y + kAB3 * s4.y, u4.y);
          un.z = fmaf(a.cdt, kAB0 * lk.z + kAB1 * p4.z + kAB2 * q4.z + kAB3 * s4.z, u4.z);
          un.w = fmaf(a.cdt, kAB0 * lk.w + kAB1 * p4.w + kAB2 * q4.w + kAB3 * s4.w, u4.w);
          const size_t gidx = goff + (static_cast<size_t>(j) * nx + t0) * M + c;
          *reinterpret_cast<float4*>(L3 + gidx) = lk;
          const bool bnd = i == 0 || i == nx - 1 || j == 0 || j == ny - 1;
          if (chunk_bnd) *reinterpret_cast<float4*>(un_s + t * kNC + c) = un;
          if (!bnd) *reinterpret_cast<float4*>(U + gidx) = un;
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

template <bool XPASS, bool X3, int MM, bool SCAT_TC>
cudaError_t launch_one(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                       const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  constexpr int NSTAGE = 1;
  const TcLayout L(XPASS ? a.nx : a.ny, X3);
  // The y-pass epilogue reuses the stage and P~ regions for its buffers.
  const size_t body = NSTAGE * static_cast<size_t>(L.stage_bytes) + kPBytes;
  const size_t smem = 1024 + (XPASS ? body : (body > kEpiBytes ? body : kEpiBytes));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc_pass_kernel<XPASS, X3, NSTAGE, MM, SCAT_TC>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 232448 - 2048);
    attr = true;
  }
  const int per_tile = kNC / a.M;
  const int lines = XPASS ? a.ny : a.nx;
  dim3 grid((lines + per_tile - 1) / per_tile, 1, a.G);
  tc_pass_kernel<XPASS, X3, NSTAGE, MM, SCAT_TC><<<grid, kThreads, smem, s>>>(a, b, U, R, L1, L2, L3, src_step,
                                                                              ring_step);
  return cudaGetLastError();
}

template <bool XPASS, bool X3>
cudaError_t launch_pass(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                        const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  const bool st = XPASS && a.tc_scatter != 0;
  if (a.M == 16)
    return st ? launch_one<XPASS, X3, 16, true>(a, b, U, R, L1, L2, L3, src_step, ring_step, s)
              : launch_one<XPASS, X3, 16, false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
  return st ? launch_one<XPASS, X3, 32, true>(a, b, U, R, L1, L2, L3, src_step, ring_step, s)
            : launch_one<XPASS, X3, 32, false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
}

}  // namespace

bool tc_supported(int nx, int ny, int M) {
  return nx >= 16 && ny >= 16 && nx <= 256 && ny <= 256 && (M == 16 || M == 32);
}

cudaError_t launch_step_tc(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                           const float* L2, float* L3, int step, cudaStream_t s, long long* launches,
                           cudaEvent_t* ev) {
  const int ring_step = b.ring_out ? step : -1;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  e = a.tc_mode == 2 ? launch_pass<true, false>(a, b, U, R, L1, L2, L3, step, ring_step, s)
                     : launch_pass<true, true>(a, b, U, R, L1, L2, L3, step, ring_step, s);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  e = a.tc_mode == 2 ? launch_pass<false, false>(a, b, U, R, L1, L2, L3, step, ring_step, s)
                     : launch_pass<false, true>(a, b, U, R, L1, L2, L3, step, ring_step, s);
  if (ev) cudaEventRecord(ev[2], s);
  if (launches) *launches += 2;
  return e;
}

cudaError_t tc_take_error(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc_error, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
}

}  // namespace rte_kern
