// Persistent, TMA-fed tcgen05 passes for sm_103a (lines of n <= 256
// positions, M in {16, 32}, TF32 operand kinds: 3xTF32 and TF32).
//
// Same arithmetic as the passes of rte_tc.cu.  x-pass: for a slab tile of
// 128 columns (grid rows j0 .. j0 + 128/M - 1 times the M ordinates) over a
// whole grid row, acc[i][c] = sum_k D_x[i][k] (-xi_m u(c, k)) on the tensor
// cores (the dense FC operator of Sec. 4.3), and R = b P~u - (a + b) u + acc
// in the epilogue (Sec. 4.1, eq. RTEAB4L).  y-pass: for a slab tile of 128
// columns (grid columns i0 .. i0 + 128/M - 1 times the M ordinates) over a
// whole grid column, acc[c][j] = sum_k (-eta_m u(c, k)) D_y[j][k], and the
// epilogue forms L^k = R + acc, the AB4 update (eq. RTEAB4), the boundary
// condition with the beam sources (eq. RTE, third line) and the exitance
// (eq. OpMed).  One CTA per SM walks its share of the tiles; its roles run
// on separate warps and hand work over through mbarriers:
//   warp 12, one lane   the copy engine.  Per K chunk (32 positions) it
//                       issues a tensor copy (cp.async.bulk.tensor over a 4D
//                       map of the state [group][row][position][ordinate])
//                       of the raw FP32 slab chunk, 128 slab columns x 32
//                       positions, into a ring of raw buffers, and a bulk
//                       copy of the split operator chunk (D hi, D lo) into a
//                       ring of operand stages;
//   warps 8-11          convert each raw chunk: scale by -xi_m (-eta_m),
//                       split into TF32 hi + lo and write the K-major
//                       128-byte-swizzle operand of the same stage (each
//                       thread keeps one slab column, so its scale is fixed);
//   warp 13, one lane   issues the MMAs of each chunk into one of two
//                       tensor-memory accumulators; the commit frees the
//                       stage, the tile's last one hands the accumulator to
//                       the epilogue;
//   warps 0-7           drain the previous tile's accumulator.  x: the FP32
//                       circulant scattering sum, absorption, R to memory.
//                       y: lane = slab column, so a node's M ordinates sit
//                       in adjacent lanes of one warp and the reflection of
//                       the boundary condition and the exitance sum are warp
//                       shuffles; every node value of u, R and the history
//                       is one coalesced load per warp, straight from memory.
// The slab never passes through registers on its way to the tensor cores,
// and the operator copy, the conversion, the MMAs and the epilogue of
// consecutive chunks and tiles overlap.  Both passes compute what the
// one-tile-per-CTA passes compute, bit for bit: the same products in the same
// order, and the same epilogue arithmetic (ab4_node, xpass_node_rhs).
// Every wait is bounded: on expiry the kernel raises the context's timeout
// word and an abort flag that ends every other role's waits; the copy engine
// waits for its copies in flight and the MMA lane for its MMAs before the
// tensor memory is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "rte_tc_common.cuh"

namespace rte_kern {

namespace {

using namespace tc;

constexpr int kEpiWarps = 8, kCvtWarps = 4;
constexpr int kWarpCopy = kEpiWarps + kCvtWarps, kWarpMMA = kWarpCopy + 1;
constexpr int kStThreads = (kWarpMMA + 1) * 32;
constexpr int kCvtThreads = kCvtWarps * 32;
constexpr int kMaxStages = 4, kRawStages = 2;
constexpr int kSmemLimit = 232448 - 2048;
constexpr int kChunkK = 32;                                   // K positions per chunk (TF32)
constexpr int kRawBytes = kNC * kChunkK * 4;                  // raw FP32 chunk: 16 KB

__device__ __forceinline__ bool st_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, 1);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// Bounded wait without the abort check: the drains before the CTA leaves.
__device__ __forceinline__ bool st_wait_plain(uint32_t bar, uint32_t parity, int* err) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Tensor copy of one box of a 4D map into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__host__ __device__ inline int stream_stages(int stage_bytes) {
  const int s = (kSmemLimit - 1024 - kRawStages * kRawBytes) / stage_bytes;
  return s > kMaxStages ? kMaxStages : s;
}

// The y epilogue's rows per accumulator load: all loads of a chunk are
// issued before any is used.
constexpr int kRowsY = 16;

// 14 warps, one CTA per SM.  The register file is split over the four SM
// sub-partitions, so with four warps on two of them a thread gets at most
// 128 registers.
template <bool XPASS, int PREC, int MM>
__global__ void __launch_bounds__(kStThreads, 1)
    tc_pass_stream(StepArgs a, BoundaryArgs b, const __grid_constant__ CUtensorMap umap, float* __restrict__ U,
                   float* __restrict__ R, const float* __restrict__ L1, const float* __restrict__ L2,
                   float* __restrict__ L3, int src_step, int ring_step) {
  using K = Kind<PREC>;
  static_assert(!K::BF && K::KC == kChunkK, "TF32 operand kinds only");
  constexpr bool X3 = K::X3;
  constexpr int M = MM;
  constexpr int per_tile = kNC / M;                 // grid rows (x) / columns (y) per tile
  extern __shared__ __align__(1024) unsigned char smraw[];
  // full_d[s], full_s[s], empty[s] (s < kMaxStages); raw_full[r],
  // raw_empty[r] (r < kRawStages); acc_full[2], acc_empty[2]; mma_done
  __shared__ __align__(8) uint64_t bars[3 * kMaxStages + 2 * kRawStages + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float pweights[64];                    // P~[k][0], the x-pass scattering weights
  const int nx = a.nx, ny = a.ny;
  const TcLayout L(XPASS ? nx : ny, X3, kChunkK);
  const int S = stream_stages(L.stage_bytes);
  const int tiles_per_group = ((XPASS ? ny : nx) + per_tile - 1) / per_tile;
  const int total = tiles_per_group * a.G;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // A launch after a timed-out one does nothing (the march reports the error).
  if (*static_cast<volatile int*>(a.err)) return;
  // x-pass: the y-pass that follows may be scheduled as soon as CTAs leave.
  if (XPASS) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int acc_cols = L.nrows_img;                 // one accumulator: n_mt * 128 columns
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  unsigned char* raw = sm + static_cast<size_t>(S) * L.stage_bytes;
  auto bar = [&](int k) { return smem_u32(&bars[k]); };
  auto full_d = [&](int s) { return bar(s); };
  auto full_s = [&](int s) { return bar(kMaxStages + s); };
  auto empty = [&](int s) { return bar(2 * kMaxStages + s); };
  auto raw_full = [&](int r) { return bar(3 * kMaxStages + r); };
  auto raw_empty = [&](int r) { return bar(3 * kMaxStages + kRawStages + r); };
  auto acc_full = [&](int b2) { return bar(3 * kMaxStages + 2 * kRawStages + b2); };
  auto acc_empty = [&](int b2) { return bar(3 * kMaxStages + 2 * kRawStages + 2 + b2); };
  const uint32_t mma_done = bar(3 * kMaxStages + 2 * kRawStages + 4);

  if (tid == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(full_d(s), 1);
      mbar_init(full_s(s), kCvtThreads);
      mbar_init(empty(s), 1);
    }
    for (int r = 0; r < kRawStages; ++r) {
      mbar_init(raw_full(r), 1);
      mbar_init(raw_empty(r), kCvtThreads);
    }
    for (int b2 = 0; b2 < 2; ++b2) {
      mbar_init(acc_full(b2), 1);
      mbar_init(acc_empty(b2), kEpiWarps * 32);
    }
    mbar_init(mma_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (XPASS)
    for (int k = tid; k < MM; k += kStThreads) pweights[k] = __ldg(a.PT + k);
  if (warp == kWarpCopy) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * acc_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abrt = &abort_flag;
  const int nrows_img = L.nrows_img;
  const size_t chunk_bytes = static_cast<size_t>(2) * nrows_img * 128;
  auto stage_ptr = [&](int s) { return sm + static_cast<size_t>(s) * L.stage_bytes; };

  if (warp == kWarpCopy) {
    // ---------------- copy engine ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&umap)) : "memory");
      const unsigned char* Dimg = static_cast<const unsigned char*>(XPASS ? a.DxImg : a.DyImg);
      int n_raw = 0, n_op = 0;                      // copies issued into each ring
      for (int tl = blockIdx.x; tl < total; tl += gridDim.x) {
        const int g = tl / tiles_per_group, t0 = (tl - g * tiles_per_group) * per_tile;
        for (int q = 0; q < L.n_kc; ++q) {
          const int r = n_raw % kRawStages, s = n_op % S;
          // the raw chunk first: the converters need it to fill the stage.
          // x: box (M, 32 positions, tile rows); y: box (M, tile columns,
          // 32 positions).
          if (!st_wait(raw_empty(r), ((n_raw / kRawStages) & 1) ^ 1, abrt, a.err)) goto copy_done;
          if (XPASS)
            tma_load_4d(smem_u32(raw + r * kRawBytes), &umap, 0, q * kChunkK, t0, g, raw_full(r), kRawBytes);
          else
            tma_load_4d(smem_u32(raw + r * kRawBytes), &umap, 0, t0, q * kChunkK, g, raw_full(r), kRawBytes);
          ++n_raw;
          if (!st_wait(empty(s), ((n_op / S) & 1) ^ 1, abrt, a.err)) goto copy_done;
          bulk_copy(smem_u32(stage_ptr(s)), Dimg + q * chunk_bytes, (X3 ? 2 : 1) * nrows_img * 128, full_d(s));
          ++n_op;
        }
      }
    copy_done:
      // every copy issued has landed before the CTA leaves
      for (int k = 0; k < kRawStages && k < n_raw; ++k) {
        const int j = n_raw - 1 - k;
        st_wait_plain(raw_full(j % kRawStages), (j / kRawStages) & 1, a.err);
      }
      for (int k = 0; k < S && k < n_op; ++k) {
        const int j = n_op - 1 - k;
        st_wait_plain(full_d(j % S), (j / S) & 1, a.err);
      }
    }
  } else if (warp == kWarpMMA) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      // idesc: D = F32, A = B = TF32, K-major, M = 128.  x: A = D_x tile
      // (128 output positions), N = 128 slab columns; y: A = slab (128 slab
      // columns), N = the output positions of the line (<= 256).
      const uint32_t idesc =
          (1u << 4) | (2u << 7) | (2u << 10) |
          (static_cast<uint32_t>((XPASS ? kNC : L.nrows_img) >> 3) << 17) | (static_cast<uint32_t>(kMT >> 4) << 24);
      int it = 0, titer = 0;
      for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
        const int b2 = titer & 1;
        if (!st_wait(acc_empty(b2), ((titer >> 1) & 1) ^ 1, abrt, a.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool fine = true;
        for (int q = 0; q < L.n_kc; ++q, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (!st_wait(full_d(s), ph, abrt, a.err) || !st_wait(full_s(s), ph, abrt, a.err)) {
            fine = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* st = stage_ptr(s);
          unsigned char* Dhi = st;
          unsigned char* Dlo = st + L.n_mt * kTileBytes;
          unsigned char* Shi = st + (X3 ? 2 : 1) * L.n_mt * kTileBytes;
          unsigned char* Slo = Shi + kTileBytes;
          const uint64_t dSh = sw128_desc(smem_u32(Shi)), dSl = sw128_desc(smem_u32(Slo));
          if (XPASS) {
            for (int t = 0; t < L.n_mt; ++t) {
              const uint64_t dDh = sw128_desc(smem_u32(Dhi + t * kTileBytes));
              const uint64_t dDl = sw128_desc(smem_u32(Dlo + t * kTileBytes));
              const uint32_t acc_t = tmem + b2 * acc_cols + t * kNC;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t o = static_cast<uint64_t>(kk * 2);   // 32 bytes per K step
                mma<false>(acc_t, dDh + o, dSh + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                if (X3) {
                  mma<false>(acc_t, dDh + o, dSl + o, idesc, 1u);
                  mma<false>(acc_t, dDl + o, dSh + o, idesc, 1u);
                }
              }
            }
          } else {
            const uint64_t dDh = sw128_desc(smem_u32(Dhi)), dDl = sw128_desc(smem_u32(Dlo));
            const uint32_t acc_t = tmem + b2 * acc_cols;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t o = static_cast<uint64_t>(kk * 2);
              mma<false>(acc_t, dSh + o, dDh + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
              if (X3) {
                mma<false>(acc_t, dSh + o, dDl + o, idesc, 1u);
                mma<false>(acc_t, dSl + o, dDh + o, idesc, 1u);
              }
            }
          }
          mma_commit(empty(s));
        }
        if (!fine) break;
        mma_commit(acc_full(b2));
      }
      // every MMA issued by this thread has completed before TMEM is freed
      mma_commit(mma_done);
      st_wait_plain(mma_done, 0, a.err);
    }
  } else if (warp >= kEpiWarps) {
    // ---------------- conversion ----------------
    // Thread ct owns slab column c = ct (line rc = c / M of the tile,
    // ordinate m) and the 8 16-byte groups of 4 positions of its operand row.
    // Raw layout x: [rc][position][m]; y: [position][rc][m] = [position][c].
    // A warp reads 32 consecutive words per position.
    const int ct = tid - kEpiWarps * 32;
    const int c = ct, rc = c / M, m = c - rc * M;
    const float sc = -__ldg((XPASS ? a.xi : a.eta) + m);
    constexpr int kPosStride = XPASS ? M : kNC;     // raw words between consecutive positions
    const int raw_off = XPASS ? rc * kChunkK * M + m : c;
    int it = 0;
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x) {
      bool fine = true;
      for (int q = 0; q < L.n_kc; ++q, ++it) {
        const int s = it % S, r = it % kRawStages;
        if (!st_wait(raw_full(r), (it / kRawStages) & 1, abrt, a.err) ||
            !st_wait(empty(s), ((it / S) & 1) ^ 1, abrt, a.err)) {
          fine = false;
          break;
        }
        const float* rw = reinterpret_cast<const float*>(raw + r * kRawBytes) + raw_off;
        unsigned char* Shi = stage_ptr(s) + (X3 ? 2 : 1) * L.n_mt * kTileBytes;
        unsigned char* Slo = Shi + kTileBytes;
        float4 v[kChunkK / 4];
#pragma unroll
        for (int grp = 0; grp < kChunkK / 4; ++grp)
          v[grp] = make_float4(rw[(4 * grp) * kPosStride], rw[(4 * grp + 1) * kPosStride],
                               rw[(4 * grp + 2) * kPosStride], rw[(4 * grp + 3) * kPosStride]);
        // The raw buffer is free once read.  The release of an mbarrier does
        // not order these generic-proxy reads before the next tensor copy
        // (async proxy) into the same buffer: without the proxy fence that
        // copy can land before the reads are performed.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(raw_empty(r));
#pragma unroll
        for (int grp = 0; grp < kChunkK / 4; ++grp) {
          float4 hi, lo;
          split4(v[grp], sc, hi, lo);
          const int off = sw128_off(c, grp);
          *reinterpret_cast<float4*>(Shi + off) = hi;
          if (X3) *reinterpret_cast<float4*>(Slo + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full_s(s));
      }
      if (!fine) break;
    }
  } else if (XPASS) {
    // ---------------- x epilogue ----------------
    // lane = output position i, columns = (row, m).  Pairs (tile t, row rc)
    // of the accumulator alternate between warps w and w + 4 (same quarter).
    const int quarter = warp & 3, half = warp >> 2;
    const int n_pairs = L.n_mt * per_tile;
    // P~[m][q] = p_{(m - q) mod M}: the symmetric circulant's first column
    // scattering weights p_k = P~[k][0], written before the CTA-wide barrier
    // that precedes the roles
    const float* pcs = pweights;
    const uint64_t pol_keep = policy_evict_last();
    int titer = 0;
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
      const int b2 = titer & 1;
      if (!st_wait(acc_full(b2), (titer >> 1) & 1, abrt, a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int g = tl / tiles_per_group, t0 = (tl - g * tiles_per_group) * per_tile;
      const size_t goff = static_cast<size_t>(g) * a.plane;
      const uint32_t tq = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + b2 * acc_cols;
      for (int p = half; p < n_pairs; p += 2) {
        const int t = p / per_tile, rc = p - t * per_tile;
        const int i = t * kMT + 32 * quarter + lane, j = t0 + rc;
        const bool valid = i < nx && j < ny;
        const size_t cell = static_cast<size_t>(j) * nx + i;
        float uu[MM];
        float ab = 0.f, bb = 0.f;
        if (valid) {
#pragma unroll
          for (int k = 0; k < MM / 8; ++k) ld8_nc(U + goff + cell * M + 8 * k, uu + 8 * k);
          bb = __ldg(a.mus + cell);
          ab = __ldg(a.mua + cell) + bb;
        } else {
#pragma unroll
          for (int k = 0; k < MM; ++k) uu[k] = 0.f;
        }
        float acc[MM];
        tmem_ld16(tq + t * kNC + rc * M, acc);
        if (MM > 16) tmem_ld16(tq + t * kNC + rc * M + 16, acc + 16);
        if (valid) {
          xpass_node_rhs<MM, true>(acc, uu, pcs, ab, bb);
          // R is read by the y-pass that follows: keep it in L2
#pragma unroll
          for (int k = 0; k < MM / 8; ++k) st8_hint(R + goff + cell * M + 8 * k, acc + 8 * k, pol_keep);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acc_empty(b2));
    }
  } else {
    // ---------------- y epilogue ----------------
    // lane = slab column c = (grid column w of the tile, ordinate m), TMEM
    // columns = grid rows j.  Chunks of kRowsY rows alternate between warps
    // w and w + 4 (same lane quarter).  Per node value: L^k = R + acc, the
    // AB4 update, then on boundary nodes the boundary condition from the
    // pre-BC values of the node (the reflected ordinate is a lane of the
    // same warp) and the exitance of each face (a fixed-order sum over the
    // node's lanes) -- the one-tile y-pass's arithmetic in the same order.
    constexpr unsigned kFull = 0xffffffffu;
    const int quarter = warp & 3, half = warp >> 2;
    const int c = 32 * quarter + lane;
    const int w = c / M, m = c - w * M;
    const int base = (lane / M) * M;              // lane of ordinate 0 of this node
    const int ring_len = 2 * ny + 2 * nx;
    const int nchunks = (ny + kRowsY - 1) / kRowsY;
    // u^{k+1} is read by the next x-pass; the history and R are read once
    const uint64_t pol_keep = policy_evict_last(), pol_once = policy_evict_first();
    int titer = 0;
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
      const int b2 = titer & 1;
      if (!st_wait(acc_full(b2), (titer >> 1) & 1, abrt, a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int g = tl / tiles_per_group, t0 = (tl - g * tiles_per_group) * per_tile;
      const size_t goff = static_cast<size_t>(g) * a.plane;
      const int i = t0 + w;
      const bool col_ok = i < nx;
      const bool lf = i == 0, rt = i == nx - 1;
      const uint32_t tq = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + b2 * acc_cols;
      float* ro = (b.ring_out && ring_step >= 0)
                      ? b.ring_out + (static_cast<size_t>(g) * b.ring_steps + ring_step) * ring_len
                      : nullptr;
      for (int ci = half; ci < nchunks; ci += 2) {
        const int j0c = ci * kRowsY;
        float acc[kRowsY];
        tmem_ld16(tq + j0c, acc);
        float uo[kRowsY], rr[kRowsY], p1[kRowsY], p2[kRowsY], p3[kRowsY];
#pragma unroll
        for (int t = 0; t < kRowsY; ++t) {
          const int j = j0c + t;
          if (col_ok && j < ny) {
            const size_t gidx = goff + (static_cast<size_t>(j) * nx + i) * M + m;
            uo[t] = ld_hint(U + gidx, pol_once);
            rr[t] = ld_hint(R + gidx, pol_once);
            p1[t] = ld_hint(L1 + gidx, pol_once);
            p2[t] = ld_hint(L2 + gidx, pol_once);
            p3[t] = ld_hint(L3 + gidx, pol_once);
          } else {
            uo[t] = rr[t] = p1[t] = p2[t] = p3[t] = 0.f;
          }
        }
        float un[kRowsY];
#pragma unroll
        for (int t = 0; t < kRowsY; ++t) {
          const float lk = rr[t] + acc[t];
          un[t] = ab4_node(a.cdt, lk, p1[t], p2[t], p3[t], uo[t]);
          const int j = j0c + t;
          if (col_ok && j < ny) L3[goff + (static_cast<size_t>(j) * nx + i) * M + m] = lk;
        }
#pragma unroll
        for (int t = 0; t < kRowsY; ++t) {
          const int j = j0c + t;
          const bool ok = col_ok && j < ny;
          const size_t gidx = goff + (static_cast<size_t>(j) * nx + i) * M + m;
          const bool bt = j == 0, tp = j == ny - 1;
          const bool bnd = ok && (lf || rt || bt || tp);
          if (__any_sync(kFull, bnd)) {
            // table: face 0..3 or corner 4..7
            const int tb = ((lf || rt) && (bt || tp)) ? 4 + (rt ? 1 : 0) + (tp ? 2 : 0)
                                                      : (lf ? 0 : rt ? 1 : bt ? 2 : 3);
            const int e = (tb < 4 ? tb : tb - 4) * M + m;
            const int refl = __ldg((tb < 4 ? b.face_refl : b.corner_refl) + e);
            const float ur = __shfl_sync(kFull, un[t], base + refl);
            float val = un[t];
            if (bnd && __ldg((tb < 4 ? b.face_act : b.corner_act) + e)) {
              const int node = lf ? j : rt ? ny + j : bt ? 2 * ny + i : 2 * ny + nx + i;
              float qv = 0.f;
              for (int k = 0; k < b.kmax; ++k) {
                const size_t gk = static_cast<size_t>(g) * b.kmax + k;
                qv = fmaf(__ldg(b.S + gk * ring_len + node) * __ldg(b.A + gk * M + m),
                          __ldg(b.T + gk * b.T_len + src_step), qv);
              }
              const float fco = __ldg((tb < 4 ? b.face_f : b.corner_f) + e);
              if (b.rho)
                qv = fmaf(1.0f - fco, __ldg(b.rho + (static_cast<size_t>(g) * b.rho_len + src_step) * ring_len + node),
                          qv);
              val = fmaf(fco, ur, qv);
            }
            if (ok) U[gidx] = val;
            if (ro) {
              if (__any_sync(kFull, bnd && (lf || rt))) {
                const int F = lf ? 0 : 1;
                float ex = 0.f;
                for (int mm = 0; mm < M; ++mm)
                  ex = fmaf(__ldg(b.wexit + F * M + mm), __shfl_sync(kFull, val, base + mm), ex);
                if (bnd && (lf || rt) && m == 0) ro[lf ? j : ny + j] = ex;
              }
              if (__any_sync(kFull, bnd && (bt || tp))) {
                const int F = bt ? 2 : 3;
                float ex = 0.f;
                for (int mm = 0; mm < M; ++mm)
                  ex = fmaf(__ldg(b.wexit + F * M + mm), __shfl_sync(kFull, val, base + mm), ex);
                if (bnd && (bt || tp) && m == 0) ro[bt ? 2 * ny + i : 2 * ny + nx + i] = ex;
              }
            }
          } else if (ok) {
            st_hint1(U + gidx, un[t], pol_keep);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acc_empty(b2));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kWarpCopy)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * acc_cols));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

template <bool XPASS, int PREC, int MM>
cudaError_t launch_stream_t(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                            const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // The state of all groups as a 4D tensor [G][ny][nx][M] (innermost first
  // below); one box is one raw chunk of one group: all M ordinates x 32
  // positions x the tile's rows (x-pass), or all M ordinates x the tile's
  // columns x 32 positions (y-pass).  Boxes past the grid read as 0.
  alignas(64) CUtensorMap map;
  const cuuint64_t dims[4] = {static_cast<cuuint64_t>(MM), static_cast<cuuint64_t>(a.nx),
                              static_cast<cuuint64_t>(a.ny), static_cast<cuuint64_t>(a.G)};
  const cuuint64_t strides[3] = {static_cast<cuuint64_t>(MM) * 4, static_cast<cuuint64_t>(a.nx) * MM * 4,
                                 static_cast<cuuint64_t>(a.plane) * 4};
  const cuuint32_t box[4] = {static_cast<cuuint32_t>(MM),
                             static_cast<cuuint32_t>(XPASS ? kChunkK : kNC / MM),
                             static_cast<cuuint32_t>(XPASS ? kNC / MM : kChunkK), 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, U, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  using K = Kind<PREC>;
  const TcLayout L(XPASS ? a.nx : a.ny, K::X3, kChunkK);
  const int S = stream_stages(L.stage_bytes);
  const size_t smem = 1024 + static_cast<size_t>(S) * L.stage_bytes + static_cast<size_t>(kRawStages) * kRawBytes;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(tc_pass_stream<XPASS, PREC, MM>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  static int sm_count[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!sm_count[dev]) cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
  const int sms = sm_count[dev] > 0 ? sm_count[dev] : 1;
  const int lines = XPASS ? a.ny : a.nx;
  const int tiles = (lines + kNC / MM - 1) / (kNC / MM) * a.G;
  const int grid = tiles < sms ? tiles : sms;
  tc_pass_stream<XPASS, PREC, MM><<<grid, kStThreads, smem, s>>>(a, b, map, U, R, L1, L2, L3, src_step, ring_step);
  return cudaGetLastError();
}

template <bool XPASS>
cudaError_t launch_stream(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                          const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  if (a.tc_mode == 1)
    return a.M == 16 ? launch_stream_t<XPASS, 1, 16>(a, b, U, R, L1, L2, L3, src_step, ring_step, s)
                     : launch_stream_t<XPASS, 1, 32>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
  return a.M == 16 ? launch_stream_t<XPASS, 2, 16>(a, b, U, R, L1, L2, L3, src_step, ring_step, s)
                   : launch_stream_t<XPASS, 2, 32>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
}

bool stream_common_ok(const StepArgs& a, int n) {
  if (!(a.tc_mode == 1 || a.tc_mode == 2) || n > 256 || !(a.M == 16 || a.M == 32)) return false;
  const TcLayout L(n, a.tc_mode == 1, kChunkK);
  return stream_stages(L.stage_bytes) >= 2;
}

}  // namespace

bool tc_stream_supported(const StepArgs& a) { return a.tc_scatter == 0 && stream_common_ok(a, a.nx); }

bool tc_ystream_supported(const StepArgs& a) { return stream_common_ok(a, a.ny); }

cudaError_t launch_xpass_stream(const StepArgs& a, const BoundaryArgs& b, const float* U, float* R,
                                cudaStream_t s) {
  return launch_stream<true>(a, b, const_cast<float*>(U), R, nullptr, nullptr, nullptr, 0, -1, s);
}

cudaError_t launch_ypass_stream(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                                const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  return launch_stream<false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
}

}  // namespace rte_kern
