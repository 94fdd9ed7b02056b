// Persistent, warp-specialised tcgen05 form of the two passes (lines of
// n <= 256 positions, M in {16, 32}) for sm_103a.
//
// Same arithmetic as rte_tc.cu.  x-pass: for a slab tile of 128 columns
// (grid rows j0 .. j0 + 128/M - 1 times the M ordinates) over a whole grid
// row, acc[i][c] = sum_k D_x[i][k] (-xi_m u(c, k)) on the tensor cores, and
// R = b P~u - (a + b) u + acc in the epilogue (Sec. 4.1, Sec. 4.3).  y-pass:
// acc[c][j] = sum_k (-eta_m u(c, k)) D_y[j][k]; the epilogue forms
// L = R + acc, the AB4 update (eq. RTEAB4), the Fresnel boundary condition
// with source injection (eq. RTE) and the exitance ring (eq. OpMed).  What
// differs from rte_tc.cu is the schedule: one CTA per SM walks its share of
// the tiles, and the roles run concurrently on separate warps, handing work
// over through mbarriers:
//   warp 10 (one lane)  bulk copies of the operator chunks into a ring of S
//                       stages (S = 2..4, by shared-memory size);
//   warps 8-9           load the slab chunk, split it into hi + lo, write it
//                       in the swizzled operand layout of the same stage;
//   warp 11 (one lane)  issues the MMAs of each chunk into one of two
//                       tensor-memory accumulators and commits them (the
//                       commit frees the stage; the last one of a tile hands
//                       the accumulator to the epilogue);
//   warps 0-7           drain the accumulator of the previous tile (two warps
//                       per 32-lane quarter) while the next tile accumulates
//                       into the other one.
// The y-pass epilogue keeps each slab column in one lane: a node's M
// ordinates sit in adjacent lanes of one warp, so the reflected ordinate of
// the boundary condition is a warp shuffle and the exitance a shuffled sum
// in ordinate order.
// Every wait is bounded: on expiry the kernel raises the context timeout word and a shared
// abort flag that ends every other role's waits, and all roles leave.
#include <cstdint>

#include "rte_tc_common.cuh"

namespace rte_kern {


namespace {

using namespace tc;

constexpr int kEpiWarps = 8, kSlabWarps = 2;
constexpr int kWarpD = kEpiWarps + kSlabWarps, kWarpMMA = kWarpD + 1;
constexpr int kWsThreads = (kWarpMMA + 1) * 32;
constexpr int kMaxStages = 4;
constexpr int kSmemLimit = 232448 - 2048;

// Bounded wait (kWaitNs, no abort check): the drains before the kernel leaves.
__device__ __forceinline__ bool ws_wait_plain(uint32_t bar, uint32_t parity, int* err) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  return true;
}

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int PREC>
__host__ __device__ inline int ws_stages(int stage_bytes) {
  const int s = (kSmemLimit - 1024) / stage_bytes;
  return s > kMaxStages ? kMaxStages : s;
}

constexpr int kTableBytes = 4096;   // y-pass boundary tables

// 12 warps: at most three per SM sub-partition, so up to 168 registers a thread.
template <bool XPASS, int PREC, int MM>
__global__ void __launch_bounds__(kWsThreads, 1)
    tc_pass_ws(StepArgs a, BoundaryArgs b, float* __restrict__ U, float* __restrict__ R,
               const float* __restrict__ L1, const float* __restrict__ L2, float* __restrict__ L3, int src_step,
               int ring_step) {
  using K = Kind<PREC>;
  constexpr bool X3 = K::X3, BF = K::BF;
  constexpr int KC = K::KC, GV = K::GV;
  constexpr int M = MM;
  constexpr int per_tile = kNC / M;
  extern __shared__ __align__(1024) unsigned char smraw[];
  // full_d[s], full_s[s], empty[s] for s < kMaxStages; acc_full[2],
  // acc_empty[2]; mma_done (all MMAs of the CTA complete)
  __shared__ __align__(8) uint64_t bars[3 * kMaxStages + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float pweights[64];                    // P~[k][0], the x-pass scattering weights
  const int nx = a.nx, ny = a.ny;
  const int n = XPASS ? nx : ny;              // line length (K and output positions)
  const int lines = XPASS ? ny : nx;          // grid rows (x) / columns (y)
  const TcLayout L(n, X3, KC);
  const int S = ws_stages<PREC>(L.stage_bytes + (XPASS ? 0 : kTableBytes));
  const int tiles_per_group = (lines + per_tile - 1) / per_tile;
  const int total = tiles_per_group * a.G;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // A launch after a timed-out one does nothing (the march reports the error).
  if (*static_cast<volatile int*>(a.err)) return;
  const int acc_cols = L.nrows_img;                    // one accumulator buffer (n_mt * 128)
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  auto bar = [&](int k) { return smem_u32(&bars[k]); };
  auto full_d = [&](int s) { return bar(s); };
  auto full_s = [&](int s) { return bar(kMaxStages + s); };
  auto empty = [&](int s) { return bar(2 * kMaxStages + s); };
  auto acc_full = [&](int b) { return bar(3 * kMaxStages + b); };
  auto acc_empty = [&](int b) { return bar(3 * kMaxStages + 2 + b); };
  const uint32_t mma_done = bar(3 * kMaxStages + 4);

  if (tid == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(full_d(s), 1);
      mbar_init(full_s(s), kSlabWarps * 32);
      mbar_init(empty(s), 1);
    }
    for (int b2 = 0; b2 < 2; ++b2) {
      mbar_init(acc_full(b2), 1);
      mbar_init(acc_empty(b2), kEpiWarps * 32);
    }
    mbar_init(mma_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // y-pass: boundary tables (faces 0..3, corners 4..7) after the stages
  float* bc_f = reinterpret_cast<float*>(sm + static_cast<size_t>(S) * L.stage_bytes);   // [8][M]
  float* bc_wexit = bc_f + 8 * M;                                                        // [4][M]
  int* bc_refl = reinterpret_cast<int*>(bc_wexit + 4 * M);                               // [8][M]
  unsigned char* bc_act = reinterpret_cast<unsigned char*>(bc_refl + 8 * M);             // [8][M]
  if (!XPASS) {
    for (int e = tid; e < 8 * M; e += kWsThreads) {
      const int tb = e / M, m = e - tb * M;
      const bool face = tb < 4;
      const int k = (face ? tb : tb - 4) * M + m;
      bc_f[e] = face ? b.face_f[k] : b.corner_f[k];
      bc_refl[e] = face ? b.face_refl[k] : b.corner_refl[k];
      bc_act[e] = face ? b.face_act[k] : b.corner_act[k];
      if (face) bc_wexit[e] = b.wexit[k];
    }
  }
  if (XPASS)
    for (int k = tid; k < MM; k += kWsThreads) pweights[k] = __ldg(a.PT + k);
  if (warp == kWarpD) {
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

  if (warp == kWarpD) {
    // ---------------- operator chunks ----------------
    if (lane == 0) {
      const unsigned char* Dimg = static_cast<const unsigned char*>(XPASS ? a.DxImg : a.DyImg);
      int it = 0;
      for (int tl = blockIdx.x; tl < total; tl += gridDim.x)
        for (int q = 0; q < L.n_kc; ++q, ++it) {
          const int s = it % S;
          if (!ws_wait(empty(s), ((it / S) & 1) ^ 1, abrt, a.err)) goto d_done;
          bulk_copy(smem_u32(stage_ptr(s)), Dimg + q * chunk_bytes, (X3 ? 2 : 1) * nrows_img * 128, full_d(s));
        }
    d_done:
      // the last copy into each stage has landed before the CTA leaves
      for (int k = 0; k < S && k < it; ++k) {
        const int j = it - 1 - k;
        ws_wait_plain(full_d(j % S), (j / S) & 1, a.err);
      }
    }
  } else if (warp == kWarpMMA) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      // idesc: D = F32, A = B = TF32 (2) or BF16 (1), K-major, M = 128;
      // N = 128 slab columns (x-pass) or all output positions (y-pass).
      constexpr uint32_t kFmt = BF ? 1u : 2u;
      const uint32_t idesc = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                             (static_cast<uint32_t>((XPASS ? kNC : nrows_img) >> 3) << 17) |
                             (static_cast<uint32_t>(kMT >> 4) << 24);
      int it = 0, titer = 0;
      for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
        const int b2 = titer & 1;
        if (!ws_wait(acc_empty(b2), ((titer >> 1) & 1) ^ 1, abrt, a.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool fine = true;
        for (int q = 0; q < L.n_kc; ++q, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (!ws_wait(full_d(s), ph, abrt, a.err) || !ws_wait(full_s(s), ph, abrt, a.err)) {
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
                mma<BF>(acc_t, dDh + o, dSh + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                if (X3) {
                  mma<BF>(acc_t, dDh + o, dSl + o, idesc, 1u);
                  mma<BF>(acc_t, dDl + o, dSh + o, idesc, 1u);
                }
              }
            }
          } else {
            const uint64_t dDh = sw128_desc(smem_u32(Dhi)), dDl = sw128_desc(smem_u32(Dlo));
            const uint32_t acc_b = tmem + b2 * acc_cols;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t o = static_cast<uint64_t>(kk * 2);
              mma<BF>(acc_b, dSh + o, dDh + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
              if (X3) {
                mma<BF>(acc_b, dSh + o, dDl + o, idesc, 1u);
                mma<BF>(acc_b, dSl + o, dDh + o, idesc, 1u);
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
      ws_wait_plain(mma_done, 0, a.err);
    }
  } else if (warp >= kEpiWarps) {
    // ---------------- slab staging ----------------
    // The 64 threads stage a chunk in units of 64 values per thread (one unit
    // per tf32 chunk, two per bf16 chunk); the next unit's values are loaded
    // while this one is split and stored, or while the stage is still busy.
    const int ltid = tid - kEpiWarps * 32;
    constexpr int kSlabThreads = kSlabWarps * 32;
    constexpr int kItems = kNC * (KC / GV) / kSlabThreads;       // items per chunk and thread
    constexpr int kUnits = BF ? 2 : 1;
    constexpr int kIU = kItems / kUnits;                        // items per unit (16 tf32, 8 bf16)
    float v[kIU][GV];
    const float* scale = XPASS ? a.xi : a.eta;
    auto load_unit = [&](int tl, int q, int h) {
      const int g = tl / tiles_per_group, t0 = (tl - g * tiles_per_group) * per_tile;
      const size_t goff = static_cast<size_t>(g) * a.plane;
      const int k0 = q * KC;
#pragma unroll
      for (int t = 0; t < kIU; ++t) {
        const int itm = ltid + (h * kIU + t) * kSlabThreads;
        const int c = itm % kNC, grp = itm / kNC;
        const int rc = c / M, m = c - rc * M;
        const int line = t0 + rc;
#pragma unroll
        for (int e = 0; e < GV; ++e) {
          const int k = k0 + grp * GV + e;
          if (line < lines && k < n) {
            // the y-pass writes U (other tiles' columns): plain loads there
            const size_t idx = XPASS ? goff + (static_cast<size_t>(line) * nx + k) * M + m
                                     : goff + (static_cast<size_t>(k) * nx + line) * M + m;
            v[t][e] = XPASS ? __ldg(U + idx) : U[idx];
          } else {
            v[t][e] = 0.f;
          }
        }
      }
    };
    int it = 0;
    if (static_cast<int>(blockIdx.x) < total) load_unit(blockIdx.x, 0, 0);
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x) {
      bool fine = true;
      for (int q = 0; q < L.n_kc; ++q, ++it) {
        const int s = it % S;
        if (!ws_wait(empty(s), ((it / S) & 1) ^ 1, abrt, a.err)) {
          fine = false;
          break;
        }
        unsigned char* Shi = stage_ptr(s) + (X3 ? 2 : 1) * L.n_mt * kTileBytes;
        unsigned char* Slo = Shi + kTileBytes;
#pragma unroll
        for (int h = 0; h < kUnits; ++h) {
#pragma unroll
          for (int t = 0; t < kIU; ++t) {
            const int itm = ltid + (h * kIU + t) * kSlabThreads;
            const int c = itm % kNC, grp = itm / kNC;
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
          // next unit: this chunk's second half, this tile's next chunk, or
          // the next tile's first chunk
          if (h + 1 < kUnits) load_unit(tl, q, h + 1);
          else if (q + 1 < L.n_kc) load_unit(tl, q + 1, 0);
          else if (tl + static_cast<int>(gridDim.x) < total) load_unit(tl + gridDim.x, 0, 0);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full_s(s));
      }
      if (!fine) break;
    }
  } else if (XPASS) {
    // ---------------- x-pass epilogue ----------------
    // lane = output position i, columns = (row, m).  Pairs (tile t, row rc)
    // of the accumulator alternate between warps w and w + 4 (same quarter).
    const int quarter = warp & 3, half = warp >> 2;
    const int n_pairs = L.n_mt * per_tile;
    // scattering weights p_k = P~[k][0], written before the CTA-wide barrier
    // that precedes the roles
    const float* pcs = pweights;
    int titer = 0;
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
      const int b2 = titer & 1;
      if (!ws_wait(acc_full(b2), (titer >> 1) & 1, abrt, a.err)) break;
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
          const float4* up = reinterpret_cast<const float4*>(U + goff + cell * M);
#pragma unroll
          for (int k = 0; k < MM / 4; ++k) {
            const float4 u4 = __ldg(up + k);
            uu[4 * k] = u4.x; uu[4 * k + 1] = u4.y; uu[4 * k + 2] = u4.z; uu[4 * k + 3] = u4.w;
          }
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
          xpass_node_rhs<MM>(acc, uu, pcs, ab, bb);
          float4* rp = reinterpret_cast<float4*>(R + goff + cell * M);
#pragma unroll
          for (int k = 0; k < MM / 4; ++k) rp[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acc_empty(b2));
    }
  } else {
    // ---------------- y-pass epilogue ----------------
    // lane = slab column c = (grid column w, ordinate m), TMEM columns = grid
    // rows j.  Chunks of 16 rows alternate between warps w and w + 4.
    constexpr unsigned kFull = 0xffffffffu;
    const int quarter = warp & 3, half = warp >> 2;
    const int c = 32 * quarter + lane;
    const int w = c / M, m = c - w * M;
    const int base = (lane / M) * M;            // lane of ordinate 0 of this node
    const int ring_len = 2 * ny + 2 * nx;
    const int nchunks = (ny + 15) / 16;
    int titer = 0;
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
      const int b2 = titer & 1;
      if (!ws_wait(acc_full(b2), (titer >> 1) & 1, abrt, a.err)) break;
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
        const int j0c = ci * 16;
        float acc[16];
        tmem_ld16(tq + j0c, acc);
        // all loads of the chunk first, then AB4 (eq. RTEAB4) and L^k
        float uo[16], rr[16], p1[16], p2[16], p3[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int j = j0c + t;
          if (col_ok && j < ny) {
            const size_t gidx = goff + (static_cast<size_t>(j) * nx + i) * M + m;
            uo[t] = U[gidx];
            rr[t] = __ldg(R + gidx);
            p1[t] = __ldg(L1 + gidx);
            p2[t] = __ldg(L2 + gidx);
            p3[t] = L3[gidx];
          } else {
            uo[t] = rr[t] = p1[t] = p2[t] = p3[t] = 0.f;
          }
        }
        float un[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const float lk = rr[t] + acc[t];
          un[t] = ab4_node(a.cdt, lk, p1[t], p2[t], p3[t], uo[t]);
          const int j = j0c + t;
          if (col_ok && j < ny) L3[goff + (static_cast<size_t>(j) * nx + i) * M + m] = lk;
        }
        // boundary condition (eq. RTE, third line) from the pre-BC values of
        // the node, then u^{k+1}; exitance of the boundary nodes (eq. OpMed)
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int j = j0c + t;
          const bool ok = col_ok && j < ny;
          const size_t gidx = goff + (static_cast<size_t>(j) * nx + i) * M + m;
          const bool bt = j == 0, tp = j == ny - 1;
          const bool bnd = ok && (lf || rt || bt || tp);
          if (__any_sync(kFull, bnd)) {
            const int tb = ((lf || rt) && (bt || tp)) ? 4 + (rt ? 1 : 0) + (tp ? 2 : 0)
                                                      : (lf ? 0 : rt ? 1 : bt ? 2 : 3);
            const float ur = __shfl_sync(kFull, un[t], base + bc_refl[tb * M + m]);
            float val = un[t];
            if (bnd && bc_act[tb * M + m]) {
              const int node = lf ? j : rt ? ny + j : bt ? 2 * ny + i : 2 * ny + nx + i;
              float qv = 0.f;
              for (int k = 0; k < b.kmax; ++k) {
                const size_t gk = static_cast<size_t>(g) * b.kmax + k;
                qv = fmaf(__ldg(b.S + gk * ring_len + node) * __ldg(b.A + gk * M + m),
                          __ldg(b.T + gk * b.T_len + src_step), qv);
              }
              const float fco = bc_f[tb * M + m];
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
                  ex = fmaf(bc_wexit[F * M + mm], __shfl_sync(kFull, val, base + mm), ex);
                if (bnd && (lf || rt) && m == 0) ro[lf ? j : ny + j] = ex;
              }
              if (__any_sync(kFull, bnd && (bt || tp))) {
                const int F = bt ? 2 : 3;
                float ex = 0.f;
                for (int mm = 0; mm < M; ++mm)
                  ex = fmaf(bc_wexit[F * M + mm], __shfl_sync(kFull, val, base + mm), ex);
                if (bnd && (bt || tp) && m == 0) ro[bt ? 2 * ny + i : 2 * ny + nx + i] = ex;
              }
            }
          } else if (ok) {
            U[gidx] = un[t];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(acc_empty(b2));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kWarpD)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * acc_cols));
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <bool XPASS, int PREC, int MM>
cudaError_t launch_ws(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                      const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  using K = Kind<PREC>;
  const TcLayout L(XPASS ? a.nx : a.ny, K::X3, K::KC);
  const int extra = XPASS ? 0 : kTableBytes;
  const int S = ws_stages<PREC>(L.stage_bytes + extra);
  const size_t smem = 1024 + static_cast<size_t>(S) * L.stage_bytes + extra;
  static bool attr = false;
  if (!attr) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, tc_pass_ws<XPASS, PREC, MM>);
    if (e != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < kWsThreads) return cudaErrorLaunchOutOfResources;
    e = cudaFuncSetAttribute(tc_pass_ws<XPASS, PREC, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int per_tile = kNC / MM;
  const int lines = XPASS ? a.ny : a.nx;
  const int total = (lines + per_tile - 1) / per_tile * a.G;
  const int grid = total < sm_count() ? total : sm_count();
  tc_pass_ws<XPASS, PREC, MM><<<grid, kWsThreads, smem, s>>>(a, b, U, R, L1, L2, L3, src_step, ring_step);
  return cudaGetLastError();
}

template <bool XPASS, int PREC>
cudaError_t launch_ws_m(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                        const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  return a.M == 16 ? launch_ws<XPASS, PREC, 16>(a, b, U, R, L1, L2, L3, src_step, ring_step, s)
                   : launch_ws<XPASS, PREC, 32>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
}

template <bool XPASS>
cudaError_t launch_ws_pass(const StepArgs& a, const BoundaryArgs& b, float* U, float* R, const float* L1,
                           const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  switch (a.tc_mode) {
    case 1: return launch_ws_m<XPASS, 1>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
    case 2: return launch_ws_m<XPASS, 2>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
    case 3: return launch_ws_m<XPASS, 3>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
    default: return launch_ws_m<XPASS, 4>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
  }
}

}  // namespace

bool tc_ws_supported(const StepArgs& a) {
  return a.tc_mode >= 1 && a.tc_mode <= 4 && a.tc_scatter == 0 && a.nx <= 256 && a.ny <= 256 &&
         (a.M == 16 || a.M == 32);
}

cudaError_t launch_pass_ws(bool xpass, const StepArgs& a, const BoundaryArgs& b, float* U, float* R,
                           const float* L1, const float* L2, float* L3, int src_step, int ring_step,
                           cudaStream_t s) {
  return xpass ? launch_ws_pass<true>(a, b, U, R, L1, L2, L3, src_step, ring_step, s)
               : launch_ws_pass<false>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
}


}  // namespace rte_kern
