// Pipelined persistent tcgen05 y-pass (lines of ny <= 256 positions,
// M in {16, 32, 64}) for sm_103a.
//
// Same arithmetic as the y-pass of rte_tc.cu: for a slab tile of 128
// columns (grid columns i0 .. i0 + 128/M - 1 times the M ordinates),
// acc[c][j] = sum_k (-eta_m u(c, k)) D_y[j][k] on the tensor cores, then
// L = R + acc, the AB4 update (eq. RTEAB4), the Fresnel boundary condition
// with source injection (eq. RTE) and the exitance ring (eq. OpMed).
//
// One CTA per SM walks its share of the tiles with two groups of eight
// warps that work on consecutive tiles at the same time:
//   warps 0-7   the main loop of rte_tc.cu: operator chunks by
//               cp.async.bulk, the slab split to hi + lo and swizzled by all
//               256 threads, one thread issuing the MMAs into one of two
//               tensor-memory accumulators;
//   warps 8-15  the epilogue of the previous tile: u, R, L1..L3 streamed in
//               8-row chunks through a four-deep cp.async ring (three chunks
//               ahead), the accumulator copied to shared memory by warps
//               8-11 (TMEM lane quarters 0-3), AB4 with float4 accesses,
//               boundary nodes finished from the pre-BC values.
// The groups synchronise internally with named barriers (1 and 2) and with
// each other through mbarriers (accumulator full / accumulator free).
// Every wait is bounded by kWaitNs of %globaltimer; on expiry the kernel
// raises the context's timeout word and an abort flag that ends the other waits.
#include <cstdint>

#include "rte_tc_common.cuh"

namespace rte_kern {


namespace {

using namespace tc;

constexpr int kPipeThreads = 512;
constexpr int kGroup = 256;                 // threads per group
constexpr int kRows = 8;                    // epilogue chunk rows
constexpr int kNBuf = 4;                    // epilogue ring depth
constexpr int kEpiArr = 5;                  // u, R, L1, L2, L3
constexpr int kChunkFloats = kEpiArr * kRows * kNC;
constexpr int kMaxM = 64;
constexpr size_t kEpiSmem = static_cast<size_t>(kNBuf) * kChunkFloats * 4 + 3 * kRows * kNC * 4 +
                            (8 + 4 + 8) * kMaxM * 4 + 8 * kMaxM;
constexpr int kSmemLimit = 232448 - 2048;

__device__ __forceinline__ bool pipe_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
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

__device__ __forceinline__ bool pipe_wait_plain(uint32_t bar, uint32_t parity, int* err) {
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

__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kGroup) : "memory");
}

__device__ __forceinline__ void cp_async_wait(int newer) {
  switch (newer) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
  }
}

template <int PREC, int MM>
__global__ void __launch_bounds__(kPipeThreads, 1)
    tc_ypass_pipe(StepArgs a, BoundaryArgs b, float* __restrict__ U, const float* __restrict__ R,
                  const float* __restrict__ L1, const float* __restrict__ L2, float* __restrict__ L3, int src_step,
                  int ring_step) {
  using K = Kind<PREC>;
  constexpr bool X3 = K::X3, BF = K::BF;
  constexpr int KC = K::KC, GV = K::GV;
  constexpr int M = MM;
  constexpr int per_tile = kNC / M;           // grid columns per tile
  extern __shared__ __align__(1024) unsigned char smraw[];
  // full (operator chunk landed), done (chunk's MMAs complete), acc_full[2],
  // acc_empty[2], mma_done
  __shared__ __align__(8) uint64_t bars[7];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int main_ok, epi_ok;             // a group leader's wait result, read after the group barrier
  const int nx = a.nx, ny = a.ny;
  const int n = ny;
  const TcLayout L(n, X3, KC);
  const int tiles_per_group = (nx + per_tile - 1) / per_tile;
  const int total = tiles_per_group * a.G;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*static_cast<volatile int*>(a.err)) return;
  const int acc_cols = L.nrows_img;
  unsigned char* sm = smraw + ((1024 - (smem_u32(smraw) & 1023)) & 1023);
  float* epi = reinterpret_cast<float*>(sm + L.stage_bytes);
  float* ebuf = epi;                                          // [kNBuf][5][kRows][128]
  float* acc_s = ebuf + kNBuf * kChunkFloats;                  // [kRows][128]
  float* un_s = acc_s + kRows * kNC;                           // [kRows][128] pre-BC u^{k+1}
  float* bc_s = un_s + kRows * kNC;                            // [kRows][128] post-BC values
  float* bc_f = bc_s + kRows * kNC;                            // [8][M]
  float* bc_wexit = bc_f + 8 * kMaxM;                          // [4][M]
  int* bc_refl = reinterpret_cast<int*>(bc_wexit + 4 * kMaxM); // [8][M]
  unsigned char* bc_act = reinterpret_cast<unsigned char*>(bc_refl + 8 * kMaxM);
  const uint32_t bar_full = smem_u32(&bars[0]), bar_done = smem_u32(&bars[1]);
  auto acc_full = [&](int k) { return smem_u32(&bars[2 + k]); };
  auto acc_empty = [&](int k) { return smem_u32(&bars[4 + k]); };
  const uint32_t mma_done = smem_u32(&bars[6]);

  if (tid == 0) {
    for (int k = 0; k < 7; ++k) mbar_init(smem_u32(&bars[k]), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < 8 * M; e += kPipeThreads) {
    const int tb = e / M, m = e - tb * M;
    const bool face = tb < 4;
    const int k = (face ? tb : tb - 4) * M + m;
    bc_f[e] = face ? b.face_f[k] : b.corner_f[k];
    bc_refl[e] = face ? b.face_refl[k] : b.corner_refl[k];
    bc_act[e] = face ? b.face_act[k] : b.corner_act[k];
    if (face) bc_wexit[e] = b.wexit[k];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * acc_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abrt = &abort_flag;
  const uint64_t pol_keep = policy_evict_last();

  if (tid < kGroup) {
    // ---------------- main loop group ----------------
    const int gtid = tid;
    constexpr uint32_t kFmt = BF ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                           (static_cast<uint32_t>(L.nrows_img >> 3) << 17) | (static_cast<uint32_t>(kMT >> 4) << 24);
    const size_t chunk_bytes = static_cast<size_t>(2) * L.nrows_img * 128;
    const unsigned char* Dimg = static_cast<const unsigned char*>(a.DyImg);
    unsigned char* Dhi = sm;
    unsigned char* Dlo = sm + L.n_mt * kTileBytes;
    unsigned char* Shi = sm + (X3 ? 2 : 1) * L.n_mt * kTileBytes;
    unsigned char* Slo = Shi + kTileBytes;
    constexpr int kItems = kNC * (KC / GV) / kGroup;          // 4
    float v[kItems][GV];
    auto load_chunk = [&](int tl, int q) {
      const int g = tl / tiles_per_group, t0 = (tl - g * tiles_per_group) * per_tile;
      const size_t goff = static_cast<size_t>(g) * a.plane;
      const int k0 = q * KC;
#pragma unroll
      for (int t = 0; t < kItems; ++t) {
        const int it = gtid + t * kGroup;
        const int c = it % kNC, grp = it / kNC;
        const int rc = c / M, m = c - rc * M;
        const int line = t0 + rc;
#pragma unroll
        for (int e = 0; e < GV; ++e) {
          const int k = k0 + grp * GV + e;
          // U of other tiles' columns is being rewritten by the epilogue
          // group: plain (coherent) loads
          v[t][e] = (line < nx && k < n) ? ld_hint(U + goff + (static_cast<size_t>(k) * nx + line) * M + m, pol_keep)
                                         : 0.f;
        }
      }
    };
    int it = 0, titer = 0, issued = 0;
    bool fine = true;
    if (static_cast<int>(blockIdx.x) < total) load_chunk(blockIdx.x, 0);
    for (int tl = blockIdx.x; tl < total && fine; tl += gridDim.x, ++titer) {
      const int b2 = titer & 1;
      for (int q = 0; q < L.n_kc; ++q, ++it) {
        // The leader waits for the previous chunk's MMAs (the stage is free
        // again) and starts the operator copy; the group follows its result.
        if (gtid == 0) {
          const bool ok0 = it < 1 || pipe_wait(bar_done, (it - 1) & 1, abrt, a.err);
          if (ok0) {
            bulk_copy(smem_u32(Dhi), Dimg + q * chunk_bytes, (X3 ? 2 : 1) * L.nrows_img * 128, bar_full);
            ++issued;
          }
          main_ok = ok0;
        }
        group_sync(1);
        if (!main_ok) {                                            // uniform over the group
          fine = false;
          break;
        }
#pragma unroll
        for (int t = 0; t < kItems; ++t) {
          const int itm = gtid + t * kGroup;
          const int c = itm % kNC, grp = itm / kNC;
          const float sc = -__ldg(a.eta + (c % M));
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
        group_sync(1);
        if (q + 1 < L.n_kc) load_chunk(tl, q + 1);
        else if (tl + static_cast<int>(gridDim.x) < total) load_chunk(tl + gridDim.x, 0);
        if (gtid == 0) {
          bool ok = true;
          if (q == 0) ok = pipe_wait(acc_empty(b2), ((titer >> 1) & 1) ^ 1, abrt, a.err);   // accumulator free
          ok = ok && pipe_wait(bar_full, it & 1, abrt, a.err);
          if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dSh = sw128_desc(smem_u32(Shi)), dSl = sw128_desc(smem_u32(Slo));
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
            mma_commit(bar_done);
            if (q == L.n_kc - 1) mma_commit(acc_full(b2));
          }
        }
      }
    }
    if (gtid == 0) {
      // every copy has landed and every MMA completed before the CTA leaves
      if (issued > 0) pipe_wait_plain(bar_full, (issued - 1) & 1, a.err);
      mma_commit(mma_done);
      pipe_wait_plain(mma_done, 0, a.err);
    }
  } else {
    // ---------------- epilogue group ----------------
    const int etid = tid - kGroup;
    const int quarter = warp & 3;                               // warps 8-11: TMEM lane quarters 0-3
    const float* srcs[kEpiArr] = {U, R, L1, L2, L3};
    const uint64_t pol_once = policy_evict_first();
    const int ring_len = 2 * ny + 2 * nx;
    const int nchunks = (ny + kRows - 1) / kRows;
    // this thread's item of a chunk: row t, four slab columns from c
    const int it_t = etid >> 5, it_c = (etid & 31) * 4;
    int titer = 0;
    for (int tl = blockIdx.x; tl < total; tl += gridDim.x, ++titer) {
      const int b2 = titer & 1;
      const int g = tl / tiles_per_group, t0 = (tl - g * tiles_per_group) * per_tile;
      const size_t goff = static_cast<size_t>(g) * a.plane;
      const int wcols = min(per_tile, nx - t0);
      const bool tile_has_xface = (t0 == 0) || (t0 + per_tile > nx - 1);
      auto issue_chunk = [&](int cc) {
        const int j = cc * kRows + it_t;
        if (it_c / M < wcols && j < ny) {
          const size_t gidx = goff + (static_cast<size_t>(j) * nx + t0) * M + it_c;
          float* base = ebuf + (cc % kNBuf) * kChunkFloats;
#pragma unroll
          for (int arr = 0; arr < kEpiArr; ++arr) {
            float* dst = base + (arr * kRows + it_t) * kNC + it_c;
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                         "l"(srcs[arr] + gidx), "l"(pol_once)
                         : "memory");
          }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      };
      // the data of the first chunks does not depend on the accumulator
      for (int cc = 0; cc < kNBuf - 1 && cc < nchunks; ++cc) issue_chunk(cc);
      if (etid == 0) epi_ok = pipe_wait(acc_full(b2), (titer >> 1) & 1, abrt, a.err);
      group_sync(2);
      const bool got = epi_ok;                                     // uniform over the group
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + b2 * acc_cols;
      for (int ci = 0; ci < nchunks; ++ci) {
        const int j0c = ci * kRows;
        if (ci + kNBuf - 1 < nchunks) issue_chunk(ci + kNBuf - 1);
        if (warp < 12) {                                          // warps 8-11 read their TMEM quarter
          float acc[8];
          tmem_ld8(tbase + j0c, acc);
          const int c = 32 * quarter + lane;
#pragma unroll
          for (int t = 0; t < kRows; ++t) acc_s[t * kNC + c] = acc[t];
        }
        cp_async_wait(min(kNBuf - 1, nchunks - 1 - ci));
        group_sync(2);
        // uniform over the group (the barriers below depend on it)
        const bool chunk_bnd = j0c == 0 || j0c + kRows > ny - 1 || tile_has_xface;
        const float* buf = ebuf + (ci % kNBuf) * kChunkFloats;
        {
          const int t = it_t, c = it_c;
          const int w = c / M, j = j0c + t, i = t0 + w;
          if (got && w < wcols && j < ny) {
            const float4 u4 = *reinterpret_cast<const float4*>(buf + (0 * kRows + t) * kNC + c);
            const float4 r4 = *reinterpret_cast<const float4*>(buf + (1 * kRows + t) * kNC + c);
            const float4 p4 = *reinterpret_cast<const float4*>(buf + (2 * kRows + t) * kNC + c);
            const float4 q4 = *reinterpret_cast<const float4*>(buf + (3 * kRows + t) * kNC + c);
            const float4 s4 = *reinterpret_cast<const float4*>(buf + (4 * kRows + t) * kNC + c);
            const float4 ac = *reinterpret_cast<const float4*>(acc_s + t * kNC + c);
            float4 lk, un;
            lk.x = r4.x + ac.x; lk.y = r4.y + ac.y; lk.z = r4.z + ac.z; lk.w = r4.w + ac.w;
            un.x = ab4_node(a.cdt, lk.x, p4.x, q4.x, s4.x, u4.x);
            un.y = ab4_node(a.cdt, lk.y, p4.y, q4.y, s4.y, u4.y);
            un.z = ab4_node(a.cdt, lk.z, p4.z, q4.z, s4.z, u4.z);
            un.w = ab4_node(a.cdt, lk.w, p4.w, q4.w, s4.w, u4.w);
            const size_t gidx = goff + (static_cast<size_t>(j) * nx + t0) * M + c;
            *reinterpret_cast<float4*>(L3 + gidx) = lk;
            const bool bnd = i == 0 || i == nx - 1 || j == 0 || j == ny - 1;
            if (chunk_bnd) *reinterpret_cast<float4*>(un_s + t * kNC + c) = un;
            if (!bnd) st_hint(U + gidx, un, pol_keep);   // u^{k+1} is read by the next x-pass
          }
        }
        if (chunk_bnd) {
          // eq. (RTE) third line on the chunk's boundary nodes from the pre-BC
          // node values: the x-face column on every row, the y-face rows on
          // every column (corners once, as x-face cells).
          group_sync(2);
          const int xcol = (t0 == 0) ? 0 : (t0 + wcols - 1 == nx - 1 ? wcols - 1 : -1);
          const int yrow0 = (j0c == 0) ? 0 : -1;
          const int yrow1 = (ny - 1 >= j0c && ny - 1 < j0c + kRows) ? ny - 1 - j0c : -1;
          const int rows = min(kRows, ny - j0c);
          const int n_xcells = xcol >= 0 ? rows : 0;
          const int n_ycells = ((yrow0 >= 0) + (yrow1 >= 0 && yrow1 != yrow0)) * wcols;
          for (int e = etid; e < (n_xcells + n_ycells) * M; e += kGroup) {
            const int cidx = e / M, m = e - cidx * M;
            int t, w;
            if (cidx < n_xcells) {
              t = cidx;
              w = xcol;
            } else {
              const int yc = cidx - n_xcells;
              t = (yc / wcols == 0 && yrow0 >= 0) ? yrow0 : yrow1;
              w = yc % wcols;
              if (xcol >= 0 && w == xcol) continue;
            }
            const int j = j0c + t, i = t0 + w;
            if (!got) continue;
            const bool lf = i == 0, rt = i == nx - 1, bt = j == 0, tp = j == ny - 1;
            int tb;
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
                qv = fmaf(1.0f - fco, __ldg(b.rho + (static_cast<size_t>(g) * b.rho_len + src_step) * ring_len + node),
                          qv);
              val = fmaf(fco, pre[bc_refl[tb * M + m]], qv);
            }
            bc_s[t * kNC + w * M + m] = val;
            U[goff + (static_cast<size_t>(j) * nx + i) * M + m] = val;
          }
          group_sync(2);
          // exitance of eq. (OpMed): one thread per (boundary node, face), in
          // a fixed summation order
          if (got && b.ring_out && ring_step >= 0) {
            float* ro = b.ring_out + (static_cast<size_t>(g) * b.ring_steps + ring_step) * ring_len;
            for (int e = etid; e < kRows * wcols * 2; e += kGroup) {
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
        group_sync(2);   // acc_s / un_s / bc_s and the ring slot are reused
      }
      // the accumulator is free again
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      group_sync(2);
      if (etid == 0) mbar_arrive(acc_empty(b2));
      if (!got) break;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // no copy in flight when the CTA leaves
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * acc_cols));
}

int pipe_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int PREC, int MM>
cudaError_t launch_pipe(const StepArgs& a, const BoundaryArgs& b, float* U, const float* R, const float* L1,
                        const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  using K = Kind<PREC>;
  const TcLayout L(a.ny, K::X3, K::KC);
  const size_t smem = 1024 + static_cast<size_t>(L.stage_bytes) + kEpiSmem;
  if (smem > static_cast<size_t>(kSmemLimit)) return cudaErrorInvalidConfiguration;
  static bool attr = false;
  if (!attr) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, tc_ypass_pipe<PREC, MM>);
    if (e != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < kPipeThreads) return cudaErrorLaunchOutOfResources;
    e = cudaFuncSetAttribute(tc_ypass_pipe<PREC, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int per_tile = kNC / MM;
  const int total = (a.nx + per_tile - 1) / per_tile * a.G;
  const int grid = total < pipe_sm_count() ? total : pipe_sm_count();
  tc_ypass_pipe<PREC, MM><<<grid, kPipeThreads, smem, s>>>(a, b, U, R, L1, L2, L3, src_step, ring_step);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_pipe_m(const StepArgs& a, const BoundaryArgs& b, float* U, const float* R, const float* L1,
                          const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  if (a.M == 16) return launch_pipe<PREC, 16>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
  if (a.M == 32) return launch_pipe<PREC, 32>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
  return launch_pipe<PREC, 64>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
}

}  // namespace

bool tc_pipe_supported(const StepArgs& a) {
  return a.tc_mode >= 1 && a.tc_mode <= 4 && a.ny <= 256 && (a.M == 16 || a.M == 32 || a.M == 64);
}

cudaError_t launch_ypass_pipe(const StepArgs& a, const BoundaryArgs& b, float* U, const float* R, const float* L1,
                              const float* L2, float* L3, int src_step, int ring_step, cudaStream_t s) {
  switch (a.tc_mode) {
    case 1: return launch_pipe_m<1>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
    case 2: return launch_pipe_m<2>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
    case 3: return launch_pipe_m<3>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
    default: return launch_pipe_m<4>(a, b, U, R, L1, L2, L3, src_step, ring_step, s);
  }
}


}  // namespace rte_kern
