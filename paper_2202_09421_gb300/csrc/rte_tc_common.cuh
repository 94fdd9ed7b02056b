// Inline-PTX helpers and operand layouts shared by the tcgen05 kernels
// (internal to the library): shared-memory matrix descriptors for the
// K-major 128-byte-swizzle layout, mbarriers, bulk copies, MMA issue,
// tensor-memory loads and the split of FP32 values into TF32 / BF16 hi + lo.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "rte_kernels.cuh"

namespace rte_kern {
namespace tc {

constexpr int kNC = 128;          // slab columns per tile (MMA N)
constexpr int kMT = 128;          // output positions per accumulator tile (MMA M)
constexpr int kThreads = 256;
constexpr int kTileBytes = 128 * 128;   // one 128-row x 128-byte operand tile
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any one wait

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr float kAB0 = 55.0f / 24.0f, kAB1 = -59.0f / 24.0f, kAB2 = 37.0f / 24.0f,
                kAB3 = -9.0f / 24.0f;

// AB4 update of one node value (eq. RTEAB4): u + c dt (55 L^k - 59 L^{k-1}
// + 37 L^{k-2} - 9 L^{k-3}) / 24 with a fixed FMA order, so that every
// y-pass schedule rounds it the same way.
__device__ __forceinline__ float ab4_node(float cdt, float lk, float l1, float l2, float l3, float u) {
  return fmaf(cdt, fmaf(kAB3, l3, fmaf(kAB2, l2, fmaf(kAB1, l1, kAB0 * lk))), u);
}

// Operand kinds of the precision modes (rte.h): 1 3xTF32, 2 TF32, 3 bf16x3,
// 4 BF16.  KC = K positions per 128-byte row, GV = values per 16-byte group.
template <int PREC>
struct Kind {
  static constexpr bool BF = PREC == 3 || PREC == 4;
  static constexpr bool X3 = PREC == 1 || PREC == 3;
  static constexpr int KC = BF ? 64 : 32;
  static constexpr int GV = BF ? 8 : 4;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row group
// stride 1024 B (start address in 16-byte units).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFF) | (static_cast<uint64_t>(1024 >> 4) << 32) |
         (static_cast<uint64_t>(1) << 46) | (static_cast<uint64_t>(2) << 61);
}

// Byte offset of the 16-byte group grp of row `row` in a K-major
// 128-byte-swizzle tile.
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

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

template <bool BF>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
  if constexpr (BF)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  else
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

// Two bf16 values in one word, the lower K index in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float k0, float k1) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(k0))) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(k1))) << 16);
}

// Splits the 8 values s*v[e] of one 16-byte group into bf16 hi and lo words.
__device__ __forceinline__ void split8_bf16(const float v[8], float s, uint4& hi, uint4& lo) {
  float h[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const float x = s * v[e];
    h[e] = __bfloat162float(__float2bfloat16_rn(x));
    l[e] = x - h[e];
  }
  hi = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
  lo = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
}

// L2 eviction priorities (createpolicy): the slab values are read again by
// the epilogue of the same CTA, the epilogue's other streams only once.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_hint(float* ptr, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_hint1(float* ptr, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(ptr), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ float ld_hint(const float* ptr, uint64_t pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
  return v;
}

// 32-byte global accesses (sm_100 and later): whole 32-byte sectors per
// thread, so a warp that walks 32 nodes of 128 B leaves no half-written
// sectors for L2 to merge.  Addresses are 32-byte aligned.
__device__ __forceinline__ void ld8_nc(const float* ptr, float* v) {
  asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(ptr));
}
__device__ __forceinline__ void st8_hint(float* ptr, const float* v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8}, %9;" ::"l"(ptr), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "l"(pol)
               : "memory");
}

// 32 lanes x 8 columns of 32-bit words from tensor memory.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 8; ++t) v[t] = __uint_as_float(r[t]);
}

// x-pass epilogue at one node (Sec. 4.1, eq. RTEAB4L): acc[m] holds the
// streaming term -xi_m (D_x u)_m from the tensor cores; on return
//   acc[m] = acc[m] - (a + b) u_m + sum_d p_d (b u_{(m - d) mod M}),
// the circulant form of b P~u with p_d = P~[d][0] (P~[m][q] = p_{(m - q) mod M},
// symmetric circulant).  The weights are read from shared memory, one
// broadcast per d for all M outputs.  The sum runs over d in order for every
// m.  PAIRED issues it on pairs of outputs (m, m + 1) with paired FP32 FMAs;
// each half is the scalar fmaf, so both forms give the same bits (for even d
// the pair reads (b u_j, b u_{j+1}) at even j, for odd d at odd j, so b u is
// kept in both pairings).  Overwrites uu with b u.
template <int MM, bool PAIRED = false>
__device__ __forceinline__ void xpass_node_rhs(float (&acc)[MM], float (&uu)[MM], const float* psm, float ab,
                                               float bb) {
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = fmaf(-ab, uu[m], acc[m]);
#pragma unroll
  for (int m = 0; m < MM; ++m) uu[m] *= bb;
  if constexpr (!PAIRED) {
#pragma unroll
    for (int d = 0; d < MM; ++d) {
      const float pd = psm[d];
#pragma unroll
      for (int m = 0; m < MM; ++m) acc[m] = fmaf(pd, uu[(m - d + MM) % MM], acc[m]);
    }
  } else {
    constexpr int H = MM / 2;
    float2 ev[H], od[H], ac[H];          // ev[k] = (bu_2k, bu_2k+1), od[k] = (bu_2k+1, bu_2k+2 mod M)
#pragma unroll
    for (int k = 0; k < H; ++k) {
      ev[k] = make_float2(uu[2 * k], uu[2 * k + 1]);
      od[k] = make_float2(uu[2 * k + 1], uu[(2 * k + 2) % MM]);
      ac[k] = make_float2(acc[2 * k], acc[2 * k + 1]);
    }
#pragma unroll
    for (int d = 0; d < MM; ++d) {
      const float pd = psm[d];
      const float2 p2 = make_float2(pd, pd);
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int j = (2 * k - d + MM) % MM;
        ac[k] = __ffma2_rn(p2, (d & 1) ? od[(j - 1) / 2] : ev[j / 2], ac[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
      acc[2 * k] = ac[k].x;
      acc[2 * k + 1] = ac[k].y;
    }
  }
}

struct TcLayout {
  int n, n_mt, n_kc, nrows_img, stage_bytes, tmem_cols;
  __host__ __device__ TcLayout(int n_, bool x3, int kc) : n(n_) {
    n_mt = (n + kMT - 1) / kMT;
    n_kc = (n + kc - 1) / kc;
    nrows_img = n_mt * kMT;
    stage_bytes = (x3 ? 2 : 1) * (n_mt + 1) * kTileBytes;   // D tiles + slab tile, hi (+ lo)
    tmem_cols = n_mt == 1 ? 128 : n_mt == 2 ? 256 : 512;    // power of two >= n_mt * 128
  }
};

}  // namespace tc
}  // namespace rte_kern
