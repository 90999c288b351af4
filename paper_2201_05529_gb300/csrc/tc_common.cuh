// tcgen05 building blocks shared by the tensor-core GEMMs of the fast path (tc_theta.cu, tc_zgemm.cu):
// mbarrier waits with an iteration limit, bulk global -> shared copies, shared-memory and instruction
// descriptors, the MMA and the TMEM load, the packed-operand geometry, and the splitting of an FP64
// value into TF32/BF16 pieces (natural split) or fixed-point BF16 slices (Ozaki, Ogita, Oishi and
// Rump's error-free splitting of matrix products).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace ptk {
namespace tcx {

constexpr int TMA = 128;            // A tile rows
constexpr int TNB = 64;             // B tile rows (columns of the product) = output tile columns
constexpr int TC_THREADS = 128;
constexpr int MAX_STAGES = 3;     // shared-memory stages of the K pipeline (2 for six slices: 227 KB)
template <int NS> struct Stages { static constexpr int value = NS >= 6 ? 2 : MAX_STAGES; };
constexpr int MAX_ITEMS = 1024;
constexpr uint32_t ROW_BYTES = 32;  // one K step of one row: 8 tf32 or 16 bf16 (two 16-byte K groups)
constexpr long long SPIN_LIMIT = 20000000;  // mbarrier polls before giving up
constexpr uint32_t NEG_A = 1u << 13;        // instruction descriptor: negate matrix A

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// true when the phase with the given parity has completed; false after SPIN_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// shared memory matrix descriptor: K-major, no swizzle, LBO = K-group stride, SBO = 8-row stride
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (a >> 4) & 0x3FFFull;
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;          // descriptor version for sm_100-class tcgen05
  return d;                        // base offset 0, layout type 0 = SWIZZLE_NONE
}

// instruction descriptor for kind::tf32 (ab_fmt = 2) or kind::f16 with bf16 inputs (ab_fmt = 1):
// FP32 accumulator, K-major A and B, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t instr_desc(uint32_t ab_fmt, int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format F32
  d |= ab_fmt << 7;                // A format
  d |= ab_fmt << 10;               // B format
  d |= (uint32_t)(N >> 3) << 17;
  d |= (uint32_t)(M >> 4) << 24;
  return d;
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
  const uint32_t en = acc ? 1u : 0u;
  if (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(en)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(en)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// packed operand geometry: one K step per chunk, 32 bytes of each row
template <bool BF16> struct Geo {
  static constexpr int EB = BF16 ? 2 : 4;       // element bytes
  static constexpr int KG = 16 / EB;            // elements per 16-byte K group
  static constexpr int KSTEP = 2 * KG;          // K per MMA instruction (8 tf32, 16 bf16)
};

__host__ __device__ __forceinline__ int cdiv(int a, int b) { return (a + b - 1) / b; }

// capacity layout of one packed operand: [row tile][K step][plane][K group][rows][16 B],
// then one int exponent per (padded) row
struct PackCap {
  int tiles, ksteps;
  size_t plane_bytes, exp_off, total;
};

__host__ __device__ __forceinline__ PackCap pack_cap(int rows_cap, int k_cap, int tile_rows, int kstep, int ns) {
  PackCap c;
  c.tiles = cdiv(rows_cap, tile_rows);
  c.ksteps = cdiv(k_cap, kstep);
  c.plane_bytes = (size_t)tile_rows * ROW_BYTES;
  c.exp_off = (size_t)c.tiles * c.ksteps * 2 * ns * c.plane_bytes;
  c.total = c.exp_off + sizeof(int) * (size_t)c.tiles * tile_rows;
  return c;
}

// the NS pieces of x (already scaled by 2^-e for slices) as TF32 or BF16 bit patterns
template <bool BF16, int NS, bool SLICE>
__device__ __forceinline__ void pieces(double x, int b, uint32_t* out) {
  if (SLICE) {
    // fixed-point slices: a_i = rint(r 2^b), r <- r 2^b - a_i; slice value a_i 2^(-b(i+1))
    double r = x;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      const double t = ldexp(r, b);
      const double a = rint(t);
      r = t - a;
      const float s = (float)ldexp(a, -b * (i + 1));      // exact: |a| <= 2^b <= 2^8
      out[i] = BF16 ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(s)) : __float_as_uint(s);
    }
  } else {
    double r = x;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      const float f = (float)r;
      if (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        out[i] = (uint32_t)__bfloat16_as_ushort(h);
        r -= (double)__bfloat162float(h);
      } else {
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(f));
        out[i] = hb;
        r -= (double)__uint_as_float(hb);
      }
    }
  }
}

// slice width: the level-0 sum over K of 2 products of |a| <= 2^b stays below 2^24
__device__ __forceinline__ int slice_bits(int K) { return K <= 512 ? 7 : (K <= 2048 ? 6 : 5); }

// exponent e with max |x| < 2^e (0 for an all-zero row)
__device__ __forceinline__ int row_exponent(double m) {
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);          // m = f 2^e, f in [0.5, 1)
  return e;
}

}  // namespace tcx
}  // namespace ptk
