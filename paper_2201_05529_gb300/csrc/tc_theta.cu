// Tensor-core theta contraction of the fast path (App. A.2 (e-f)) on sm_103a: tcgen05 + TMEM.
//
//   theta[(u,p),(v,q)] = sum_c (R_L[u,(p,c)] lambda_c) L_R[(c,q),v]      (complex)
//   D[(u,p'),(q',v)]   = sum_{p,q} G[(p' q'),(p q)] theta[(u,p),(v,q)]   (gate in the epilogue)
//
// Complex products use the 3M scheme (T1 = Ar Br, T2 = Ai Bi, T3 = (Ar+Ai)(Br+Bi);
// Re = T1 - T2, Im = T3 - T1 - T2), each real product split into hi/lo parts for accuracy:
//   TF32x3: x = hi + lo with hi = tf32(x), lo = tf32(x - hi); X Y ~ Xh Yh + Xh Yl + Xl Yh
//   BF16x3: the same with bf16 parts;  TF32x1: Xh Yh only.
// A pack kernel writes every operand plane already in the tcgen05 canonical K-major no-swizzle
// layout (8-row x 16-byte core matrices; K-groups of the 128-row tile are contiguous), so one
// cp.async.bulk per plane and K-chunk stages a tile in shared memory. One elected thread issues
// tcgen05.mma (M = 128, N = 128, FP32 accumulators in TMEM: three 128-column accumulators); the
// four warps read TMEM back (tcgen05.ld 32x32b) and apply the 16x16 gate across 4-lane groups in
// FP32 (theta is FP32-accurate; an FP64 gate would cost ~1M DFMA per tile at GB300's FP64 rate).
// Every mbarrier wait has an iteration limit: on expiry the kernel records ST_TIMEOUT, frees its
// TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.h"

namespace ptk {

namespace {

constexpr int TM = 128;             // tile rows (u,p)
constexpr int TN = 128;             // tile cols (v,q)
constexpr int TC_THREADS = 128;
constexpr int PLANES = 6;           // Ar_h, Ar_l, Ai_h, Ai_l, As_h, As_l (As = Ar + Ai)
constexpr long long SPIN_LIMIT = 20000000;  // mbarrier polls before giving up

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

// packed operand geometry (elements of 4 bytes for tf32, 2 bytes for bf16)
template <bool BF16> struct Geo {
  static constexpr int EB = BF16 ? 2 : 4;           // element bytes
  static constexpr int KG = 16 / EB;                // elements per core-matrix row (K group)
  static constexpr int KC = BF16 ? 64 : 32;         // K elements per chunk
  static constexpr int KSTEP = BF16 ? 16 : 8;       // K per MMA instruction
  static constexpr uint32_t CHUNK_BYTES = (uint32_t)TM * KC * EB;   // one plane, one chunk, one tile
};

}  // namespace

// ------------------------------------------------------------------ packing (FP64 -> split planes)
// Operand A rows (u,p) = u*4+p, K index c: A[(u,p), c] = R_L[u, p*chc + c] lambda_c.
// Operand B rows (v,q) = v*4+q, K index c: B[(v,q), c] = L_R[(c*4+q), v].
// Output per bond: [row tile][K chunk][plane][K group][128 rows][KG elements] (bulk-copy ready).
template <bool BF16>
__global__ void k_tc_pack(Tables T, const BondWork* work, int n_work, int which, int rt_cap, int kc_cap) {
  using G = Geo<BF16>;
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const int BL = W.lam_l, BC = BL + 1, BR = BL + 2;
  const int sL = W.site_l, sR = sL + 1;
  const int chl = T.lam_chi[BL], chc = T.lam_chi[BC], chr = T.lam_chi[BR];
  const int kL = T.site_kappa[sL], kR = T.site_kappa[sR];
  const int mL = chl * kL, nL = 4 * chc, mR = 4 * chc, nR = kR * chr;
  const bool qrL = mL > nL, lqR = nR > mR;
  const int rL = qrL ? nL : mL, rR = lqR ? mR : nR;
  const int rows = which == 0 ? 4 * rL : 4 * rR;
  const int n_rt = (rows + TM - 1) / TM, n_kc = (chc + G::KC - 1) / G::KC;
  if (n_rt > rt_cap || n_kc > kc_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  const double* lamC = T.lam_ptr[BC];
  const double2* RLp = qrL ? W.RL : W.QL;
  const int ldRL = qrL ? nL : mL;
  const double2* LRp = lqR ? W.LR : W.QR;
  const int ldLR = lqR ? mR : nR;
  unsigned char* out = (unsigned char*)(which == 0 ? W.TA : W.TB);
  const size_t tile_bytes = (size_t)PLANES * G::CHUNK_BYTES;
  const size_t total = (size_t)n_rt * n_kc * TM * G::KC;     // (tile, chunk, row, k) elements
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % G::KC);
    size_t t = idx / G::KC;
    const int m = (int)(t % TM);
    t /= TM;
    const int kc = (int)(t % n_kc);
    const int rt = (int)(t / n_kc);
    const int row = rt * TM + m, c = kc * G::KC + k;
    double2 v = make_double2(0.0, 0.0);
    if (row < rows && c < chc) {
      if (which == 0) {
        const int u = row >> 2, p = row & 3;
        v = RLp[u + (size_t)(p * chc + c) * ldRL];
        v.x *= lamC[c];
        v.y *= lamC[c];
      } else {
        const int vv = row >> 2, q = row & 3;
        const double2 x = LRp[vv + (size_t)(c * 4 + q) * ldLR];   // L_R(row, v) = conj(...)
        v = make_double2(x.x, -x.y);
      }
    }
    const double comps[3] = {v.x, v.y, v.x + v.y};
    unsigned char* base = out + ((size_t)rt * n_kc + kc) * tile_bytes;
    const size_t in_plane = ((size_t)(k / G::KG) * TM + m) * 16 + (size_t)(k % G::KG) * G::EB;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float f = (float)comps[q];
      unsigned char* ph = base + (size_t)(2 * q) * G::CHUNK_BYTES + in_plane;
      unsigned char* pl = base + (size_t)(2 * q + 1) * G::CHUNK_BYTES + in_plane;
      if (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        const __nv_bfloat16 l = __float2bfloat16_rn((float)(comps[q] - (double)__bfloat162float(h)));
        *(__nv_bfloat16*)ph = h;
        *(__nv_bfloat16*)pl = l;
      } else {
        // tf32 hi: round to 10 mantissa bits; lo: the remainder (also consumed as tf32)
        uint32_t hb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(f));
        const float h = __uint_as_float(hb);
        const float l = (float)(comps[q] - (double)h);
        uint32_t lb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(l));
        *(uint32_t*)ph = hb;
        *(uint32_t*)pl = lb;
      }
    }
  }
}

// ------------------------------------------------------------------ GEMM + gate epilogue
// grid: (row tiles of A) x (row tiles of B) x items; 128 threads.
template <bool BF16, int NSPLIT>
__global__ void __launch_bounds__(TC_THREADS) k_tc_theta(Tables T, const BondWork* work, int n_work, int rt_cap,
                                                         int kc_cap) {
  using G = Geo<BF16>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ float2 gate_s[256];           // the 16x16 gate in FP32 (theta is FP32-accurate)
  const int w = blockIdx.z;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const int BL = W.lam_l, BC = BL + 1, BR = BL + 2;
  const int sL = W.site_l, sR = sL + 1;
  const int chl = T.lam_chi[BL], chc = T.lam_chi[BC], chr = T.lam_chi[BR];
  const int kL = T.site_kappa[sL], kR = T.site_kappa[sR];
  const int mL = chl * kL, nL = 4 * chc, mR = 4 * chc, nR = kR * chr;
  const bool qrL = mL > nL, lqR = nR > mR;
  const int rL = qrL ? nL : mL, rR = lqR ? mR : nR;
  const int mD = 4 * rL, nD = 4 * rR;
  const int n_kc = (chc + G::KC - 1) / G::KC;
  const int rt = blockIdx.x, ct = blockIdx.y;
  const bool fits = (mD + TM - 1) / TM <= rt_cap && (nD + TN - 1) / TN <= rt_cap && n_kc <= kc_cap &&
                    mD <= W.mD_cap && nD <= W.nD_cap;
  const bool tr = mD < nD;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    W.info[0] = fits ? mD : 0;          // 0: the SVD and the following stages skip this bond
    W.info[1] = fits ? nD : 0;
    W.info[2] = tr ? 1 : 0;
  }
  if (!fits || rt * TM >= mD || ct * TN >= nD) return;     // outside the live matrix
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* sA = smem;                                   // PLANES chunks of A
  unsigned char* sB = smem + PLANES * G::CHUNK_BYTES;         // PLANES chunks of B
  for (int i = tid; i < 256; i += blockDim.x)
    gate_s[i] = make_float2((float)W.gate[i].x, (float)W.gate[i].y);
  if (tid == 0) {
    mbar_init(&bar_load, 1);
    mbar_init(&bar_mma, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_s))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const size_t tile_bytes = (size_t)PLANES * G::CHUNK_BYTES;
  const unsigned char* gA = (const unsigned char*)W.TA;
  const unsigned char* gB = (const unsigned char*)W.TB;
  const uint32_t idesc = instr_desc(BF16 ? 1u : 2u, TM, TN);
  const uint32_t LBO = TM * 16, SBO = 128;
  uint32_t phase = 0;
  for (int kc = 0; kc < n_kc; ++kc) {
    if (tid == 0) {
      mbar_expect_tx(&bar_load, (uint32_t)(2 * tile_bytes));
      const unsigned char* srcA = gA + ((size_t)rt * n_kc + kc) * tile_bytes;
      const unsigned char* srcB = gB + ((size_t)ct * n_kc + kc) * tile_bytes;
      for (int pl = 0; pl < PLANES; ++pl) {
        bulk_g2s(sA + pl * G::CHUNK_BYTES, srcA + pl * G::CHUNK_BYTES, G::CHUNK_BYTES, &bar_load);
        bulk_g2s(sB + pl * G::CHUNK_BYTES, srcB + pl * G::CHUNK_BYTES, G::CHUNK_BYTES, &bar_load);
      }
      bool ok = mbar_wait(&bar_load, phase);
      bool mma_issued = false;
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // T1 = Ar Br (cols 0..127), T2 = Ai Bi (cols 128..255), T3 = As Bs (cols 256..383)
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
          const unsigned char* ah = sA + (2 * comp) * G::CHUNK_BYTES;
          const unsigned char* al = sA + (2 * comp + 1) * G::CHUNK_BYTES;
          const unsigned char* bh = sB + (2 * comp) * G::CHUNK_BYTES;
          const unsigned char* bl = sB + (2 * comp + 1) * G::CHUNK_BYTES;
          const uint32_t d = tmem + comp * TN;
          for (int ks = 0; ks < G::KC / G::KSTEP; ++ks) {
            const uint32_t koff = ks * 2 * LBO;              // two 16-byte K groups per MMA
            const bool first = (kc == 0 && ks == 0);
            mma<BF16>(d, smem_desc(ah + koff, LBO, SBO), smem_desc(bh + koff, LBO, SBO), idesc, !first);
            if (NSPLIT >= 3) {
              mma<BF16>(d, smem_desc(ah + koff, LBO, SBO), smem_desc(bl + koff, LBO, SBO), idesc, true);
              mma<BF16>(d, smem_desc(al + koff, LBO, SBO), smem_desc(bh + koff, LBO, SBO), idesc, true);
            }
          }
        }
        mma_commit(&bar_mma);
        mma_issued = true;
        ok = mbar_wait(&bar_mma, phase);
      }
      if (!ok) {
        // give the copies / MMAs still in flight one more bounded wait before leaving
        atomicOr(T.status, ST_TIMEOUT);
        abort_s = 1;
        if (mma_issued) mbar_wait(&bar_mma, phase);
        else mbar_wait(&bar_load, phase);
      }
    }
    __syncthreads();
    phase ^= 1;
    if (abort_s) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!abort_s) {
    // epilogue: thread = row (u,p) of the tile; 8 columns (2 v x 4 q) per TMEM load
    const int row = rt * TM + warp * 32 + lane;
    const int u = row >> 2, p = row & 3;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < TN; c0 += 8) {
      float t1[8], t2[8], t3[8];
      tmem_ld8(tmem + lane_base + 0 * TN + c0, t1);
      tmem_ld8(tmem + lane_base + 1 * TN + c0, t2);
      tmem_ld8(tmem + lane_base + 2 * TN + c0, t3);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int col = ct * TN + c0 + half * 4;             // (v, q=0) of this group
        const int v = col >> 2;
        // theta[(u,p),(v,q)] for q = 0..3 held by this lane; lanes 4k..4k+3 hold p = 0..3
        float re[4], im[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float a = t1[half * 4 + q], b = t2[half * 4 + q], s = t3[half * 4 + q];
          re[q] = a - b;
          im[q] = s - a - b;
        }
        float2 out[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) out[qq] = make_float2(0.f, 0.f);
        const int base_lane = lane & ~3;
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float tr_ = __shfl_sync(0xffffffffu, re[q], base_lane + pp);
            const float ti_ = __shfl_sync(0xffffffffu, im[q], base_lane + pp);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const float2 g = gate_s[(p * 4 + qq) * 16 + pp * 4 + q];
              out[qq].x = fmaf(g.x, tr_, fmaf(-g.y, ti_, out[qq].x));
              out[qq].y = fmaf(g.x, ti_, fmaf(g.y, tr_, out[qq].y));
            }
          }
        }
        if (row < mD && v < rR) {
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int Drow = u * 4 + p, Dcol = qq * rR + v;
            if (!tr) W.A[Drow + (size_t)Dcol * mD] = make_double2(out[qq].x, out[qq].y);
            else W.A[Dcol + (size_t)Drow * nD] = make_double2(out[qq].x, -out[qq].y);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ launchers
size_t tc_pack_bytes(int rows_cap, int k_cap, int precision) {
  const bool bf = precision == 2;
  const int KC = bf ? Geo<true>::KC : Geo<false>::KC;
  const size_t chunk = bf ? Geo<true>::CHUNK_BYTES : Geo<false>::CHUNK_BYTES;
  const int rt = (rows_cap + TM - 1) / TM, kc = (k_cap + KC - 1) / KC;
  return (size_t)rt * kc * PLANES * chunk;
}

void tc_caps(int rows_cap, int k_cap, int precision, int* rt_cap, int* kc_cap) {
  const bool bf = precision == 2;
  const int KC = bf ? Geo<true>::KC : Geo<false>::KC;
  *rt_cap = (rows_cap + TM - 1) / TM;
  *kc_cap = (k_cap + KC - 1) / KC;
}

void launch_tc_theta(const Tables& T, const BondWork* work, int n_work, int rt_cap, int kc_cap, int precision,
                     cudaStream_t st) {
  const int gx = 64;
  const bool bf = precision == 2;
  // operand planes plus a 32 KB guard so every descriptor-addressed read stays inside the allocation
  const size_t smem = 2 * (size_t)PLANES * (bf ? Geo<true>::CHUNK_BYTES : Geo<false>::CHUNK_BYTES) + 32768;
  if (bf) {
    k_tc_pack<true><<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, 0, rt_cap, kc_cap);
    k_tc_pack<true><<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, 1, rt_cap, kc_cap);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_tc_theta<true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    k_tc_theta<true, 3><<<dim3(rt_cap, rt_cap, n_work), TC_THREADS, smem, st>>>(T, work, n_work, rt_cap, kc_cap);
  } else {
    k_tc_pack<false><<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, 0, rt_cap, kc_cap);
    k_tc_pack<false><<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, 1, rt_cap, kc_cap);
    static bool attr3 = false, attr1 = false;
    if (precision == 3) {
      if (!attr1) {
        cudaFuncSetAttribute(k_tc_theta<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr1 = true;
      }
      k_tc_theta<false, 1><<<dim3(rt_cap, rt_cap, n_work), TC_THREADS, smem, st>>>(T, work, n_work, rt_cap, kc_cap);
    } else {
      if (!attr3) {
        cudaFuncSetAttribute(k_tc_theta<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr3 = true;
      }
      k_tc_theta<false, 3><<<dim3(rt_cap, rt_cap, n_work), TC_THREADS, smem, st>>>(T, work, n_work, rt_cap, kc_cap);
    }
  }
}

}  // namespace ptk
