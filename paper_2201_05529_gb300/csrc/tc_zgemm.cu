// Batched complex GEMM on the tensor cores with an FP64-class result, for the large products of
// the fast path's bond SVD (App. A.2): the randomized range finder's sketches D Omega and
// D^H Q, the projection Q^H D, and the singular vectors of D built from those of the small factor.
//
//   C_i = opA(A_i) opB(B_i)        (M_i x N_i, inner dimension K_i; op = as stored, T or H)
//
// for a list of items whose live dims sit in device memory: a plan kernel writes the list from the
// bonds' info words, so one CUDA graph replays every step unchanged.
//
// Arithmetic (the error-free splitting of Ozaki, Ogita, Oishi and Rump, as in the theta GEMM):
// every row of opA(A) and every column of opB(B) is scaled by a power of two 2^-e so its entries
// lie in (-1, 1), then cut into six BF16 fixed-point slices a_s 2^(-7(s+1)) with integer
// |a_s| <= 2^7. Slice products are exact in FP32, and K is accumulated in chunks of 512 so that the
// level-0 and level-1 sums of a chunk stay integers below 2^24: the tensor cores' FP32 accumulation
// is exact there, the deeper levels carry only their own rounding, and the chunks are added in
// FP64 in the output. Products of slice
// pairs (s, t) accumulate in TMEM by level min(s + t, 3), real and imaginary parts separately
// (Re = Ar Br - Ai Bi via the MMA's negate-A bit, Im = Ar Bi + Ai Br); the epilogue adds the
// levels in FP64 and applies 2^(e_row + e_col). The result is accurate to ~1e-12 of the scale
// of the rows and columns it combines (per 512-long chunk of K).
//
// Data flow: two passes per operand (row exponents, then the 12 slice planes in the tcgen05
// K-major no-swizzle layout: A in 128-row tiles, B in 64-column tiles, one 16-element K step per
// block, so one cp.async.bulk stages each), then one persistent GEMM launch (one CTA per SM) that
// walks the live 128 x 64 output tiles of all items with a two-stage bulk-copy / MMA pipeline.
// Every mbarrier wait is bounded: on expiry the kernel records ST_TIMEOUT in *status, waits
// (bounded) for its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"
#include "tc_common.cuh"

namespace ptk {

using namespace tcx;

namespace {

constexpr int ZNS = 6;                        // BF16 slices per value
constexpr int ZBITS = 7;                      // slice width
constexpr int ZKC_STEPS = 32;                 // K steps (16 each) per exact accumulation chunk: K = 512
using ZG = Geo<true>;                         // BF16 geometry: 16-element K steps

__host__ __device__ __forceinline__ PackCap zcap(const ZGemmItem& it, int which) {
  return which == 0 ? pack_cap(it.cap_m, it.cap_k, TMA, ZG::KSTEP, ZNS)
                    : pack_cap(it.cap_n, it.cap_k, TNB, ZG::KSTEP, ZNS);
}

__device__ __forceinline__ bool item_live(const ZGemmItem& it) { return it.M > 0 && it.N > 0 && it.K > 0; }

__device__ __forceinline__ bool item_fits(const ZGemmItem& it) {
  return it.M <= it.cap_m && it.N <= it.cap_n && it.K <= it.cap_k;
}

// row m, column k of opA(A)
__device__ __forceinline__ double2 a_elem(const ZGemmItem& it, int m, int k) {
  if (it.opA == ZOP_N) return it.A[m + (size_t)k * it.lda];
  double2 v = it.A[k + (size_t)m * it.lda];
  if (it.opA == ZOP_C) v.y = -v.y;
  return v;
}

// row k, column n of opB(B) (column n read from column bcol[n] when a map is given)
__device__ __forceinline__ double2 b_elem(const ZGemmItem& it, int n, int k) {
  const int c = it.bcol ? it.bcol[n] : n;
  if (it.opB == ZOP_N) return it.B[k + (size_t)c * it.ldb];
  double2 v = it.B[c + (size_t)k * it.ldb];
  if (it.opB == ZOP_C) v.y = -v.y;
  return v;
}

__device__ __forceinline__ double2 op_elem(const ZGemmItem& it, int which, int r, int k) {
  return which == 0 ? a_elem(it, r, k) : b_elem(it, r, k);
}

}  // namespace

// Pass 1: e with max |entry| < 2^e for every row of opA(A) (which = 0) or column of opB(B) (1).
// grid: (x: rows, y: items)
// which = -1: operand A even where the item marks it as already packed (a pack-only launch)
__global__ void k_zg_rowexp(const ZGemmItem* items, int n_items, int which) {
  const int i = blockIdx.y;
  if (i >= n_items) return;
  const ZGemmItem it = items[i];
  const bool force = which < 0;
  if (force) which = 0;
  if (!item_live(it) || !item_fits(it) || (which == 0 && it.skip_a > 0 && !force)) return;
  const int rows = which == 0 ? it.M : it.N, tr = which == 0 ? TMA : TNB;
  const PackCap cp = zcap(it, which);
  int* ex = (int*)((which == 0 ? it.TA : it.TB) + cp.exp_off);
  const int padded = cdiv(rows, tr) * tr;
  const bool k_contiguous = which == 0 ? it.opA != ZOP_N : it.opB == ZOP_N;
  if (k_contiguous) {
    // a row's entries are contiguous in memory: one warp per row, its lanes striding K (the
    // maximum does not depend on the order, so the exponent is the same as a sequential scan's)
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < padded; r += gridDim.x * wpb) {
      double m = 0.0;
      if (r < rows)
        for (int k = lane; k < it.K; k += 32) {
          const double2 v = op_elem(it, which, r, k);
          m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) ex[r] = row_exponent(m);
    }
    return;
  }
  // consecutive rows are contiguous: one thread per row, consecutive threads on consecutive rows
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < padded; r += gridDim.x * blockDim.x) {
    double m = 0.0;
    if (r < rows)
      for (int k = 0; k < it.K; ++k) {
        const double2 v = op_elem(it, which, r, k);
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
      }
    ex[r] = row_exponent(m);
  }
}

// Pass 2: one thread per (row, 8-element K group): the 12 slice planes of its 8 entries, 16 bytes
// each; consecutive threads take consecutive rows, so reads of column-major operands and the
// 16-byte writes of a plane are both contiguous. grid: (x: elements, y: items)
__global__ void k_zg_pack(const ZGemmItem* items, int n_items, int which, int* status) {
  const int i = blockIdx.y;
  if (i >= n_items) return;
  const ZGemmItem it = items[i];
  const bool force = which < 0;
  if (force) which = 0;
  if (!item_live(it) || (which == 0 && it.skip_a > 0 && !force)) return;
  if (!item_fits(it)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_CAPACITY);
    return;
  }
  const int rows = which == 0 ? it.M : it.N, tr = which == 0 ? TMA : TNB;
  constexpr int NS = ZNS;
  const PackCap cp = zcap(it, which);
  unsigned char* out = which == 0 ? it.TA : it.TB;
  const int* ex = (const int*)(out + cp.exp_off);
  const int n_rt = cdiv(rows, tr), n_ks = cdiv(it.K, ZG::KSTEP);
  const int padded = n_rt * tr, n_grp = 2 * n_ks;
  const int b = ZBITS;         // the GEMM accumulates K in chunks of 512: 7-bit slices stay exact
  const size_t total = (size_t)padded * n_grp;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % padded), grp = (int)(idx / padded);
    const int rt = r / tr, m = r % tr, ks = grp >> 1, half = grp & 1;
    const int e = ex[r];
    uint32_t pr[NS][4], pi[NS][4];       // 8 BF16 per plane, two per word
#pragma unroll
    for (int j = 0; j < ZG::KG; ++j) {
      const int k = ks * ZG::KSTEP + half * ZG::KG + j;
      double2 v = make_double2(0.0, 0.0);
      if (r < rows && k < it.K) v = op_elem(it, which, r, k);
      uint32_t sr[NS], si[NS];
      pieces<true, NS, true>(ldexp(v.x, -e), b, sr);
      pieces<true, NS, true>(ldexp(v.y, -e), b, si);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if ((j & 1) == 0) {
          pr[s][j >> 1] = sr[s];
          pi[s][j >> 1] = si[s];
        } else {
          pr[s][j >> 1] |= sr[s] << 16;
          pi[s][j >> 1] |= si[s] << 16;
        }
      }
    }
    unsigned char* base = out + ((size_t)rt * cp.ksteps + ks) * (2 * NS) * cp.plane_bytes +
                          ((size_t)half * tr + m) * 16;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      *(uint4*)(base + (size_t)s * cp.plane_bytes) = make_uint4(pr[s][0], pr[s][1], pr[s][2], pr[s][3]);
      *(uint4*)(base + (size_t)(NS + s) * cp.plane_bytes) = make_uint4(pi[s][0], pi[s][1], pi[s][2], pi[s][3]);
    }
  }
}

// The GEMM: persistent, one CTA per SM over the live 128 x 64 tiles of every item. K runs in chunks
// of 512 (32 MMA steps): each chunk's four levels accumulate exactly enough in TMEM, and the
// epilogue adds the chunk to C in FP64 (the first chunk writes C, or C - product for acc < 0).
__global__ void __launch_bounds__(TC_THREADS, 1) k_zgemm(const ZGemmItem* items, int n_items, int* status) {
  constexpr uint32_t A_PLANE = TMA * ROW_BYTES, B_PLANE = TNB * ROW_BYTES;
  constexpr uint32_t A_STAGE = 2 * ZNS * A_PLANE, B_STAGE = 2 * ZNS * B_PLANE, STAGE = A_STAGE + B_STAGE;
  constexpr int STAGES = Stages<ZNS>::value;
  constexpr int NLEV = 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bar_full[MAX_STAGES], bar_empty[MAX_STAGES];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ int col_exp[TNB];
  __shared__ int tile_off[MAX_ITEMS + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (n_items > MAX_ITEMS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(status, ST_CAPACITY);
    return;
  }
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  for (int i = tid; i < n_items; i += blockDim.x) {
    const ZGemmItem& it = items[i];
    tile_off[i + 1] = (item_live(it) && item_fits(it)) ? cdiv(it.M, TMA) * cdiv(it.N, TNB) : 0;
  }
  if (tid == 0) {
    tile_off[0] = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int i = 0; i < n_items; ++i) tile_off[i + 1] += tile_off[i];
  __syncthreads();
  const int total = tile_off[n_items];
  if ((int)blockIdx.x >= total) return;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_s))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = instr_desc(1u, TMA, TNB);
  constexpr uint32_t LBO_A = TMA * 16, LBO_B = TNB * 16, SBO = 128;
  uint32_t g = 0;                 // K steps processed by this CTA (stage = g % STAGES)
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const ZGemmItem& it = items[lo];
    const PackCap ca = zcap(it, 0), cb = zcap(it, 1);
    const int nt_b = cdiv(it.N, TNB);
    const int rt = (t - tile_off[lo]) / nt_b, ct = (t - tile_off[lo]) % nt_b;
    const int n_ks = cdiv(it.K, ZG::KSTEP);
    if (tid < TNB) col_exp[tid] = ((const int*)(it.TB + cb.exp_off))[ct * TNB + tid];
    const unsigned char* gA = it.TA + (size_t)rt * ca.ksteps * A_STAGE;
    const unsigned char* gB = it.TB + (size_t)ct * cb.ksteps * B_STAGE;
    const int m = rt * TMA + warp * 32 + lane;
    const int e_m = ((const int*)(it.TA + ca.exp_off))[m];
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool bad = false;
    for (int ks0 = 0; ks0 < n_ks; ks0 += ZKC_STEPS) {
      const int nk = min(ZKC_STEPS, n_ks - ks0);
      if (tid == 0) {
        auto load = [&](int ks, uint32_t gg) {
          unsigned char* st = smem + (gg % STAGES) * STAGE;
          uint64_t* bar = &bar_full[gg % STAGES];
          mbar_expect_tx(bar, STAGE);
          bulk_g2s(st, gA + (size_t)(ks0 + ks) * A_STAGE, A_STAGE, bar);
          bulk_g2s(st + A_STAGE, gB + (size_t)(ks0 + ks) * B_STAGE, B_STAGE, bar);
        };
        auto par = [](uint32_t gg) { return (gg / STAGES) & 1u; };
        bool ok = true;
        uint32_t loaded = g, waited = g, committed = 0;
        bool any_commit = false;
        bool init[NLEV] = {false, false, false, false};
        // prologue: the chunk's first STAGES - 1 steps (their stages were freed by the last wait)
        for (int ks = 0; ks < nk && ks < STAGES - 1; ++ks) {
          load(ks, g + ks);
          loaded = g + ks + 1;
        }
        for (int ks = 0; ks < nk && ok; ++ks) {
          const uint32_t gg = g + ks;
          ok = mbar_wait(&bar_full[gg % STAGES], par(gg));
          if (!ok) break;
          waited = gg + 1;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned char* sa = smem + (gg % STAGES) * STAGE;
          const unsigned char* sb = sa + A_STAGE;
#pragma unroll
          for (int s = 0; s < ZNS; ++s) {
#pragma unroll
            for (int u = 0; u < ZNS - s; ++u) {
              const int L = (s + u) < NLEV - 1 ? (s + u) : NLEV - 1;
              const uint32_t dre = tmem + (2 * L) * TNB, dim = dre + TNB;
              const uint64_t ar = smem_desc(sa + s * A_PLANE, LBO_A, SBO);
              const uint64_t ai = smem_desc(sa + (ZNS + s) * A_PLANE, LBO_A, SBO);
              const uint64_t br = smem_desc(sb + u * B_PLANE, LBO_B, SBO);
              const uint64_t bi = smem_desc(sb + (ZNS + u) * B_PLANE, LBO_B, SBO);
              mma<true>(dre, ar, br, idesc, init[L]);
              mma<true>(dre, ai, bi, idesc | NEG_A, true);
              mma<true>(dim, ar, bi, idesc, init[L]);
              mma<true>(dim, ai, br, idesc, true);
              init[L] = true;
            }
          }
          mma_commit(&bar_empty[gg % STAGES]);
          committed = gg;
          any_commit = true;
          const int nx = ks + STAGES - 1;
          if (nx < nk) {
            if (ks >= 1) ok = mbar_wait(&bar_empty[(gg - 1) % STAGES], par(gg - 1));
            if (!ok) break;
            load(nx, g + nx);
            loaded = g + nx + 1;
          }
        }
        if (ok && any_commit) ok = mbar_wait(&bar_empty[committed % STAGES], par(committed));
        if (!ok) {
          atomicOr(status, ST_TIMEOUT);
          abort_s = 1;
          for (uint32_t q = waited; q < loaded; ++q) mbar_wait(&bar_full[q % STAGES], par(q));
          if (any_commit) mbar_wait(&bar_empty[committed % STAGES], par(committed));
        }
      }
      g += nk;
      __syncthreads();
      if (abort_s) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // epilogue of the chunk: thread = row m of the tile, 8 columns per TMEM load
      const bool first = ks0 == 0;
      for (int c0 = 0; c0 < TNB; c0 += 8) {
        double re[8], im[8];
        {
          float x[8], y[8];
          tmem_ld8(tmem + lane_base + c0, x);
          tmem_ld8(tmem + lane_base + TNB + c0, y);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            re[j] = (double)x[j];
            im[j] = (double)y[j];
          }
#pragma unroll
          for (int L = 1; L < NLEV; ++L) {
            tmem_ld8(tmem + lane_base + (2 * L) * TNB + c0, x);
            tmem_ld8(tmem + lane_base + (2 * L + 1) * TNB + c0, y);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              re[j] += (double)x[j];
              im[j] += (double)y[j];
            }
          }
        }
        if (m < it.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = ct * TNB + c0 + j;
            if (n >= it.N) continue;
            const int e = e_m + col_exp[c0 + j];
            double2 v = make_double2(ldexp(re[j], e), ldexp(im[j], e));
            if (it.acc < 0) v = make_double2(-v.x, -v.y);
            double2* cp = it.C + m + (size_t)n * it.ldc;
            if (!first || it.acc < 0) {
              const double2 o = *cp;
              v = make_double2(o.x + v.x, o.y + v.y);
            }
            bad |= !(isfinite(v.x) && isfinite(v.y));
            *cp = v;
          }
        }
      }
      // TMEM reads complete before the next chunk's MMAs overwrite the accumulators
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (abort_s) break;
    if (bad && it.flag) *it.flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

size_t zgemm_pack_bytes(int rows_cap, int k_cap, int which) {
  return pack_cap(std::max(1, rows_cap), std::max(1, k_cap), which == 0 ? TMA : TNB, ZG::KSTEP, ZNS).total;
}

int zgemm_max_items() { return MAX_ITEMS; }

int zgemm_tile_cap(int m_cap, int n_cap) { return cdiv(std::max(1, m_cap), TMA) * cdiv(std::max(1, n_cap), TNB); }

namespace {
constexpr int ZMAX_DEV = 64;
bool g_zattr_done[ZMAX_DEV] = {};
}  // namespace

void launch_zgemm_pack_a(const ZGemmItem* items, int n_items, int m_cap_max, int* status, cudaStream_t st) {
  if (n_items <= 0) return;
  const int bx_a = std::min(1024, cdiv(std::max(1, m_cap_max), 4));     // four rows per block when a warp takes a row
  k_zg_rowexp<<<dim3(bx_a, n_items), 128, 0, st>>>(items, n_items, -1);
  k_zg_pack<<<dim3(128, n_items), 256, 0, st>>>(items, n_items, -1, status);
}

void launch_zgemm(const ZGemmItem* items, int n_items, int tile_cap, int m_cap_max, int n_cap_max, int* status,
                  cudaStream_t st) {
  if (n_items <= 0) return;
  // four rows per block when a warp takes a row (rows contiguous in K), else 128
  const int bx_a = std::min(1024, cdiv(std::max(1, m_cap_max), 4)), bx_b = std::min(1024, cdiv(std::max(1, n_cap_max), 4));
  k_zg_rowexp<<<dim3(bx_a, n_items), 128, 0, st>>>(items, n_items, 0);
  k_zg_rowexp<<<dim3(bx_b, n_items), 128, 0, st>>>(items, n_items, 1);
  k_zg_pack<<<dim3(128, n_items), 256, 0, st>>>(items, n_items, 0, status);
  k_zg_pack<<<dim3(64, n_items), 256, 0, st>>>(items, n_items, 1, status);
  const size_t smem = (size_t)Stages<ZNS>::value * 2 * ZNS * (TMA + TNB) * ROW_BYTES + 1024;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (dev >= 0 && dev < ZMAX_DEV && !g_zattr_done[dev]) {
    cudaFuncSetAttribute(k_zgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    g_zattr_done[dev] = true;
  }
  const int grid = std::max(1, std::min(sms > 0 ? sms : 152, tile_cap));
  k_zgemm<<<grid, TC_THREADS, smem, st>>>(items, n_items, status);
}

}  // namespace ptk
