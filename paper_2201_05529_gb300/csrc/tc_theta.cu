// Tensor-core theta + gate of the fast path (App. A.2) on sm_103a: tcgen05 + TMEM.
//
// The two-site gate acts on the Liouville legs p (left) and q (right) of
//   theta[(u,p),(q,v)] = sum_c R_L[u,(p,c)] lambda_c L_R[(c,q),v],
//   D[(u,p'),(q',v)]   = sum_{p,q} G[(p' q'),(p q)] theta[(u,p),(q,v)].
// Folding the gate into the right operand turns theta + gate into ONE complex GEMM with K = 4 chi:
//   A[u, k]    = R_L[u, k] lambda_{k mod chi}                         (k = p chi + c)
//   B'[n', k]  = sum_q G[(p' q'),(p q)] L_R[(c,q), v]                 (n' = (q' rR + v) 4 + p')
//   D[u 4 + p', q' rR + v] = sum_k A[u, k] B'[n', k].
// B' is formed in FP64 by the pack kernel; the GEMM runs on the tensor cores.
//
// Precision. Each operand row is represented as a sum of NS pieces:
//   * natural split (PT_TF32X3, PT_BF16X3, PT_TF32X1): x = x0 + x1 + x2, each piece the TF32/BF16
//     rounding of the remainder;
//   * fixed-point slices (PT_BF16_OZAKI; Ozaki, Ogita, Oishi and Rump's error-free splitting of
//     matrix products): the row is scaled by a power of two 2^-e_row so every entry lies in (-1, 1),
//     then cut into NS = 6 slices a_i 2^(-b(i+1)) with integer a_i, |a_i| <= 2^b (b = 7 while
//     K <= 512). A product of two slices is exact in FP32 and the sum over K of the level-0 (and
//     level-1) slice products is an integer multiple of one power of two below 2^24, so the tensor
//     cores' FP32 accumulation of those levels is exact; level 2 and the levels beyond carry only
//     their own rounding, ~2^-24 of quantities 2^-2b and 2^-3b smaller. The product is accurate to
//     ~1e-12 relative to the rows' scale (FP32 accumulation of unscaled pieces gives ~1e-6 there),
//     which also keeps the exact null space of a rank-deficient D at that level, below the
//     rank-revealing stop of the pivoted QR that follows.
// Complex products take four real products (Re = Ar Br - Ai Bi with the MMA's negate-A bit,
// Im = Ar Bi + Ai Br). The piece products accumulate in TMEM accumulator pairs by level
// (i + j = 0, 1, 2, >= 3; two levels 0, 1-2 for three pieces); the epilogue adds them in FP64 and
// applies 2^(e_row(A) + e_row(B')).
//
// Data flow. Pack kernels write each operand's 2 NS planes (real/imaginary x pieces) in the tcgen05
// canonical K-major no-swizzle layout (8-row x 16-byte core matrices), one block per plane, row tile
// (A: 128 rows, B': 64 rows) and K step, so one cp.async.bulk stages each. The GEMM kernel is
// persistent: one CTA per SM walks the list of live 128 x 64 output tiles of every bond of the
// layer (live dims read on the device, so a CUDA graph replays it unchanged). Three shared-memory
// stages pipeline the K steps: one thread issues the bulk copies of step g+1 while the tensor cores
// run step g, and tcgen05.commit on a per-stage mbarrier frees a stage. Four warps read TMEM back
// (tcgen05.ld 32x32b). Every mbarrier wait has an iteration limit: on expiry the kernel records
// ST_TIMEOUT, waits (bounded) for its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "kernels.h"
#include "tc_common.cuh"

namespace ptk {

using namespace tcx;

namespace {

// live dims of one bond's theta + gate GEMM
struct GemmDims {
  int rL, rR, mD, nD, chc, K;   // A rows = rL, B' rows = 4 nD, K = 4 chc
  bool qrL, lqR;
};

__device__ __forceinline__ GemmDims gemm_dims(const Tables& T, const BondWork& W) {
  const int BL = W.lam_l, BC = BL + 1, BR = BL + 2;
  const int sL = W.site_l, sR = sL + 1;
  const int chl = T.lam_chi[BL], chc = T.lam_chi[BC], chr = T.lam_chi[BR];
  const int kL = T.site_kappa[sL], kR = T.site_kappa[sR];
  const int mL = chl * kL, nL = 4 * chc, mR = 4 * chc, nR = kR * chr;
  GemmDims d;
  d.qrL = mL > nL;
  d.lqR = nR > mR;
  d.rL = d.qrL ? nL : mL;
  d.rR = d.lqR ? mR : nR;
  d.mD = 4 * d.rL;
  d.nD = 4 * d.rR;
  d.chc = chc;
  d.K = 4 * chc;
  return d;
}

// operand capacities of a bond: A rows = rL_cap = mD_cap / 4, B' rows = 4 nD_cap, K = 4 chi_cap
__host__ __device__ __forceinline__ PackCap cap_a(const BondWork& W, int kstep, int ns) {
  return pack_cap(W.mD_cap / 4, W.nL_cap, TMA, kstep, ns);
}
__host__ __device__ __forceinline__ PackCap cap_b(const BondWork& W, int kstep, int ns) {
  return pack_cap(4 * W.nD_cap, W.nL_cap, TNB, kstep, ns);
}

// sources of operand A (which = 0) and B' (which = 1) in FP64
struct OpSrc {
  const double2* RLp;
  int ldRL;
  const double2* LRp;
  int ldLR;
  const double* lamC;
  int chc, rR;
};

__device__ __forceinline__ double2 op_elem(const OpSrc& s, const double2* gate, int which, int row, int k) {
  if (which == 0) {
    const double2 v = s.RLp[row + (size_t)k * s.ldRL];
    const double l = s.lamC[k % s.chc];
    return make_double2(v.x * l, v.y * l);
  }
  // n' = Dcol 4 + p', Dcol = q' rR + v; k = p chc + c
  const int pp = row & 3, dcol = row >> 2;
  const int qq = dcol / s.rR, v = dcol - qq * s.rR;
  const int p = k / s.chc, c = k - p * s.chc;
  double2 acc = make_double2(0.0, 0.0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 g = gate[(pp * 4 + qq) * 16 + p * 4 + q];
    const double2 x = s.LRp[v + (size_t)(c * 4 + q) * s.ldLR];   // L_R(c q, v) = conj(x)
    acc.x = fma(g.x, x.x, fma(g.y, x.y, acc.x));
    acc.y = fma(g.y, x.x, fma(-g.x, x.y, acc.y));
  }
  return acc;
}

__device__ __forceinline__ OpSrc op_src(const Tables& T, const BondWork& W, const GemmDims& d) {
  OpSrc s;
  s.RLp = d.qrL ? W.RL : W.QL;
  s.ldRL = d.qrL ? 4 * d.chc : T.lam_chi[W.lam_l] * T.site_kappa[W.site_l];
  s.LRp = d.lqR ? W.LR : W.QR;
  s.ldLR = d.lqR ? 4 * d.chc : T.site_kappa[W.site_l + 1] * T.lam_chi[W.lam_l + 2];
  s.lamC = T.lam_ptr[W.lam_l + 1];
  s.chc = d.chc;
  s.rR = d.rR;
  return s;
}

}  // namespace

// ------------------------------------------------------------------ packing (FP64 -> pieces)
// Pass 1 (slices only): the power-of-two exponent of every row of A (which = 0) or B' (which = 1).
// grid: (x: rows, y: bonds)
__global__ void k_tc_rowexp(Tables T, const BondWork* work, int n_work, int which, int kstep, int ns) {
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const GemmDims d = gemm_dims(T, W);
  const int rows = which == 0 ? d.rL : 4 * d.nD;
  const int tile_rows = which == 0 ? TMA : TNB;
  const PackCap cp = which == 0 ? cap_a(W, kstep, ns) : cap_b(W, kstep, ns);
  __shared__ double2 gate[256];
  if (which == 1)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) gate[i] = W.gate[i];
  __syncthreads();
  if (cdiv(rows, tile_rows) > cp.tiles || cdiv(d.K, kstep) > cp.ksteps) return;   // pack reports it
  const OpSrc s = op_src(T, W, d);
  int* ex = (int*)((unsigned char*)(which == 0 ? W.TA : W.TB) + cp.exp_off);
  const int padded = cdiv(rows, tile_rows) * tile_rows;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < padded; row += gridDim.x * blockDim.x) {
    double m = 0.0;
    if (row < rows)
      for (int k = 0; k < d.K; ++k) {
        const double2 v = op_elem(s, gate, which, row, k);
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
      }
    ex[row] = row_exponent(m);
  }
}

// Pass 2: every element of the live tiles -> NS pieces of its real and imaginary parts.
// grid: (x: elements, y: bonds)
template <bool BF16, int NS, bool SLICE>
__global__ void k_tc_pack(Tables T, const BondWork* work, int n_work, int which) {
  using G = Geo<BF16>;
  const int w = blockIdx.y;
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const GemmDims d = gemm_dims(T, W);
  const int tile_rows = which == 0 ? TMA : TNB;
  const int rows = which == 0 ? d.rL : 4 * d.nD;
  const PackCap cp = which == 0 ? cap_a(W, G::KSTEP, NS) : cap_b(W, G::KSTEP, NS);
  const int n_rt = cdiv(rows, tile_rows), n_ks = cdiv(d.K, G::KSTEP);
  if (n_rt > cp.tiles || n_ks > cp.ksteps) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  __shared__ double2 gate[256];
  if (which == 1)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) gate[i] = W.gate[i];
  __syncthreads();
  const OpSrc s = op_src(T, W, d);
  unsigned char* out = (unsigned char*)(which == 0 ? W.TA : W.TB);
  const int* ex = (const int*)(out + cp.exp_off);
  const int b = slice_bits(d.K);
  const size_t per_step = (size_t)2 * NS * cp.plane_bytes;
  // element order (k within the step fastest, then row, step, tile): consecutive threads write
  // consecutive bytes of one 16-byte K group
  const size_t total = (size_t)n_rt * n_ks * tile_rows * G::KSTEP;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % G::KSTEP);
    size_t t = idx / G::KSTEP;
    const int m = (int)(t % tile_rows);
    t /= tile_rows;
    const int ks = (int)(t % n_ks);
    const int rt = (int)(t / n_ks);
    const int row = rt * tile_rows + m, k = ks * G::KSTEP + kk;
    double2 v = make_double2(0.0, 0.0);
    if (row < rows && k < d.K) v = op_elem(s, gate, which, row, k);
    if (SLICE) {
      const int e = ex[row];
      v.x = ldexp(v.x, -e);
      v.y = ldexp(v.y, -e);
    } else if (kk == 0 && ks == 0) {
      ((int*)(out + cp.exp_off))[row] = 0;     // natural split: no row scaling
    }
    uint32_t pr[NS], pi[NS];
    pieces<BF16, NS, SLICE>(v.x, b, pr);
    pieces<BF16, NS, SLICE>(v.y, b, pi);
    unsigned char* base = out + ((size_t)rt * cp.ksteps + ks) * per_step;
    const size_t in_plane = ((size_t)(kk / G::KG) * tile_rows + m) * 16 + (size_t)(kk % G::KG) * G::EB;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      unsigned char* a = base + (size_t)q * cp.plane_bytes + in_plane;
      unsigned char* c = base + (size_t)(NS + q) * cp.plane_bytes + in_plane;
      if (BF16) {
        *(uint16_t*)a = (uint16_t)pr[q];
        *(uint16_t*)c = (uint16_t)pi[q];
      } else {
        *(uint32_t*)a = pr[q];
        *(uint32_t*)c = pi[q];
      }
    }
  }
}

// ------------------------------------------------------------------ GEMM, FP64 epilogue
// Persistent: grid = min(SMs, tile capacity); each CTA walks the live 128 x 64 tiles of every bond.
template <bool BF16, int NS>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_theta(Tables T, const BondWork* work, int n_work) {
  using G = Geo<BF16>;
  constexpr uint32_t A_PLANE = TMA * ROW_BYTES, B_PLANE = TNB * ROW_BYTES;
  constexpr uint32_t A_STAGE = 2 * NS * A_PLANE, B_STAGE = 2 * NS * B_PLANE, STAGE = A_STAGE + B_STAGE;
  constexpr int STAGES = Stages<NS>::value;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t bar_full[MAX_STAGES], bar_empty[MAX_STAGES];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ int col_exp[TNB];
  __shared__ int tile_off[MAX_ITEMS + 1];   // prefix of live tiles per bond
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (n_work > MAX_ITEMS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // live tiles of every bond (every CTA computes the same list); CTA 0 publishes the SVD shapes
  for (int w = tid; w < n_work; w += blockDim.x) {
    const BondWork& W = work[w];
    const GemmDims d = gemm_dims(T, W);
    const PackCap ca = cap_a(W, G::KSTEP, NS), cb = cap_b(W, G::KSTEP, NS);
    const int nt_a = cdiv(d.rL, TMA), nt_b = cdiv(4 * d.nD, TNB), n_ks = cdiv(d.K, G::KSTEP);
    const bool fits = nt_a <= ca.tiles && nt_b <= cb.tiles && n_ks <= ca.ksteps && d.mD <= W.mD_cap &&
                      d.nD <= W.nD_cap;
    tile_off[w + 1] = fits ? nt_a * nt_b : 0;
    if (blockIdx.x == 0) {
      W.info[0] = fits ? d.mD : 0;      // 0: the SVD and the following stages skip this bond
      W.info[1] = fits ? d.nD : 0;
      W.info[2] = d.mD < d.nD ? 1 : 0;
    }
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
    for (int w = 0; w < n_work; ++w) tile_off[w + 1] += tile_off[w];
  __syncthreads();
  const int total = tile_off[n_work];
  if ((int)blockIdx.x >= total) return;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_s))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  // accumulator pairs by level L = min(i + j, NLEV - 1): columns [2 L TNB, (2 L + 1) TNB) hold the
  // real part, the next TNB columns the imaginary part (4 levels x 2 x 64 columns = all of TMEM)
  const uint32_t idesc = instr_desc(BF16 ? 1u : 2u, TMA, TNB);
  constexpr uint32_t LBO_A = TMA * 16, LBO_B = TNB * 16, SBO = 128;
  constexpr int NLEV = NS == 1 ? 1 : (NS <= 3 ? 3 : 4);
  uint32_t g = 0;                 // K steps processed by this CTA (stage = g % STAGES)
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = n_work - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const int w = lo;
    const BondWork& W = work[w];
    const GemmDims d = gemm_dims(T, W);
    const PackCap ca = cap_a(W, G::KSTEP, NS), cb = cap_b(W, G::KSTEP, NS);
    const int nt_b = cdiv(4 * d.nD, TNB);
    const int rt = (t - tile_off[w]) / nt_b, ct = (t - tile_off[w]) % nt_b;
    const int n_ks = cdiv(d.K, G::KSTEP);
    if (tid < TNB) col_exp[tid] = ((const int*)((const unsigned char*)W.TB + cb.exp_off))[ct * TNB + tid];
    if (tid == 0) {
      const unsigned char* gA = (const unsigned char*)W.TA + (size_t)rt * ca.ksteps * A_STAGE;
      const unsigned char* gB = (const unsigned char*)W.TB + (size_t)ct * cb.ksteps * B_STAGE;
      auto load = [&](int ks, uint32_t gg) {
        unsigned char* st = smem + (gg % STAGES) * STAGE;
        uint64_t* bar = &bar_full[gg % STAGES];
        mbar_expect_tx(bar, STAGE);
        bulk_g2s(st, gA + (size_t)ks * A_STAGE, A_STAGE, bar);
        bulk_g2s(st + A_STAGE, gB + (size_t)ks * B_STAGE, B_STAGE, bar);
      };
      auto par = [](uint32_t gg) { return (gg / STAGES) & 1u; };
      bool ok = true;
      uint32_t loaded = g, waited = g, committed = 0;
      bool any_commit = false;
      bool init[4] = {false, false, false, false};
      // prologue: the first STAGES - 1 steps (their stages were freed by the previous tile's end)
      for (int ks = 0; ks < n_ks && ks < STAGES - 1; ++ks) {
        load(ks, g + ks);
        loaded = g + ks + 1;
      }
      for (int ks = 0; ks < n_ks && ok; ++ks) {
        const uint32_t gg = g + ks;
        ok = mbar_wait(&bar_full[gg % STAGES], par(gg));
        if (!ok) break;
        waited = gg + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned char* sa = smem + (gg % STAGES) * STAGE;
        const unsigned char* sb = sa + A_STAGE;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
#pragma unroll
          for (int j = 0; j < NS - i; ++j) {
            const int L = (i + j) < NLEV - 1 ? (i + j) : NLEV - 1;
            const uint32_t dre = tmem + (2 * L) * TNB, dim = dre + TNB;
            const uint64_t ar = smem_desc(sa + i * A_PLANE, LBO_A, SBO);
            const uint64_t ai = smem_desc(sa + (NS + i) * A_PLANE, LBO_A, SBO);
            const uint64_t br = smem_desc(sb + j * B_PLANE, LBO_B, SBO);
            const uint64_t bi = smem_desc(sb + (NS + j) * B_PLANE, LBO_B, SBO);
            // Re += Ar Br - Ai Bi, Im += Ar Bi + Ai Br
            mma<BF16>(dre, ar, br, idesc, init[L]);
            mma<BF16>(dre, ai, bi, idesc | NEG_A, true);
            mma<BF16>(dim, ar, bi, idesc, init[L]);
            mma<BF16>(dim, ai, br, idesc, true);
            init[L] = true;
          }
        }
        mma_commit(&bar_empty[gg % STAGES]);
        committed = gg;
        any_commit = true;
        // refill: step ks + STAGES - 1 goes into the stage read by step ks - 1
        const int nk = ks + STAGES - 1;
        if (nk < n_ks) {
          if (ks >= 1) ok = mbar_wait(&bar_empty[(gg - 1) % STAGES], par(gg - 1));
          if (!ok) break;
          load(nk, g + nk);
          loaded = g + nk + 1;
        }
      }
      // all MMAs of the tile complete before the epilogue reads TMEM
      if (ok && any_commit) ok = mbar_wait(&bar_empty[committed % STAGES], par(committed));
      if (!ok) {
        // give the copies and MMAs in flight one more bounded wait before leaving
        atomicOr(T.status, ST_TIMEOUT);
        abort_s = 1;
        for (uint32_t q = waited; q < loaded; ++q) mbar_wait(&bar_full[q % STAGES], par(q));
        if (any_commit) mbar_wait(&bar_empty[committed % STAGES], par(committed));
      }
    }
    g += n_ks;
    __syncthreads();
    if (abort_s) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: thread = row u of the tile; 8 columns (two D columns x four p') per TMEM load
    const int u = rt * TMA + warp * 32 + lane;
    const int e_u = ((const int*)((const unsigned char*)W.TA + ca.exp_off))[u];
    const bool tr = d.mD < d.nD;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
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
      if (u < d.rL) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int np = ct * TNB + c0 + j;          // n' = Dcol 4 + p'
          if (np >= 4 * d.nD) continue;
          const int e = e_u + col_exp[c0 + j];
          const double2 v = make_double2(ldexp(re[j], e), ldexp(im[j], e));
          if (!(isfinite(v.x) && isfinite(v.y))) W.info[7] = 1;   // k_nan_guard stops this bond
          const int Drow = u * 4 + (np & 3), Dcol = np >> 2;
          if (!tr) W.A[Drow + (size_t)Dcol * d.mD] = v;
          else W.A[Dcol + (size_t)Drow * d.nD] = make_double2(v.x, -v.y);
        }
      }
    }
    // TMEM reads complete before the next tile's MMAs overwrite the accumulators
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ launchers
namespace {
struct Mode {
  bool bf16;
  int ns;
};
Mode mode_of(int precision) {
  switch (precision) {
    case 1: return {false, 3};   // TF32x3: natural split
    case 2: return {true, 3};    // BF16x3: natural split
    case 3: return {false, 1};   // TF32x1
    default: return {true, 6};   // BF16 fixed-point slices (Ozaki)
  }
}

constexpr int MAX_DEV = 64;
bool g_attr_done[MAX_DEV][5] = {};

template <bool BF16, int NS, bool SLICE>
void launch_mode(const Tables& T, const BondWork* work, int n_work, int tile_cap, int precision, cudaStream_t st) {
  constexpr int KSTEP = Geo<BF16>::KSTEP;
  const int gx = 64;
  if (SLICE) {
    // one thread per row: A has r_L <= 512 rows, B' up to 4 n_D = 8192 (the gate-folded rows)
    k_tc_rowexp<<<dim3(4, n_work), 128, 0, st>>>(T, work, n_work, 0, KSTEP, NS);
    k_tc_rowexp<<<dim3(64, n_work), 128, 0, st>>>(T, work, n_work, 1, KSTEP, NS);
  }
  k_tc_pack<BF16, NS, SLICE><<<dim3(gx, n_work), 256, 0, st>>>(T, work, n_work, 0);
  k_tc_pack<BF16, NS, SLICE><<<dim3(4 * gx, n_work), 256, 0, st>>>(T, work, n_work, 1);
  const size_t smem = (size_t)Stages<NS>::value * 2 * NS * (TMA + TNB) * ROW_BYTES + 1024;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the large dynamic shared memory limit is a per-device function attribute
  if (dev >= 0 && dev < MAX_DEV && !g_attr_done[dev][precision]) {
    cudaFuncSetAttribute(k_tc_theta<BF16, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    g_attr_done[dev][precision] = true;
  }
  const int grid = std::max(1, std::min(sms > 0 ? sms : 152, tile_cap));
  k_tc_theta<BF16, NS><<<grid, TC_THREADS, smem, st>>>(T, work, n_work);
}
}  // namespace

size_t tc_pack_bytes(const BondWork& W, int which, int precision) {
  const Mode m = mode_of(precision);
  const int kstep = m.bf16 ? Geo<true>::KSTEP : Geo<false>::KSTEP;
  return (which == 0 ? cap_a(W, kstep, m.ns) : cap_b(W, kstep, m.ns)).total;
}

int tc_tile_cap(const BondWork& W, int precision) {
  const Mode m = mode_of(precision);
  const int kstep = m.bf16 ? Geo<true>::KSTEP : Geo<false>::KSTEP;
  return cap_a(W, kstep, m.ns).tiles * cap_b(W, kstep, m.ns).tiles;
}

void launch_tc_theta(const Tables& T, const BondWork* work, int n_work, int tile_cap, int precision,
                     cudaStream_t st) {
  switch (precision) {
    case 1: launch_mode<false, 3, false>(T, work, n_work, tile_cap, precision, st); break;
    case 2: launch_mode<true, 3, false>(T, work, n_work, tile_cap, precision, st); break;
    case 3: launch_mode<false, 1, false>(T, work, n_work, tile_cap, precision, st); break;
    default: launch_mode<true, 6, true>(T, work, n_work, tile_cap, 4, st); break;
  }
}

}  // namespace ptk
