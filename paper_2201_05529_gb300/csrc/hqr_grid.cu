// Whole-GPU Householder QR of the outer blocks of every bond of a layer (App. A.2: the exact
// reductions B_L = Q_L R_L and B_R^H = Q_R^H L_R^H that shrink the two-site block before the SVD).
//
// On the 21-site chain one layer holds ~20 such blocks of up to 2048 x 512: O(m n^2) FP64 work
// each, far too much for one CTA per block. Here one cooperative launch (one 512-thread CTA per SM)
// factors all of them at once. The columns of all blocks are dealt to the CTAs cyclically (global
// column g goes to CTA g mod G), so every CTA keeps work as the factorisation retires columns, and
// each warp updates its columns in place in global memory (L2). Step j applies reflector j of every
// block to the block's columns k > j; the warp that owns column j+1 applies it there first and then
// forms reflector j+1 from that column (look-ahead), so one grid barrier per step suffices.
// Afterwards every warp copies R out of its columns and forms its columns of the explicit
// Q = P_0 ... P_{n-1} [I; 0]: column k needs only the stored reflectors 0..k, so that phase runs
// without barriers.
//
// Reflectors P_j = I - tau_j u_j u_j^H with u_j[j] = 1: the column x it was formed from is kept raw
// in HH (rows > j) and the scale 1 / u_jj in HH[j, j]; tau_j in aux (B_L) or sig (B_R^H), the
// diagonal of R = beta_j. Every grid barrier wait is bounded.
#include "grid_sync.cuh"
#include "kernels.h"

namespace ptk {

namespace {

constexpr int HQ_THREADS = 512;
constexpr int HQ_WARPS = HQ_THREADS / 32;
constexpr int HQ_MAX_PAIRS = 384;           // (block, column) pairs one CTA may own
constexpr int HQ_MAX_ITEMS = 2048;          // blocks: two per bond
constexpr int HQ_U = 8;                     // rows per lane per block: loads in flight per lane
constexpr int HQ_ROWS = 32 * HQ_U;          // rows per block

using HMat = QRItem;

// block `item` (bond item / 2, side item % 2) of the layer, if it needs a reduction
__device__ __forceinline__ bool hmat_of(const Tables& T, const BondWork* work, int item, HMat* M) {
  const BondWork& W = work[item >> 1];
  const BondDims d = bond_dims(T, W);
  if (!bond_fits(d, W)) return false;
  if ((item & 1) == 0) {
    if (!d.qrL) return false;
    *M = HMat{W.QL, W.HH, W.RL, W.aux, d.mL, d.nL};
  } else {
    if (!d.lqR) return false;
    *M = HMat{W.QR, W.HH + (size_t)W.mL_cap * W.nL_cap, W.LR, W.sig, d.nR, d.mR};
  }
  return true;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reflector storage: P_j = I - tau_j u_j u_j^H with u_j[j] = 1 and u_j[r] = x_r s_j for r > j,
// where x is column j as it stood when the reflector was formed (kept raw in H[:, j], rows > j) and
// s_j = 1 / (alpha - beta) is kept in H[j, j] (the slot of the implicit unit entry); so forming a
// reflector needs no pass of its own over the column.

// y <- P_j y on rows j.. (one warp). HQ_U rows per lane per block: that many independent L2 loads
// in flight per lane (the loops are latency-bound, not bandwidth-bound). With NORM, also return
// ||y_new[j+1..]||^2 and alpha = y_new[j+1], and copy y_new[j+2..] raw into H[:, j+1] (the next
// reflector's column).
template <bool NORM>
__device__ __forceinline__ void apply_reflector(const HMat& M, int j, double2* y, int lane, double* nrm2_out = nullptr,
                                                double2* alpha_out = nullptr) {
  const double t = __ldcg(M.tau + j);
  if (t == 0.0 && !NORM) return;
  const double2* x = M.H + (size_t)j * M.m;
  const double2 sj = __ldcg(x + j);
  double2* hn = M.H + (size_t)(j + 1) * M.m;
  // rows j+1 .. m-1 in blocks of HQ_ROWS (lane + 32 q, q < HQ_U); the block count is the same for every
  // lane, the last block's rows are predicated: no lane-dependent loop bounds
  const int r0 = j + 1 + lane;
  const int nblk = (M.m - (j + 1) + HQ_ROWS - 1) / HQ_ROWS;
  // pass 1: conj(x) . y over rows > j
  double sr0 = 0.0, si0 = 0.0, sr1 = 0.0, si1 = 0.0;
  if (t != 0.0) {
    for (int i = 0; i < nblk; ++i) {
      const int r = r0 + i * HQ_ROWS;
      double2 a[HQ_U], b[HQ_U];
#pragma unroll
      for (int q = 0; q < HQ_U; ++q) {
        const bool in = r + 32 * q < M.m;
        a[q] = in ? __ldcg(x + r + 32 * q) : make_double2(0.0, 0.0);
        b[q] = in ? __ldcg(y + r + 32 * q) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int q = 0; q < HQ_U; q += 2) {
        sr0 = fma(a[q].x, b[q].x, fma(a[q].y, b[q].y, sr0));
        si0 = fma(a[q].x, b[q].y, fma(-a[q].y, b[q].x, si0));
        sr1 = fma(a[q + 1].x, b[q + 1].x, fma(a[q + 1].y, b[q + 1].y, sr1));
        si1 = fma(a[q + 1].x, b[q + 1].y, fma(-a[q + 1].y, b[q + 1].x, si1));
      }
    }
  }
  const double dr = warp_sum(sr0 + sr1), di = warp_sum(si0 + si1);
  // u^H y = y_j + conj(s) (x^H y)_{r > j};  c = tau u^H y;  y_j -= c, y_r -= x_r (s c)
  const double2 yj = __ldcg(y + j);
  const double2 d = make_double2(yj.x + sj.x * dr + sj.y * di, yj.y + sj.x * di - sj.y * dr);
  const double2 c = make_double2(t * d.x, t * d.y);
  const double2 sc = make_double2(sj.x * c.x - sj.y * c.y, sj.x * c.y + sj.y * c.x);
  __syncwarp();
  if (lane == 0 && t != 0.0) __stcg(y + j, make_double2(yj.x - c.x, yj.y - c.y));
  double n0 = 0.0, n1 = 0.0;
  double2 alpha = make_double2(0.0, 0.0);
  for (int i = 0; i < nblk; ++i) {
    const int r = r0 + i * HQ_ROWS;
    double2 a[HQ_U], b[HQ_U];
#pragma unroll
    for (int q = 0; q < HQ_U; ++q) {
      const bool in = r + 32 * q < M.m;
      a[q] = in ? __ldcg(x + r + 32 * q) : make_double2(0.0, 0.0);
      b[q] = in ? __ldcg(y + r + 32 * q) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < HQ_U; ++q) {
      const int rr = r + 32 * q;
      if (rr >= M.m) continue;
      if (t != 0.0) {
        b[q].x -= a[q].x * sc.x - a[q].y * sc.y;
        b[q].y -= a[q].x * sc.y + a[q].y * sc.x;
        __stcg(y + rr, b[q]);
      }
      if (NORM) {
        if (rr == j + 1) alpha = b[q];
        else __stcg(hn + rr, b[q]);
        if (q & 1) n1 = fma(b[q].x, b[q].x, fma(b[q].y, b[q].y, n1));
        else n0 = fma(b[q].x, b[q].x, fma(b[q].y, b[q].y, n0));
      }
    }
  }
  if (NORM) {
    *nrm2_out = warp_sum(n0 + n1);
    // row j + 1 is lane 0's first row
    alpha.x = __shfl_sync(0xffffffffu, alpha.x, 0);
    alpha.y = __shfl_sync(0xffffffffu, alpha.y, 0);
    *alpha_out = alpha;
  }
  __syncwarp();
}

// reflector j from the squared norm of column j (rows j..) and its entry alpha = x_j: tau_j, the
// scale s_j into H[j, j], beta into the diagonal of R (H[:, j] rows > j already hold x raw)
__device__ __forceinline__ void finish_reflector(const HMat& M, int j, double nrm2, double2 alpha, int lane) {
  if (lane == 0) {
    const double aabs = sqrt(alpha.x * alpha.x + alpha.y * alpha.y);
    const double nrm = sqrt(nrm2);
    double t = 0.0;
    double2 s = make_double2(0.0, 0.0), beta = alpha;
    if (nrm > 0.0) {
      const double2 ph = aabs > 0.0 ? make_double2(alpha.x / aabs, alpha.y / aabs) : make_double2(1.0, 0.0);
      beta = make_double2(-ph.x * nrm, -ph.y * nrm);
      const double2 uj = make_double2(ph.x * (aabs + nrm), ph.y * (aabs + nrm));      // alpha - beta
      const double uj2 = uj.x * uj.x + uj.y * uj.y;
      t = 2.0 * uj2 / (nrm2 - aabs * aabs + uj2);
      s = make_double2(uj.x / uj2, -uj.y / uj2);                                    // 1 / (alpha - beta)
    }
    __stcg(M.tau + j, t);
    __stcg(M.H + j + (size_t)j * M.m, s);
    M.R[j + (size_t)j * M.n] = beta;
  }
  __syncwarp();
}

// reflector 0 straight from column 0: one pass (norm, raw copy into H)
__device__ __forceinline__ void first_reflector(const HMat& M, int lane) {
  const double2* x = M.A;
  double n0 = 0.0;
  for (int r = 1 + lane; r < M.m; r += 32) {
    const double2 v = __ldcg(x + r);
    __stcg(M.H + r, v);
    n0 = fma(v.x, v.x, fma(v.y, v.y, n0));
  }
  const double2 a0 = __ldcg(x);
  const double nrm2 = warp_sum(n0) + a0.x * a0.x + a0.y * a0.y;
  finish_reflector(M, 0, nrm2, a0, lane);
}

}  // namespace

// The factorisation proper over n_items matrices, matrix `it` given by get(it, &M) (false: none).
template <class Get>
__device__ __forceinline__ void hqr_body(const Get& get, int n_items, GridSync gs, int* status) {
  __shared__ HMat s_mat[HQ_MAX_PAIRS];
  __shared__ int s_col[HQ_MAX_PAIRS];
  __shared__ int s_cnt, s_maxn;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x;
  if (n_items > HQ_MAX_ITEMS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(status, ST_CAPACITY);
    return;
  }
  // the (block, column) pairs of this CTA: global column g = prefix + k goes to CTA g mod G
  if (tid == 0) {
    int cnt = 0, maxn = 0;
    long long prefix = 0;
    bool over = false;
    for (int it = 0; it < n_items; ++it) {
      HMat M;
      if (!get(it, &M)) continue;
      maxn = max(maxn, M.n);
      int k0 = (int)(((long long)blockIdx.x - prefix) % G);
      if (k0 < 0) k0 += G;
      for (int k = k0; k < M.n; k += G) {
        if (cnt < HQ_MAX_PAIRS) {
          s_mat[cnt] = M;
          s_col[cnt] = k;
        } else {
          over = true;
        }
        ++cnt;
      }
      prefix += M.n;
    }
    if (over) atomicOr(status, ST_CAPACITY);
    s_cnt = over ? 0 : cnt;
    s_maxn = maxn;
  }
  __syncthreads();
  const int cnt = s_cnt, maxn = s_maxn;
  // reflector 0 of every block
  for (int t = wid; t < cnt; t += HQ_WARPS)
    if (s_col[t] == 0) first_reflector(s_mat[t], lane);
  if (!grid_barrier(gs, status)) return;
  // step j: reflector j on columns k > j; the owner of column j + 1 forms reflector j + 1 from the
  // same pass (its norm and raw copy)
  for (int j = 0; j + 1 < maxn; ++j) {
    for (int t = wid; t < cnt; t += HQ_WARPS) {
      const HMat& M = s_mat[t];
      const int k = s_col[t];
      if (k <= j || j + 1 >= M.n) continue;
      if (k == j + 1) {
        double nrm2;
        double2 alpha;
        apply_reflector<true>(M, j, M.A + (size_t)k * M.m, lane, &nrm2, &alpha);
        finish_reflector(M, j + 1, nrm2, alpha, lane);
      } else {
        apply_reflector<false>(M, j, M.A + (size_t)k * M.m, lane);
      }
    }
    if (!grid_barrier(gs, status)) return;
  }
  // R (strict upper part of each column) out, then the explicit Q column by column
  for (int t = wid; t < cnt; t += HQ_WARPS) {
    const HMat& M = s_mat[t];
    const int k = s_col[t];
    double2* a = M.A + (size_t)k * M.m;
    for (int r = lane; r < M.n; r += 32)
      if (r != k) M.R[r + (size_t)k * M.n] = r < k ? __ldcg(a + r) : make_double2(0.0, 0.0);
    __syncwarp();
    for (int r = lane; r < M.m; r += 32) __stcg(a + r, make_double2(r == k ? 1.0 : 0.0, 0.0));
    __syncwarp();
    for (int j = min(k, M.n - 1); j >= 0; --j) apply_reflector<false>(M, j, a, lane);
  }
}

__global__ void __launch_bounds__(HQ_THREADS, 1)
    k_hqr_grid(Tables T, const BondWork* work, int n_work, GridSync gs) {
  hqr_body([&](int it, HMat* M) { return hmat_of(T, work, it, M); }, 2 * n_work, gs, T.status);
}

// the same factorisation over a list of matrices (m >= n each; m or n = 0: skipped)
__global__ void __launch_bounds__(HQ_THREADS, 1)
    k_hqr_items(const QRItem* items, int n_items, GridSync gs, int* status) {
  hqr_body(
      [&](int it, HMat* M) {
        const QRItem q = items[it];
        if (q.m <= 0 || q.n <= 0 || q.n > q.m) return false;
        *M = q;
        return true;
      },
      n_items, gs, status);
}

int hqr_grid_fits(int total_cols_cap, int n_items, int blocks) {
  return blocks > 0 && n_items <= HQ_MAX_ITEMS && (total_cols_cap + blocks - 1) / blocks <= HQ_MAX_PAIRS;
}

int hqr_grid_ok() {
  int a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_hqr_grid, HQ_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a >= 1;
}

void launch_hqr_grid(const Tables& T, const BondWork* work, int n_work, int blocks, unsigned* sync3,
                     cudaStream_t st) {
  cudaMemsetAsync(sync3, 0, sizeof(unsigned), st);
  cudaMemsetAsync(sync3 + 2, 0, sizeof(unsigned), st);
  GridSync gs{sync3, (int*)(sync3 + 2), GRID_WAIT_LIMIT_CYCLES};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(HQ_THREADS, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_hqr_grid, T, work, n_work, gs);
}

void launch_hqr_items(const QRItem* items, int n_items, int blocks, unsigned* sync3, int* status, cudaStream_t st) {
  cudaMemsetAsync(sync3, 0, sizeof(unsigned), st);
  cudaMemsetAsync(sync3 + 2, 0, sizeof(unsigned), st);
  GridSync gs{sync3, (int*)(sync3 + 2), GRID_WAIT_LIMIT_CYCLES};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(HQ_THREADS, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_hqr_items, items, n_items, gs, status);
}

int hqr_items_ok() {
  int a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_hqr_items, HQ_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a >= 1;
}

}  // namespace ptk
