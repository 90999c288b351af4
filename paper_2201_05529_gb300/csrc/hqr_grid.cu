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
// Reflectors as in k_householder: P_j = I - tau_j u_j u_j^H with u_j[j] = 1 (stored in HH), tau_j in
// aux (B_L) or sig (B_R^H), the diagonal of R = beta_j. Every grid barrier wait is bounded.
#include "grid_sync.cuh"
#include "kernels.h"

namespace ptk {

namespace {

constexpr int HQ_THREADS = 512;
constexpr int HQ_WARPS = HQ_THREADS / 32;
constexpr int HQ_MAX_PAIRS = 384;           // (block, column) pairs one CTA may own
constexpr int HQ_MAX_ITEMS = 2048;          // blocks: two per bond

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

// y <- P_j y on rows j.. (one warp). Four rows per lane per iteration: four independent L2 loads
// in flight per lane (the loops are latency-bound, not bandwidth-bound)
__device__ __forceinline__ void apply_reflector(const HMat& M, int j, double2* y, int lane) {
  const double t = __ldcg(M.tau + j);
  if (t == 0.0) return;
  const double2* u = M.H + (size_t)j * M.m;
  double sr0 = 0.0, si0 = 0.0, sr1 = 0.0, si1 = 0.0;
  int r = j + lane;
  for (; r + 96 < M.m; r += 128) {
    const double2 a0 = __ldcg(u + r), b0 = __ldcg(y + r);
    const double2 a1 = __ldcg(u + r + 32), b1 = __ldcg(y + r + 32);
    const double2 a2 = __ldcg(u + r + 64), b2 = __ldcg(y + r + 64);
    const double2 a3 = __ldcg(u + r + 96), b3 = __ldcg(y + r + 96);
    sr0 = fma(a0.x, b0.x, fma(a0.y, b0.y, sr0));              // conj(u) y
    si0 = fma(a0.x, b0.y, fma(-a0.y, b0.x, si0));
    sr1 = fma(a1.x, b1.x, fma(a1.y, b1.y, sr1));
    si1 = fma(a1.x, b1.y, fma(-a1.y, b1.x, si1));
    sr0 = fma(a2.x, b2.x, fma(a2.y, b2.y, sr0));
    si0 = fma(a2.x, b2.y, fma(-a2.y, b2.x, si0));
    sr1 = fma(a3.x, b3.x, fma(a3.y, b3.y, sr1));
    si1 = fma(a3.x, b3.y, fma(-a3.y, b3.x, si1));
  }
  for (; r < M.m; r += 32) {
    const double2 a = __ldcg(u + r), b = __ldcg(y + r);
    sr0 = fma(a.x, b.x, fma(a.y, b.y, sr0));
    si0 = fma(a.x, b.y, fma(-a.y, b.x, si0));
  }
  const double sr = warp_sum(sr0 + sr1) * t;
  const double si = warp_sum(si0 + si1) * t;
  r = j + lane;
  for (; r + 96 < M.m; r += 128) {
    double2 a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = __ldcg(u + r + 32 * q);
      b[q] = __ldcg(y + r + 32 * q);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      b[q].x -= a[q].x * sr - a[q].y * si;
      b[q].y -= a[q].x * si + a[q].y * sr;
      __stcg(y + r + 32 * q, b[q]);
    }
  }
  for (; r < M.m; r += 32) {
    const double2 a = __ldcg(u + r);
    double2 b = __ldcg(y + r);
    b.x -= a.x * sr - a.y * si;
    b.y -= a.x * si + a.y * sr;
    __stcg(y + r, b);
  }
  __syncwarp();
}

// reflector j from column j of A (rows j..), one warp
__device__ __forceinline__ void make_reflector(const HMat& M, int j, int lane) {
  const double2* x = M.A + (size_t)j * M.m;
  double p0 = 0.0, p1 = 0.0;
  int r = j + lane;
  for (; r + 96 < M.m; r += 128) {
    const double2 v0 = __ldcg(x + r), v1 = __ldcg(x + r + 32), v2 = __ldcg(x + r + 64), v3 = __ldcg(x + r + 96);
    p0 = fma(v0.x, v0.x, fma(v0.y, v0.y, p0));
    p1 = fma(v1.x, v1.x, fma(v1.y, v1.y, p1));
    p0 = fma(v2.x, v2.x, fma(v2.y, v2.y, p0));
    p1 = fma(v3.x, v3.x, fma(v3.y, v3.y, p1));
  }
  for (; r < M.m; r += 32) {
    const double2 v = __ldcg(x + r);
    p0 = fma(v.x, v.x, fma(v.y, v.y, p0));
  }
  const double nrm2 = warp_sum(p0 + p1);
  const double2 alpha = __ldcg(x + j);
  const double aabs = sqrt(alpha.x * alpha.x + alpha.y * alpha.y);
  const double nrm = sqrt(nrm2);
  double t = 0.0;
  double2 uj = make_double2(1.0, 0.0), beta = alpha;
  if (nrm > 0.0) {
    const double2 ph = aabs > 0.0 ? make_double2(alpha.x / aabs, alpha.y / aabs) : make_double2(1.0, 0.0);
    beta = make_double2(-ph.x * nrm, -ph.y * nrm);
    uj = make_double2(ph.x * (aabs + nrm), ph.y * (aabs + nrm));      // u_j = alpha - beta
    const double uj2 = uj.x * uj.x + uj.y * uj.y;
    t = 2.0 * uj2 / (nrm2 - aabs * aabs + uj2);
  }
  const double inv = 1.0 / (uj.x * uj.x + uj.y * uj.y);
  const double2 ujinv = make_double2(uj.x * inv, -uj.y * inv);        // 1 / u_j
  double2* u = M.H + (size_t)j * M.m;
  for (r = j + lane; r < M.m; r += 32) {
    double2 v = make_double2(1.0, 0.0);
    if (r != j) {
      const double2 xr = __ldcg(x + r);
      v = nrm > 0.0 ? make_double2(xr.x * ujinv.x - xr.y * ujinv.y, xr.x * ujinv.y + xr.y * ujinv.x)
                    : make_double2(0.0, 0.0);
    }
    __stcg(u + r, v);
  }
  if (lane == 0) {
    __stcg(M.tau + j, t);
    M.R[j + (size_t)j * M.n] = beta;
  }
  __syncwarp();
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
    if (s_col[t] == 0) make_reflector(s_mat[t], 0, lane);
  if (!grid_barrier(gs, status)) return;
  // step j: reflector j on columns k > j; the owner of column j + 1 forms reflector j + 1
  for (int j = 0; j + 1 < maxn; ++j) {
    for (int t = wid; t < cnt; t += HQ_WARPS) {
      const HMat& M = s_mat[t];
      const int k = s_col[t];
      if (k <= j || j + 1 >= M.n) continue;
      apply_reflector(M, j, M.A + (size_t)k * M.m, lane);
      if (k == j + 1) make_reflector(M, j + 1, lane);
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
    for (int j = min(k, M.n - 1); j >= 0; --j) apply_reflector(M, j, a, lane);
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
