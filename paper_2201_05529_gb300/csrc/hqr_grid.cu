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

struct HMat {
  double2* A;      // m x n column-major: B on entry, Q on exit
  double2* H;      // reflector vectors, m x n column-major
  double2* R;      // n x n column-major
  double* tau;     // n
  int m, n;
};

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

// y <- P_j y on rows j.. (one warp)
__device__ __forceinline__ void apply_reflector(const HMat& M, int j, double2* y, int lane) {
  const double t = __ldcg(M.tau + j);
  if (t == 0.0) return;
  const double2* u = M.H + (size_t)j * M.m;
  double sr = 0.0, si = 0.0;
  for (int r = j + lane; r < M.m; r += 32) {
    const double2 a = __ldcg(u + r), b = __ldcg(y + r);
    sr = fma(a.x, b.x, fma(a.y, b.y, sr));              // conj(u) y
    si = fma(a.x, b.y, fma(-a.y, b.x, si));
  }
  sr = warp_sum(sr) * t;
  si = warp_sum(si) * t;
  for (int r = j + lane; r < M.m; r += 32) {
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
  double part = 0.0;
  for (int r = j + lane; r < M.m; r += 32) {
    const double2 v = __ldcg(x + r);
    part += v.x * v.x + v.y * v.y;
  }
  const double nrm2 = warp_sum(part);
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
  for (int r = j + lane; r < M.m; r += 32) {
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

__global__ void __launch_bounds__(HQ_THREADS, 1)
    k_hqr_grid(Tables T, const BondWork* work, int n_work, GridSync gs) {
  __shared__ HMat s_mat[HQ_MAX_PAIRS];
  __shared__ int s_col[HQ_MAX_PAIRS];
  __shared__ int s_cnt, s_maxn;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int G = gridDim.x;
  const int n_items = 2 * n_work;
  if (n_items > HQ_MAX_ITEMS) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(T.status, ST_CAPACITY);
    return;
  }
  // the (block, column) pairs of this CTA: global column g = prefix + k goes to CTA g mod G
  if (tid == 0) {
    int cnt = 0, maxn = 0;
    long long prefix = 0;
    bool over = false;
    for (int it = 0; it < n_items; ++it) {
      HMat M;
      if (!hmat_of(T, work, it, &M)) continue;
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
    if (over) atomicOr(T.status, ST_CAPACITY);
    s_cnt = over ? 0 : cnt;
    s_maxn = maxn;
  }
  __syncthreads();
  const int cnt = s_cnt, maxn = s_maxn;
  // reflector 0 of every block
  for (int t = wid; t < cnt; t += HQ_WARPS)
    if (s_col[t] == 0) make_reflector(s_mat[t], 0, lane);
  if (!grid_barrier(gs, T.status)) return;
  // step j: reflector j on columns k > j; the owner of column j + 1 forms reflector j + 1
  for (int j = 0; j + 1 < maxn; ++j) {
    for (int t = wid; t < cnt; t += HQ_WARPS) {
      const HMat& M = s_mat[t];
      const int k = s_col[t];
      if (k <= j || j + 1 >= M.n) continue;
      apply_reflector(M, j, M.A + (size_t)k * M.m, lane);
      if (k == j + 1) make_reflector(M, j + 1, lane);
    }
    if (!grid_barrier(gs, T.status)) return;
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

}  // namespace ptk
