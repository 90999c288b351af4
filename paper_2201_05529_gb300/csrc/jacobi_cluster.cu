// Cluster-parallel one-sided Jacobi SVD (App. A.2: the SVD of D).
//
// One thread-block cluster (up to 16 CTAs of 1024 threads) works on one matrix held column-major
// in global memory (L2-resident at these sizes). Each round of the round-robin tournament is a set
// of disjoint column pairs; the pairs are spread over every warp of the cluster and the rounds are
// separated by cluster barriers (release/acquire at cluster scope). A sweep-parity counter in
// global memory tells every CTA whether the sweep rotated anything. The scalar type R is double
// for the FP64 path and float for the FP32 preconditioning sweeps of the fast path.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace ptk {

template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };

template <typename C2> __device__ __forceinline__ auto c_abs2(C2 a) { return a.x * a.x + a.y * a.y; }

template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__device__ __forceinline__ R r_sqrt(R x) { return sqrt(x); }

// Rotate columns i, j of A (Ma rows) and V (Na rows) so that they become orthogonal.
template <typename R>
__device__ __forceinline__ bool jac_pair(typename CT<R>::T* A, typename CT<R>::T* V, int Ma, int Na,
                                         int i, int j, R tol, R floor2, int lane) {
  using C2 = typename CT<R>::T;
  C2* ai = A + (size_t)i * Ma;
  C2* aj = A + (size_t)j * Ma;
  R al = 0, be = 0, gr = 0, gi = 0;
  for (int r = lane; r < Ma; r += 32) {
    const C2 x = __ldcg(ai + r), y = __ldcg(aj + r);
    al = fma(x.x, x.x, fma(x.y, x.y, al));
    be = fma(y.x, y.x, fma(y.y, y.y, be));
    gr = fma(x.x, y.x, fma(x.y, y.y, gr));     // conj(x) * y
    gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
  }
  al = wsum(al);
  be = wsum(be);
  gr = wsum(gr);
  gi = wsum(gi);
  const R g2 = gr * gr + gi * gi;
  // columns at the rounding-noise level of the matrix (|a|^2 <= floor2) are not rotated: they can
  // never become orthogonal relative to their own norm and carry no information at this precision
  if (!(g2 > tol * tol * al * be) || g2 == R(0) || !(fmin(al, be) > floor2)) return false;
  const R g = r_sqrt(g2), h = be - al;
  // tan(theta) = 2 g sign(h) / (|h| + sqrt(h^2 + 4 g^2)), the smaller root of the rotation equation
  const R t = (h >= R(0) ? R(2) : R(-2)) * g / (fabs(h) + r_sqrt(h * h + R(4) * g2));
  const R c = R(1) / r_sqrt(R(1) + t * t), s = c * t;
  // e = exp(-i phi) = conj(gamma) / |gamma|
  const R er = gr / g, ei = -gi / g;
  const R ser = s * er, sei = s * ei, cer = c * er, cei = c * ei;
  for (int r = lane; r < Ma; r += 32) {
    const C2 x = __ldcg(ai + r), y = __ldcg(aj + r);
    C2 nx, ny;
    nx.x = c * x.x - (ser * y.x - sei * y.y);
    nx.y = c * x.y - (ser * y.y + sei * y.x);
    ny.x = s * x.x + (cer * y.x - cei * y.y);
    ny.y = s * x.y + (cer * y.y + cei * y.x);
    __stcg(ai + r, nx);
    __stcg(aj + r, ny);
  }
  C2* vi = V + (size_t)i * Na;
  C2* vj = V + (size_t)j * Na;
  for (int r = lane; r < Na; r += 32) {
    const C2 x = __ldcg(vi + r), y = __ldcg(vj + r);
    C2 nx, ny;
    nx.x = c * x.x - (ser * y.x - sei * y.y);
    nx.y = c * x.y - (ser * y.y + sei * y.x);
    ny.x = s * x.x + (cer * y.x - cei * y.y);
    ny.y = s * x.y + (cer * y.y + cei * y.x);
    __stcg(vi + r, nx);
    __stcg(vj + r, ny);
  }
  return true;
}

// Whole SVD of one matrix by one cluster. cnt: 2 ints of global scratch (sweep-parity counters).
// On exit: A columns normalised (left vectors), V right vectors, sig norms, perm by descending sig.
template <typename R>
__device__ void jacobi_cluster_svd(typename CT<R>::T* A, typename CT<R>::T* V, R* sig, int* perm,
                                   R* aux, int* cnt, int Ma, int Na, int max_sweeps, bool init_v,
                                   R tol, R unit_roundoff, int* sweeps_out, int* status) {
  using C2 = typename CT<R>::T;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), ncta = (int)cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwb = blockDim.x >> 5;
  const int gw = wid * ncta + rank, ngw = ncta * nwb;     // pairs interleaved over the CTAs
  const int gt = rank * blockDim.x + tid, ngt = ncta * blockDim.x;
  if (init_v)
    for (size_t idx = gt; idx < (size_t)Na * Na; idx += ngt) {
      C2 v;
      v.x = ((idx % Na) == (idx / Na)) ? R(1) : R(0);
      v.y = R(0);
      V[idx] = v;
    }
  if (rank == 0 && tid == 0) {
    cnt[0] = 0;
    cnt[1] = 0;
  }
  // ||A||_F^2 (invariant under the rotations), summed in a fixed order for reproducibility
  for (int c = gw; c < Na; c += ngw) {
    const C2* a = A + (size_t)c * Ma;
    R s2 = 0;
    for (int r = lane; r < Ma; r += 32) s2 += c_abs2(__ldcg(a + r));
    s2 = wsum(s2);
    if (lane == 0) __stcg(aux + c, s2);
  }
  cl.sync();
  __shared__ R fro_s;
  if (wid == 0) {
    R acc = 0;
    for (int k = lane; k < Na; k += 32) acc += __ldcg(aux + k);
    acc = wsum(acc);
    if (lane == 0) fro_s = acc;
  }
  __syncthreads();
  const R floor2 = unit_roundoff * unit_roundoff * fro_s;
  const int Np = Na + (Na & 1);
  int sweep = 0;
  bool converged = Na < 2;
  cl.sync();
  while (!converged && sweep < max_sweeps) {
    const int par = sweep & 1;
    if (rank == 0 && tid == 0) cnt[par ^ 1] = 0;     // nobody touches the other counter this sweep
    int mine = 0;
    for (int round = 0; round < Np - 1; ++round) {
      for (int q = gw; q < Np / 2; q += ngw) {
        int i, j;
        if (q == 0) { i = Np - 1; j = round; }
        else { i = (round + q) % (Np - 1); j = (round - q + Np - 1) % (Np - 1); }
        if (i > j) { const int t = i; i = j; j = t; }
        if (j >= Na) continue;
        mine += jac_pair<R>(A, V, Ma, Na, i, j, tol, floor2, lane) ? 1 : 0;
      }
      cl.sync();
    }
    if (lane == 0 && mine) atomicAdd(&cnt[par], mine);
    cl.sync();
    converged = (*(volatile int*)&cnt[par]) == 0;
    ++sweep;
    cl.sync();
  }
  if (rank == 0 && tid == 0) {
    *sweeps_out = converged ? sweep : -sweep;
    if (!converged) atomicOr(status, ST_SVD_NOCONV);
  }
  for (int c = gw; c < Na; c += ngw) {
    C2* a = A + (size_t)c * Ma;
    R s2 = 0;
    for (int r = lane; r < Ma; r += 32) s2 += c_abs2(__ldcg(a + r));
    s2 = wsum(s2);
    const R s = r_sqrt(s2);
    if (lane == 0) sig[c] = s;
    if (s > R(0)) {
      const R inv = R(1) / s;
      for (int r = lane; r < Ma; r += 32) {
        C2 x = __ldcg(a + r);
        x.x *= inv;
        x.y *= inv;
        __stcg(a + r, x);
      }
    }
    if (lane == 0 && !(s == s)) atomicOr(status, ST_NAN);
  }
  cl.sync();
  for (int c = gt; c < Na; c += ngt) {
    // a NaN ranks as -1 so the ranks stay a permutation (perm indexes columns downstream)
    R sc = __ldcg(sig + c);
    if (!(sc == sc)) sc = R(-1);
    int rk = 0;
    for (int k = 0; k < Na; ++k) {
      R sk = __ldcg(sig + k);
      if (!(sk == sk)) sk = R(-1);
      rk += (sk > sc) || (sk == sc && k < c);
    }
    perm[rk] = c;
  }
  cl.sync();
}

// FP64 bond SVDs: one cluster per work item (blockIdx.x / cluster size).
__global__ void __launch_bounds__(1024) k_jacobi_cluster(const BondWork* work, int n_work, int max_sweeps,
                                                         int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int w = blockIdx.x / cl.num_blocks();
  if (w >= n_work) return;
  const BondWork& W = work[w];
  const int mD = W.info[0], nD = W.info[1];
  if (mD <= 0 || nD <= 0) return;
  const bool tr = W.info[2] != 0;
  const int Ma = tr ? nD : mD, Na = tr ? mD : nD;
  jacobi_cluster_svd<double>(W.A, W.V, W.sig, W.perm, W.aux, W.info + 4, Ma, Na, max_sweeps, true,
                             (double)Ma * 1.1102230246251565e-16, 1.1102230246251565e-16, W.info + 3,
                             status);
}

static cudaLaunchConfig_t jac_cfg(int n_work, int cluster, cudaStream_t st, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_work * cluster, 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Largest cluster size (16, 8, 4, 2, 1) the device can co-schedule for the bond SVD kernel.
int jacobi_cluster_size(int want) {
  cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= 1; c >>= 1) {
    if (c > want) continue;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = jac_cfg(1, c, 0, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_jacobi_cluster, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

void launch_jacobi_cluster(const BondWork* work, int n_work, int cluster, int max_sweeps, int* status,
                           cudaStream_t st) {
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = jac_cfg(n_work, cluster, st, at);
  cudaLaunchKernelEx(&cfg, k_jacobi_cluster, work, n_work, max_sweeps, status);
}

}  // namespace ptk
